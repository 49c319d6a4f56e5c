/*
 * FP64 CPU oracle for the D3Q19 BGK lattice Boltzmann update.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct
 * reference that the CUDA path is checked against. Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product library never links, calls or falls back to it. It shares no code,
 * table or helper with the CUDA sources.
 *
 * What it computes (Sec. 2 of Habich et al., "Performance engineering for the
 * lattice Boltzmann method on GPGPUs"):
 *   - moments rho = sum f_i, j = sum f_i e_i                (Sec. 2, step 1)
 *   - the D3Q19 equilibrium of Qian et al. (cited in Sec. 2)
 *   - BGK relaxation f* = f - (f - f_eq)/tau                (Eq. 1, Sec. 2 step 2)
 *   - propagation to x + e_i                                (Sec. 2, step 3)
 *   - bounce-back at non-fluid cells, folded into the stream (Sec. 2, Ziegler rule)
 * Readings where the paper is silent (each is listed in the design notes):
 *   - Eq. 1 prints a doubled minus; a single minus is meant, as in the inline
 *     collide formula of Sec. 2.
 *   - u = (j + F/2)/rho (compressible Qian equilibrium, Guo forcing).
 *   - the body force is Guo, Zheng & Shi (2002): the source term
 *     S_i = (1 - 1/(2 tau)) w_i [3 (e_i - u) + 9 (e_i.u) e_i] . F.
 *   - bounce-back is the halfway rule: a population pushed into a solid cell
 *     returns to its origin with the opposite velocity in the same step.
 *   - a solid cell flagged 2 is a wall moving with velocity u_w (the paper's
 *     lid-driven cavity, Sec. 7): the reflected population loses
 *     2 w_i rho_w (e_i . u_w) / c_s^2 = 6 w_i (e_i . u_w), with the wall
 *     density rho_w taken as the reference density 1 (Ladd's rule).
 *   - all three axes are periodic; walls are solid flag layers.
 *   - model 1 is the incompressible equilibrium of He & Luo (1997), the
 *     reading of the paper's "incompressible flow solver" wording with the
 *     1/rho of its velocity moment left out (Sec. 1, Sec. 2 step 1): the
 *     velocity terms carry the reference density rho0 = 1 instead of rho and
 *     u = j + F/2. Model 0 is the Qian equilibrium above.
 * The state is the pre-collision populations f^n (push form), canonical layout
 * f[i][z][y][x], x fastest. Solid cells hold zeros.
 *
 * Storage-rounding emulation (optional, fmt != 0): after every stream step the
 * shifted deviation s_i = f_i - w_i of every fluid entry is rounded to the
 * nearest value of a narrower IEEE format (ties to even), written from the
 * format's definition (sign, exponent range, mantissa width).
 *
 * Moment-split storage (fmt 4: binary16, fmt 5: bfloat16; a storage format of
 * this library, not of the paper): the 19 post-collision values P_i of a cell
 * are kept as their momentum J = sum_i P_i e_i and the remainders
 * g_i = (P_i - w_i) - 3 w_i (e_i . J~), where J~ is J rounded to the element
 * format; g_i is rounded too, and a reader rebuilds
 * P~_i = w_i + 3 w_i (e_i . J~) + g~_i. The rebuilt value is off by the
 * rounding of g_i alone, which is small next to the deviation itself in a
 * flow whose populations are near their linear equilibrium part. The rounding
 * is applied where a cell's values are written: to the post-collision values
 * of every fluid cell before they stream, and to the initial state grouped as
 * the values each cell holds for its neighbours to pull.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19

/* D3Q19 velocity set (Qian et al., cited in Sec. 2). Order: rest, six axis
 * directions +x,-x,+y,-y,+z,-z, then the twelve edge diagonals in the groups
 * (+-1,+-1,0), (+-1,0,+-1), (0,+-1,+-1) with + before -. */
static const int E[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {1, -1, 0}, {-1, 1, 0}, {-1, -1, 0},
    {1, 0, 1},  {1, 0, -1}, {-1, 0, 1}, {-1, 0, -1},
    {0, 1, 1},  {0, 1, -1}, {0, -1, 1}, {0, -1, -1},
};

/* Weights: 1/3 rest, 1/18 axis, 1/36 diagonal (Qian et al.). */
static double weight(int i)
{
    if (i == 0) return 1.0 / 3.0;
    if (i <= 6) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

/* Index of the velocity -e_i, found by search. */
static int opposite(int i)
{
    for (int k = 0; k < Q; ++k)
        if (E[k][0] == -E[i][0] && E[k][1] == -E[i][1] && E[k][2] == -E[i][2])
            return k;
    return -1;
}

static int wrap(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

static int64_t cell(int x, int y, int z, int nx, int ny)
{
    return (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
}

/* Export of the table above, so that a test can compare it with the table
 * the CUDA library was compiled with. */
void oracle_lattice(int *e /* [19][3] */, double *w /* [19] */, int *opp /* [19] */)
{
    for (int i = 0; i < Q; ++i) {
        for (int a = 0; a < 3; ++a) e[3 * i + a] = E[i][a];
        w[i] = weight(i);
        opp[i] = opposite(i);
    }
}

/* f_eq_i(rho, u) = w_i rho [1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u] (Qian et al.). */
void oracle_equilibrium(double rho, const double *u, double *feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; ++i) {
        double eu = E[i][0] * u[0] + E[i][1] * u[1] + E[i][2] * u[2];
        feq[i] = weight(i) * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* He & Luo incompressible equilibrium (model 1): the density enters only the
 * zeroth-order term, the velocity terms are those of the reference density 1:
 *   f_eq_i(rho, u) = w_i [rho + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u]. */
void oracle_equilibrium_incompressible(double rho, const double *u, double *feq)
{
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; ++i) {
        double cu = E[i][0] * u[0] + E[i][1] * u[1] + E[i][2] * u[2];
        feq[i] = weight(i) * (rho + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
    }
}

/* Moments of one cell for the incompressible model: rho = sum f_i, and the
 * velocity is the momentum over the reference density 1, u = sum f_i e_i + F/2. */
void oracle_moments_incompressible(const double *f, const double *F, double *rho_out, double *u_out)
{
    double r = 0.0, mom[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
        r += f[i];
        for (int a = 0; a < 3; ++a) mom[a] += E[i][a] * f[i];
    }
    *rho_out = r;
    for (int a = 0; a < 3; ++a) u_out[a] = mom[a] + F[a] / 2.0;
}

/* Moments of one cell: rho = sum f_i, u = (sum f_i e_i + F/2) / rho. */
void oracle_moments(const double *f, const double *F, double *rho_out, double *u_out)
{
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
        rho += f[i];
        for (int a = 0; a < 3; ++a) j[a] += f[i] * E[i][a];
    }
    *rho_out = rho;
    for (int a = 0; a < 3; ++a) u_out[a] = (j[a] + 0.5 * F[a]) / rho;
}

/* Collide one cell (Eq. 1 with the Guo source term): fout = f - (f - feq)/tau + S,
 * with the moments and equilibrium of `model` (0 Qian, 1 incompressible). */
void oracle_collide_cell_model(int model, const double *f, double tau, const double *F, double *fout)
{
    double rho, u[3], feq[Q];
    if (model == 1) {
        oracle_moments_incompressible(f, F, &rho, u);
        oracle_equilibrium_incompressible(rho, u, feq);
    } else {
        oracle_moments(f, F, &rho, u);
        oracle_equilibrium(rho, u, feq);
    }
    double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    for (int i = 0; i < Q; ++i) {
        double eu = E[i][0] * u[0] + E[i][1] * u[1] + E[i][2] * u[2];
        double eF = E[i][0] * F[0] + E[i][1] * F[1] + E[i][2] * F[2];
        double S = (1.0 - 1.0 / (2.0 * tau)) * weight(i) * (3.0 * (eF - uF) + 9.0 * eu * eF);
        fout[i] = f[i] - (f[i] - feq[i]) / tau + S;
    }
}

void oracle_collide_cell(const double *f, double tau, const double *F, double *fout)
{
    oracle_collide_cell_model(0, f, tau, F, fout);
}

/* Force at cell c: uniform (F_per_cell == 0, F = [3]) or a field F[3][N]. */
static void force_at(const double *F, int F_per_cell, int64_t c, int64_t N, double *out)
{
    for (int a = 0; a < 3; ++a) {
        if (!F) out[a] = 0.0;
        else if (F_per_cell) out[a] = F[a * N + c];
        else out[a] = F[a];
    }
}

static int is_fluid(const uint8_t *flags, int64_t c)
{
    return flags == NULL || flags[c] == 0;
}

static int is_moving_wall(const uint8_t *flags, int64_t c)
{
    return flags != NULL && flags[c] == 2;
}

/* ---- storage rounding emulation (ties to even) ---------------------------
 * A binary format with `mant` stored mantissa bits and smallest normal
 * exponent emin: values in [2^e, 2^(e+1)) are spaced 2^(max(e,emin) - mant)
 * apart; nearbyint() in the default rounding mode rounds to nearest, ties to
 * even. Values beyond the largest finite `maxval` become infinities. */
static double round_format(double v, int mant, int emin, double maxval)
{
    if (v == 0.0 || !isfinite(v)) return v;
    int ex;
    frexp(v, &ex); /* |v| = m 2^ex, m in [0.5, 1) */
    int e = ex - 1;
    if (e < emin) e = emin;
    double q = ldexp(1.0, e - mant);
    double r = nearbyint(v / q) * q;
    if (fabs(r) > maxval) r = copysign(INFINITY, v);
    return r;
}

/* fmt: 1 = IEEE binary32, 2 = IEEE binary16, 3 = bfloat16; the moment-split
 * formats 4 and 5 round their elements as binary16 and bfloat16. */
double oracle_round(double v, int fmt)
{
    switch (fmt) {
    case 1: return round_format(v, 23, -126, 3.4028234663852886e38);
    case 2: case 4: return round_format(v, 10, -14, 65504.0);
    case 3: case 5: return round_format(v, 7, -126, 3.3895313892515355e38);
    default: return v;
    }
}

static int is_split(int fmt) { return fmt == 4 || fmt == 5; }

/* The 19 values P[i] one cell stores, through the moment-split format fmt:
 * J = sum_i P_i e_i rounded, g_i = (P_i - w_i) - 3 w_i (e_i . J~) rounded,
 * P_i <- w_i + (3 w_i (e_i . J~) + g~_i). */
void oracle_split_round(double *P, int fmt)
{
    double J[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < 3; ++a) J[a] += P[i] * E[i][a];
    for (int a = 0; a < 3; ++a) J[a] = oracle_round(J[a], fmt);
    for (int i = 0; i < Q; ++i) {
        double w = weight(i);
        double base = 3.0 * w * (E[i][0] * J[0] + E[i][1] * J[1] + E[i][2] * J[2]);
        double g = oracle_round((P[i] - w) - base, fmt);
        P[i] = w + (base + g);
    }
}

/* Storage rounding of the elementwise formats (1-3): every fluid entry's
 * deviation s_i = f_i - w_i, after each stream step and at init. */
static void round_storage(double *f, const uint8_t *flags, int64_t N, int fmt)
{
    if (!fmt || is_split(fmt)) return;
    for (int i = 0; i < Q; ++i) {
        double w = weight(i);
        for (int64_t c = 0; c < N; ++c)
            if (is_fluid(flags, c)) f[i * N + c] = w + oracle_round(f[i * N + c] - w, fmt);
    }
}

/* A pre-collision state f (push form) as it is held in moment-split storage
 * by cells that each store the values their neighbours pull: fluid cell x
 * holds P_i(x) = f_i(x + e_i) when x + e_i is fluid, else f_opp(i)(x) (the
 * halfway bounce-back of x's own population). Each fluid cell's 19 values go
 * through oracle_split_round, and f is rebuilt from them: f_i(y) = P_i(y - e_i)
 * when y - e_i is fluid, else P_opp(i)(y). Returns -1 if scratch allocation
 * failed. */
static int store_split(int nx, int ny, int nz, const uint8_t *flags, double *f, int fmt)
{
    int64_t N = (int64_t)nx * ny * nz;
    double *P = (double *)malloc(sizeof(double) * Q * N);
    if (!P) return -1;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t c = cell(x, y, z, nx, ny);
                if (!is_fluid(flags, c)) continue;
                double v[Q];
                for (int i = 0; i < Q; ++i) {
                    int64_t d = cell(wrap(x + E[i][0], nx), wrap(y + E[i][1], ny), wrap(z + E[i][2], nz), nx, ny);
                    v[i] = is_fluid(flags, d) ? f[i * N + d] : f[opposite(i) * N + c];
                }
                oracle_split_round(v, fmt);
                for (int i = 0; i < Q; ++i) P[i * N + c] = v[i];
            }
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t c = cell(x, y, z, nx, ny);
                if (!is_fluid(flags, c)) continue;
                for (int i = 0; i < Q; ++i) {
                    int64_t s = cell(wrap(x - E[i][0], nx), wrap(y - E[i][1], ny), wrap(z - E[i][2], nz), nx, ny);
                    f[i * N + c] = is_fluid(flags, s) ? P[i * N + s] : P[opposite(i) * N + c];
                }
            }
    free(P);
    return 0;
}

/* A state f written to storage format fmt (as lbm_set_state would hold it):
 * the elementwise rounding of formats 1-3, or the moment-split storage of
 * formats 4 and 5. Returns 0, or -1 if scratch allocation failed. */
int oracle_store(int nx, int ny, int nz, const uint8_t *flags, double *f, int fmt)
{
    if (is_split(fmt)) return store_split(nx, ny, nz, flags, f, fmt);
    round_storage(f, flags, (int64_t)nx * ny * nz, fmt);
    return 0;
}

/* f[i][c] = f_eq_i(rho0(c), u0(c)) at fluid cells, 0 at solid cells, with the
 * equilibrium of `model`. rho0 may be NULL (rho0 = 1). Optional storage
 * rounding as in oracle_store. Returns 0, or -1 if scratch allocation failed. */
int oracle_init(int nx, int ny, int nz, const uint8_t *flags, const double *rho0,
                const double *u0 /* [3][N] */, double *f /* [19][N] */, int fmt, int model)
{
    int64_t N = (int64_t)nx * ny * nz;
    for (int64_t c = 0; c < N; ++c) {
        double feq[Q], u[3] = {0.0, 0.0, 0.0}, rho = 1.0;
        if (is_fluid(flags, c)) {
            if (rho0) rho = rho0[c];
            for (int a = 0; a < 3; ++a) u[a] = u0[a * N + c];
            if (model == 1)
                oracle_equilibrium_incompressible(rho, u, feq);
            else
                oracle_equilibrium(rho, u, feq);
        } else {
            for (int i = 0; i < Q; ++i) feq[i] = 0.0;
        }
        for (int i = 0; i < Q; ++i) f[i * N + c] = feq[i];
    }
    return oracle_store(nx, ny, nz, flags, f, fmt);
}

/* One collide-and-push step from cur to nxt (Sec. 2 steps 1-3 plus the
 * bounce-back rule). Every fluid entry of nxt is written exactly once. */
static void step_once(int nx, int ny, int nz, double tau, const uint8_t *flags,
                      const double *F, int F_per_cell, const double *u_wall, const double *cur,
                      double *nxt, int nthreads, int model, int fmt)
{
    int64_t N = (int64_t)nx * ny * nz;
    memset(nxt, 0, sizeof(double) * Q * N);
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (int z = 0; z < nz; ++z) {
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                int64_t c = cell(x, y, z, nx, ny);
                if (!is_fluid(flags, c)) continue;
                double f[Q], fs[Q], Fc[3];
                for (int i = 0; i < Q; ++i) f[i] = cur[i * N + c];
                force_at(F, F_per_cell, c, N, Fc);
                oracle_collide_cell_model(model, f, tau, Fc, fs);
                if (is_split(fmt)) oracle_split_round(fs, fmt); /* stored where computed */
                for (int i = 0; i < Q; ++i) {
                    int xd = wrap(x + E[i][0], nx), yd = wrap(y + E[i][1], ny),
                        zd = wrap(z + E[i][2], nz);
                    int64_t d = cell(xd, yd, zd, nx, ny);
                    if (is_fluid(flags, d)) {
                        nxt[i * N + d] = fs[i];        /* stream to x + e_i */
                    } else {
                        double moving = 0.0;           /* halfway bounce-back */
                        if (u_wall && is_moving_wall(flags, d))
                            moving = 6.0 * weight(i) *
                                     (E[i][0] * u_wall[0] + E[i][1] * u_wall[1] + E[i][2] * u_wall[2]);
                        nxt[opposite(i) * N + c] = fs[i] - moving;
                    }
                }
            }
        }
    }
    (void)nthreads;
}

/* Advance f (in place) by nsteps with the collision of `model`; u_wall
 * (nullable) is the velocity of the cells flagged 2. Returns 0, or -1 if
 * scratch allocation failed. */
int oracle_run(int nx, int ny, int nz, double tau, const uint8_t *flags, const double *F,
               int F_per_cell, const double *u_wall, double *f, int nsteps, int fmt, int nthreads, int model)
{
    int64_t N = (int64_t)nx * ny * nz;
    double *tmp = (double *)malloc(sizeof(double) * Q * N);
    if (!tmp) return -1;
    if (nthreads < 1) nthreads = 1;
    double *a = f, *b = tmp;
    for (int s = 0; s < nsteps; ++s) {
        step_once(nx, ny, nz, tau, flags, F, F_per_cell, u_wall, a, b, nthreads, model, fmt);
        round_storage(b, flags, N, fmt);
        double *t = a; a = b; b = t;
    }
    if (a != f) memcpy(f, a, sizeof(double) * Q * N);
    free(tmp);
    return 0;
}

/* Moments of one cell under `model`. */
static void moments_of(int model, const double *f, const double *F, double *rho, double *u)
{
    if (model == 1)
        oracle_moments_incompressible(f, F, rho, u);
    else
        oracle_moments(f, F, rho, u);
}

/* Macroscopic fields at state f: rho [N] and u [3][N]; 0 at solid cells. */
void oracle_macros(int nx, int ny, int nz, const uint8_t *flags, const double *F,
                   int F_per_cell, const double *f, double *rho, double *u, int model)
{
    int64_t N = (int64_t)nx * ny * nz;
    for (int64_t c = 0; c < N; ++c) {
        double fc[Q], Fc[3], r = 0.0, uc[3] = {0.0, 0.0, 0.0};
        if (is_fluid(flags, c)) {
            for (int i = 0; i < Q; ++i) fc[i] = f[i * N + c];
            force_at(F, F_per_cell, c, N, Fc);
            moments_of(model, fc, Fc, &r, uc);
        }
        if (rho) rho[c] = r;
        for (int a = 0; a < 3; ++a) u[a * N + c] = uc[a];
    }
}

/* Totals over fluid cells: out = {sum rho, and the three components of the
 * sum of the momentum j + F/2} (rho u for model 0, u for model 1).
 * Accumulated in cell order. */
void oracle_sums(int nx, int ny, int nz, const uint8_t *flags, const double *F, int F_per_cell,
                 const double *f, double *out, int model)
{
    int64_t N = (int64_t)nx * ny * nz;
    for (int k = 0; k < 4; ++k) out[k] = 0.0;
    for (int64_t c = 0; c < N; ++c) {
        if (!is_fluid(flags, c)) continue;
        double fc[Q], Fc[3], r, uc[3];
        for (int i = 0; i < Q; ++i) fc[i] = f[i * N + c];
        force_at(F, F_per_cell, c, N, Fc);
        moments_of(model, fc, Fc, &r, uc);
        out[0] += r;
        for (int a = 0; a < 3; ++a) out[1 + a] += model == 1 ? uc[a] : r * uc[a];
    }
}

/* Number of threads OpenMP would use (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
