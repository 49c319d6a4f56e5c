// Discrete adjoint of the D3Q19 BGK + Guo update (not in the paper; the
// transpose of the forward kernels in lbm_kernels.cuh), and the final stage
// of the FP64 reduction.
//
// Forward step n at fluid cell x, in shifted populations s:
//   f^{n+1} = G(C(f^n)),  C: s*_k = (1 - w) s_k + w seq_k(rho, j') + S_k(u, F)
// with w = 1/tau, j' = j + F/2, u = j'/rho, and G the streaming/bounce-back
// permutation. The adjoint lambda^n = dL/df^n obeys
//   mu = G^T lambda^{n+1}:  mu_k(x) = lambda_k(x + e_k) if x + e_k is fluid,
//                                     lambda_{opp(k)}(x) otherwise,
//   lambda^n_m(x) = sum_k mu_k ds*_k/ds_m
//                 = (1 - w) mu_m + [w a - d.u/rho] + [w b + d/rho] . e_m,
// where, with A_k = d f_eq_k / d rho (at fixed j'), B_k = grad_j' f_eq_k and
// D_k = grad_u S_k:
//   a = sum mu_k A_k,  A_k = w_k [1 - 9/2 (e_k.u)^2 + 3/2 u.u]
//   b = sum mu_k B_k,  B_k = w_k [3 e_k + 9 (e_k.u) e_k - 3 u]
//   d = sum mu_k D_k,  D_k = (1 - w/2) w_k [-3 F + 9 (e_k.F) e_k]
// and the force gradient of that step is dL/dF(x) += b + d / (2 rho).
// In the incompressible model (He & Luo: u = j', f_eq with the reference
// density 1 in its velocity terms) A_k = w_k, u does not depend on rho, so
//   lambda^n_m = (1 - w) mu_m + w sum_k mu_k w_k + [w b + d] . e_m,
// and dL/dF(x) += b + d / 2 (B_k and D_k are unchanged).
// Only (rho, u) of f^n enter, so the forward pass records just those.
#include "lbm_launch.h"

namespace lbm {

__device__ __forceinline__ double warp_sum_final(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum RED_BLOCKS x 4 partials in a fixed order (one block).
__global__ void __launch_bounds__(RED_THREADS) k_reduce_final(const double *__restrict__ partials, int nblocks,
                                                             double *__restrict__ out) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += partials[b * 4 + k];
    __shared__ double sm[RED_THREADS / 32][4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double v = warp_sum_final(acc[k]);
        if (lane == 0) sm[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) t += sm[w][threadIdx.x];
        out[threadIdx.x] = t;
    }
}

// lambda^n of one cell from mu = G^T lambda^{n+1}, the recorded (rho, u) and
// the force (see the header comment); adds this step's dL/dF to g.
template <class R, bool FORCE>
__device__ __forceinline__ void adj_collide(R mu[Q], R rho, R ux, R uy, R uz, R Fx, R Fy, R Fz, R om, R &gx, R &gy,
                                            R &gz, bool incomp) {
    const R usq = ux * ux + uy * uy + uz * uz;
    // P = sum_k w_k mu_k; A4 = sum over pairs w p (e.u)^2; b = sum w (3 q + 9 (e.u) p) e;
    // d = sum w p (e.F) e; with p = mu_i + mu_opp(i), q = mu_i - mu_opp(i)
    R P = R(1.0 / 3.0) * mu[0], A4 = R(0);
    R bx = R(0), by = R(0), bz = R(0), dx = R(0), dy = R(0), dz = R(0);
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) {
        const int i = pair_first(p), o = opp(i);
        const R w = i <= 6 ? R(1.0 / 18.0) : R(1.0 / 36.0);
        const R pp = mu[i] + mu[o], qq = mu[i] - mu[o];
        const R eu = R(ex(i)) * ux + R(ey(i)) * uy + R(ez(i)) * uz;
        P += w * pp;
        A4 += w * pp * eu * eu;
        const R t = w * (R(3) * qq + R(9) * eu * pp);
        bx += t * R(ex(i));
        by += t * R(ey(i));
        bz += t * R(ez(i));
        if (FORCE) {
            const R eF = R(ex(i)) * Fx + R(ey(i)) * Fy + R(ez(i)) * Fz;
            const R td = w * pp * eF;
            dx += td * R(ex(i));
            dy += td * R(ey(i));
            dz += td * R(ez(i));
        }
    }
    const R a = incomp ? P : P * (R(1) + R(1.5) * usq) - R(4.5) * A4;
    bx -= R(3) * ux * P;
    by -= R(3) * uy * P;
    bz -= R(3) * uz * P;
    if (FORCE) {
        const R cF = R(1) - R(0.5) * om;
        dx = cF * (R(9) * dx - R(3) * Fx * P);
        dy = cF * (R(9) * dy - R(3) * Fy * P);
        dz = cF * (R(9) * dz - R(3) * Fz * P);
    }
    const R inv = incomp ? R(1) : R(1) / rho;
    const R alpha = incomp ? om * a : om * a - (dx * ux + dy * uy + dz * uz) * inv;
    const R betx = om * bx + dx * inv, bety = om * by + dy * inv, betz = om * bz + dz * inv;
    const R keep = R(1) - om;
#pragma unroll
    for (int i = 0; i < Q; ++i) mu[i] = keep * mu[i] + alpha + R(ex(i)) * betx + R(ey(i)) * bety + R(ez(i)) * betz;
    const R h = R(0.5) * inv;
    gx = bx + dx * h;
    gy = by + dy * h;
    gz = bz + dz * h;
}

// One reverse step for the two x-adjacent cells x0, x0 + 1 of a row, in the
// layout of the forward step kernel. mu = G^T lambda^{n+1} is gathered with the
// push mask (bit i: x + e_i is solid, so mu_i(x) = lambda_opp(i)(x) from the
// cell itself); threads whose two cells are solid skip everything.
// Resident 256-thread blocks per SM: FP64 1; FP32 2 (128 registers hold the
// early grad_F loads without spilling: 149 us per step on the walled channel,
// against 168 us at 3 blocks with the loads at the end and 181 us at 3 blocks
// with them early and spilled).
template <class R> struct AdjBlocks {
    static constexpr int value = sizeof(R) == 8 ? 1 : 2;
};

// FLAT: the launch of d.PF (pairs in plane order), else of d.P (whole rows).
template <class R, bool FLAGS, bool FORCE, bool FLAT>
__global__ void __launch_bounds__(256, AdjBlocks<R>::value)
    k_adj_step(const Dev d, const R *__restrict__ lam_in, R *__restrict__ lam_out, const R *__restrict__ tape,
               R *__restrict__ grad_F) {
    int x0, y, z;
    if (!pair_cell<FLAT>(d.g, FLAT ? d.PF : d.P, blockDim.x, blockDim.y, blockIdx.x, blockIdx.y, threadIdx.x,
                         threadIdx.y, x0, y, z))
        return;
    const Geom &g = d.g;
    const bool has1 = x0 + 1 < g.nx;
    const int c = cell_index(g, x0, y, z);
    const long long qs = g.qs;
    uint32_t m0 = 0u, m1 = has1 ? 0u : SOLID_BIT;
    if (FLAGS) {
        const uint2 mm = ld_resident2(d.mask + c);
        m0 = mm.x;
        m1 |= mm.y;
    }
    const bool live0 = !(m0 & SOLID_BIT), live1 = !(m1 & SOLID_BIT);
    if (FLAGS && !live0 && !live1) return;
    // mu_i(x) = lambda_i(x + e_i): source columns of the e_x = +-1 populations
    const int xa = wrap1(x0 - 1, g.nx);              // e_x = -1, cell x0 (e_x = -1 of x0 + 1 reads x0)
    const int xb = wrap1(x0 + 1, g.nx);              // e_x = +1, cell x0
    const int xc = has1 ? wrap1(x0 + 2, g.nx) : x0;  // e_x = +1, cell x0 + 1
    // this step's dL/dF is added to grad_F, which only this thread touches:
    // load it now, with the gather, not after the collision
    const long long N = d.n_cells, cc = canon_index(g, x0, y, z);
    R G0x = R(0), G0y = R(0), G0z = R(0), G1x = R(0), G1y = R(0), G1z = R(0);
    if (grad_F) {
        if (live0) {
            G0x = grad_F[cc];
            G0y = grad_F[N + cc];
            G0z = grad_F[2 * N + cc];
        }
        if (live1) {
            G1x = grad_F[cc + 1];
            G1y = grad_F[N + cc + 1];
            G1z = grad_F[2 * N + cc + 1];
        }
    }
    R mu0[Q], mu1[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int row = (wrap1(z + ez(i), g.nz) * g.ny + wrap1(y + ey(i), g.ny)) * g.pitch;
        const R *Li = lam_in + (long long)i * qs + row;
        const R *Lo = lam_in + (long long)opp(i) * qs + c;  // own cell, opposite population
        const bool b0 = FLAGS && i > 0 && ((m0 >> i) & 1u);
        const bool b1 = FLAGS && i > 0 && ((m1 >> i) & 1u);
        if (ex(i) == 0) {
            if (b0 == b1) {
                ld2_real(b0 ? Lo : Li + x0, mu0[i], mu1[i]);
            } else {
                mu0[i] = __ldg(b0 ? Lo : Li + x0);
                mu1[i] = __ldg(b1 ? Lo + 1 : Li + x0 + 1);
            }
        } else {
            mu0[i] = __ldg(b0 ? Lo : Li + (ex(i) > 0 ? xb : xa));
            mu1[i] = __ldg(b1 ? Lo + 1 : Li + (ex(i) > 0 ? xc : x0));
        }
    }
    R rho0, rho1, ux0, ux1, uy0, uy1, uz0, uz1;
    ld2_real(tape + c, rho0, rho1);
    ld2_real(tape + qs + c, ux0, ux1);
    ld2_real(tape + 2 * qs + c, uy0, uy1);
    ld2_real(tape + 3 * qs + c, uz0, uz1);
    R F0x = R(0), F0y = R(0), F0z = R(0), F1x = R(0), F1y = R(0), F1z = R(0);
    if (FORCE) {
        if (d.Ffield) {
            const R *F = static_cast<const R *>(d.Ffield);
            ld2_real(F + c, F0x, F1x);
            ld2_real(F + qs + c, F0y, F1y);
            ld2_real(F + 2 * qs + c, F0z, F1z);
        } else {
            F0x = F1x = DevR<R>::F(d, 0);
            F0y = F1y = DevR<R>::F(d, 1);
            F0z = F1z = DevR<R>::F(d, 2);
        }
    }
    const R om = DevR<R>::omega(d);
    R g0x, g0y, g0z, g1x, g1y, g1z;
    adj_collide<R, FORCE>(mu0, rho0, ux0, uy0, uz0, F0x, F0y, F0z, om, g0x, g0y, g0z, d.incomp);
    adj_collide<R, FORCE>(mu1, rho1, ux1, uy1, uz1, F1x, F1y, F1z, om, g1x, g1y, g1z, d.incomp);
    // (a solid cell of a mixed pair gets a value nobody reads)
#pragma unroll
    for (int i = 0; i < Q; ++i) st2_real(lam_out + (long long)i * qs + c, mu0[i], mu1[i]);
    if (grad_F) {
        if (live0) {
            grad_F[cc] = G0x + g0x;
            grad_F[N + cc] = G0y + g0y;
            grad_F[2 * N + cc] = G0z + g0z;
        }
        if (live1) {
            grad_F[cc + 1] = G1x + g1x;
            grad_F[N + cc + 1] = G1y + g1y;
            grad_F[2 * N + cc + 1] = G1z + g1z;
        }
    }
}

// The FP32 reverse step with one cell per thread: a warp's 4-byte loads of 32
// consecutive cells already fill whole 128-byte lines, so FP32 needs no cell
// pairs, and one cell's 19 adjoint populations, tape and gradient fit in 64
// registers, so 4 blocks of 256 threads are resident per SM (the paired
// kernel holds 2 at 128 registers, and its long-scoreboard waits were the
// top stall). Threads take the cells of a plane's box rows in order, across
// row ends. A solid cell stores zeros (its slots are never read), so that
// every 32-byte sector of a lattice row is written whole.
// I: the index type of the lattice, tape and gradient offsets; int where
// every offset fits (19 qs and 3 nx ny nz below 2^31), so that each address is
// one 32-bit index and one wide multiply-add.
constexpr int ADJ1_BLOCKS = 4;

template <bool FLAGS, bool FORCE, class I>
__global__ void __launch_bounds__(256, ADJ1_BLOCKS)
    k_adj_step1(const Dev d, const float *__restrict__ lam_in, float *__restrict__ lam_out,
                const float *__restrict__ tape, float *__restrict__ grad_F) {
    const Geom &g = d.g;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = k / g.nx;
    if (r >= d.P.nyr) return;
    const int bz = d.zrev ? (int)gridDim.y - 1 - (int)blockIdx.y : (int)blockIdx.y;  // (see k_step)
    const int x = k - r * g.nx, y = d.P.y0 + r, z = d.P.z0 + bz;
    const int c = cell_index(g, x, y, z);
    const I qs = (I)g.qs;
    uint32_t m = 0u;
    if (FLAGS) {
        m = __ldg(d.mask + c);
        if (m & SOLID_BIT) {
#pragma unroll
            for (int i = 0; i < Q; ++i) lam_out[(I)i * qs + c] = 0.0f;
            return;
        }
    }
    const I N = (I)d.n_cells, cc = (I)canon_index(g, x, y, z);
    float Gx = 0.0f, Gy = 0.0f, Gz = 0.0f;
    if (grad_F) {  // loaded with the gather, not after the collision
        Gx = grad_F[cc];
        Gy = grad_F[N + cc];
        Gz = grad_F[2 * N + cc];
    }
    float mu[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        // mu_i(x) = lambda_i(x + e_i), or lambda_opp(i)(x) where x + e_i is solid
        const int src = (wrap1(z + ez(i), g.nz) * g.ny + wrap1(y + ey(i), g.ny)) * g.pitch + wrap1(x + ex(i), g.nx);
        const bool b = FLAGS && i > 0 && ((m >> i) & 1u);
        mu[i] = __ldg(lam_in + (b ? (I)opp(i) * qs + c : (I)i * qs + src));
    }
    const float rho = __ldg(tape + c), ux = __ldg(tape + qs + c), uy = __ldg(tape + 2 * qs + c),
                uz = __ldg(tape + 3 * qs + c);
    float Fx = 0.0f, Fy = 0.0f, Fz = 0.0f;
    if (FORCE) {
        if (d.Ffield) {
            const float *F = static_cast<const float *>(d.Ffield);
            Fx = __ldg(F + c);
            Fy = __ldg(F + qs + c);
            Fz = __ldg(F + 2 * qs + c);
        } else {
            Fx = DevR<float>::F(d, 0);
            Fy = DevR<float>::F(d, 1);
            Fz = DevR<float>::F(d, 2);
        }
    }
    float gx, gy, gz;
    adj_collide<float, FORCE>(mu, rho, ux, uy, uz, Fx, Fy, Fz, DevR<float>::omega(d), gx, gy, gz, d.incomp);
#pragma unroll
    for (int i = 0; i < Q; ++i) __stcs(lam_out + (I)i * qs + c, mu[i]);
    if (grad_F) {
        grad_F[cc] = Gx + gx;
        grad_F[N + cc] = Gy + gy;
        grad_F[2 * N + cc] = Gz + gz;
    }
}

// dL/du0 and dL/drho0 through f^0 = f_eq(rho0, u0):
//   dL/du0 = rho0 sum_i lambda_i w_i [3 e_i + 9 (e_i.u0) e_i - 3 u0]
//   dL/drho0 = sum_i lambda_i w_i [1 + 3 e_i.u0 + 9/2 (e_i.u0)^2 - 3/2 u0.u0]
// (incompressible model: no rho0 factor in dL/du0, dL/drho0 = sum lambda_i w_i)
template <class R, bool FLAGS>
__global__ void __launch_bounds__(256)
    k_adj_init_grad(const Dev d, const R *__restrict__ lam, const R *__restrict__ rho0, const R *__restrict__ u0,
                    R *__restrict__ grad_u0, R *__restrict__ grad_rho0) {
    int x, y, z;
    if (!row_cell(d.g, d.L.nxb, blockDim.x, blockDim.y, blockIdx.x, blockIdx.y, threadIdx.x,
                  threadIdx.y, x, y, z))
        return;
    const int c = cell_index(d.g, x, y, z);
    const long long N = d.n_cells, cc = canon_index(d.g, x, y, z), qs = d.g.qs;
    if (FLAGS && d.flags[c]) {
        grad_u0[cc] = grad_u0[N + cc] = grad_u0[2 * N + cc] = R(0);
        if (grad_rho0) grad_rho0[cc] = R(0);
        return;
    }
    const R r0 = rho0 ? rho0[cc] : R(1);
    const R ux = u0[cc], uy = u0[N + cc], uz = u0[2 * N + cc];
    const R usq = ux * ux + uy * uy + uz * uz;
    R gx = R(0), gy = R(0), gz = R(0), gr = R(0), P = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const R l = lam[i * qs + c] * R(weight(i));
        const R eu = R(ex(i)) * ux + R(ey(i)) * uy + R(ez(i)) * uz;
        const R t = l * (R(3) + R(9) * eu);
        gx += t * R(ex(i));
        gy += t * R(ey(i));
        gz += t * R(ez(i));
        P += l;
        gr += l * (R(3) * eu + R(4.5) * eu * eu);
    }
    // d f_eq / d u carries rho0 in the Qian equilibrium, the reference
    // density 1 in the incompressible one, where d f_eq / d rho0 = w
    const R ru = d.incomp ? R(1) : r0;
    grad_u0[cc] = ru * (gx - R(3) * ux * P);
    grad_u0[N + cc] = ru * (gy - R(3) * uy * P);
    grad_u0[2 * N + cc] = ru * (gz - R(3) * uz * P);
    if (grad_rho0) grad_rho0[cc] = d.incomp ? P : P * (R(1) - R(1.5) * usq) + gr;
}

static dim3 grid_of(const Dev &d) { return dim3(d.L.nxb * d.L.nyb, d.g.nz); }
static dim3 block_of(const Dev &d) { return dim3(d.L.bx_threads, d.L.by_threads); }
// The reverse step runs on the paired launch of the forward step kernels:
// flat where whole rows would leave lanes idle.
template <class R, bool FLAGS, bool FLAT>
static cudaError_t launch_adj_step2(const Dev &d, const void *li, void *lo, const void *tape, void *gF) {
    const RowLaunch &P = FLAT ? d.PF : d.P;
    const dim3 grid(P.nxb * P.nyb, P.nzr), block(P.bx_threads, P.by_threads);
    if (d.force_on)
        k_adj_step<R, FLAGS, true, FLAT><<<grid, block, 0, d.stream>>>(
            d, static_cast<const R *>(li), static_cast<R *>(lo), static_cast<const R *>(tape), static_cast<R *>(gF));
    else
        k_adj_step<R, FLAGS, false, FLAT><<<grid, block, 0, d.stream>>>(
            d, static_cast<const R *>(li), static_cast<R *>(lo), static_cast<const R *>(tape), static_cast<R *>(gF));
    return cudaGetLastError();
}

template <class R, bool FLAGS>
static cudaError_t launch_adj_step(const Dev &d, const void *li, void *lo, const void *tape, void *gF) {
    return d.flat_step ? launch_adj_step2<R, FLAGS, true>(d, li, lo, tape, gF)
                       : launch_adj_step2<R, FLAGS, false>(d, li, lo, tape, gF);
}

// FP32: one cell per thread over the cells of the fluid box's rows.
template <bool FLAGS>
static cudaError_t launch_adj_step1(const Dev &d, const void *li, void *lo, const void *tape, void *gF) {
    const dim3 grid((unsigned)(((long long)d.P.nyr * d.g.nx + 255) / 256), d.P.nzr);
    const float *a = static_cast<const float *>(li);
    const float *t = static_cast<const float *>(tape);
    float *b = static_cast<float *>(lo), *G = static_cast<float *>(gF);
    const bool small = (long long)Q * d.g.qs < (1LL << 31) && 3 * d.n_cells < (1LL << 31);
    if (small) {
        if (d.force_on)
            k_adj_step1<FLAGS, true, int><<<grid, 256, 0, d.stream>>>(d, a, b, t, G);
        else
            k_adj_step1<FLAGS, false, int><<<grid, 256, 0, d.stream>>>(d, a, b, t, G);
    } else {
        if (d.force_on)
            k_adj_step1<FLAGS, true, long long><<<grid, 256, 0, d.stream>>>(d, a, b, t, G);
        else
            k_adj_step1<FLAGS, false, long long><<<grid, 256, 0, d.stream>>>(d, a, b, t, G);
    }
    return cudaGetLastError();
}

template <class R>
cudaError_t AdjOps<R>::step(const Dev &d, const void *lam_in, void *lam_out, const void *tape_k, void *grad_F) {
    if (d.flags && !d.mask) return cudaErrorInvalidValue;  // the reverse gather reads the push masks
    if (sizeof(R) == 4)
        return d.flags ? launch_adj_step1<true>(d, lam_in, lam_out, tape_k, grad_F)
                       : launch_adj_step1<false>(d, lam_in, lam_out, tape_k, grad_F);
    return d.flags ? launch_adj_step<R, true>(d, lam_in, lam_out, tape_k, grad_F)
                   : launch_adj_step<R, false>(d, lam_in, lam_out, tape_k, grad_F);
}

template <class R>
cudaError_t AdjOps<R>::init_grad(const Dev &d, const void *lam, const void *rho0, const void *u0, void *grad_u0,
                                 void *grad_rho0) {
    if (d.flags)
        k_adj_init_grad<R, true><<<grid_of(d), block_of(d), 0, d.stream>>>(
            d, static_cast<const R *>(lam), static_cast<const R *>(rho0), static_cast<const R *>(u0),
            static_cast<R *>(grad_u0), static_cast<R *>(grad_rho0));
    else
        k_adj_init_grad<R, false><<<grid_of(d), block_of(d), 0, d.stream>>>(
            d, static_cast<const R *>(lam), static_cast<const R *>(rho0), static_cast<const R *>(u0),
            static_cast<R *>(grad_u0), static_cast<R *>(grad_rho0));
    return cudaGetLastError();
}

template struct AdjOps<double>;
template struct AdjOps<float>;

}  // namespace lbm
