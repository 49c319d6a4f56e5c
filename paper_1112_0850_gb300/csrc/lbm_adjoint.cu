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

template <class R, bool FLAGS, bool FORCE>
__global__ void __launch_bounds__(256, sizeof(R) == 8 ? 2 : 4)
    k_adj_step(const Dev d, const R *__restrict__ lam_in, R *__restrict__ lam_out, const R *__restrict__ tape,
               R *__restrict__ grad_F) {
    int x, y, z;
    if (!row_cell(d.g, d.L.nxb, blockDim.x, blockDim.y, blockIdx.x, blockIdx.y, threadIdx.x,
                  threadIdx.y, x, y, z))
        return;
    const int c = cell_index(d.g, x, y, z);
    if (FLAGS && d.flags[c]) return;
    const long long qs = d.g.qs;
    // mu = G^T lambda^{n+1}
    R mu[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int t = push_dst(d.g, x, y, z, i);
        long long off = (long long)i * qs + t;
        if (FLAGS && i > 0 && d.flags[t]) off = (long long)opp(i) * qs + c;
        mu[i] = __ldg(lam_in + off);
    }
    const R rho = __ldg(tape + c), ux = __ldg(tape + qs + c), uy = __ldg(tape + 2 * qs + c),
            uz = __ldg(tape + 3 * qs + c);
    R Fx = R(0), Fy = R(0), Fz = R(0);
    if (FORCE) {
        if (d.Ffield) {
            const R *F = static_cast<const R *>(d.Ffield);
            Fx = F[c];
            Fy = F[qs + c];
            Fz = F[2 * qs + c];
        } else {
            Fx = R(d.F[0]);
            Fy = R(d.F[1]);
            Fz = R(d.F[2]);
        }
    }
    const R om = R(d.omega);
    const R usq = ux * ux + uy * uy + uz * uz;
    // P = sum_k w_k mu_k; A4 = sum over pairs w p (e.u)^2; bv = sum w (3 q + 9 (e.u) p) e;
    // dv = sum w p (e.F) e; with p = mu_i + mu_opp(i), q = mu_i - mu_opp(i).
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
    const R a = P * (R(1) + R(1.5) * usq) - R(4.5) * A4;
    bx -= R(3) * ux * P;
    by -= R(3) * uy * P;
    bz -= R(3) * uz * P;
    const R cF = R(1) - R(0.5) * om;
    if (FORCE) {
        dx = cF * (R(9) * dx - R(3) * Fx * P);
        dy = cF * (R(9) * dy - R(3) * Fy * P);
        dz = cF * (R(9) * dz - R(3) * Fz * P);
    }
    const R inv = R(1) / rho;
    const R alpha = om * a - (dx * ux + dy * uy + dz * uz) * inv;
    const R betx = om * bx + dx * inv, bety = om * by + dy * inv, betz = om * bz + dz * inv;
    const R keep = R(1) - om;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        __stcs(lam_out + (long long)i * qs + c,
               keep * mu[i] + alpha + R(ex(i)) * betx + R(ey(i)) * bety + R(ez(i)) * betz);
    if (grad_F) {
        const long long N = d.n_cells, cc = canon_index(d.g, x, y, z);
        const R h = R(0.5) * inv;
        grad_F[cc] += bx + dx * h;
        grad_F[N + cc] += by + dy * h;
        grad_F[2 * N + cc] += bz + dz * h;
    }
}

// dL/du0 and dL/drho0 through f^0 = f_eq(rho0, u0):
//   dL/du0 = rho0 sum_i lambda_i w_i [3 e_i + 9 (e_i.u0) e_i - 3 u0]
//   dL/drho0 = sum_i lambda_i w_i [1 + 3 e_i.u0 + 9/2 (e_i.u0)^2 - 3/2 u0.u0]
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
    grad_u0[cc] = r0 * (gx - R(3) * ux * P);
    grad_u0[N + cc] = r0 * (gy - R(3) * uy * P);
    grad_u0[2 * N + cc] = r0 * (gz - R(3) * uz * P);
    if (grad_rho0) grad_rho0[cc] = P * (R(1) - R(1.5) * usq) + gr;
}

static dim3 grid_of(const Dev &d) { return dim3(d.L.nxb * d.L.nyb, d.g.nz); }
static dim3 block_of(const Dev &d) { return dim3(d.L.bx_threads, d.L.by_threads); }

template <class R, bool FLAGS>
static cudaError_t launch_adj_step(const Dev &d, const void *li, void *lo, const void *tape, void *gF) {
    if (d.force_on)
        k_adj_step<R, FLAGS, true><<<grid_of(d), block_of(d), 0, d.stream>>>(
            d, static_cast<const R *>(li), static_cast<R *>(lo), static_cast<const R *>(tape), static_cast<R *>(gF));
    else
        k_adj_step<R, FLAGS, false><<<grid_of(d), block_of(d), 0, d.stream>>>(
            d, static_cast<const R *>(li), static_cast<R *>(lo), static_cast<const R *>(tape), static_cast<R *>(gF));
    return cudaGetLastError();
}

template <class R>
cudaError_t AdjOps<R>::step(const Dev &d, const void *lam_in, void *lam_out, const void *tape_k, void *grad_F) {
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
