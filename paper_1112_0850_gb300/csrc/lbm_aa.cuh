// AA-pattern stream-collide: one lattice A updated in place.
//
// The fused update of Sec. 2 needs two grids when populations move to their
// neighbours in every step. The AA pattern (Bailey et al., 2009) alternates
// two kinds of step on one lattice instead, each moving the same bytes as a
// two-grid step. Two layouts of the pre-collision state f^n alternate:
//   natural (before an even step): slot i of cell x holds f^n_i(x);
//   swapped (before an odd step):  slot opp(i) of x holds P^{n-1}_i(x), the
//     post-collision value of the even step, so f^n_i(x) is slot opp(i) of
//     x - e_i if that cell is fluid, else slot i of x itself (halfway
//     bounce-back, plus the moving-wall term).
// Even step: cell x reads slot i of x, collides, and writes P_i(x) to slot
// opp(i) of x; no neighbour is touched. Odd step: cell x gathers from the
// swapped layout, collides, and writes P_i(x) to slot i of x + e_i (where the
// next even step reads f_i(x + e_i)); if x + e_i is solid, the bounced value
// goes to slot opp(i) of x instead. In both steps a fluid cell writes the
// slots it read, each read before it is written by the same thread, and (the
// odd step's mask-free scatter) solid slots that no one reads, so the
// in-place update has no races (and the read-only load path is safe: no
// fluid cell reads a slot after it is written within a launch).
//
// Halfway bounce-back needs only the odd step: where x - e_j is solid (bit
// opp(j) of the push mask, i.e. x + e_opp(j) is solid too) population j is
// read from slot j of x itself, and population opp(j) is written back there.
// Solid cells' values are never used; the even step stores their lanes with
// the rest of the pair (whole 32-byte sectors). The odd step's two forms
// (aa_odd_pair) either leave solid cells alone or let a solid lane load
// values it discards (slots a neighbour may be rewriting) and let fluid
// cells store into solid slots that only they read.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

// Live lanes of the pair (x0, x0 + 1): fluid and inside the row.
template <bool FLAGS>
__device__ __forceinline__ void pair_live(const Dev &d, int c, bool has1, bool &live0, bool &live1) {
    live0 = true;
    live1 = has1;
    if (FLAGS) {
        const uchar2 fl = __ldg(reinterpret_cast<const uchar2 *>(d.flags + c));
        live0 = !fl.x;
        live1 = has1 && !fl.y;
    }
}

template <class R, int FORCE, bool TFORM>
__device__ __forceinline__ void pair_force(const Dev &d, int c, typename Pair2<R>::V &Fx, typename Pair2<R>::V &Fy,
                                           typename Pair2<R>::V &Fz, Guo2<R> &G) {
    Fx = Fy = Fz = vsplat(R(0));
    if (FORCE == 1) {
        Fx = vsplat(DevR<R>::F(d, 0));
        Fy = vsplat(DevR<R>::F(d, 1));
        Fz = vsplat(DevR<R>::F(d, 2));
        G = uniform_guo<R, TFORM>(d);
    } else if (FORCE == 2) {
        const R *F = static_cast<const R *>(d.Ffield);
        ld2_real(F + c, Fx.x, Fx.y);
        ld2_real(F + d.g.qs + c, Fy.x, Fy.y);
        ld2_real(F + 2 * d.g.qs + c, Fz.x, Fz.y);
        G = guo2<R>(TFORM ? DevR<R>::cs(d) : R(1) - R(0.5) * DevR<R>::omega(d), Fx, Fy, Fz);
    }
}

template <class R, bool RECORD>
__device__ __forceinline__ void pair_check_record(const Dev &d, int c, bool live0, bool live1, const Mom2<R> &m,
                                                  R *tape) {
    const bool bad0 = live0 && !(m.rho.x > R(0) && m.rho.x < R(1e30));
    const bool bad1 = live1 && !(m.rho.y > R(0) && m.rho.y < R(1e30));
    if (bad0 || bad1) atomicOr(d.status, LBM_STATUS_DIVERGED);
    if (RECORD) {
        const long long qs = d.g.qs;
        st2_real(tape + c, m.rho.x, m.rho.y);
        st2_real(tape + qs + c, m.ux.x, m.ux.y);
        st2_real(tape + 2 * qs + c, m.uy.x, m.uy.y);
        st2_real(tape + 3 * qs + c, m.uz.x, m.uz.y);
    }
}

// Even step (natural -> swapped): local, every access an aligned pair.
// FLAT (both AA kernels): the launch of d.PF (pairs in plane order), else of d.P.
// RED: also add the pair's pre-collision totals to red[4] (pair_add_totals).
template <int S, bool FLAGS, int FORCE, bool RECORD, bool FLAT, bool RED>
__device__ __forceinline__ void aa_even_pair(const Dev &d, typename Stor<S>::T *__restrict__ A,
                                             typename Stor<S>::R *__restrict__ tape, double *red) {
    typedef typename Stor<S>::R R;
    typedef typename Pair2<R>::V V;
    int x0, y, z;
    // alternating plane order (see k_step) on walled lattices only: without
    // flags the 16-bit forms spill 16 more bytes at 64 registers for it (the
    // 512^3 box lost 2.4%, and a lattice that size keeps no plane in L2)
    const int bz = FLAGS && d.zrev ? (int)gridDim.y - 1 - (int)blockIdx.y : (int)blockIdx.y;
    if (!pair_cell<FLAT>(d.g, FLAT ? d.PF : d.P, blockDim.x, blockDim.y, blockIdx.x, bz, threadIdx.x, threadIdx.y,
                         x0, y, z))
        return;
    const long long qs = d.g.qs;
    const int c = cell_index(d.g, x0, y, z);
    bool live0, live1;
    pair_live<FLAGS>(d, c, x0 + 1 < d.g.nx, live0, live1);
    // (solid cells load, collide and store like the others: an early exit on
    // the flags would put a dependent load before the gather)
    const R nan = quiet_nan<R>();
    V s[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) Stor<S>::ld2(A + (long long)i * qs + c, s[i].x, s[i].y);
    V Fx, Fy, Fz;
    Guo2<R> G;
    pair_force<R, FORCE, relax_about_t(S)>(d, c, Fx, Fy, Fz, G);
    const Mom2<R> m = moments2<R, FORCE != 0>(s, Fx, Fy, Fz, d.incomp);
    if (RED) pair_add_totals<R>(m, live0, live1, d.incomp, red);
    pair_check_record<R, RECORD>(d, c, live0, live1, m, tape);
    collide2<R, FORCE != 0, relax_about_t(S)>(s, m, DevR<R>::omega(d), DevR<R>::cs(d), Fx, Fy, Fz, G, d.incomp);
    // a solid lane writes its NaN back (its slots stay marked). FP32: a
    // 32-byte sector whose 8 cells are all solid skips its stores instead (as
    // in the two-grid step: no reader takes a solid slot's value), found by
    // one ballot over the sector's four pairs on lanes 4k .. 4k + 3
    bool skip = false;
    if constexpr (FLAGS && S == LBM_F32) {
        if ((d.g.pitch & 7) == 0 && (((d.g.nx + 1) / 2) & 3) == 0) {
            const unsigned sb = __ballot_sync(__activemask(), !live0 && !live1);
            skip = ((sb >> ((threadIdx.x & 31) & ~3u)) & 0xFu) == 0xFu;
        }
    }
    if (!skip) {
#pragma unroll
        for (int i = 0; i < Q; ++i)
            Stor<S>::st2(A + (long long)opp(i) * qs + c, !FLAGS || live0 ? s[i].x : nan,
                         !FLAGS || live1 ? s[i].y : nan);
    }
}

template <int S, bool FLAGS, int FORCE, bool RECORD, bool FLAT>
__global__ void __launch_bounds__(256, StepBlocks<S>::value)
    k_aa_even(const Dev d, typename Stor<S>::T *__restrict__ A, typename Stor<S>::R *__restrict__ tape) {
    aa_even_pair<S, FLAGS, FORCE, RECORD, FLAT, false>(d, A, tape, nullptr);
}

// The even step with the totals of its pre-collision state summed per block
// (every thread, in the lattice or not, reaches the block sum).
template <int S, bool FLAGS, int FORCE, bool FLAT>
__global__ void __launch_bounds__(256, StepBlocks<S>::value)
    k_aa_even_reduce(const Dev d, typename Stor<S>::T *__restrict__ A, double *__restrict__ partials) {
    double red[4] = {0.0, 0.0, 0.0, 0.0};
    aa_even_pair<S, FLAGS, FORCE, false, FLAT, true>(d, A, nullptr, red);
    block_partials(red, partials);
}

// Resident 256-thread blocks per SM the odd step is compiled for. With flags
// both of its forms (aa_odd_pair) need more registers: 2 blocks (128
// registers) ran the walled channel at 33.2 vs 26.7 GFLUPS in FP16 with
// selected addresses, and at 32.8 vs 32.1 in FP32 with the mask-free gather
// (3 blocks spill about 110 bytes there).
template <int S, bool FLAGS> struct AaOddBlocks {
    static constexpr int value = S == LBM_F64 ? 1 : (FLAGS ? 2 : StepBlocks<S>::value);
};

// Odd step (swapped -> natural): gather from the neighbours, scatter to them.
// Halfway bounce-back (push mask bit j: x + e_j is solid):
//  - loads: population i comes from slot i of x itself when bit opp(i) is set,
//    from slot opp(i) of x - e_i otherwise; every load address is a select,
//    so the gather is one branch-free sequence that waits for the mask.
//  - stores, in one of two forms per storage format: selected (FP64), P_i(x)
//    to slot opp(i) of x itself when bit i is set, else to slot i of x + e_i;
//    or the mask-free scatter (FP32, 16-bit storage): every population of a
//    live cell is stored to its neighbour's slot, a solid neighbour's
//    included (slot i of a solid x + e_i is written by x alone and read by no
//    one: x itself reads its own slot there), and the bounced ones are then
//    stored to the cell's own slots.
// Walled channel, GFLUPS, FP32 / FP16: selected stores 31.1 / 35.0, the
// mask-free scatter 33.1 / 38.0. Also measured: a mask-free gather (every
// population loaded from its neighbour without waiting for the mask, the
// bounced ones reloaded from the own slots after) with the mask-free scatter
// 32.8 / 32.1, with selected stores 30.9 / 33.2; a NaN-driven fix-up with
// separate store paths twice as slow (its code size and divergence made it
// instruction-bound).
template <int S> __host__ __device__ constexpr bool aa_free_scatter() { return S != LBM_F64; }

template <int S, bool FLAGS, int FORCE, bool RECORD, bool FLAT, bool RED>
__device__ __forceinline__ void aa_odd_pair(const Dev &d, typename Stor<S>::T *__restrict__ A,
                                            typename Stor<S>::R *__restrict__ tape, double *red) {
    typedef typename Stor<S>::T T;
    typedef typename Stor<S>::R R;
    typedef typename Pair2<R>::V V;
    constexpr bool FREE_ST = aa_free_scatter<S>();
    int x0, y, z;
    // alternating plane order (see k_step) on walled lattices only: without
    // flags the 16-bit forms spill 16 more bytes at 64 registers for it (the
    // 512^3 box lost 2.4%, and a lattice that size keeps no plane in L2)
    const int bz = FLAGS && d.zrev ? (int)gridDim.y - 1 - (int)blockIdx.y : (int)blockIdx.y;
    if (!pair_cell<FLAT>(d.g, FLAT ? d.PF : d.P, blockDim.x, blockDim.y, blockIdx.x, bz, threadIdx.x, threadIdx.y,
                         x0, y, z))
        return;
    const Geom &g = d.g;
    const long long qs = g.qs;
    const bool has1 = x0 + 1 < g.nx;
    const int c = cell_index(g, x0, y, z);
    uint32_t m0 = 0u, m1 = has1 ? 0u : SOLID_BIT;
    if (FLAGS) {
        const uint2 mm = ld_resident2(d.mask + c);
        m0 = mm.x;
        m1 |= mm.y;
    }
    const bool live0 = !(m0 & SOLID_BIT), live1 = !(m1 & SOLID_BIT);
    if (!live0 && !live1) return;  // (the selected gather waits for the mask anyway)
    // neighbour columns: x0 - 1, x0 + 1, x0 + 2 (the last only for a full pair)
    const int xa = wrap1(x0 - 1, g.nx);
    const int xb = wrap1(x0 + 1, g.nx);
    const int xc = has1 ? wrap1(x0 + 2, g.nx) : x0;
    V s[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        // f_i(x) = slot opp(i) of x - e_i, or slot i of x if x - e_i is solid
        const int row = (wrap1(z - ez(i), g.nz) * g.ny + wrap1(y - ey(i), g.ny)) * g.pitch;
        const T *Pn = A + (long long)opp(i) * qs + row;
        const T *Po = A + (long long)i * qs + c;
        const bool b0 = FLAGS && i > 0 && ((m0 >> opp(i)) & 1u);
        const bool b1 = FLAGS && i > 0 && ((m1 >> opp(i)) & 1u);
        if (ex(i) == 0) {
            if (b0 == b1) {
                Stor<S>::ld2(b0 ? Po : Pn + x0, s[i].x, s[i].y);
            } else {
                s[i].x = Stor<S>::ld(b0 ? Po : Pn + x0);
                s[i].y = Stor<S>::ld(b1 ? Po + 1 : Pn + x0 + 1);
            }
        } else {
            s[i].x = Stor<S>::ld(b0 ? Po : Pn + (ex(i) > 0 ? xa : xb));
            s[i].y = Stor<S>::ld(b1 ? Po + 1 : Pn + (ex(i) > 0 ? x0 : xc));
        }
    }
    const bool bounce_st = FLAGS && FREE_ST && ((m0 | m1) & 0x7fffeu);
    const bool mv = FLAGS && d.moving_on && ((m0 | m1) & MOVING_BIT);
    if (mv) {
        // bounced off a moving wall: plus 6 w_i (e_i . u_w)
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if (((m0 >> opp(i)) & 1u) && d.flags[pull_src(g, x0, y, z, i)] == 2) s[i].x += wall_term<R>(d, i);
            if (((m1 >> opp(i)) & 1u) && d.flags[pull_src(g, x0 + 1, y, z, i)] == 2) s[i].y += wall_term<R>(d, i);
        }
    }
    V Fx, Fy, Fz;
    Guo2<R> G;
    pair_force<R, FORCE, relax_about_t(S)>(d, c, Fx, Fy, Fz, G);
    const Mom2<R> m = moments2<R, FORCE != 0>(s, Fx, Fy, Fz, d.incomp);
    if (RED) pair_add_totals<R>(m, live0, live1, d.incomp, red);
    pair_check_record<R, RECORD>(d, c, live0, live1, m, tape);
    collide2<R, FORCE != 0, relax_about_t(S)>(s, m, DevR<R>::omega(d), DevR<R>::cs(d), Fx, Fy, Fz, G, d.incomp);
    // P_i(x) to slot i of x + e_i, or to slot opp(i) of x if x + e_i is solid
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int row = (wrap1(z + ez(i), g.nz) * g.ny + wrap1(y + ey(i), g.ny)) * g.pitch;
        T *Pn = A + (long long)i * qs + row;
        T *Po = A + (long long)opp(i) * qs + c;
        const bool b0 = FLAGS && !FREE_ST && i > 0 && ((m0 >> i) & 1u);
        const bool b1 = FLAGS && !FREE_ST && i > 0 && ((m1 >> i) & 1u);
        if (ex(i) == 0 && b0 == b1 && live0 && live1) {
            Stor<S>::st2(b0 ? Po : Pn + x0, s[i].x, s[i].y);
        } else {
            if (live0) Stor<S>::st(b0 ? Po : Pn + (ex(i) > 0 ? xb : (ex(i) < 0 ? xa : x0)), s[i].x);
            if (live1) Stor<S>::st(b1 ? Po + 1 : Pn + (ex(i) > 0 ? xc : (ex(i) < 0 ? x0 : x0 + 1)), s[i].y);
        }
    }
    if (bounce_st) {
        // the mask-free scatter's bounced values, to the own slots
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            T *Po = A + (long long)opp(i) * qs + c;
            if (live0 && ((m0 >> i) & 1u)) Stor<S>::st(Po, s[i].x);
            if (live1 && ((m1 >> i) & 1u)) Stor<S>::st(Po + 1, s[i].y);
        }
    }
    if (mv) {
        // a population bounced back from a moving wall arrives as opp(i) and
        // carries 6 w_opp(i) (e_opp(i) . u_w) = -6 w_i (e_i . u_w): rewrite
        // the own slots just stored (same thread, so this store is the last)
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            T *Po = A + (long long)opp(i) * qs + c;
            if (live0 && ((m0 >> i) & 1u) && d.flags[push_dst(g, x0, y, z, i)] == 2)
                Stor<S>::st(Po, s[i].x - wall_term<R>(d, i));
            if (live1 && ((m1 >> i) & 1u) && d.flags[push_dst(g, x0 + 1, y, z, i)] == 2)
                Stor<S>::st(Po + 1, s[i].y - wall_term<R>(d, i));
        }
    }
}

template <int S, bool FLAGS, int FORCE, bool RECORD, bool FLAT>
__global__ void __launch_bounds__(256, AaOddBlocks<S, FLAGS>::value)
    k_aa_odd(const Dev d, typename Stor<S>::T *__restrict__ A, typename Stor<S>::R *__restrict__ tape) {
    aa_odd_pair<S, FLAGS, FORCE, RECORD, FLAT, false>(d, A, tape, nullptr);
}

// The odd step with the totals of its pre-collision state summed per block.
template <int S, bool FLAGS, int FORCE, bool FLAT>
__global__ void __launch_bounds__(256, AaOddBlocks<S, FLAGS>::value)
    k_aa_odd_reduce(const Dev d, typename Stor<S>::T *__restrict__ A, double *__restrict__ partials) {
    double red[4] = {0.0, 0.0, 0.0, 0.0};
    aa_odd_pair<S, FLAGS, FORCE, false, FLAT, true>(d, A, nullptr, red);
    block_partials(red, partials);
}

template <int S, bool FLAGS, int FORCE, bool FLAT>
static cudaError_t launch_aa4(const Dev &d, void *A, int odd, void *tape) {
    typedef typename Stor<S>::T T;
    typedef typename Stor<S>::R R;
    T *a = static_cast<T *>(A);
    R *t = static_cast<R *>(tape);
    const RowLaunch &P = FLAT ? d.PF : d.P;
    const dim3 grid(P.nxb * P.nyb, P.nzr), block(P.bx_threads, P.by_threads);
    if (odd) {
        if (tape)
            k_aa_odd<S, FLAGS, FORCE, true, FLAT><<<grid, block, 0, d.stream>>>(d, a, t);
        else
            k_aa_odd<S, FLAGS, FORCE, false, FLAT><<<grid, block, 0, d.stream>>>(d, a, nullptr);
    } else {
        if (tape)
            k_aa_even<S, FLAGS, FORCE, true, FLAT><<<grid, block, 0, d.stream>>>(d, a, t);
        else
            k_aa_even<S, FLAGS, FORCE, false, FLAT><<<grid, block, 0, d.stream>>>(d, a, nullptr);
    }
    return cudaGetLastError();
}

// The AA kernels run flat only where whole rows would leave lanes idle (with
// whole-warp rows their flat forms compile to no fewer spills).
template <int S, bool FLAGS, int FORCE>
static cudaError_t launch_aa3(const Dev &d, void *A, int odd, void *tape) {
    return d.flat_step ? launch_aa4<S, FLAGS, FORCE, true>(d, A, odd, tape)
                       : launch_aa4<S, FLAGS, FORCE, false>(d, A, odd, tape);
}

template <int S, bool FLAGS>
static cudaError_t launch_aa2(const Dev &d, void *A, int odd, void *tape) {
    if (d.Ffield) return launch_aa3<S, FLAGS, 2>(d, A, odd, tape);
    if (d.force_on) return launch_aa3<S, FLAGS, 1>(d, A, odd, tape);
    return launch_aa3<S, FLAGS, 0>(d, A, odd, tape);
}

template <int S, bool FLAGS, int FORCE, bool FLAT>
static cudaError_t launch_aa_reduce4(const Dev &d, void *A, int odd, double *partials, double *out) {
    typedef typename Stor<S>::T T;
    T *a = static_cast<T *>(A);
    const RowLaunch &P = FLAT ? d.PF : d.P;
    const dim3 grid(P.nxb * P.nyb, P.nzr), block(P.bx_threads, P.by_threads);
    if (odd)
        k_aa_odd_reduce<S, FLAGS, FORCE, FLAT><<<grid, block, 0, d.stream>>>(d, a, partials);
    else
        k_aa_even_reduce<S, FLAGS, FORCE, FLAT><<<grid, block, 0, d.stream>>>(d, a, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, RED_THREADS, 0, d.stream>>>(partials, (int)(grid.x * grid.y), out);
    return cudaGetLastError();
}

template <int S, bool FLAGS>
static cudaError_t launch_aa_reduce2(const Dev &d, void *A, int odd, double *partials, double *out) {
    if (d.Ffield)
        return d.flat_step ? launch_aa_reduce4<S, FLAGS, 2, true>(d, A, odd, partials, out)
                           : launch_aa_reduce4<S, FLAGS, 2, false>(d, A, odd, partials, out);
    if (d.force_on)
        return d.flat_step ? launch_aa_reduce4<S, FLAGS, 1, true>(d, A, odd, partials, out)
                           : launch_aa_reduce4<S, FLAGS, 1, false>(d, A, odd, partials, out);
    return d.flat_step ? launch_aa_reduce4<S, FLAGS, 0, true>(d, A, odd, partials, out)
                       : launch_aa_reduce4<S, FLAGS, 0, false>(d, A, odd, partials, out);
}

template <int S>
cudaError_t AaOps<S>::step_reduce(const Dev &d, void *A, int odd, double *partials, double *out) {
    if (d.flags && !d.mask) return cudaErrorInvalidValue;
    return d.flags ? launch_aa_reduce2<S, true>(d, A, odd, partials, out)
                   : launch_aa_reduce2<S, false>(d, A, odd, partials, out);
}

template <int S>
cudaError_t AaOps<S>::step(const Dev &d, void *A, int odd, void *tape) {
    if (d.flags && !d.mask) return cudaErrorInvalidValue;  // the odd step selects with the push masks
    return d.flags ? launch_aa2<S, true>(d, A, odd, tape) : launch_aa2<S, false>(d, A, odd, tape);
}

}  // namespace lbm
