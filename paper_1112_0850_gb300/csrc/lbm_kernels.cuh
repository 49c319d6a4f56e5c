// Kernels of the D3Q19 BGK path, templated on the population storage format.
// Included by one translation unit per format (lbm_ops_*.cu), which
// instantiates Ops<S>.
//
// Data layout (HBM): two padded structure-of-arrays lattices of 19 arrays
// each, P[i][z][y][pitch]; the kernels keep the post-collision populations
// P^n at the cell where they were computed and gather them at the start of
// the next step (Sec. 6: loads from the neighbours, aligned coalesced stores
// to the local cell, two grids). With halfway bounce-back folded into the
// gather (Sec. 2: bounce-back combined with streaming):
//   f^{n+1}_i(x) = P^n_i(x - e_i)        if x - e_i is fluid
//                = P^n_{opp(i)}(x)        otherwise.
#pragma once

#include "lbm_launch.h"

namespace lbm {

// Element access of canonical arrays in a storage format (values are
// converted through double, rounding to nearest even when narrowing).
template <int D> struct IOFmt;
template <> struct IOFmt<LBM_F64> {
    typedef double T;
    static __device__ __forceinline__ double get(const T *p) { return *p; }
    static __device__ __forceinline__ void put(T *p, double v) { *p = v; }
};
template <> struct IOFmt<LBM_F32> {
    typedef float T;
    static __device__ __forceinline__ double get(const T *p) { return (double)*p; }
    static __device__ __forceinline__ void put(T *p, double v) { *p = __double2float_rn(v); }
};
template <> struct IOFmt<LBM_F16S> {
    typedef __half T;
    static __device__ __forceinline__ double get(const T *p) { return (double)__half2float(*p); }
    static __device__ __forceinline__ void put(T *p, double v) { *p = __double2half(v); }
};
template <> struct IOFmt<LBM_BF16S> {
    typedef __nv_bfloat16 T;
    static __device__ __forceinline__ double get(const T *p) { return (double)__bfloat162float(*p); }
    static __device__ __forceinline__ void put(T *p, double v) { *p = __double2bfloat16(v); }
};

// Canonical state arrays of a moment-split context hold plain shifted
// deviations in the format's 16-bit element type.
template <> struct IOFmt<LBM_F16M> : IOFmt<LBM_F16S> {};
template <> struct IOFmt<LBM_BF16M> : IOFmt<LBM_BF16S> {};

// ---------------------------------------------------------------------------
// Moment-split storage (LBM_F16M, LBM_BF16M): a cell holds, for its 19
// post-collision values P_i, the momentum word J (SplitJ) and the remainders
// g_i = s_i - K_i (e_i . J) (s_i = P_i - w_i, J as stored), rebuilt as
// s_i = K_i (e_i . J) + g_i with one fused multiply-add. K_i = 3 w_i, taken as
// the momentum-exact pair of OddK (2 K_axis + 8 K_diag = 1 exactly, so the
// base parts carry J itself). Writing e_i = sigma e'_i with the first non-zero
// component of e'_i equal to +1, K_i (e_i . J) = (sigma K_i)(e'_i . J): e'_i . J
// is one component or one sum / difference (edot_first), the same value in the
// packed step kernel and the per-cell readers.
LBM_HD constexpr bool first_positive(int i) {
    return ex(i) > 0 || (ex(i) == 0 && (ey(i) > 0 || (ey(i) == 0 && ez(i) > 0)));
}
// e'_i: the member of the pair (i, opp(i)) whose first non-zero component is +1.
LBM_HD constexpr int split_first(int i) { return first_positive(i) ? i : opp(i); }
// sigma K_i (0 for the rest population).
LBM_HD constexpr float split_k(int i) {
    return i == 0 ? 0.0f : (first_positive(i) ? 1.0f : -1.0f) * (i <= 6 ? OddK<float>::AXIS : OddK<float>::DIAG);
}

// e'_i . J of one cell's momentum word (scalar; the association of edot_first).
template <int S> __device__ __forceinline__ float split_edot(int i, uint2 w) {
    const float jx = SplitJ<S>::lo(w.x), jy = SplitJ<S>::hi(w.x), jz = SplitJ<S>::lo(w.y);
    if (ex(i)) {
        if (ey(i)) return ey(i) > 0 ? __fadd_rn(jx, jy) : __fsub_rn(jx, jy);
        if (ez(i)) return ez(i) > 0 ? __fadd_rn(jx, jz) : __fsub_rn(jx, jz);
        return jx;
    }
    if (ey(i)) {
        if (ez(i)) return ez(i) > 0 ? __fadd_rn(jy, jz) : __fsub_rn(jy, jz);
        return jy;
    }
    return jz;
}

// Momentum words of a moment-split lattice P (one uint2 per padded cell).
template <class T> __device__ __forceinline__ const uint2 *split_words(const Dev &d, const T *P) {
    return reinterpret_cast<const uint2 *>(P + d.jo);
}
template <class T> __device__ __forceinline__ uint2 *split_words(const Dev &d, T *P) {
    return reinterpret_cast<uint2 *>(P + d.jo);
}

// In a row of odd length the padding cell after the last cell holds a copy of
// the momentum word of the row's first cell (x = 0): the lone last cell of the
// row, whose thread loads the word pair (nx - 1, nx), pulls its e_x = -1
// values from cell 0 (periodic in x). Every writer of cell 0's word keeps it.
__device__ __forceinline__ void split_ghost(const Dev &d, uint2 *J, int x, int c, uint2 w) {
    if ((d.g.nx & 1) && x == 0) J[c + d.g.nx] = w;
}

// Round to the 16-bit format (nearest even) from float or double.
template <int S> __device__ __forceinline__ unsigned split_pack(float a, float b) { return SplitJ<S>::pack(a, b); }
template <int S> __device__ __forceinline__ unsigned split_pack(double a, double b) {
    union {
        unsigned short h[2];
        unsigned u;
    } v;
    if (S == LBM_F16M) {
        v.h[0] = __half_as_ushort(__double2half(a));
        v.h[1] = __half_as_ushort(__double2half(b));
    } else {
        v.h[0] = __bfloat16_as_ushort(__double2bfloat16(a));
        v.h[1] = __bfloat16_as_ushort(__double2bfloat16(b));
    }
    return v.u;
}

// Write one cell's 19 shifted values v (float or double) at cell c of a
// moment-split lattice: J = sum_i v_i e_i rounded to the format, then the
// remainders g_i = v_i - K_i (e_i . J) rounded.
template <int S, class V>
__device__ __forceinline__ void split_store(const Dev &d, typename Stor<S>::T *P, int x, int c, const V v[Q]) {
    V jx = V(0), jy = V(0), jz = V(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (ex(i)) jx += ex(i) > 0 ? v[i] : -v[i];
        if (ey(i)) jy += ey(i) > 0 ? v[i] : -v[i];
        if (ez(i)) jz += ez(i) > 0 ? v[i] : -v[i];
    }
    const unsigned wx = split_pack<S>(jx, jy), wy = split_pack<S>(jz, V(0));
    const uint2 w = make_uint2(wx, wy);
    IOFmt<S>::put(P + c, (double)v[0]);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const V g = fma(V(-split_k(i)), V(split_edot<S>(split_first(i), w)), v[i]);
        IOFmt<S>::put(P + (long long)i * d.g.qs + c, (double)g);
    }
    split_words(d, P)[c] = w;
    split_ghost(d, split_words(d, P), x, c, w);
}

__device__ __forceinline__ bool is_solid(const uint8_t *flags, int c) { return flags && flags[c]; }

// Moving-wall term of a population bounced into direction i: 6 w_i (e_i . u_w).
template <class R> __device__ __forceinline__ R wall_term(const Dev &d, int i);
template <> __device__ __forceinline__ float wall_term<float>(const Dev &d, int i) { return d.wcf[i]; }
template <> __device__ __forceinline__ double wall_term<double>(const Dev &d, int i) { return d.wc[i]; }

template <class R> __device__ __forceinline__ void force_at(const Dev &d, int c, R &Fx, R &Fy, R &Fz) {
    if (d.Ffield) {
        const R *F = static_cast<const R *>(d.Ffield);
        Fx = F[c];
        Fy = F[d.g.qs + c];
        Fz = F[2 * d.g.qs + c];
    } else {
        Fx = DevR<R>::F(d, 0);
        Fy = DevR<R>::F(d, 1);
        Fz = DevR<R>::F(d, 2);
    }
}

// Gather the 19 pre-collision populations of fluid cell (x, y, z) from P in
// the layout d.layout. In the link form a solid source's slot already holds
// the bounced value (what the next step will read), so the gather there
// ignores flags; the AA swapped layout is the pull layout with slot i and
// slot opp(i) exchanged.
template <int S, bool FLAGS>
__device__ __forceinline__ void gather(const Dev &d, const typename Stor<S>::T *P, int x, int y, int z,
                                       int c, typename Stor<S>::R s[Q]) {
    const long long qs = d.g.qs;
    if constexpr (is_split(S)) {
        // rebuild each value from its source cell's momentum word; a bounced
        // one is the cell's own opposite value, rebuilt from its own word
        const uint2 *J = split_words(d, P);
        s[0] = Stor<S>::ld(P + c);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int src = pull_src(d.g, x, y, z, i);
            const uint8_t f = FLAGS ? d.flags[src] : 0;
            if (!f) {
                s[i] = __fmaf_rn(split_k(i), split_edot<S>(split_first(i), __ldg(J + src)),
                                 Stor<S>::ld(P + (long long)i * qs + src));
            } else {
                s[i] = __fmaf_rn(split_k(opp(i)), split_edot<S>(split_first(i), __ldg(J + c)),
                                 Stor<S>::ld(P + (long long)opp(i) * qs + c));
                if (f == 2 && d.moving_on) s[i] += wall_term<typename Stor<S>::R>(d, i);
            }
        }
        return;
    }
    if (d.layout == LAYOUT_AA_NAT) {
#pragma unroll
        for (int i = 0; i < Q; ++i) s[i] = Stor<S>::ld(P + (long long)i * qs + c);
        return;
    }
    const bool mirror = d.layout == LAYOUT_AA_SWAP;
    const bool flag_free = bounce_in_solid(S) && !mirror;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int src = pull_src(d.g, x, y, z, i);
        long long off = (long long)(mirror ? opp(i) : i) * qs + src;
        uint8_t f = 0;
        if (FLAGS && i > 0 && !flag_free) f = d.flags[src];
        if (f) off = (long long)(mirror ? i : opp(i)) * qs + c;
        s[i] = Stor<S>::ld(P + off);
        if (f == 2 && d.moving_on) s[i] += wall_term<typename Stor<S>::R>(d, i);
    }
}

// NaN marks solid slots in the NaN-mark form and in the AA pattern. (In the
// AA pattern they are hygiene only: the odd step's mask-free scatter stores
// into solid slots, and no reader takes a solid slot's value.)
template <int S> __device__ __forceinline__ bool nan_marked(const Dev &d) {
    return bounce_mode(S) == BB_NANS || d.layout != LAYOUT_PULL;
}

// ---------------------------------------------------------------------------
// Fused stream-collide (Sec. 2 steps 1-3, Eq. 1; Sec. 6 pull-style update).
//
// Each thread updates the two x-adjacent cells x0, x0 + 1 of one row, so the
// populations with e_x = 0 (rest, +-y, +-z and the yz diagonals) move as one
// aligned pair per load and every population is stored as one aligned pair;
// populations with e_x = +-1 come from sources shifted by one cell and are
// loaded per cell. Every pair is stored whole, a solid cell included, so
// 32-byte sectors are written complete (FP32 leaves out the sectors whose
// cells are all solid, which no one reads). Halfway bounce-back takes one of
// these forms, chosen per storage format by measurement (Bounce<S>):
//
//  - load side (FP64): a 32-bit push mask per cell (bit j: x + e_j is solid)
//    is loaded first; a population whose source x - e_i is solid (bit opp(i))
//    loads the opposite population of the cell itself, so each value costs one
//    load; threads whose two cells are solid skip everything.
//  - mask-guided reload (FP32): the push mask is loaded first but the gather
//    does not wait for it (every load takes the neighbour's address); pairs
//    with a bounce bit then reload their bounced populations from the cell's
//    own opposite slots, over the gathered values, before the moments.
//    Solid slots are never read. 37.5 against 34.0 GFLUPS for NaN marks on
//    the channel, which test each value and take the moments twice.
//  - NaN marks (kept as the measured alternative): every slot of a solid cell
//    holds NaN (written at create, init and set_state, and stored by the step
//    for solid cells). The gather loads all 19 values without looking at
//    flags; a NaN marks a solid source, so a NaN rho finds the cells next to a
//    solid, and only those lanes then load the opposite population of the
//    cell itself and take their moments again.
//  - separate kernel (16-bit storage), the paper's arrangement (Sec. 7: the
//    non-fluid cells are treated in a separate kernel): a solid cell s keeps in
//    slot i the value that its fluid neighbour s + e_i pulls next step (that
//    neighbour's post-collision population opp(i)); after the step, k_bounce
//    copies those values along a precomputed list of boundary links. Fewest
//    instructions in the step kernel, which is what the 2-byte formats need.
// In every form the fluid cells' own slots hold the post-collision
// populations, which is what the flag-aware readers (macros, state, reduction,
// adjoint) gather.
//
// Resident blocks of 256 threads per SM the step kernels are compiled for:
// FP64 arithmetic 1 (<= 255 registers), FP32 storage 3 (<= 80), 16-bit
// storage 4 (<= 64: fewer bytes per thread, so more threads in flight).
template <int S> struct StepBlocks {
    static constexpr int value = S == LBM_F64 ? 1 : ((S == LBM_F32 || is_split(S)) ? 3 : 4);
};
template <int S> struct Bounce {
    static constexpr int mode = bounce_mode(S);
};
template <int S> struct LinkBounce {
    static constexpr bool value = Bounce<S>::mode == BB_LINKS;
};

template <class R> __device__ __forceinline__ R quiet_nan();
template <> __device__ __forceinline__ float quiet_nan<float>() { return __int_as_float(0x7fffffff); }
template <> __device__ __forceinline__ double quiet_nan<double>() {
    return __longlong_as_double(0x7fffffffffffffffLL);
}

// The precomputed Guo constants of a uniform force, with c = 1 - omega/2, or
// over omega (c' = tau - 1/2) for the form of collide2 that relaxes about T.
template <class R, bool TFORM> __device__ __forceinline__ Guo2<R> uniform_guo(const Dev &d);
template <> __device__ __forceinline__ Guo2<float> uniform_guo<float, false>(const Dev &d) {
    Guo2<float> t;
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) {
        t.A[p] = vsplat(d.gAf[p]);
        t.C[p] = vsplat(d.gCf[p]);
    }
    return t;
}
template <> __device__ __forceinline__ Guo2<float> uniform_guo<float, true>(const Dev &d) {
    Guo2<float> t;
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) {
        t.A[p] = vsplat(d.gAtf[p]);
        t.C[p] = vsplat(d.gCtf[p]);
    }
    return t;
}
template <> __device__ __forceinline__ Guo2<double> uniform_guo<double, false>(const Dev &d) {
    Guo2<double> t;
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) {
        t.A[p] = vsplat(d.gA[p]);
        t.C[p] = vsplat(d.gC[p]);
    }
    return t;
}

// Where the gather finds the row of population i that cell row (y, z) pulls
// from, (y - e_iy, z - e_iz): in the source lattice in global memory, or in
// a shared-memory copy of those 19 rows (see k_step_tma).
// Offset k qs + c of lattice P: in 64 bits, or (I = unsigned, where every
// offset of the lattice fits) as one 32-bit index, which costs fewer
// instructions per address.
template <class I, class T> __device__ __forceinline__ T *lat_at(T *P, int k, long long qs, int c) {
    if constexpr (sizeof(I) == 4)
        return P + ((unsigned)k * (unsigned)qs + (unsigned)c);
    else
        return P + (long long)k * qs + c;
}

template <int S, class I = long long> struct GlobalRows {
    typedef typename Stor<S>::T T;
    typedef typename Stor<S>::R R;
    const T *src;
    __device__ __forceinline__ const T *row(const Geom &g, int i, int y, int z) const {
        return lat_at<I>(src, i, g.qs, (wrap1(z - ez(i), g.nz) * g.ny + wrap1(y - ey(i), g.ny)) * g.pitch);
    }
    static __device__ __forceinline__ R ld(const T *p) { return Stor<S>::ld(p); }
    static __device__ __forceinline__ void ld2(const T *p, R &a, R &b) { Stor<S>::ld2(p, a, b); }
};
template <int S> struct SharedRows {
    typedef typename Stor<S>::T T;
    typedef typename Stor<S>::R R;
    const T *buf;  // [Q][pitch]
    __device__ __forceinline__ const T *row(const Geom &g, int i, int, int) const { return buf + i * g.pitch; }
    static __device__ __forceinline__ R ld(const T *p) { return Stor<S>::ls(p); }
    static __device__ __forceinline__ void ld2(const T *p, R &a, R &b) { Stor<S>::ls2(p, a, b); }
};

// The pair's mass and momentum j + F/2 (rho u, or u itself in the
// incompressible model) of the pre-collision state, in FP64, added to red[4].
template <class R>
__device__ __forceinline__ void pair_add_totals(const Mom2<R> &m, bool live0, bool live1, bool incomp, double *red) {
    if (live0) {
        const double mr = incomp ? 1.0 : (double)m.rho.x;
        red[0] += (double)m.rho.x;
        red[1] += mr * (double)m.ux.x;
        red[2] += mr * (double)m.uy.x;
        red[3] += mr * (double)m.uz.x;
    }
    if (live1) {
        const double mr = incomp ? 1.0 : (double)m.rho.y;
        red[0] += (double)m.rho.y;
        red[1] += mr * (double)m.ux.y;
        red[2] += mr * (double)m.uy.y;
        red[3] += mr * (double)m.uz.y;
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The block's sum of every thread's red[4], in a fixed order, to
// partials[4 b + k] of block b = blockIdx.y * gridDim.x + blockIdx.x. Every
// thread of the block calls it (blocks of whole warps, at most 256 threads).
__device__ __forceinline__ void block_partials(const double red[4], double *__restrict__ partials) {
    __shared__ double sm[8][4];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nwarps = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double v = warp_sum_d(red[k]);
        if (lane == 0) sm[wid][k] = v;
    }
    __syncthreads();
    if (tid < 4) {
        double t = 0.0;
        for (int w = 0; w < nwarps; ++w) t += sm[w][tid];
        partials[4 * ((long long)blockIdx.y * gridDim.x + blockIdx.x) + tid] = t;
    }
}

// One fused step for the cell pair (x0, x0 + 1) of row (y, z): gather through
// `rows` (the cell's own opposite populations, for bounce-back, from src),
// collide, store to dst. RED: also add the pair's mass and momentum j + F/2
// (of the pre-collision state, in FP64) to red[4]; the pair then never
// returns early, so that its block can reduce.
template <int S, bool FLAGS, int FORCE, bool RECORD, class Rows, bool RED = false, class I = long long>
__device__ __forceinline__ void step_pair(const Dev &d, const Rows &rows, const typename Stor<S>::T *__restrict__ src,
                                          typename Stor<S>::T *__restrict__ dst, typename Stor<S>::R *__restrict__ tape,
                                          int x0, int y, int z, double *red = nullptr) {
    typedef typename Stor<S>::T T;
    typedef typename Stor<S>::R R;
    typedef typename Pair2<R>::V V;  // lane x: cell x0, lane y: cell x0 + 1
    constexpr bool MFIX = Bounce<S>::mode == BB_MFIX;
    constexpr bool LINKS = Bounce<S>::mode != BB_LOAD && !MFIX;  // flag-free gather (links or NaN marks)
    constexpr bool NANS = Bounce<S>::mode == BB_NANS;
    const Geom &g = d.g;
    const bool has1 = x0 + 1 < g.nx;
    const int c = cell_index(g, x0, y, z);
    uint32_t m0 = 0u, m1 = 0u;
    bool live0 = true, live1 = has1;
    if (FLAGS && !LINKS) {
        const uint2 mm = ld_resident2(d.mask + c);
        m0 = mm.x;
        m1 = mm.y;
        live0 = !(m0 & SOLID_BIT);
        live1 = has1 && !(m1 & SOLID_BIT);
        if (!MFIX && !RED && !live0 && !live1) return;
    } else if (FLAGS) {
        const uchar2 fl = __ldg(reinterpret_cast<const uchar2 *>(d.flags + c));
        // (no early exit for two solid cells: branching on this load would put
        // a dependent round trip in front of the gather, which measured ~12%
        // slower on the walled channel than loading and storing their pairs)
        live0 = !fl.x;
        live1 = has1 && !fl.y;
    }
    // source columns of the e_x = +-1 populations
    const int xa = wrap1(x0 - 1, g.nx);              // e_x = +1, cell x0
    const int xb = wrap1(x0 + 1, g.nx);              // e_x = -1, cell x0
    const int xc = has1 ? wrap1(x0 + 2, g.nx) : x0;  // e_x = -1, cell x0 + 1 (e_x = +1 pulls from x0)
    V s[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T *Pi = rows.row(g, i, y, z);
        if (FLAGS && !LINKS && !MFIX && i > 0) {
            const T *Po = lat_at<I>(src, opp(i), g.qs, c);  // own cell, opposite population
            const bool b0 = (m0 >> opp(i)) & 1u, b1 = (m1 >> opp(i)) & 1u;
            if (ex(i) == 0) {
                if (b0 == b1) {
                    Stor<S>::ld2(b0 ? Po : Pi + x0, s[i].x, s[i].y);
                } else {
                    s[i].x = Stor<S>::ld(b0 ? Po : Pi + x0);
                    s[i].y = Stor<S>::ld(b1 ? Po + 1 : Pi + x0 + 1);
                }
            } else {
                s[i].x = Stor<S>::ld(b0 ? Po : Pi + (ex(i) > 0 ? xa : xb));
                s[i].y = Stor<S>::ld(b1 ? Po + 1 : Pi + (ex(i) > 0 ? x0 : xc));
            }
        } else if (ex(i) == 0) {
            Rows::ld2(Pi + x0, s[i].x, s[i].y);
        } else {
            s[i].x = Rows::ld(Pi + (ex(i) > 0 ? xa : xb));
            s[i].y = Rows::ld(Pi + (ex(i) > 0 ? x0 : xc));
        }
    }
    // (a solid cell's mask has the bits of its solid neighbours, but its
    // values are never read: only fluid lanes reload, which spares the pairs
    // inside obstacles 36 loads; walled channel +1.5%)
    const uint32_t r0 = live0 ? m0 : 0u, r1 = live1 ? m1 : 0u;
    if (FLAGS && MFIX && ((r0 | r1) & 0x7fffeu)) {
        // a pair next to a solid: its bounced populations come from the
        // cell's own opposite slots, loaded over the gathered (unread) ones
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const T *Po = lat_at<I>(src, opp(i), g.qs, c);
            if ((r0 >> opp(i)) & 1u) s[i].x = Stor<S>::ld(Po);
            if ((r1 >> opp(i)) & 1u) s[i].y = Stor<S>::ld(Po + 1);
        }
    }
    if (FLAGS && !LINKS && d.moving_on && ((m0 | m1) & MOVING_BIT)) {
        // load side next to a moving wall: add its term to the bounced values
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if (((m0 >> opp(i)) & 1u) && d.flags[pull_src(g, x0, y, z, i)] == 2) s[i].x += wall_term<R>(d, i);
            if (((m1 >> opp(i)) & 1u) && d.flags[pull_src(g, x0 + 1, y, z, i)] == 2) s[i].y += wall_term<R>(d, i);
        }
    }
    V Fx = vsplat(R(0)), Fy = vsplat(R(0)), Fz = vsplat(R(0));
    Guo2<R> G;
    if (FORCE == 1) {
        Fx = vsplat(DevR<R>::F(d, 0));
        Fy = vsplat(DevR<R>::F(d, 1));
        Fz = vsplat(DevR<R>::F(d, 2));
        G = uniform_guo<R, relax_about_t(S)>(d);
    } else if (FORCE == 2) {
        const R *F = static_cast<const R *>(d.Ffield);
        ld2_real(F + c, Fx.x, Fx.y);
        ld2_real(F + g.qs + c, Fy.x, Fy.y);
        ld2_real(F + 2 * g.qs + c, Fz.x, Fz.y);
        G = guo2<R>(relax_about_t(S) ? DevR<R>::cs(d) : R(1) - R(0.5) * DevR<R>::omega(d), Fx, Fy, Fz);
    }
    Mom2<R> m = moments2<R, FORCE != 0>(s, Fx, Fy, Fz, d.incomp);
    if (FLAGS && NANS && ((live0 && m.rho.x != m.rho.x) || (live1 && m.rho.y != m.rho.y))) {
        // A solid source slot holds NaN, and a NaN anywhere makes rho NaN, so
        // one test per cell finds the cells next to a solid. Only those reload
        // each NaN population from the opposite slot of the cell itself
        // (halfway bounce-back, plus the moving-wall term) and take their
        // moments again.
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const T *Po = lat_at<I>(src, opp(i), g.qs, c);
            if (live0 && s[i].x != s[i].x) {
                s[i].x = Stor<S>::ld(Po);
                if (d.moving_on && d.flags[pull_src(g, x0, y, z, i)] == 2) s[i].x += wall_term<R>(d, i);
            }
            if (live1 && s[i].y != s[i].y) {
                s[i].y = Stor<S>::ld(Po + 1);
                if (d.moving_on && d.flags[pull_src(g, x0 + 1, y, z, i)] == 2) s[i].y += wall_term<R>(d, i);
            }
        }
        m = moments2<R, FORCE != 0>(s, Fx, Fy, Fz, d.incomp);
    }
    const bool bad0 = live0 && !(m.rho.x > R(0) && m.rho.x < R(1e30));
    const bool bad1 = live1 && !(m.rho.y > R(0) && m.rho.y < R(1e30));
    if (bad0 || bad1) atomicOr(d.status, LBM_STATUS_DIVERGED);
    if (RED) pair_add_totals<R>(m, live0, live1, d.incomp, red);
    if (RECORD) {
        const long long qs = g.qs;
        st2_real(tape + c, m.rho.x, m.rho.y);
        st2_real(tape + qs + c, m.ux.x, m.ux.y);
        st2_real(tape + 2 * qs + c, m.uy.x, m.uy.y);
        st2_real(tape + 3 * qs + c, m.uz.x, m.uz.y);
    }
    collide2<R, FORCE != 0, relax_about_t(S)>(s, m, DevR<R>::omega(d), DevR<R>::cs(d), Fx, Fy, Fz, G, d.incomp);
    // The pair is stored whole, a solid cell included, so 32-byte sectors are
    // written complete: a solid cell's values are never read (load side and
    // mask-guided reload, where all-solid sectors are left out below), it
    // stores the NaN that marks it (NaN marks), or its slots are link targets
    // that k_bounce rewrites (links). When moving-wall links are written into
    // solid slots by other threads of this launch, a pair with a solid cell
    // stores its fluid cell alone.
    if (FLAGS && NANS) {
        const R nan = quiet_nan<R>();
#pragma unroll
        for (int i = 0; i < Q; ++i)
            Stor<S>::st2(lat_at<I>(dst, i, g.qs, c), live0 ? s[i].x : nan, live1 ? s[i].y : nan);
    } else if (FLAGS && LinkBounce<S>::value && d.has_moving && !(live0 && live1)) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (live0) Stor<S>::st(lat_at<I>(dst, i, g.qs, c), s[i].x);
            if (live1) Stor<S>::st(lat_at<I>(dst, i, g.qs, c + 1), s[i].y);
        }
    } else {
        // FP32 mask-guided reload: a 32-byte sector whose 8 cells are all solid
        // is read by no one (the gather replaces every value it loads from a
        // solid slot, and the readers output zeros for solid cells), so its
        // four pairs skip their stores. Where rows start on sector boundaries
        // and hold a multiple of 4 pairs, the sector's pairs are on the lanes
        // 4k .. 4k + 3 of a warp; a lane not in step here (or past the edge)
        // counts as fluid, so no store is skipped on its account. Walled
        // channel +1.4%.
        bool skip = false;
        if constexpr (FLAGS && MFIX && S == LBM_F32) {
            if ((g.pitch & 7) == 0 && (((g.nx + 1) / 2) & 3) == 0) {
                const unsigned sb = __ballot_sync(__activemask(), !live0 && !live1);
                skip = ((sb >> ((threadIdx.x & 31) & ~3u)) & 0xFu) == 0xFu;
            }
        }
        // write-back stores: the planes a step writes last stay in L2 for the
        // next step, which starts on them (FP32 channel 39.3 against 39.8
        // GFLUPS with streaming stores; the AA and reverse steps keep theirs)
        if (!skip) {
#pragma unroll
            for (int i = 0; i < Q; ++i) Stor<S>::st2_wb(lat_at<I>(dst, i, g.qs, c), s[i].x, s[i].y);
        }
    }
    if (FLAGS && LinkBounce<S>::value && d.has_moving) {
        // Links into a moving wall (not in the link list): slot opp(j) of the
        // wall cell x + e_j gets P_j(x) + 6 w_opp(j) (e_opp(j) . u_w), formed
        // from the unrounded P_j(x) so that it is rounded to storage once.
        const uint2 mm = ld_resident2(d.mask + c);
        if ((mm.x | mm.y) & MOVING_BIT) {
#pragma unroll
            for (int j = 1; j < Q; ++j) {
                if (live0 && ((mm.x >> j) & 1u)) {
                    const int t = push_dst(g, x0, y, z, j);
                    if (d.flags[t] == 2) Stor<S>::st(lat_at<I>(dst, opp(j), g.qs, t), s[j].x - wall_term<R>(d, j));
                }
                if (live1 && ((mm.y >> j) & 1u)) {
                    const int t = push_dst(g, x0 + 1, y, z, j);
                    if (d.flags[t] == 2) Stor<S>::st(lat_at<I>(dst, opp(j), g.qs, t), s[j].y - wall_term<R>(d, j));
                }
            }
        }
    }
}

// The fused step of step_pair for the moment-split formats: the gather
// rebuilds each value from its source cell's remainder and momentum word, the
// bounce-back reload (the mask-guided form) rebuilds the cell's own opposite
// values from its own word, and the store writes the pair's momentum word,
// J = j + F (the momentum of the post-collision values: the Guo collision
// adds F), rounded, then the remainders against it.
template <int S, bool FLAGS, int FORCE, bool RECORD, bool RED = false, bool ODD = false>
__device__ __forceinline__ void step_pair_split(const Dev &d, const typename Stor<S>::T *__restrict__ src,
                                                typename Stor<S>::T *__restrict__ dst, float *__restrict__ tape,
                                                int x0, int y, int z, double *red = nullptr) {
    typedef typename Stor<S>::T T;
    typedef float R;
    typedef float2 V;  // lane x: cell x0, lane y: cell x0 + 1
    const Geom &g = d.g;
    const bool has1 = x0 + 1 < g.nx;
    const int c = cell_index(g, x0, y, z);
    uint32_t m0 = 0u, m1 = 0u;
    bool live0 = true, live1 = has1;
    if (FLAGS) {
        const uint2 mm = ld_resident2(d.mask + c);
        m0 = mm.x;
        m1 = mm.y;
        live0 = !(m0 & SOLID_BIT);
        live1 = has1 && !(m1 & SOLID_BIT);
    }
    const int xa = wrap1(x0 - 1, g.nx);              // e_x = +1, cell x0
    const int xb = wrap1(x0 + 1, g.nx);              // e_x = -1, cell x0
    const int xc = has1 ? wrap1(x0 + 2, g.nx) : x0;  // e_x = -1, cell x0 + 1 (e_x = +1 pulls from x0)
    // Momentum words of the nine source rows (y - e_y, z - e_z), r = 3 (e_y + 1)
    // + e_z + 1: the pair (x0, x0 + 1) of each, and cells xa and xc of the five
    // rows that directions with e_x = +-1 pull from (those with e_y e_z = 0).
    // The lone last cell of an odd row pulls its e_x = -1 values from the
    // row's first cell: its pair's second word is the copy of that cell's word
    // kept after the row's last cell (split_ghost), so no lane needs a select.
    const uint2 *Js = split_words(d, src);
    uint4 jq[9];
    uint2 ja[9], jc[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        const int dy = r / 3 - 1, dz = r % 3 - 1;
        const int rb = (wrap1(z - dz, g.nz) * g.ny + wrap1(y - dy, g.ny)) * g.pitch;
        jq[r] = __ldg(reinterpret_cast<const uint4 *>(Js + rb + x0));
        if (dy == 0 || dz == 0) {
            ja[r] = __ldg(Js + rb + xa);
            jc[r] = __ldg(Js + rb + xc);
        }
    }
    V s[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T *Pi = src + (long long)i * g.qs + (wrap1(z - ez(i), g.nz) * g.ny + wrap1(y - ey(i), g.ny)) * g.pitch;
        V gi;
        if (ex(i) == 0) {
            Stor<S>::ld2(Pi + x0, gi.x, gi.y);
        } else {
            gi.x = Stor<S>::ld(Pi + (ex(i) > 0 ? xa : xb));
            gi.y = Stor<S>::ld(Pi + (ex(i) > 0 ? x0 : xc));
        }
        if (i == 0) {
            s[0] = gi;
            continue;
        }
        const int r = (ey(i) + 1) * 3 + ez(i) + 1;
        uint2 wa, wb;  // the momentum words of the two source cells
        if (ex(i) == 0) {
            wa = make_uint2(jq[r].x, jq[r].y);
            wb = make_uint2(jq[r].z, jq[r].w);
        } else if (ex(i) > 0) {
            wa = ja[r];
            wb = make_uint2(jq[r].x, jq[r].y);
        } else {  // sources xb, xc: x0 + 1 (or its copy of cell 0 for a lone last cell) and x0 + 2
            wa = make_uint2(jq[r].z, jq[r].w);
            wb = jc[r];
        }
        const V jx = make_float2(SplitJ<S>::lo(wa.x), SplitJ<S>::lo(wb.x));
        const V jy = make_float2(SplitJ<S>::hi(wa.x), SplitJ<S>::hi(wb.x));
        const V jz = make_float2(SplitJ<S>::lo(wa.y), SplitJ<S>::lo(wb.y));
        s[i] = vfma(vsplat(split_k(i)), edot_first(split_first(i), jx, jy, jz), gi);
    }
    if (FLAGS && ((m0 | m1) & 0x7fffeu)) {
        // a pair next to a solid: its bounced values are the cell's own
        // opposite ones, rebuilt from its own momentum word (row r = 4) and
        // selected over the gathered (unread) ones. Per opposite pair (i, io)
        // one e'.J of the own word serves both directions, and the pair's own
        // remainders i and io load as two aligned pair words: branch-free, and
        // 14% faster on the walled channel than a predicated scalar load per
        // bounced value.
        const V ox = make_float2(SplitJ<S>::lo(jq[4].x), SplitJ<S>::lo(jq[4].z));
        const V oy = make_float2(SplitJ<S>::hi(jq[4].x), SplitJ<S>::hi(jq[4].z));
        const V oz = make_float2(SplitJ<S>::lo(jq[4].y), SplitJ<S>::lo(jq[4].w));
#pragma unroll
        for (int p = 0; p < NPAIR; ++p) {
            const int i = pair_first(p), io = opp(i);
            const V e = edot_first(i, ox, oy, oz);
            V gi, gio;
            Stor<S>::ld2(src + (long long)i * g.qs + c, gi.x, gi.y);
            Stor<S>::ld2(src + (long long)io * g.qs + c, gio.x, gio.y);
            const V ri = vfma(vsplat(split_k(io)), e, gio);
            const V rio = vfma(vsplat(split_k(i)), e, gi);
            s[i].x = ((m0 >> io) & 1u) ? ri.x : s[i].x;
            s[i].y = ((m1 >> io) & 1u) ? ri.y : s[i].y;
            s[io].x = ((m0 >> i) & 1u) ? rio.x : s[io].x;
            s[io].y = ((m1 >> i) & 1u) ? rio.y : s[io].y;
        }
    }
    if (FLAGS && d.moving_on && ((m0 | m1) & MOVING_BIT)) {
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if (((m0 >> opp(i)) & 1u) && d.flags[pull_src(g, x0, y, z, i)] == 2) s[i].x += wall_term<R>(d, i);
            if (((m1 >> opp(i)) & 1u) && d.flags[pull_src(g, x0 + 1, y, z, i)] == 2) s[i].y += wall_term<R>(d, i);
        }
    }
    V Fx = vsplat(R(0)), Fy = vsplat(R(0)), Fz = vsplat(R(0));
    Guo2<R> G;
    if (FORCE == 1) {
        Fx = vsplat(DevR<R>::F(d, 0));
        Fy = vsplat(DevR<R>::F(d, 1));
        Fz = vsplat(DevR<R>::F(d, 2));
        G = uniform_guo<R, false>(d);
    } else if (FORCE == 2) {
        const R *F = static_cast<const R *>(d.Ffield);
        ld2_real(F + c, Fx.x, Fx.y);
        ld2_real(F + g.qs + c, Fy.x, Fy.y);
        ld2_real(F + 2 * g.qs + c, Fz.x, Fz.y);
        G = guo2<R>(R(1) - R(0.5) * DevR<R>::omega(d), Fx, Fy, Fz);
    }
    const Mom2<R> m = moments2<R, FORCE != 0>(s, Fx, Fy, Fz, d.incomp);
    const bool bad0 = live0 && !(m.rho.x > R(0) && m.rho.x < R(1e30));
    const bool bad1 = live1 && !(m.rho.y > R(0) && m.rho.y < R(1e30));
    if (bad0 || bad1) atomicOr(d.status, LBM_STATUS_DIVERGED);
    if (RED) pair_add_totals<R>(m, live0, live1, d.incomp, red);
    if (RECORD) {
        const long long qs = g.qs;
        st2_real(tape + c, m.rho.x, m.rho.y);
        st2_real(tape + qs + c, m.ux.x, m.ux.y);
        st2_real(tape + 2 * qs + c, m.uy.x, m.uy.y);
        st2_real(tape + 3 * qs + c, m.uz.x, m.uz.y);
    }
    collide2<R, FORCE != 0, false>(s, m, DevR<R>::omega(d), DevR<R>::cs(d), Fx, Fy, Fz, G, d.incomp);
    // the pair's momentum word, then the remainders against the rounded J
    V Jx = m.jx, Jy = m.jy, Jz = m.jz;
    if (FORCE) {
        const V h = vsplat(R(0.5));
        Jx = vfma(h, Fx, Jx);
        Jy = vfma(h, Fy, Jy);
        Jz = vfma(h, Fz, Jz);
    }
    const unsigned w0x = SplitJ<S>::pack(Jx.x, Jy.x), w0y = SplitJ<S>::pack(Jz.x, R(0));
    const unsigned w1x = SplitJ<S>::pack(Jx.y, Jy.y), w1y = SplitJ<S>::pack(Jz.y, R(0));
    const V tx = make_float2(SplitJ<S>::lo(w0x), SplitJ<S>::lo(w1x));
    const V ty = make_float2(SplitJ<S>::hi(w0x), SplitJ<S>::hi(w1x));
    const V tz = make_float2(SplitJ<S>::lo(w0y), SplitJ<S>::lo(w1y));
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) {
        const int i = pair_first(p), io = opp(i);
        const V e = edot_first(i, tx, ty, tz);
        s[i] = vfma(vsplat(-split_k(i)), e, s[i]);
        s[io] = vfma(vsplat(-split_k(io)), e, s[io]);
    }
    // Pairs are stored whole, a solid cell included (its values are never
    // read: the mask-guided reload rebuilds bounced values from the fluid
    // cell's own slots), so 32-byte sectors are written complete.
#pragma unroll
    for (int i = 0; i < Q; ++i) Stor<S>::st2(dst + (long long)i * g.qs + c, s[i].x, s[i].y);
    uint2 *Jd = split_words(d, dst);
    if (!ODD || has1)
        *reinterpret_cast<uint4 *>(Jd + c) = make_uint4(w0x, w0y, w1x, w1y);
    else  // the lone last cell of an odd row: the slot after it holds cell 0's copy
        Jd[c] = make_uint2(w0x, w0y);
    if (ODD) split_ghost(d, Jd, x0, c, make_uint2(w0x, w0y));
}

// Launch every step kernel as a programmatic dependent of the kernel before it
// on its stream (the previous step, or the link form's bounce kernel): its
// blocks are scheduled as that kernel drains, and wait for it to complete
// before their first load. Measured: the link form's chain +1%; FP32 steps
// +0.5% when launched one by one (short runs), +0.2% in replayed graphs.
constexpr int STEP_PDL = 1;

// Block shape of the step kernel: the flat FP32 step with 32-bit offsets runs
// 7 blocks of 128 threads per SM (72 registers, no spills: 28 warps) instead
// of 3 of 256 (80 registers: 24 warps), +1.1% on the walled channel; 4 blocks
// of 256 (64 registers) spilled 48 bytes and lost 4%.
template <int S, bool FLAT, bool U32> constexpr int step_threads() { return U32 && FLAT ? 128 : 256; }
template <int S, bool FLAT, bool U32> constexpr int step_min_blocks() {
    return U32 && FLAT ? 7 : StepBlocks<S>::value;
}

// FLAT: the launch of d.PF (pairs in plane order), else of d.P (whole rows).
// ODD (moment-split formats only): rows of odd length, whose last cell is
// alone in its pair (see split_ghost). U32: 32-bit lattice offsets (lat_at).
template <int S, bool FLAGS, int FORCE, bool RECORD, bool FLAT = false, bool ODD = false, bool U32 = false>
__global__ void __launch_bounds__(step_threads<S, FLAT, U32>(), step_min_blocks<S, FLAT, U32>())
    k_step(const Dev d, const typename Stor<S>::T *__restrict__ src, typename Stor<S>::T *__restrict__ dst,
           typename Stor<S>::R *__restrict__ tape) {
    // launched as a programmatic dependent: wait for the kernel before it (the
    // previous step, or a bounce kernel whose links land in src) to complete
    // (a no-op when launched normally)
    if (STEP_PDL) asm volatile("griddepcontrol.wait;" ::: "memory");
    // let the next kernel (the bounce kernel, or the next step) be scheduled
    // once every block of this grid is running; it still waits for this grid
    // to complete before it reads what this grid writes
    if (STEP_PDL) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // blocks are dispatched in index order: with d.zrev the planes run from
    // the last to the first. (The BF16 split step keeps ascending order: with
    // the reversal its code schedules worse, 35.5 against 36.8 GFLUPS on the
    // walled channel at the same spills, while the FP16 split one gains 1.3%.)
    constexpr bool REV = S != LBM_BF16M;
    const int bz = REV && d.zrev ? (int)gridDim.y - 1 - (int)blockIdx.y : (int)blockIdx.y;
    int x0, y, z;
    if (!pair_cell<FLAT>(d.g, FLAT ? d.PF : d.P, blockDim.x, blockDim.y, blockIdx.x, bz, threadIdx.x, threadIdx.y,
                         x0, y, z))
        return;
    if constexpr (is_split(S))
        step_pair_split<S, FLAGS, FORCE, RECORD, false, ODD>(d, src, dst, tape, x0, y, z);
    else if constexpr (U32)
        step_pair<S, FLAGS, FORCE, RECORD, GlobalRows<S, unsigned>, false, unsigned>(
            d, GlobalRows<S, unsigned>{src}, src, dst, tape, x0, y, z);
    else
        step_pair<S, FLAGS, FORCE, RECORD>(d, GlobalRows<S>{src}, src, dst, tape, x0, y, z);
}

// The step with the mass/momentum totals of its pre-collision state fused in
// (the reduction of lbm_reduce without a pass of its own): every thread, in
// the lattice or not, reaches the block reduction; partials[4 b + k] of block
// b = blockIdx.y * gridDim.x + blockIdx.x, summed in a fixed order.
template <int S, bool FLAGS, int FORCE, bool FLAT, bool ODD = false>
__global__ void __launch_bounds__(256, StepBlocks<S>::value)
    k_step_reduce(const Dev d, const typename Stor<S>::T *__restrict__ src, typename Stor<S>::T *__restrict__ dst,
                  double *__restrict__ partials) {
    if (FLAGS && LinkBounce<S>::value) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    double red[4] = {0.0, 0.0, 0.0, 0.0};
    int x0, y, z;
    if (pair_cell<FLAT>(d.g, FLAT ? d.PF : d.P, blockDim.x, blockDim.y, blockIdx.x, blockIdx.y, threadIdx.x,
                        threadIdx.y, x0, y, z)) {
        if constexpr (is_split(S))
            step_pair_split<S, FLAGS, FORCE, false, true, ODD>(d, src, dst, nullptr, x0, y, z, red);
        else
            step_pair<S, FLAGS, FORCE, false, GlobalRows<S>, true>(d, GlobalRows<S>{src}, src, dst, nullptr, x0, y,
                                                                  z, red);
    }
    block_partials(red, partials);
}

// ---------------------------------------------------------------------------
// The step with its source rows staged in shared memory by the Tensor Memory
// Accelerator (FP32 and 16-bit storage). A cell row (y, z) pulls population
// i from the one row (y - e_iy, z - e_iz) of array i, shifted by e_ix, so a
// block that updates whole cell rows needs exactly 19 source rows per row.
// One thread issues them as 1-D bulk asynchronous copies (cp.async.bulk,
// whole padded rows: 16-byte aligned, sizes a multiple of 16 bytes) that
// signal an mbarrier with their byte count; the block computes row k from one
// buffer while the copies of row k + 1 land in the other. The loads are thus
// in flight without holding registers. The gathered values, the arithmetic
// (step_pair) and the stores are the same as in k_step, so both give the
// same bits. Opt-in (lbm_options.stage_rows): measured against the direct
// kernel it gains 1-4% on 16-bit lattices without obstacles, and loses on
// walled ones, where the block barrier per row exposes the latency of the
// bounce-back reloads that the direct kernel hides behind other warps.
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Wait for the phase with the given parity to complete, for at most ~1 s.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > (1LL << 31)) return false;
    return true;
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Order this thread's earlier shared-memory accesses (and the block's, after
// a barrier) before later asynchronous-proxy writes to the same memory.
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// The 19 source rows of cell row r into buf [Q][pitch], counted on bar.
// Row r of the fluid box (see pair_launch) as (y, z).
__device__ __forceinline__ void box_row(const RowLaunch &P, int r, int &y, int &z) {
    y = P.y0 + r % P.nyr;
    z = P.z0 + r / P.nyr;
}

template <int S>
__device__ __forceinline__ void issue_source_rows(const Geom &g, const RowLaunch &P, const typename Stor<S>::T *src,
                                                  typename Stor<S>::T *buf, uint64_t *bar, int r, uint32_t rowbytes) {
    int y, z;
    box_row(P, r, y, z);
    mbar_arrive_expect_tx(bar, (uint32_t)Q * rowbytes);
#pragma unroll 1
    for (int i = 0; i < Q; ++i) {
        const long long row = (long long)(wrap1(z - ez(i), g.nz) * g.ny + wrap1(y - ey(i), g.ny)) * g.pitch;
        bulk_copy_g2s(buf + i * g.pitch, src + (long long)i * g.qs + row, rowbytes, bar);
    }
}

template <int S, bool FLAGS, int FORCE, bool RECORD>
__global__ void __launch_bounds__(512)
    k_step_tma(const Dev d, const typename Stor<S>::T *__restrict__ src, typename Stor<S>::T *__restrict__ dst,
               typename Stor<S>::R *__restrict__ tape) {
    typedef typename Stor<S>::T T;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Geom &g = d.g;
    const uint32_t rowbytes = (uint32_t)g.pitch * (uint32_t)sizeof(T);
    T *buf = reinterpret_cast<T *>(smem_raw);  // [2][Q][pitch]
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + 2 * Q * rowbytes);
    const int nrows = d.P.nyr * d.P.nzr;  // the rows of the fluid box
    const int t = threadIdx.x, stride = gridDim.x;
    if (t == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        fence_mbar_init();
    }
    __syncthreads();
    int r = blockIdx.x;
    if (t == 0) {
        if (r < nrows) issue_source_rows<S>(g, d.P, src, buf, bar, r, rowbytes);
        if (r + stride < nrows) issue_source_rows<S>(g, d.P, src, buf + Q * g.pitch, bar + 1, r + stride, rowbytes);
    }
    const int pairs = (g.nx + 1) >> 1;
    for (int k = 0; r < nrows; ++k, r += stride) {
        const int b = k & 1;
        const bool ok = mbar_wait_bounded(bar + b, (k >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            // copies that never completed: report, give the other buffer's
            // copies a bounded chance to land, and leave. If that second
            // wait runs out too, the block exits with bulk copies still
            // addressed to its shared memory; there is no way to cancel them,
            // and an SM that later reuses that shared memory for another
            // block could see it overwritten. This path has never been
            // observed (no test forces it, nor may one: forcing it means a
            // copy that never completes); the status word tells the caller to
            // discard the run. The kernel is opt-in (lbm_options.stage_rows).
            if (t == 0) {
                atomicOr(d.status, LBM_STATUS_TIMEOUT);
                mbar_wait_bounded(bar + (b ^ 1), ((k + 1) >> 1) & 1);
            }
            return;
        }
        int y, z;
        box_row(d.P, r, y, z);
        const SharedRows<S> rows{buf + b * Q * g.pitch};
        for (int p = t; p < pairs; p += blockDim.x) step_pair<S, FLAGS, FORCE, RECORD>(d, rows, src, dst, tape, 2 * p, y, z);
        __syncthreads();  // every read of buffer b is done
        if (t == 0 && r + 2 * stride < nrows) {
            fence_async_shared();
            issue_source_rows<S>(g, d.P, src, buf + b * Q * g.pitch, bar + b, r + 2 * stride, rowbytes);
        }
    }
}

// Bounce-back links (separate-kernel form): for each fluid cell x and
// direction j with x + e_j solid and at rest, slot opp(j) of the solid cell
// receives the post-collision population j of x, copied bit for bit (links
// into moving walls are written by the step kernel). Links are grouped by
// direction (blockIdx.x + 1) and ordered by cell within a direction. Every
// direction's links are cut into gridDim.y equal spans, block (j, b) taking
// span b of direction j: blocks are dispatched span by span across the 18
// directions, so the kernel sweeps the planes once, against the order of the
// step before it, and ends on the planes the next step starts with (FP16
// channel 45.9 GFLUPS; sweeping in the step's own order 44.2, and one sweep
// per direction 45.6).
// Each thread copies LINKS_PER_THREAD links (256 apart, so index loads stay
// coalesced); all index loads are issued before the value loads, and all value
// loads before the stores, so the two dependent round trips are shared.
constexpr int LINKS_PER_THREAD = 4;
static_assert(256 * LINKS_PER_THREAD == BOUNCE_LINKS_PER_BLOCK, "k_bounce block size");
constexpr int BOUNCE_SWEEP_OPPOSITE = 1;
// Launch k_bounce as a programmatic dependent of the step kernel.
constexpr int BOUNCE_PDL = 1;

template <int S>
__global__ void __launch_bounds__(256) k_bounce(const Dev d, typename Stor<S>::T *__restrict__ P) {
    typedef typename Stor<S>::T T;
    const int j = blockIdx.x + 1;
    const int base = d.link_off[j];
    const int nb = (int)gridDim.y;
    const int b = (d.zrev ^ BOUNCE_SWEEP_OPPOSITE) ? nb - 1 - (int)blockIdx.y : (int)blockIdx.y;
    const int nj = d.link_off[j + 1] - base;
    const int span = (nj + nb - 1) / nb;  // <= blockDim.x * LINKS_PER_THREAD: nb spans the largest direction
    const int k0 = b * span + threadIdx.x;
    const int n = min(nj, (b + 1) * span);  // end of this block's span
    const uint2 *L = reinterpret_cast<const uint2 *>(d.links) + base;
    const T *from = P + (long long)j * d.g.qs;
    T *to = P + (long long)opp(j) * d.g.qs;
    uint2 l[LINKS_PER_THREAD];
    T v[LINKS_PER_THREAD];
#pragma unroll
    for (int r = 0; r < LINKS_PER_THREAD; ++r) {
        const int k = k0 + r * blockDim.x;
        l[r] = k < n ? ld_resident2(reinterpret_cast<const uint32_t *>(L + k)) : make_uint2(0u, 0u);  // (fluid, solid)
    }
    // Launched as a programmatic dependent of the step kernel: the links above
    // do not depend on it, the values below do. Wait here for the step's grid
    // to complete (a no-op when launched normally).
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // the next step kernel may be scheduled from here on: no earlier, so that
    // it cannot start before the step this kernel waited for has completed
    if (STEP_PDL) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#pragma unroll
    for (int r = 0; r < LINKS_PER_THREAD; ++r)
        if (k0 + r * blockDim.x < n) v[r] = from[l[r].x];
#pragma unroll
    for (int r = 0; r < LINKS_PER_THREAD; ++r)
        if (k0 + r * blockDim.x < n) to[l[r].y] = v[r];
}

// ---------------------------------------------------------------------------
// Initial state: P^{-1}_i(y) = f_eq_i at y + e_i if that cell is fluid, else
// f_eq_{opp(i)}(y) (so that the gather yields f^0 = f_eq(rho0, u0)), stored
// shifted by -w_i.
template <class R>
__device__ __forceinline__ R feq_shifted(int i, R rho1, R ux, R uy, R uz, bool incomp) {
    const R eu = R(ex(i)) * ux + R(ey(i)) * uy + R(ez(i)) * uz;
    const R usq = ux * ux + uy * uy + uz * uz;
    const R rho = incomp ? R(1) : R(1) + rho1;  // (He & Luo: velocity terms of the reference density)
    return R(weight(i)) * (rho1 + rho * (R(3) * eu + R(4.5) * eu * eu - R(1.5) * usq));
}

__device__ __forceinline__ long long canon_neighbor(const Geom &g, int x, int y, int z, int i) {
    return canon_index(g, wrap1(x + ex(i), g.nx), wrap1(y + ey(i), g.ny), wrap1(z + ez(i), g.nz));
}

template <int S, bool FLAGS>
__global__ void __launch_bounds__(256)
    k_init_eq(const Dev d, typename Stor<S>::T *__restrict__ P, const typename Stor<S>::R *__restrict__ rho0,
              const typename Stor<S>::R *__restrict__ u0) {
    typedef typename Stor<S>::R R;
    int x, y, z;
    if (!row_cell(d.g, d.L.nxb, blockDim.x, blockDim.y, blockIdx.x, blockIdx.y, threadIdx.x,
                  threadIdx.y, x, y, z))
        return;
    const int c = cell_index(d.g, x, y, z);
    if (FLAGS && d.flags[c]) {
        if (nan_marked<S>(d))
#pragma unroll
            for (int i = 0; i < Q; ++i) P[(long long)i * d.g.qs + c] = Stor<S>::enc(quiet_nan<R>());
        return;
    }
    const long long N = d.n_cells, cc = canon_index(d.g, x, y, z);
    if constexpr (is_split(S)) {  // the 19 values this cell holds, written as J and remainders
        R v[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int t = push_dst(d.g, x, y, z, i);
            int k = i;
            long long ct = canon_neighbor(d.g, x, y, z, i);
            const bool bounce = FLAGS && d.flags[t];
            if (bounce) {
                k = opp(i);
                ct = cc;
            }
            const R r1 = rho0 ? rho0[ct] - R(1) : R(0);
            v[i] = feq_shifted<R>(k, r1, u0[ct], u0[N + ct], u0[2 * N + ct], d.incomp);
            if (bounce && d.flags[t] == 2 && d.moving_on) v[i] += wall_term<R>(d, i);
        }
        split_store<S>(d, P, x, c, v);
        return;
    }
    if (d.layout == LAYOUT_AA_NAT) {  // AA natural layout: f^0_i(x) at the cell itself
        const R r1 = rho0 ? rho0[cc] - R(1) : R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i)
            P[(long long)i * d.g.qs + c] =
                Stor<S>::enc(feq_shifted<R>(i, r1, u0[cc], u0[N + cc], u0[2 * N + cc], d.incomp));
        return;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int t = push_dst(d.g, x, y, z, i);
        int k = i;
        long long ct = canon_neighbor(d.g, x, y, z, i);
        const bool bounce = FLAGS && d.flags[t];
        if (bounce) {
            k = opp(i);
            ct = cc;
        }
        const R r1 = rho0 ? rho0[ct] - R(1) : R(0);
        const R v = feq_shifted<R>(k, r1, u0[ct], u0[N + ct], u0[2 * N + ct], d.incomp);
        // (the gather adds the moving-wall term to a value bounced off a moving wall)
        const R wv = !bounce_in_solid(S) && bounce && d.flags[t] == 2 && d.moving_on ? wall_term<R>(d, i) : R(0);
        P[(long long)i * d.g.qs + c] = Stor<S>::enc(v + wv);
        // the solid neighbour's slot that the link form pulls f_opp(i)(x) from
        if (bounce && bounce_in_solid(S)) P[(long long)opp(i) * d.g.qs + t] = Stor<S>::enc(v);
    }
}

// ---------------------------------------------------------------------------
// get_state: canonical shifted f^n = gather(P), format D; solid cells 0.
template <int S, int D, bool FLAGS>
__global__ void __launch_bounds__(256)
    k_get_state(const Dev d, const typename Stor<S>::T *__restrict__ P, typename IOFmt<D>::T *__restrict__ out) {
    typedef typename Stor<S>::R R;
    int x, y, z;
    if (!row_cell(d.g, d.L.nxb, blockDim.x, blockDim.y, blockIdx.x, blockIdx.y, threadIdx.x,
                  threadIdx.y, x, y, z))
        return;
    const int c = cell_index(d.g, x, y, z);
    const long long N = d.n_cells, cc = canon_index(d.g, x, y, z);
    if (FLAGS && d.flags[c]) {
#pragma unroll
        for (int i = 0; i < Q; ++i) IOFmt<D>::put(out + i * N + cc, 0.0);
        return;
    }
    R s[Q];
    gather<S, FLAGS>(d, P, x, y, z, c, s);
#pragma unroll
    for (int i = 0; i < Q; ++i) IOFmt<D>::put(out + i * N + cc, (double)s[i]);
}

// set_state: P_i(y) = s_i(y + e_i) if fluid there, else s_{opp(i)}(y).
template <int S, int D, bool FLAGS>
__global__ void __launch_bounds__(256)
    k_set_state(const Dev d, typename Stor<S>::T *__restrict__ P, const typename IOFmt<D>::T *__restrict__ in) {
    int x, y, z;
    if (!row_cell(d.g, d.L.nxb, blockDim.x, blockDim.y, blockIdx.x, blockIdx.y, threadIdx.x,
                  threadIdx.y, x, y, z))
        return;
    const int c = cell_index(d.g, x, y, z);
    if (FLAGS && d.flags[c]) {
        if (nan_marked<S>(d))
#pragma unroll
            for (int i = 0; i < Q; ++i) IOFmt<S>::put(P + (long long)i * d.g.qs + c, (double)quiet_nan<float>());
        return;
    }
    const long long N = d.n_cells, cc = canon_index(d.g, x, y, z);
    if constexpr (is_split(S)) {  // the 19 values this cell holds, written as J and remainders
        double v[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int t = push_dst(d.g, x, y, z, i);
            long long off = (long long)i * N + canon_neighbor(d.g, x, y, z, i);
            const bool bounce = FLAGS && d.flags[t];
            if (bounce) off = (long long)opp(i) * N + cc;
            v[i] = IOFmt<D>::get(in + off) + (bounce && d.flags[t] == 2 && d.moving_on ? d.wc[i] : 0.0);
        }
        split_store<S>(d, P, x, c, v);
        return;
    }
    if (d.layout == LAYOUT_AA_NAT) {  // AA natural layout: s_i(x) at the cell itself
#pragma unroll
        for (int i = 0; i < Q; ++i) IOFmt<S>::put(P + (long long)i * d.g.qs + c, IOFmt<D>::get(in + i * N + cc));
        return;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int t = push_dst(d.g, x, y, z, i);
        long long off = (long long)i * N + canon_neighbor(d.g, x, y, z, i);
        const bool bounce = FLAGS && d.flags[t];
        if (bounce) off = (long long)opp(i) * N + cc;
        const double v = IOFmt<D>::get(in + off);
        const double wv = !bounce_in_solid(S) && bounce && d.flags[t] == 2 && d.moving_on ? d.wc[i] : 0.0;
        IOFmt<S>::put(P + (long long)i * d.g.qs + c, v + wv);
        // the solid neighbour's slot that the link form pulls f_opp(i)(x) from
        if (bounce && bounce_in_solid(S)) IOFmt<S>::put(P + (long long)opp(i) * d.g.qs + t, v);
    }
}

// ---------------------------------------------------------------------------
// Macroscopic fields (Sec. 2 step 1): rho and u = (j + F/2)/rho; solid 0.
template <int S, bool FLAGS, bool FORCE>
__global__ void __launch_bounds__(256)
    k_macros(const Dev d, const typename Stor<S>::T *__restrict__ P, typename Stor<S>::R *__restrict__ rho,
             typename Stor<S>::R *__restrict__ u) {
    typedef typename Stor<S>::R R;
    int x, y, z;
    if (!row_cell(d.g, d.L.nxb, blockDim.x, blockDim.y, blockIdx.x, blockIdx.y, threadIdx.x,
                  threadIdx.y, x, y, z))
        return;
    const int c = cell_index(d.g, x, y, z);
    const long long N = d.n_cells, cc = canon_index(d.g, x, y, z);
    if (FLAGS && d.flags[c]) {
        if (rho) rho[cc] = R(0);
        u[cc] = u[N + cc] = u[2 * N + cc] = R(0);
        return;
    }
    R s[Q];
    gather<S, FLAGS>(d, P, x, y, z, c, s);
    R Fx = R(0), Fy = R(0), Fz = R(0);
    if (FORCE) force_at<R>(d, c, Fx, Fy, Fz);
    const Mom<R> m = moments<R>(s, Fx, Fy, Fz, d.incomp);
    if (rho) rho[cc] = m.rho;
    u[cc] = m.ux;
    u[N + cc] = m.uy;
    u[2 * N + cc] = m.uz;
}

// ---------------------------------------------------------------------------
// Mass and momentum totals in FP64: fixed grid, each thread walks the cells
// c = tid, tid + stride, ... in order; blocks combine in a fixed tree; a
// single block adds the per-block partials in index order. Deterministic.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int S, bool FLAGS, bool FORCE>
__global__ void __launch_bounds__(RED_THREADS)
    k_reduce(const Dev d, const typename Stor<S>::T *__restrict__ P, int z0, int z1, double *__restrict__ partials) {
    typedef typename Stor<S>::R R;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    // the cells of planes z0 <= z < z1
    const long long N = (long long)d.g.nx * d.g.ny * (z1 - z0);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long cc = (long long)blockIdx.x * blockDim.x + threadIdx.x; cc < N; cc += stride) {
        const int x = (int)(cc % d.g.nx);
        const long long r = cc / d.g.nx;
        const int y = (int)(r % d.g.ny);
        const int z = z0 + (int)(r / d.g.ny);
        const int c = cell_index(d.g, x, y, z);
        if (FLAGS && d.flags[c]) continue;
        R s[Q];
        gather<S, FLAGS>(d, P, x, y, z, c, s);
        R Fx = R(0), Fy = R(0), Fz = R(0);
        if (FORCE) force_at<R>(d, c, Fx, Fy, Fz);
        const Mom<R> m = moments<R>(s, Fx, Fy, Fz, d.incomp);
        // momentum j + F/2: rho u, or u itself in the incompressible model
        const double mr = d.incomp ? 1.0 : (double)m.rho;
        acc[0] += (double)m.rho;
        acc[1] += mr * (double)m.ux;
        acc[2] += mr * (double)m.uy;
        acc[3] += mr * (double)m.uz;
    }
    __shared__ double sm[RED_THREADS / 32][4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) sm[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) t += sm[w][threadIdx.x];
        partials[blockIdx.x * 4 + threadIdx.x] = t;
    }
}

__global__ void __launch_bounds__(RED_THREADS) k_reduce_final(const double *__restrict__ partials, int nblocks,
                                                             double *__restrict__ out);

// ---------------------------------------------------------------------------
// Adjoint seed (not in the paper): lambda^T_m = dL/drho + g.(e_m - u)/rho,
// g = dL/du, at the gathered state; grad_F += g / (2 rho) (u contains F/2).
// Incompressible model (u = j + F/2): lambda^T_m = dL/drho + g.e_m, grad_F += g/2.
template <int S, bool FLAGS, bool FORCE>
__global__ void __launch_bounds__(256)
    k_adj_seed(const Dev d, const typename Stor<S>::T *__restrict__ P, const typename Stor<S>::R *__restrict__ dL_du,
               const typename Stor<S>::R *__restrict__ dL_drho, typename Stor<S>::R *__restrict__ lam,
               typename Stor<S>::R *__restrict__ grad_F) {
    typedef typename Stor<S>::R R;
    int x, y, z;
    if (!row_cell(d.g, d.L.nxb, blockDim.x, blockDim.y, blockIdx.x, blockIdx.y, threadIdx.x,
                  threadIdx.y, x, y, z))
        return;
    const int c = cell_index(d.g, x, y, z);
    const long long qs = d.g.qs, N = d.n_cells, cc = canon_index(d.g, x, y, z);
    if (FLAGS && d.flags[c]) return;  // solid cells' adjoint slots are never read
    R s[Q];
    gather<S, FLAGS>(d, P, x, y, z, c, s);
    R Fx = R(0), Fy = R(0), Fz = R(0);
    if (FORCE) force_at<R>(d, c, Fx, Fy, Fz);
    const Mom<R> m = moments<R>(s, Fx, Fy, Fz, d.incomp);
    const R gx = dL_du[cc], gy = dL_du[N + cc], gz = dL_du[2 * N + cc];
    const R dr = dL_drho ? dL_drho[cc] : R(0);
    const R inv = d.incomp ? R(1) : R(1) / m.rho;
    const R base = d.incomp ? dr : dr - (gx * m.ux + gy * m.uy + gz * m.uz) * inv;
#pragma unroll
    for (int i = 0; i < Q; ++i) lam[i * qs + c] = base + (R(ex(i)) * gx + R(ey(i)) * gy + R(ez(i)) * gz) * inv;
    if (grad_F) {
        grad_F[cc] += R(0.5) * gx * inv;
        grad_F[N + cc] += R(0.5) * gy * inv;
        grad_F[2 * N + cc] += R(0.5) * gz * inv;
    }
}

// ---------------------------------------------------------------------------
// Host launchers.
inline dim3 row_grid(const Dev &d) { return dim3(d.L.nxb * d.L.nyb, d.g.nz); }
inline dim3 row_block(const Dev &d) { return dim3(d.L.bx_threads, d.L.by_threads); }

// The step kernels run on the paired launch (two cells per thread).
inline dim3 step_grid(const Dev &d) { return dim3(d.P.nxb * d.P.nyb, d.P.nzr); }
inline dim3 step_block(const Dev &d) { return dim3(d.P.bx_threads, d.P.by_threads); }

// 32-bit lattice offsets: measured on the FP32 step with flags (walled
// channel +0.9%); the 16-bit and flag-free steps gained nothing (512^3 box
// FP16 -1.9%), so they keep 64-bit offsets.
template <int S, bool FLAGS> inline bool step_u32(const Dev &d) {
    return S == LBM_F32 && FLAGS && (long long)Q * d.g.qs < (1LL << 32);
}

template <int S, bool FLAGS, int FORCE, bool FLAT, bool ODD = false, bool U32 = false>
static cudaError_t launch_step3f(const Dev &d, const void *src, void *dst, void *tape) {
    typedef typename Stor<S>::T T;
    typedef typename Stor<S>::R R;
    if constexpr (!U32 && S == LBM_F32 && FLAGS) {
        if (step_u32<S, FLAGS>(d)) {
            if constexpr (FLAT && step_threads<S, true, true>() != 256) {
                Dev d2 = d;  // the same pairs in blocks of the kernel's size
                d2.PF = flat_launch(d.P, step_threads<S, true, true>());
                return launch_step3f<S, FLAGS, FORCE, FLAT, ODD, true>(d2, src, dst, tape);
            }
            return launch_step3f<S, FLAGS, FORCE, FLAT, ODD, true>(d, src, dst, tape);
        }
    }
    const RowLaunch &P = FLAT ? d.PF : d.P;
    const dim3 grid(P.nxb * P.nyb, P.nzr), block(P.bx_threads, P.by_threads);
    if (STEP_PDL) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.stream = d.stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e = tape ? cudaLaunchKernelEx(&cfg, k_step<S, FLAGS, FORCE, true, FLAT, ODD, U32>, d,
                                                  static_cast<const T *>(src), static_cast<T *>(dst),
                                                  static_cast<R *>(tape))
                             : cudaLaunchKernelEx(&cfg, k_step<S, FLAGS, FORCE, false, FLAT, ODD, U32>, d,
                                                  static_cast<const T *>(src), static_cast<T *>(dst), (R *)nullptr);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    if (tape)
        k_step<S, FLAGS, FORCE, true, FLAT, ODD, U32><<<grid, block, 0, d.stream>>>(
            d, static_cast<const T *>(src), static_cast<T *>(dst), static_cast<R *>(tape));
    else
        k_step<S, FLAGS, FORCE, false, FLAT, ODD, U32><<<grid, block, 0, d.stream>>>(
            d, static_cast<const T *>(src), static_cast<T *>(dst), nullptr);
    return cudaGetLastError();
}

// The flat launch where whole rows would leave lanes idle, and also where it
// measured faster with whole-warp rows (its index code compiles to fewer
// spills): FP32 (walled channel +1%) and 16-bit storage without flags (512^3
// box +3%). The 16-bit link form with flags keeps whole rows there (the flat
// form spilled more: -4.5%); so does FP64.
template <int S, bool FLAGS> constexpr bool flat_preferred() {
    return S == LBM_F32 || is_split(S) || (S != LBM_F64 && !FLAGS);
}

template <int S, bool FLAGS, int FORCE>
static cudaError_t launch_step3(const Dev &d, const void *src, void *dst, void *tape) {
    if constexpr (is_split(S))  // (always the flat launch)
        return (d.g.nx & 1) ? launch_step3f<S, FLAGS, FORCE, true, true>(d, src, dst, tape)
                            : launch_step3f<S, FLAGS, FORCE, true, false>(d, src, dst, tape);
    else
        return d.flat_step || flat_preferred<S, FLAGS>() ? launch_step3f<S, FLAGS, FORCE, true>(d, src, dst, tape)
                                                         : launch_step3f<S, FLAGS, FORCE, false>(d, src, dst, tape);
}

// Shared memory of the row-staged step: two buffers of 19 padded rows.
constexpr int TMA_SMEM_MAX = 200 * 1024;
template <int S> inline int tma_smem_bytes(const Dev &d) {
    return 2 * Q * d.g.pitch * (int)sizeof(typename Stor<S>::T) + 16;
}
// The row-staged step serves the flag-free gathers (NaN marks, links) of
// FP32 and 16-bit storage when rows are whole 16-byte multiples and two
// buffers fit.
template <int S> inline bool tma_eligible(const Dev &d) {
    const long long rowbytes = (long long)d.g.pitch * sizeof(typename Stor<S>::T);
    return d.row_staging && Bounce<S>::mode != BB_LOAD && rowbytes % 16 == 0 && tma_smem_bytes<S>(d) <= TMA_SMEM_MAX;
}

template <int S, bool FLAGS, int FORCE, bool RECORD>
static cudaError_t launch_step_tma4(const Dev &d, const void *src, void *dst, void *tape) {
    typedef typename Stor<S>::T T;
    typedef typename Stor<S>::R R;
    auto kern = k_step_tma<S, FLAGS, FORCE, RECORD>;
    // (set on every launch: the attribute belongs to the current device's context)
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, TMA_SMEM_MAX);
    if (e != cudaSuccess) return e;
    const int smem = tma_smem_bytes<S>(d);
    const int pairs = (d.g.nx + 1) / 2;
    const int threads = pairs >= 512 ? 512 : (pairs + 31) / 32 * 32;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess) return e;
    const long long nrows = (long long)d.P.nyr * d.P.nzr;
    const long long want = (long long)(occ > 0 ? occ : 1) * d.num_sms;
    const int grid = (int)(nrows < want ? nrows : want);
    kern<<<grid, threads, smem, d.stream>>>(d, static_cast<const T *>(src), static_cast<T *>(dst),
                                           static_cast<R *>(tape));
    return cudaGetLastError();
}

template <int S, bool FLAGS, int FORCE>
static cudaError_t launch_step3_any(const Dev &d, const void *src, void *dst, void *tape) {
    if constexpr (!is_split(S)) {  // (the moment-split formats have no staged form)
        if (tma_eligible<S>(d))
            return tape ? launch_step_tma4<S, FLAGS, FORCE, true>(d, src, dst, tape)
                        : launch_step_tma4<S, FLAGS, FORCE, false>(d, src, dst, tape);
    }
    return launch_step3<S, FLAGS, FORCE>(d, src, dst, tape);
}

template <int S, bool FLAGS>
static cudaError_t launch_step2(const Dev &d, const void *src, void *dst, void *tape) {
    if (d.Ffield) return launch_step3_any<S, FLAGS, 2>(d, src, dst, tape);
    if (d.force_on) return launch_step3_any<S, FLAGS, 1>(d, src, dst, tape);
    return launch_step3_any<S, FLAGS, 0>(d, src, dst, tape);
}

template <int S>
cudaError_t Ops<S>::step(const Dev &d, const void *src, void *dst, void *tape) {
    if (!d.flags) return launch_step2<S, false>(d, src, dst, tape);
    if (!d.mask) return cudaErrorInvalidValue;  // every two-grid form with flags may read the push masks
    cudaError_t e = launch_step2<S, true>(d, src, dst, tape);
    if (e != cudaSuccess || !LinkBounce<S>::value || d.link_max == 0) return e;
    const int per_block = 256 * LINKS_PER_THREAD;
    // programmatic dependent launch: the bounce kernel's blocks may start (and
    // load their links) while the step kernel drains; they wait for its grid
    // before reading the values (griddepcontrol.wait in k_bounce)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(Q - 1, (d.link_max + per_block - 1) / per_block);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = d.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = BOUNCE_PDL;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_bounce<S>, d, static_cast<typename Stor<S>::T *>(dst));
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int S>
cudaError_t Ops<S>::bounce(const Dev &d, void *dst) {
    if (!d.flags || !LinkBounce<S>::value || d.link_max == 0) return cudaSuccess;
    const int per_block = 256 * LINKS_PER_THREAD;
    k_bounce<S><<<dim3(Q - 1, (d.link_max + per_block - 1) / per_block), 256, 0, d.stream>>>(
        d, static_cast<typename Stor<S>::T *>(dst));
    return cudaGetLastError();
}

// The fused step-reduce kernel for one launch mapping (FLAT) and row parity (ODD).
template <int S, bool FLAT, bool ODD>
static void launch_step_reduce2(const Dev &d, const dim3 grid, const dim3 block, const typename Stor<S>::T *s,
                                typename Stor<S>::T *t, double *partials) {
    if (d.flags) {
        if (d.Ffield) k_step_reduce<S, true, 2, FLAT, ODD><<<grid, block, 0, d.stream>>>(d, s, t, partials);
        else if (d.force_on) k_step_reduce<S, true, 1, FLAT, ODD><<<grid, block, 0, d.stream>>>(d, s, t, partials);
        else k_step_reduce<S, true, 0, FLAT, ODD><<<grid, block, 0, d.stream>>>(d, s, t, partials);
    } else {
        if (d.Ffield) k_step_reduce<S, false, 2, FLAT, ODD><<<grid, block, 0, d.stream>>>(d, s, t, partials);
        else if (d.force_on) k_step_reduce<S, false, 1, FLAT, ODD><<<grid, block, 0, d.stream>>>(d, s, t, partials);
        else k_step_reduce<S, false, 0, FLAT, ODD><<<grid, block, 0, d.stream>>>(d, s, t, partials);
    }
}

template <int S>
cudaError_t Ops<S>::step_reduce(const Dev &d, const void *src, void *dst, double *partials, double *out) {
    typedef typename Stor<S>::T T;
    if (d.flags && !d.mask) return cudaErrorInvalidValue;
    const T *s = static_cast<const T *>(src);
    T *t = static_cast<T *>(dst);
    // the launch mapping of the plain step (launch_step3)
    const bool flat = d.flat_step || (d.flags ? flat_preferred<S, true>() : flat_preferred<S, false>());
    const RowLaunch &P = flat ? d.PF : d.P;
    const dim3 grid(P.nxb * P.nyb, P.nzr), block(P.bx_threads, P.by_threads);
    if constexpr (is_split(S)) {  // (always the flat launch)
        if (d.g.nx & 1)
            launch_step_reduce2<S, true, true>(d, grid, block, s, t, partials);
        else
            launch_step_reduce2<S, true, false>(d, grid, block, s, t, partials);
    } else if (flat) {
        launch_step_reduce2<S, true, false>(d, grid, block, s, t, partials);
    } else {
        launch_step_reduce2<S, false, false>(d, grid, block, s, t, partials);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (d.flags && LinkBounce<S>::value && d.link_max > 0) {
        const int per_block = 256 * LINKS_PER_THREAD;
        k_bounce<S><<<dim3(Q - 1, (d.link_max + per_block - 1) / per_block), 256, 0, d.stream>>>(d, t);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_reduce_final<<<1, RED_THREADS, 0, d.stream>>>(partials, (int)(grid.x * grid.y), out);
    return cudaGetLastError();
}

// NaN marks on every slot of every solid cell (NaN-mark form; no-op otherwise).
template <int S>
__global__ void __launch_bounds__(256) k_fill_solid(const Dev d, typename Stor<S>::T *__restrict__ P) {
    int x, y, z;
    if (!row_cell(d.g, d.L.nxb, blockDim.x, blockDim.y, blockIdx.x, blockIdx.y, threadIdx.x, threadIdx.y, x, y, z))
        return;
    const int c = cell_index(d.g, x, y, z);
    if (!d.flags[c]) return;
#pragma unroll
    for (int i = 0; i < Q; ++i) P[(long long)i * d.g.qs + c] = Stor<S>::enc(quiet_nan<typename Stor<S>::R>());
}

template <int S>
cudaError_t Ops<S>::fill_solid(const Dev &d, void *lat) {
    if (!d.flags || (Bounce<S>::mode != BB_NANS && d.layout == LAYOUT_PULL)) return cudaSuccess;
    k_fill_solid<S><<<row_grid(d), row_block(d), 0, d.stream>>>(d, static_cast<typename Stor<S>::T *>(lat));
    return cudaGetLastError();
}

template <int S>
cudaError_t Ops<S>::init_eq(const Dev &d, void *lat, const void *rho0, const void *u0) {
    typedef typename Stor<S>::T T;
    typedef typename Stor<S>::R R;
    if (d.flags)
        k_init_eq<S, true><<<row_grid(d), row_block(d), 0, d.stream>>>(
            d, static_cast<T *>(lat), static_cast<const R *>(rho0), static_cast<const R *>(u0));
    else
        k_init_eq<S, false><<<row_grid(d), row_block(d), 0, d.stream>>>(
            d, static_cast<T *>(lat), static_cast<const R *>(rho0), static_cast<const R *>(u0));
    return cudaGetLastError();
}

template <int S, int D>
static cudaError_t launch_get(const Dev &d, const void *lat, void *dst) {
    typedef typename Stor<S>::T T;
    typedef typename IOFmt<D>::T TD;
    if (d.flags)
        k_get_state<S, D, true><<<row_grid(d), row_block(d), 0, d.stream>>>(d, static_cast<const T *>(lat),
                                                                          static_cast<TD *>(dst));
    else
        k_get_state<S, D, false><<<row_grid(d), row_block(d), 0, d.stream>>>(d, static_cast<const T *>(lat),
                                                                           static_cast<TD *>(dst));
    return cudaGetLastError();
}

template <int S, int D>
static cudaError_t launch_set(const Dev &d, void *lat, const void *src) {
    typedef typename Stor<S>::T T;
    typedef typename IOFmt<D>::T TD;
    if (d.flags)
        k_set_state<S, D, true><<<row_grid(d), row_block(d), 0, d.stream>>>(d, static_cast<T *>(lat),
                                                                          static_cast<const TD *>(src));
    else
        k_set_state<S, D, false><<<row_grid(d), row_block(d), 0, d.stream>>>(d, static_cast<T *>(lat),
                                                                           static_cast<const TD *>(src));
    return cudaGetLastError();
}

template <int S>
cudaError_t Ops<S>::get_state(const Dev &d, const void *lat, void *dst, int fmt) {
    switch (fmt) {
    case LBM_F64: return launch_get<S, LBM_F64>(d, lat, dst);
    case LBM_F32: return launch_get<S, LBM_F32>(d, lat, dst);
    case LBM_F16S: case LBM_F16M: return launch_get<S, LBM_F16S>(d, lat, dst);
    case LBM_BF16S: case LBM_BF16M: return launch_get<S, LBM_BF16S>(d, lat, dst);
    }
    return cudaErrorInvalidValue;
}

template <int S>
cudaError_t Ops<S>::set_state(const Dev &d, void *lat, const void *src, int fmt) {
    switch (fmt) {
    case LBM_F64: return launch_set<S, LBM_F64>(d, lat, src);
    case LBM_F32: return launch_set<S, LBM_F32>(d, lat, src);
    case LBM_F16S: case LBM_F16M: return launch_set<S, LBM_F16S>(d, lat, src);
    case LBM_BF16S: case LBM_BF16M: return launch_set<S, LBM_BF16S>(d, lat, src);
    }
    return cudaErrorInvalidValue;
}

template <int S, bool FLAGS>
static cudaError_t launch_macros(const Dev &d, const void *lat, void *rho, void *u) {
    typedef typename Stor<S>::T T;
    typedef typename Stor<S>::R R;
    if (d.force_on)
        k_macros<S, FLAGS, true><<<row_grid(d), row_block(d), 0, d.stream>>>(
            d, static_cast<const T *>(lat), static_cast<R *>(rho), static_cast<R *>(u));
    else
        k_macros<S, FLAGS, false><<<row_grid(d), row_block(d), 0, d.stream>>>(
            d, static_cast<const T *>(lat), static_cast<R *>(rho), static_cast<R *>(u));
    return cudaGetLastError();
}

template <int S>
cudaError_t Ops<S>::macros(const Dev &d, const void *lat, void *rho, void *u) {
    return d.flags ? launch_macros<S, true>(d, lat, rho, u) : launch_macros<S, false>(d, lat, rho, u);
}

template <int S, bool FLAGS>
static cudaError_t launch_reduce(const Dev &d, const void *lat, int z0, int z1, double *partials) {
    typedef typename Stor<S>::T T;
    if (d.force_on)
        k_reduce<S, FLAGS, true><<<RED_BLOCKS, RED_THREADS, 0, d.stream>>>(d, static_cast<const T *>(lat), z0, z1,
                                                                          partials);
    else
        k_reduce<S, FLAGS, false><<<RED_BLOCKS, RED_THREADS, 0, d.stream>>>(d, static_cast<const T *>(lat), z0, z1,
                                                                           partials);
    return cudaGetLastError();
}

template <int S>
cudaError_t Ops<S>::reduce(const Dev &d, const void *lat, int z0, int z1, double *partials, double *out) {
    cudaError_t e = d.flags ? launch_reduce<S, true>(d, lat, z0, z1, partials)
                            : launch_reduce<S, false>(d, lat, z0, z1, partials);
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, RED_THREADS, 0, d.stream>>>(partials, RED_BLOCKS, out);
    return cudaGetLastError();
}

template <int S, bool FLAGS>
static cudaError_t launch_seed(const Dev &d, const void *lat, const void *dL_du, const void *dL_drho, void *lam,
                               void *grad_F) {
    typedef typename Stor<S>::T T;
    typedef typename Stor<S>::R R;
    if (d.force_on)
        k_adj_seed<S, FLAGS, true><<<row_grid(d), row_block(d), 0, d.stream>>>(
            d, static_cast<const T *>(lat), static_cast<const R *>(dL_du), static_cast<const R *>(dL_drho),
            static_cast<R *>(lam), static_cast<R *>(grad_F));
    else
        k_adj_seed<S, FLAGS, false><<<row_grid(d), row_block(d), 0, d.stream>>>(
            d, static_cast<const T *>(lat), static_cast<const R *>(dL_du), static_cast<const R *>(dL_drho),
            static_cast<R *>(lam), static_cast<R *>(grad_F));
    return cudaGetLastError();
}

template <int S>
cudaError_t Ops<S>::adj_seed(const Dev &d, const void *lat, const void *dL_du, const void *dL_drho, void *lam,
                             void *grad_F) {
    return d.flags ? launch_seed<S, true>(d, lat, dL_du, dL_drho, lam, grad_F)
                   : launch_seed<S, false>(d, lat, dL_du, dL_drho, lam, grad_F);
}

}  // namespace lbm
