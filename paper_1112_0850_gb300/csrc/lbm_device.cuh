// Device-side building blocks of the D3Q19 BGK kernels: the lattice table,
// population storage formats, the padded structure-of-arrays geometry and the
// per-cell collision (Sec. 2 of Habich et al.; Eq. 1 with the Qian
// equilibrium and, as this library's reading, the Guo body force).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lbm_capi.h"

#define LBM_HD __host__ __device__ __forceinline__

namespace lbm {

constexpr int Q = 19;

// Velocity set, in the order documented in lbm_capi.h: component a of e_i is
// stored as a + 1 in bits 2i..2i+1 of one 64-bit constant per axis, so that
// host and device code fold ex(i), ey(i), ez(i) to literals once loops unroll.
LBM_HD constexpr int ex(int i) { return int((0x1542829549ULL >> (2 * i)) & 3ULL) - 1; }
LBM_HD constexpr int ey(int i) { return int((0x295489495ULL >> (2 * i)) & 3ULL) - 1; }
LBM_HD constexpr int ez(int i) { return int((0x888954955ULL >> (2 * i)) & 3ULL) - 1; }

// Index of -e_i: axis pairs (1,2), (3,4), (5,6); the diagonals come in groups
// of four (7-10, 11-14, 15-18) where member k pairs with member 3 - k.
LBM_HD constexpr int opp(int i) {
    return i == 0 ? 0
                  : (i <= 6 ? ((i & 1) ? i + 1 : i - 1)
                            : (7 + 4 * ((i - 7) / 4)) + 3 - (i - (7 + 4 * ((i - 7) / 4))));
}

LBM_HD constexpr double weight(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

// The nine opposite pairs (i, opp(i)) with i the member listed first.
constexpr int NPAIR = 9;
LBM_HD constexpr int pair_first(int p) { return p < 3 ? 1 + 2 * p : (p < 5 ? 4 + p : (p < 7 ? 6 + p : 8 + p)); }

// ---------------------------------------------------------------------------
// Storage formats. Every format stores the shifted deviation s = f - w.
// R is the arithmetic type (double for LBM_F64, float otherwise).
template <int S> struct Stor;

// ld2/st2 move the values of two x-adjacent cells (p 2-element aligned).
template <> struct Stor<LBM_F64> {
    typedef double T;
    typedef double R;
    static __device__ __forceinline__ R ld(const T *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(T *p, R v) { __stcs(p, v); }
    static __device__ __forceinline__ T enc(R v) { return v; }
    static __device__ __forceinline__ void ld2(const T *p, R &a, R &b) {
        const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ void st2(T *p, R a, R b) {
        __stcs(reinterpret_cast<double2 *>(p), make_double2(a, b));
    }
    // a write-back store: the line stays in L2 for a later reader
    static __device__ __forceinline__ void st2_wb(T *p, R a, R b) {
        *reinterpret_cast<double2 *>(p) = make_double2(a, b);
    }
    // plain loads (shared memory)
    static __device__ __forceinline__ R ls(const T *p) { return *p; }
    static __device__ __forceinline__ void ls2(const T *p, R &a, R &b) {
        const double2 v = *reinterpret_cast<const double2 *>(p);
        a = v.x;
        b = v.y;
    }
};

template <> struct Stor<LBM_F32> {
    typedef float T;
    typedef float R;
    static __device__ __forceinline__ R ld(const T *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(T *p, R v) { __stcs(p, v); }
    static __device__ __forceinline__ T enc(R v) { return v; }
    static __device__ __forceinline__ void ld2(const T *p, R &a, R &b) {
        const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ void st2(T *p, R a, R b) {
        __stcs(reinterpret_cast<float2 *>(p), make_float2(a, b));
    }
    static __device__ __forceinline__ void st2_wb(T *p, R a, R b) {
        *reinterpret_cast<float2 *>(p) = make_float2(a, b);
    }
    static __device__ __forceinline__ R ls(const T *p) { return *p; }
    static __device__ __forceinline__ void ls2(const T *p, R &a, R &b) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        a = v.x;
        b = v.y;
    }
};

template <> struct Stor<LBM_F16S> {
    typedef __half T;
    typedef float R;
    // (16-bit pairs are stored write-back already)
    static __device__ __forceinline__ void st2_wb(T *p, R a, R b) { st2(p, a, b); }
    static __device__ __forceinline__ R ld(const T *p) {
        return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short *>(p))));
    }
    static __device__ __forceinline__ void st(T *p, R v) {
        __stcs(reinterpret_cast<unsigned short *>(p), __half_as_ushort(__float2half_rn(v)));
    }
    static __device__ __forceinline__ T enc(R v) { return __float2half_rn(v); }
    // pairs move as one 32-bit word and convert with one packed instruction
    static __device__ __forceinline__ void ld2(const T *p, R &a, R &b) {
        union {
            unsigned u;
            __half2 h;
        } v;
        v.u = __ldg(reinterpret_cast<const unsigned *>(p));
        const float2 f = __half22float2(v.h);
        a = f.x;
        b = f.y;
    }
    static __device__ __forceinline__ void st2(T *p, R a, R b) {
        union {
            unsigned u;
            __half2 h;
        } v;
        v.h = __floats2half2_rn(a, b);
        *reinterpret_cast<unsigned *>(p) = v.u;  // (write-back: +1% over streaming stores)
    }
    static __device__ __forceinline__ R ls(const T *p) { return __half2float(*p); }
    static __device__ __forceinline__ void ls2(const T *p, R &a, R &b) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(p));
        a = f.x;
        b = f.y;
    }
};

template <> struct Stor<LBM_BF16S> {
    typedef __nv_bfloat16 T;
    typedef float R;
    // (16-bit pairs are stored write-back already)
    static __device__ __forceinline__ void st2_wb(T *p, R a, R b) { st2(p, a, b); }
    static __device__ __forceinline__ R ld(const T *p) {
        return __bfloat162float(
            __ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short *>(p))));
    }
    static __device__ __forceinline__ void st(T *p, R v) {
        __stcs(reinterpret_cast<unsigned short *>(p), __bfloat16_as_ushort(__float2bfloat16_rn(v)));
    }
    static __device__ __forceinline__ T enc(R v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ void ld2(const T *p, R &a, R &b) {
        union {
            unsigned u;
            __nv_bfloat162 h;
        } v;
        v.u = __ldg(reinterpret_cast<const unsigned *>(p));
        const float2 f = __bfloat1622float2(v.h);
        a = f.x;
        b = f.y;
    }
    static __device__ __forceinline__ void st2(T *p, R a, R b) {
        union {
            unsigned u;
            __nv_bfloat162 h;
        } v;
        v.h = __floats2bfloat162_rn(a, b);
        *reinterpret_cast<unsigned *>(p) = v.u;  // (write-back: +1% over streaming stores)
    }
    static __device__ __forceinline__ R ls(const T *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void ls2(const T *p, R &a, R &b) {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
        a = f.x;
        b = f.y;
    }
};

// The moment-split formats store their 19 remainders as the 16-bit format
// of the same name does; their per-cell momentum words are handled by SplitJ.
LBM_HD constexpr bool is_split(int s) { return s == LBM_F16M || s == LBM_BF16M; }
template <> struct Stor<LBM_F16M> : Stor<LBM_F16S> {};
template <> struct Stor<LBM_BF16M> : Stor<LBM_BF16S> {};

// Momentum J of a cell in a moment-split lattice: one 8-byte word per cell,
// (J_x, J_y) in its first 32-bit half and (J_z, 0) in its second, each a
// 16-bit value of the format (rounded to nearest even). lo/hi give the value
// in the low/high 16 bits of a 32-bit half as float (exact).
template <int S> struct SplitJ;
template <> struct SplitJ<LBM_F16M> {
    static __device__ __forceinline__ unsigned pack(float a, float b) {
        union {
            unsigned u;
            __half2 h;
        } v;
        v.h = __floats2half2_rn(a, b);
        return v.u;
    }
    static __device__ __forceinline__ float lo(unsigned w) {
        return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu)));
    }
    static __device__ __forceinline__ float hi(unsigned w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }
};
template <> struct SplitJ<LBM_BF16M> {
    static __device__ __forceinline__ unsigned pack(float a, float b) {
        union {
            unsigned u;
            __nv_bfloat162 h;
        } v;
        v.h = __floats2bfloat162_rn(a, b);
        return v.u;
    }
    static __device__ __forceinline__ float lo(unsigned w) { return __uint_as_float(w << 16); }
    static __device__ __forceinline__ float hi(unsigned w) { return __uint_as_float(w & 0xffff0000u); }
};

// Two 32-bit words of a small array read every step (the push masks of a
// cell pair, 4 B a cell; a bounce-back link), loaded with an L2 evict-last
// policy: while the lattices stream through L2 every step, these arrays stay
// resident, so the loads that bounce-back waits on hit L2 (measured +2% on the
// walled channel in FP32, +1% in 16-bit storage).
__device__ __forceinline__ uint2 ld_resident2(const uint32_t *p) {
    unsigned long long pol;
    uint2 m;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    asm("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(m.x), "=r"(m.y) : "l"(p), "l"(pol));
    return m;
}

// Pairs of arithmetic-type values (force field, tape) at an even index.
__device__ __forceinline__ void ld2_real(const float *p, float &a, float &b) {
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void ld2_real(const double *p, double &a, double &b) {
    const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void st2_real(float *p, float a, float b) {
    __stcs(reinterpret_cast<float2 *>(p), make_float2(a, b));
}
__device__ __forceinline__ void st2_real(double *p, double a, double b) {
    __stcs(reinterpret_cast<double2 *>(p), make_double2(a, b));
}

// Bytes of one stored population value (a remainder, for the split formats).
inline size_t storage_bytes(lbm_storage s) { return s == LBM_F64 ? 8 : (s == LBM_F32 ? 4 : 2); }

// Element offset of the momentum words in a moment-split lattice: after the
// 19 remainder arrays, rounded up to a 16-byte boundary (8 elements).
LBM_HD long long split_j_offset(long long qs) { return (19 * qs + 7) / 8 * 8; }

// Bytes of one padded lattice of qs cells in storage s.
inline size_t lattice_bytes_of(lbm_storage s, long long qs) {
    if (is_split(s)) return (size_t)split_j_offset(qs) * 2 + (size_t)qs * 8;
    return (size_t)19 * (size_t)qs * storage_bytes(s);
}

// ---------------------------------------------------------------------------
// Geometry of the padded structure-of-arrays store: population i of cell
// (x, y, z) lives at base + i * qs + (z * ny + y) * pitch + x. Rows are padded
// to `pitch` elements so that each starts on a 128-byte boundary (Sec. 6,
// padding cells after each stripe); padding cells are never computed.
struct Geom {
    int nx, ny, nz, pitch;
    long long qs;  // nz * ny * pitch: elements per population array (< 2^31)
};

LBM_HD int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

LBM_HD int cell_index(const Geom &g, int x, int y, int z) { return (z * g.ny + y) * g.pitch + x; }

// Row-oriented launch: block (bx, by) = (x_block + nxb * y_group, z), threads
// (tx, ty); each thread owns one cell. Used by every per-cell kernel.
struct RowLaunch {
    int bx_threads, by_threads;  // block shape
    int nxb, nyb;                // x blocks per row, y groups
    int y0, z0, nyr, nzr;        // paired launch: the rows y0 .. y0 + nyr - 1 of planes z0 .. z0 + nzr - 1
    int W;                       // flat paired launch: pairs per row
};

inline RowLaunch row_launch(const Geom &g) {
    RowLaunch L;
    int w = 32;  // power of two in [32, 256] covering a row, so blocks hold 256 threads
    while (w < g.nx && w < 256) w *= 2;
    L.bx_threads = w;
    L.by_threads = 256 / w;
    L.nxb = (g.nx + w - 1) / w;
    L.nyb = (g.ny + L.by_threads - 1) / L.by_threads;
    L.y0 = L.z0 = 0;
    L.nyr = g.ny;
    L.nzr = g.nz;
    L.W = 0;
    return L;
}

// Paired launch of the step kernels: each thread owns the two x-adjacent cells
// x0 = 2 (xb * bx_threads + tx) and x0 + 1 of row (y, z). A row's pairs are
// split into the fewest blocks of at most 256 threads, each a multiple of 32
// wide, so few lanes idle when nx is not a power of two; rows stack in y up to
// 256 threads per block.
// The paired launch covers whole rows of the box y0 <= y < y0 + nyr,
// z0 <= z < z0 + nzr (the whole lattice by default; the step kernels get the
// smallest box holding every fluid cell, since rows of solid cells need no
// update).
inline RowLaunch pair_launch(const Geom &g, int y0 = 0, int nyr = -1, int z0 = 0, int nzr = -1) {
    RowLaunch L;
    const int half = (g.nx + 1) / 2;
    L.nxb = (half + 255) / 256;
    const int per = (half + L.nxb - 1) / L.nxb;
    L.bx_threads = (per + 31) / 32 * 32;
    L.by_threads = 256 / L.bx_threads;
    L.y0 = y0;
    L.z0 = z0;
    L.nyr = nyr < 0 ? g.ny : nyr;
    L.nzr = nzr < 0 ? g.nz : nzr;
    L.nyb = (L.nyr + L.by_threads - 1) / L.by_threads;
    L.W = (g.nx + 1) / 2;
    return L;
}

// Whole rows per block leave the last warp of a row partly idle when the row's
// pairs are not a multiple of 32 (n = 200: 28 of 128 threads). The flat launch
// gives consecutive threads consecutive pairs of a plane's rows, across row
// ends (with rows padded only to pairs, consecutive rows are adjacent in
// memory, so such warps still load contiguous runs): blocks of threads x 1
// (256 unless a kernel is compiled for another block size).
inline bool rows_leave_lanes_idle(const RowLaunch &P) { return P.nxb * P.bx_threads != P.W; }
inline RowLaunch flat_launch(const RowLaunch &rows, int threads = 256) {
    RowLaunch L = rows;
    L.nxb = 1;
    L.bx_threads = threads;
    L.by_threads = 1;
    L.nyb = (int)(((long long)L.nyr * L.W + threads - 1) / threads);
    return L;
}

template <bool FLAT = false>
LBM_HD bool pair_cell(const Geom &g, const RowLaunch &P, int bdx, int bdy, int bx, int bz, int tx, int ty, int &x0,
                      int &y, int &z) {
    if (FLAT) {  // thread k of the plane takes pair k of the box rows
        const int k = bx * (bdx * bdy) + ty * bdx + tx;
        const int r = k / P.W;
        x0 = 2 * (k - r * P.W);
        y = P.y0 + r;
        z = P.z0 + bz;
        return r < P.nyr && z < P.z0 + P.nzr;
    }
    const int xb = bx % P.nxb;
    const int yg = bx / P.nxb;
    x0 = 2 * (xb * bdx + tx);
    y = P.y0 + yg * bdy + ty;
    z = P.z0 + bz;
    return x0 < g.nx && y < P.y0 + P.nyr && z < P.z0 + P.nzr;
}

// Push mask of a cell (precomputed on the host from the flags): bit j,
// 1 <= j <= 18, is set when the neighbour x + e_j is solid, so population j
// bounces back; SOLID_BIT is set on solid cells and on row padding.
constexpr uint32_t SOLID_BIT = 0x80000000u;
// Set in the push mask of a cell with a moving-wall neighbour.
constexpr uint32_t MOVING_BIT = 0x40000000u;

// Cell owned by thread (tx, ty) of block (bx, bz); false for threads past the edge.
LBM_HD bool row_cell(const Geom &g, int nxb, int bdx, int bdy, int bx, int bz, int tx, int ty,
                     int &x, int &y, int &z) {
    int xb = bx % nxb;
    int yg = bx / nxb;
    x = xb * bdx + tx;
    y = yg * bdy + ty;
    z = bz;
    return x < g.nx && y < g.ny && z < g.nz;
}

// Index of the cell (x + dx, y + dy, z + dz), periodic, |d| <= 1.
LBM_HD int neighbor_index(const Geom &g, int x, int y, int z, int dx, int dy, int dz) {
    return cell_index(g, wrap1(x + dx, g.nx), wrap1(y + dy, g.ny), wrap1(z + dz, g.nz));
}

// Cell that population i of cell (x, y, z) is pulled from: x - e_i.
LBM_HD int pull_src(const Geom &g, int x, int y, int z, int i) {
    return neighbor_index(g, x, y, z, -ex(i), -ey(i), -ez(i));
}

// Cell that population i of cell (x, y, z) streams to: x + e_i.
LBM_HD int push_dst(const Geom &g, int x, int y, int z, int i) {
    return neighbor_index(g, x, y, z, ex(i), ey(i), ez(i));
}

// Canonical (unpadded) index of cell (x, y, z).
LBM_HD long long canon_index(const Geom &g, int x, int y, int z) {
    return (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
}

// ---------------------------------------------------------------------------
// Collision of one cell in shifted form (Eq. 1, Qian equilibrium, Guo force):
//   rho - 1 = sum s_i,  j = sum s_i e_i,  u = (j + F/2) / rho
//   s*_i = s_i + omega (seq_i - s_i) + S_i,
//   seq_i = f_eq_i - w_i = w_i [(rho - 1) + rho (3 e.u + 9/2 (e.u)^2 - 3/2 u.u)]
//   S_i = (1 - omega/2) w_i [3 (e_i - u) + 9 (e_i.u) e_i] . F
// Opposite directions share the even part and flip the odd part.
// Correctly rounded 1/x (the same value as an IEEE division 1/x).
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }

template <class R> struct Mom {
    R rho1, rho, ux, uy, uz;
};

// incomp: the incompressible model of He & Luo, u = j + F/2 (the momentum of
// the reference density 1); otherwise u = (j + F/2)/rho.
template <class R>
__device__ __forceinline__ Mom<R> moments(const R s[Q], R Fx, R Fy, R Fz, bool incomp = false) {
    Mom<R> m;
    // rho - 1 summed over opposite pairs first: the odd (velocity) parts of
    // s_i and s_opp(i) cancel exactly before any rounding of the total
    R r = s[0];
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) r += s[pair_first(p)] + s[opp(pair_first(p))];
    // the association of moments2, so the two agree bit for bit
    R jx = (((s[1] - s[2]) + (s[7] - s[10])) + ((s[8] - s[9]) + (s[11] - s[14]))) + (s[12] - s[13]);
    R jy = (((s[3] - s[4]) + (s[7] - s[10])) + ((s[9] - s[8]) + (s[15] - s[18]))) + (s[16] - s[17]);
    R jz = (((s[5] - s[6]) + (s[11] - s[14])) + ((s[13] - s[12]) + (s[15] - s[18]))) + (s[17] - s[16]);
    m.rho1 = r;
    m.rho = R(1) + r;
    if (incomp) {
        m.ux = jx + R(0.5) * Fx;
        m.uy = jy + R(0.5) * Fy;
        m.uz = jz + R(0.5) * Fz;
        return m;
    }
    R inv = rcp_rn(m.rho);
    m.ux = (jx + R(0.5) * Fx) * inv;
    m.uy = (jy + R(0.5) * Fy) * inv;
    m.uz = (jz + R(0.5) * Fz) * inv;
    return m;
}

// ---------------------------------------------------------------------------
// Arithmetic on the two cells of a pair at once: lane x is cell x0, lane y is
// cell x0 + 1. FP32 uses the packed FP32x2 instructions of sm_100 and later
// (one instruction for both cells, each lane rounded as its scalar operation
// would be); FP64 works lane by lane. vsub is b * (-1) + a fused: the product
// is exact, so it rounds once, like a - b.
template <class R> struct Pair2;
template <> struct Pair2<float> {
    typedef float2 V;
};
template <> struct Pair2<double> {
    typedef double2 V;
};

__device__ __forceinline__ float2 vsplat(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 vrcp(float2 a) { return make_float2(rcp_rn(a.x), rcp_rn(a.y)); }

__device__ __forceinline__ double2 vsplat(double a) { return make_double2(a, a); }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) {
    return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
}
__device__ __forceinline__ double2 vmul(double2 a, double2 b) {
    return make_double2(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y));
}
__device__ __forceinline__ double2 vfma(double2 a, double2 b, double2 c) {
    return make_double2(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 vsub(double2 a, double2 b) {
    return make_double2(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y));
}
__device__ __forceinline__ double2 vrcp(double2 a) { return make_double2(rcp_rn(a.x), rcp_rn(a.y)); }

// e_i . v for i = pair_first(p): the first non-zero component of e_i is +1,
// the second 0 or +-1, so this is one component or one sum/difference.
template <class V> __device__ __forceinline__ V edot_first(int i, V vx, V vy, V vz) {
    if (ex(i)) {
        if (ey(i)) return ey(i) > 0 ? vadd(vx, vy) : vsub(vx, vy);
        if (ez(i)) return ez(i) > 0 ? vadd(vx, vz) : vsub(vx, vz);
        return vx;
    }
    if (ey(i)) {
        if (ez(i)) return ez(i) > 0 ? vadd(vy, vz) : vsub(vy, vz);
        return vy;
    }
    return vz;
}

template <class R> struct Mom2 {
    typedef typename Pair2<R>::V V;
    V rho1, rho, ux, uy, uz;
    V jx, jy, jz;  // j + F/2 (= rho u, or u itself in the incompressible model)
    V inv;         // 1/rho (1 in the incompressible model): u = j' inv
};

// Moments of both cells: rho - 1 summed over opposite pairs first (the odd
// parts of s_i and s_opp(i) cancel exactly before the total is rounded),
// u = (j + F/2) / rho, or u = j + F/2 for the incompressible model.
template <class R, bool FORCE>
__device__ __forceinline__ Mom2<R> moments2(const typename Pair2<R>::V s[Q], typename Pair2<R>::V Fx,
                                            typename Pair2<R>::V Fy, typename Pair2<R>::V Fz, bool incomp) {
    typedef typename Pair2<R>::V V;
    Mom2<R> m;
    V r = s[0];
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) r = vadd(r, vadd(s[pair_first(p)], s[opp(pair_first(p))]));
    V jx = vadd(vadd(vadd(vsub(s[1], s[2]), vsub(s[7], s[10])), vadd(vsub(s[8], s[9]), vsub(s[11], s[14]))),
                vsub(s[12], s[13]));
    V jy = vadd(vadd(vadd(vsub(s[3], s[4]), vsub(s[7], s[10])), vadd(vsub(s[9], s[8]), vsub(s[15], s[18]))),
                vsub(s[16], s[17]));
    V jz = vadd(vadd(vadd(vsub(s[5], s[6]), vsub(s[11], s[14])), vadd(vsub(s[13], s[12]), vsub(s[15], s[18]))),
                vsub(s[17], s[16]));
    if (FORCE) {
        const V h = vsplat(R(0.5));
        jx = vfma(h, Fx, jx);
        jy = vfma(h, Fy, jy);
        jz = vfma(h, Fz, jz);
    }
    m.rho1 = r;
    m.rho = vadd(vsplat(R(1)), r);
    m.jx = jx;
    m.jy = jy;
    m.jz = jz;
    if (incomp) {
        m.ux = jx;
        m.uy = jy;
        m.uz = jz;
        m.inv = vsplat(R(1));
        return m;
    }
    const V inv = vrcp(m.rho);
    m.inv = inv;
    m.ux = vmul(jx, inv);
    m.uy = vmul(jy, inv);
    m.uz = vmul(jz, inv);
    return m;
}

// Guo source with c = 1 - omega/2 (or c' = c/omega = tau - 1/2 for the form of
// collide2 that adds S/omega to the equilibrium): rest S_0 = -c u.F
// (3 w_0 = 1), and per opposite pair p (direction i = pair_first(p)):
//   even part  (e_i.u) A_p - 3 c w_p (u.F),   odd part  C_p,
//   A_p = 9 c w_p (e_i.F),  C_p = 3 c w_p (e_i.F).
// A and C depend only on F and tau: a uniform force passes them in precomputed.
template <class R> struct Guo2 {
    typedef typename Pair2<R>::V V;
    V A[NPAIR], C[NPAIR];
};

template <class R>
__device__ __forceinline__ Guo2<R> guo2(R cF, typename Pair2<R>::V Fx, typename Pair2<R>::V Fy,
                                        typename Pair2<R>::V Fz) {
    Guo2<R> t;
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) {
        const int i = pair_first(p);
        const R w = i <= 6 ? R(1.0 / 18.0) : R(1.0 / 36.0);
        const typename Pair2<R>::V eF = edot_first(i, Fx, Fy, Fz);
        t.A[p] = vmul(vsplat(R(9) * cF * w), eF);
        t.C[p] = vmul(vsplat(R(3) * cF * w), eF);
    }
    return t;
}

// 3 w_i of the odd part of the equilibrium, P_i = 3 w_i (e_i . j'): 1/6 for
// the axis pairs and 1/12 for the diagonal ones, rounded so that the momentum
// they carry, (2 K_AXIS + 8 K_DIAG) j', is j' with no rounding (the nearest
// 1/6 and 1/12 give j' (1 + 3e-8) in FP32). A relative bias of that size in
// every cell's momentum, repeated every step of a slowly varying flow, adds
// up linearly over the steps.
template <class R> struct OddK;
template <> struct OddK<float> {
    static constexpr float AXIS = 0x1.555554p-3f, DIAG = 0x1.555556p-4f;
};
template <> struct OddK<double> {
    static constexpr double AXIS = 0x1.5555555555554p-3, DIAG = 0x1.5555555555556p-4;
};

// BGK relaxation (Eq. 1) with the Qian equilibrium and the Guo source, both
// cells of the pair, populations in shifted form. Per opposite pair
// (i, opp(i)), with weight w, e = e_i . u and t = 9/2 e^2 - 3/2 u.u, both forms
// below compute E and P, the even and odd parts of the equilibrium plus the
// source, and differ in how the relaxation is rounded.
//
// TFORM (FP32 storage): s_i <- T_i + (1 - omega)(s_i - T_i) with
// T_i = s_eq_i + S_i / omega, the same update as (1 - omega) s_i + omega s_eq_i
// + S_i. Near tau = 1/2 the two terms of the latter are about twice the result
// and of opposite sign; this form rounds terms of the size of s_i, so T's mass
// and momentum carry over. With j' = j + F/2 (= rho u) and e = (e_i . j')/rho:
//   T_i, T_opp(i) = E +- P,   E = a + b t [+ e A],   P = K (e_i . j') [+ C],
//   a = w rho1 [- 3 w c' u.F],   b = w rho,   K = 3 w (OddK),
// A, C and c' = tau - 1/2 those of the source over omega (guo2).
//
// Otherwise (FP64, 16-bit storage): s_i <- (1 - omega) s_i + E + P and
// s_opp(i) <- (1 - omega) s_opp(i) + E - P, with omega folded in:
//   E = a + b t [+ e A],   P = 3 b e [+ C],   a = omega w rho1 [- 3 w c u.F],
//   b = omega w rho,   c = 1 - omega/2,
// so without a force E +- P = a + b (t +- 3e).
//
// Bracketed terms only with a force. a and b are formed per weight class, the
// diagonal ones (w = 1/36) by halving the axis ones (w = 1/18), so only one
// class's factors are held at a time. The incompressible model (He & Luo)
// has the reference density 1 in place of rho in b, and j' = u.
template <class R, bool FORCE, bool TFORM>
__device__ __forceinline__ void collide2(typename Pair2<R>::V s[Q], const Mom2<R> &m, R omega, R cs,
                                         typename Pair2<R>::V Fx, typename Pair2<R>::V Fy,
                                         typename Pair2<R>::V Fz, const Guo2<R> &G, bool incomp) {
    typedef typename Pair2<R>::V V;
    const V rho_e = incomp ? vsplat(R(1)) : m.rho;
    const V omc = vsplat(R(1) - omega);
    const V nusq15 = vmul(vsplat(R(-1.5)), vfma(m.uz, m.uz, vfma(m.uy, m.uy, vmul(m.ux, m.ux))));
    // the factors of the equilibrium: w, or omega w with omega folded in
    const R k3 = TFORM ? R(1.0 / 3.0) : omega * R(1.0 / 3.0);
    const R k18 = TFORM ? R(1.0 / 18.0) : omega * R(1.0 / 18.0);
    const R cF = TFORM ? cs : R(1) - R(0.5) * omega;  // Guo factor (over omega for TFORM)
    V uF = vsplat(R(0));
    if (FORCE) uF = vfma(m.uz, Fz, vfma(m.uy, Fy, vmul(m.ux, Fx)));
    {  // rest population, w = 1/3 (3 w c = c)
        V a0 = vmul(vsplat(k3), m.rho1);
        if (FORCE) a0 = vfma(vsplat(-cF), uF, a0);
        const V T0 = vfma(vmul(vsplat(k3), rho_e), nusq15, a0);
        s[0] = TFORM ? vfma(omc, vsub(s[0], T0), T0) : vfma(omc, s[0], T0);
    }
    V a = vmul(vsplat(k18), m.rho1);
    if (FORCE) a = vfma(vsplat(R(-1.0 / 6.0) * cF), uF, a);
    V b = vmul(vsplat(k18), rho_e);
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) {
        const int i = pair_first(p), io = opp(i);
        if (p == 3) {  // first diagonal pair: w halves
            a = vmul(vsplat(R(0.5)), a);
            b = vmul(vsplat(R(0.5)), b);
        }
        if (TFORM) {
            const V ej = edot_first(i, m.jx, m.jy, m.jz);
            const V e = vmul(ej, m.inv);
            const V K = vsplat(p < 3 ? OddK<R>::AXIS : OddK<R>::DIAG);
            const V t = vfma(vsplat(R(4.5)), vmul(e, e), nusq15);
            V E = vfma(b, t, a);
            V P;
            if (FORCE) {
                E = vfma(e, G.A[p], E);
                P = vfma(K, ej, G.C[p]);
            } else {
                P = vmul(K, ej);
            }
            const V Ti = vadd(E, P), To = vsub(E, P);
            s[i] = vfma(omc, vsub(s[i], Ti), Ti);
            s[io] = vfma(omc, vsub(s[io], To), To);
        } else {
            const V e = edot_first(i, m.ux, m.uy, m.uz);
            const V t = vfma(vsplat(R(4.5)), vmul(e, e), nusq15);
            if (FORCE) {
                const V E = vfma(e, G.A[p], vfma(b, t, a));
                const V P = vfma(vmul(vsplat(R(3)), b), e, G.C[p]);
                s[i] = vfma(omc, s[i], vadd(E, P));
                s[io] = vfma(omc, s[io], vsub(E, P));
            } else {
                s[i] = vfma(omc, s[i], vfma(b, vfma(vsplat(R(3)), e, t), a));
                s[io] = vfma(omc, s[io], vfma(b, vfma(vsplat(R(-3)), e, t), a));
            }
        }
    }
}

}  // namespace lbm
