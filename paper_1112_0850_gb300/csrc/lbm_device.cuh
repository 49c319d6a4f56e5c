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
};

template <> struct Stor<LBM_F16S> {
    typedef __half T;
    typedef float R;
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
        __stcs(reinterpret_cast<unsigned *>(p), v.u);
    }
};

template <> struct Stor<LBM_BF16S> {
    typedef __nv_bfloat16 T;
    typedef float R;
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
        __stcs(reinterpret_cast<unsigned *>(p), v.u);
    }
};

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

inline size_t storage_bytes(lbm_storage s) { return s == LBM_F64 ? 8 : (s == LBM_F32 ? 4 : 2); }

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
};

inline RowLaunch row_launch(const Geom &g) {
    RowLaunch L;
    int w = 32;  // power of two in [32, 256] covering a row, so blocks hold 256 threads
    while (w < g.nx && w < 256) w *= 2;
    L.bx_threads = w;
    L.by_threads = 256 / w;
    L.nxb = (g.nx + w - 1) / w;
    L.nyb = (g.ny + L.by_threads - 1) / L.by_threads;
    return L;
}

// Paired launch of the step kernels: each thread owns the two x-adjacent cells
// x0 = 2 (xb * bx_threads + tx) and x0 + 1 of row (y, z). A row's pairs are
// split into the fewest blocks of at most 256 threads, each a multiple of 32
// wide, so few lanes idle when nx is not a power of two; rows stack in y up to
// 256 threads per block.
inline RowLaunch pair_launch(const Geom &g) {
    RowLaunch L;
    const int half = (g.nx + 1) / 2;
    L.nxb = (half + 255) / 256;
    const int per = (half + L.nxb - 1) / L.nxb;
    L.bx_threads = (per + 31) / 32 * 32;
    L.by_threads = 256 / L.bx_threads;
    L.nyb = (g.ny + L.by_threads - 1) / L.by_threads;
    return L;
}

LBM_HD bool pair_cell(const Geom &g, int nxb, int bdx, int bdy, int bx, int bz, int tx, int ty, int &x0, int &y,
                      int &z) {
    const int xb = bx % nxb;
    const int yg = bx / nxb;
    x0 = 2 * (xb * bdx + tx);
    y = yg * bdy + ty;
    z = bz;
    return x0 < g.nx && y < g.ny && z < g.nz;
}

// Push mask of a cell (precomputed on the host from the flags): bit j,
// 1 <= j <= 18, is set when the neighbour x + e_j is solid, so population j
// bounces back; SOLID_BIT is set on solid cells and on row padding.
constexpr uint32_t SOLID_BIT = 0x80000000u;

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
template <class R> struct Mom {
    R rho1, rho, ux, uy, uz;
};

template <class R>
__device__ __forceinline__ Mom<R> moments(const R s[Q], R Fx, R Fy, R Fz) {
    Mom<R> m;
    // rho - 1 summed over opposite pairs first: the odd (velocity) parts of
    // s_i and s_opp(i) cancel exactly before any rounding of the total
    R r = s[0];
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) r += s[pair_first(p)] + s[opp(pair_first(p))];
    R jx = (s[1] - s[2]) + (s[7] - s[10]) + (s[8] - s[9]) + (s[11] - s[14]) + (s[12] - s[13]);
    R jy = (s[3] - s[4]) + (s[7] - s[10]) + (s[9] - s[8]) + (s[15] - s[18]) + (s[16] - s[17]);
    R jz = (s[5] - s[6]) + (s[11] - s[14]) + (s[13] - s[12]) + (s[15] - s[18]) + (s[17] - s[16]);
    m.rho1 = r;
    m.rho = R(1) + r;
    R inv = R(1) / m.rho;
    m.ux = (jx + R(0.5) * Fx) * inv;
    m.uy = (jy + R(0.5) * Fy) * inv;
    m.uz = (jz + R(0.5) * Fz) * inv;
    return m;
}

// Guo source of one cell with c = 1 - omega/2: rest S_0 = -c uF (3 w_0 = 1),
// and per opposite pair p (direction i = pair_first(p)):
//   even part  (e_i.u) A_p - 3 c w_p (u.F),   odd part  C_p,
//   A_p = 9 c w_p (e_i.F),  C_p = 3 c w_p (e_i.F).
// A and C depend only on F and tau: a uniform force passes them in precomputed.
template <class R> struct Guo {
    R A[NPAIR], C[NPAIR];
};

template <class R>
__device__ __forceinline__ Guo<R> guo_terms(R omega, R Fx, R Fy, R Fz) {
    Guo<R> t;
    const R cF = R(1) - R(0.5) * omega;
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) {
        const int i = pair_first(p);
        const R w = i <= 6 ? R(1.0 / 18.0) : R(1.0 / 36.0);
        const R eF = R(ex(i)) * Fx + R(ey(i)) * Fy + R(ez(i)) * Fz;
        t.A[p] = R(9) * cF * w * eF;
        t.C[p] = R(3) * cF * w * eF;
    }
    return t;
}

template <class R, bool FORCE>
__device__ __forceinline__ void collide(R s[Q], const Mom<R> &m, R omega, R Fx, R Fy, R Fz, const Guo<R> &G) {
    const R usq15 = R(1.5) * (m.ux * m.ux + m.uy * m.uy + m.uz * m.uz);
    const R cF = R(1) - R(0.5) * omega;
    const R uF = FORCE ? (m.ux * Fx + m.uy * Fy + m.uz * Fz) : R(0);
    {
        const R w = R(1.0 / 3.0);
        R seq = w * (m.rho1 - m.rho * usq15);
        R src = FORCE ? -cF * uF : R(0);
        s[0] = s[0] + omega * (seq - s[0]) + src;
    }
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) {
        const int i = pair_first(p), o = opp(i);
        const R w = i <= 6 ? R(1.0 / 18.0) : R(1.0 / 36.0);
        const R eu = R(ex(i)) * m.ux + R(ey(i)) * m.uy + R(ez(i)) * m.uz;
        const R even = w * (m.rho1 + m.rho * (R(4.5) * eu * eu - usq15));
        const R odd = w * R(3) * m.rho * eu;
        R fe = R(0), fo = R(0);
        if (FORCE) {
            fe = eu * G.A[p] - (R(3) * w) * cF * uF;
            fo = G.C[p];
        }
        const R a = s[i], b = s[o];
        s[i] = a + omega * (even + odd - a) + (fe + fo);
        s[o] = b + omega * (even - odd - b) + (fe - fo);
    }
}

}  // namespace lbm
