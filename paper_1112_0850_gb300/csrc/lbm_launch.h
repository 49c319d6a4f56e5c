// Host-side interface between the C-ABI layer (lbm_capi.cu) and the kernel
// translation units. Each storage format S is compiled in its own unit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_device.cuh"

namespace lbm {

// How the state f^n sits in the lattice the readers and writers are given:
//   LAYOUT_PULL     post-collision P^{n-1} at its cell; f^n = gather (two lattices)
//   LAYOUT_AA_NAT   AA pattern before an even step: slot i of cell x holds f^n_i(x)
//   LAYOUT_AA_SWAP  AA pattern before an odd step: slot opp(i) of x holds
//                   P^{n-1}_i(x); f^n = the pull gather with mirrored slots
enum { LAYOUT_PULL = 0, LAYOUT_AA_NAT = 1, LAYOUT_AA_SWAP = 2 };

// Everything a launch needs to know about a context, by value.
struct Dev {
    Geom g;
    RowLaunch L;           // one cell per thread
    RowLaunch P;           // two x-adjacent cells per thread (step kernels)
    RowLaunch PF;          // the same pairs in plane order (flat_launch), for the two-grid step
    bool flat_step;        // the two-grid step uses PF: whole rows would leave lanes idle
    const uint8_t *flags;  // padded [qs] (1 = solid, also on padding), or nullptr = all fluid
    const uint32_t *mask;  // padded [qs] push masks (SOLID_BIT, bounce bits), null iff flags is
    const void *Ffield;    // padded [3][qs] of R, or nullptr
    double F[3];           // uniform force (used when Ffield == nullptr)
    double gA[9], gC[9];   // Guo constants of the uniform force per opposite pair (see guo2)
    float gAf[9], gCf[9];  // the same, rounded to float
    float gAtf[9], gCtf[9];  // the same over omega, rounded to float (the FP32 form of collide2)
    bool has_moving;       // some cell is a moving wall (flag 2)
    bool moving_on;        // has_moving and the wall velocity is nonzero
    double wc[19];         // moving-wall term 6 w_i (e_i . u_w) added to a population bounced into direction i
    float wcf[19];         // the same, rounded to float
    const uint32_t *links; // bounce-back links (cell, solid neighbour) grouped by direction, or null
    int link_off[20];      // links of direction j: [link_off[j], link_off[j + 1]), j = 1..18
    int link_max;          // largest per-direction count
    bool force_on;         // Ffield != nullptr or F != 0
    double omega;          // 1 / tau
    double cs;             // tau - 1/2: the Guo factor 1 - omega/2 over omega
    float omega_f, cs_f;   // the same, and F, rounded to float on the host: a conversion from
    float F_f[3];          // double in every thread costs the narrow FP64 pipe (28% busy in the FP32 step)
    unsigned *status;      // device status word
    cudaStream_t stream;
    long long n_cells;     // nx * ny * nz
    int layout;            // LAYOUT_* of the lattice passed to readers and writers
    bool incomp;           // incompressible equilibrium (He & Luo) instead of Qian's
    bool row_staging;      // use the TMA row-staged step kernel where it applies
    int num_sms;           // multiprocessors of the device (grid of persistent kernels)
    long long jo;          // moment-split formats: element offset of the momentum words in a lattice
    int zrev;              // step kernels: take the planes in descending order (alternates by step)
};

// omega, tau - 1/2 and the uniform force in the arithmetic type R.
template <class R> struct DevR;
template <> struct DevR<float> {
    static __device__ __forceinline__ float omega(const Dev &d) { return d.omega_f; }
    static __device__ __forceinline__ float cs(const Dev &d) { return d.cs_f; }
    static __device__ __forceinline__ float F(const Dev &d, int a) { return d.F_f[a]; }
};
template <> struct DevR<double> {
    static __device__ __forceinline__ double omega(const Dev &d) { return d.omega; }
    static __device__ __forceinline__ double cs(const Dev &d) { return d.cs; }
    static __device__ __forceinline__ double F(const Dev &d, int a) { return d.F[a]; }
};

// Bounce-back form per storage format (see k_step), the measured fastest on
// the walled channel: FP64 load side, FP32 mask-guided reload, 16-bit link
// kernel (BB_NANS, NaN marks with a rho-gated fix-up, is kept as the
// measured alternative). The moment-split formats take the mask-guided
// reload: a bounced value is rebuilt from the cell's own momentum, which a
// copy into a solid slot could not carry.
enum { BB_LOAD = 0, BB_LINKS = 1, BB_NANS = 2, BB_MFIX = 3 };
__host__ __device__ constexpr int bounce_mode(int s) {
    return s == LBM_F64 ? BB_LOAD : ((s == LBM_F32 || is_split(s)) ? BB_MFIX : BB_LINKS);
}
// The form in which a solid cell's slot holds the value bounced into it, so
// the gather needs no flags (links).
__host__ __device__ constexpr bool bounce_in_solid(int s) { return bounce_mode(s) == BB_LINKS; }

// The collision's rounding form per storage format (collide2): FP32 relaxes
// about T = s_eq + S/omega with the momentum-exact odd part, which keeps
// rounding from biasing mass and momentum step after step; FP64 (bias at the
// 1e-16 level, ALU-bound) and 16-bit storage (error set by the storage
// rounding) keep the cheaper omega-scaled form.
__host__ __device__ constexpr bool relax_about_t(int s) { return s == LBM_F32; }

// Links each k_bounce block copies at most (256 threads x 4), and the most
// blocks per direction its grid has (gridDim.y): the link form's limit.
constexpr int BOUNCE_LINKS_PER_BLOCK = 1024;
constexpr long long BOUNCE_MAX_LINKS = 65535LL * BOUNCE_LINKS_PER_BLOCK;

constexpr int RED_BLOCKS = 152 * 8;  // fixed grid of the reduction: deterministic order
constexpr int RED_THREADS = 256;

template <int S> struct Ops {
    // One fused stream-collide step: dst = C(G(src)); tape (nullable) gets
    // (rho, ux, uy, uz) of the pre-collision state, padded [4][qs] of R.
    static cudaError_t step(const Dev &d, const void *src, void *dst, void *tape);
    // Mark the solid cells of lat for the NaN-mark form of bounce-back and the
    // AA pattern (no-op otherwise).
    static cudaError_t fill_solid(const Dev &d, void *lat);
    // lat = P^{-1} such that gathering it gives f_eq(rho0, u0); rho0 nullable.
    static cudaError_t init_eq(const Dev &d, void *lat, const void *rho0, const void *u0);
    // Canonical shifted state of format fmt <-> lattice (gather / inverse gather).
    static cudaError_t get_state(const Dev &d, const void *lat, void *dst, int fmt);
    static cudaError_t set_state(const Dev &d, void *lat, const void *src, int fmt);
    static cudaError_t macros(const Dev &d, const void *lat, void *rho, void *u);
    // The link bounce of a step alone (link form with flags; no-op otherwise):
    // the solid slots of dst the next step gathers.
    static cudaError_t bounce(const Dev &d, void *dst);
    // Totals over the fluid cells of planes z0 <= z < z1. partials: RED_BLOCKS * 4
    // doubles of scratch; out: 4 doubles (device).
    static cudaError_t reduce(const Dev &d, const void *lat, int z0, int z1, double *partials, double *out);
    // One step (as step, no tape) that also sums the totals of reduce for its
    // pre-collision state into out (4 doubles, device); partials: 4 doubles per
    // block of the step grid.
    static cudaError_t step_reduce(const Dev &d, const void *src, void *dst, double *partials, double *out);
    // lambda^T from dL/du, dL/drho at the current state; grad_F += explicit term.
    static cudaError_t adj_seed(const Dev &d, const void *lat, const void *dL_du,
                                const void *dL_drho, void *lam, void *grad_F);
};

// The AA-pattern update (one lattice, in place); every solid slot holds NaN.
template <int S> struct AaOps {
    // One step on lattice A: the local (even) step if odd == 0, which takes
    // the natural layout to the swapped one, else the neighbour (odd) step,
    // which takes it back. tape as in Ops<S>::step.
    static cudaError_t step(const Dev &d, void *A, int odd, void *tape);
    // The same step, with the mass/momentum totals of the state it starts from
    // summed by its blocks (partials: 4 doubles per block of the launch) and
    // finished into out[4] (device), as Ops<S>::step_reduce.
    static cudaError_t step_reduce(const Dev &d, void *A, int odd, double *partials, double *out);
};

// Set-up: push masks of every padded cell from the padded flags (device).
cudaError_t build_push_mask(const Geom &g, const uint8_t *flags, uint32_t *mask, cudaStream_t st);
// z-slab halo copy between plane z of the lattice and a packed buffer of the
// five populations with e_z = dir (lbm_halo.cu); unpack writes fluid cells only.
cudaError_t launch_halo(const Geom &g, void *lat, int elem_bytes, void *buf, int z, int dir, bool unpack,
                        const uint8_t *flags, int num_sms, cudaStream_t s);

// Adjoint kernels that only depend on the arithmetic type R (double or float).
template <class R> struct AdjOps {
    static cudaError_t step(const Dev &d, const void *lam_in, void *lam_out, const void *tape_k,
                            void *grad_F);
    static cudaError_t init_grad(const Dev &d, const void *lam, const void *rho0, const void *u0,
                                 void *grad_u0, void *grad_rho0);
};

}  // namespace lbm
