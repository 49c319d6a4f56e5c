// Host-side interface between the C-ABI layer (lbm_capi.cu) and the kernel
// translation units. Each storage format S is compiled in its own unit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_device.cuh"

namespace lbm {

// Everything a launch needs to know about a context, by value.
struct Dev {
    Geom g;
    RowLaunch L;           // one cell per thread
    RowLaunch P;           // two x-adjacent cells per thread (step kernels)
    const uint8_t *flags;  // padded [qs] (1 = solid, also on padding), or nullptr = all fluid
    const uint32_t *mask;  // padded [qs] push masks (SOLID_BIT, bounce bits), null iff flags is
    const void *Ffield;    // padded [3][qs] of R, or nullptr
    double F[3];           // uniform force (used when Ffield == nullptr)
    double gA[9], gC[9];   // Guo constants of the uniform force per opposite pair (see collide)
    float gAf[9], gCf[9];  // the same, rounded to float
    const uint32_t *links; // bounce-back links (cell, solid neighbour) grouped by direction, or null
    int link_off[20];      // links of direction j: [link_off[j], link_off[j + 1]), j = 1..18
    int link_max;          // largest per-direction count
    bool force_on;         // Ffield != nullptr or F != 0
    double omega;          // 1 / tau
    unsigned *status;      // device status word
    cudaStream_t stream;
    long long n_cells;     // nx * ny * nz
};

constexpr int RED_BLOCKS = 152 * 8;  // fixed grid of the reduction: deterministic order
constexpr int RED_THREADS = 256;

template <int S> struct Ops {
    // One fused stream-collide step: dst = C(G(src)); tape (nullable) gets
    // (rho, ux, uy, uz) of the pre-collision state, padded [4][qs] of R.
    static cudaError_t step(const Dev &d, const void *src, void *dst, void *tape);
    // lat = P^{-1} such that gathering it gives f_eq(rho0, u0); rho0 nullable.
    static cudaError_t init_eq(const Dev &d, void *lat, const void *rho0, const void *u0);
    // Canonical shifted state of format fmt <-> lattice (gather / inverse gather).
    static cudaError_t get_state(const Dev &d, const void *lat, void *dst, int fmt);
    static cudaError_t set_state(const Dev &d, void *lat, const void *src, int fmt);
    static cudaError_t macros(const Dev &d, const void *lat, void *rho, void *u);
    // partials: RED_BLOCKS * 4 doubles of scratch; out: 4 doubles (device).
    static cudaError_t reduce(const Dev &d, const void *lat, double *partials, double *out);
    // lambda^T from dL/du, dL/drho at the current state; grad_F += explicit term.
    static cudaError_t adj_seed(const Dev &d, const void *lat, const void *dL_du,
                                const void *dL_drho, void *lam, void *grad_F);
};

// Adjoint kernels that only depend on the arithmetic type R (double or float).
template <class R> struct AdjOps {
    static cudaError_t step(const Dev &d, const void *lam_in, void *lam_out, const void *tape_k,
                            void *grad_F);
    static cudaError_t init_grad(const Dev &d, const void *lam, const void *rho0, const void *u0,
                                 void *grad_u0, void *grad_rho0);
};

}  // namespace lbm
