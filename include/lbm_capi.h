/*
 * lbm_capi.h: C interface of the GB300 D3Q19 BGK lattice Boltzmann library.
 *
 * The library advances the D3Q19 lattice Boltzmann equation with the BGK
 * collision operator (Habich et al., "Performance engineering for the lattice
 * Boltzmann method on GPGPUs", Sec. 2, Eq. 1), fusing the stream and collide
 * steps into one pass over two lattices (Sec. 2 and Sec. 6, "stream-collide"
 * with two grids), with bounce-back at cells flagged as obstacles (Sec. 2,
 * the Ziegler rule, folded into streaming) and a body force. The equilibrium
 * is the D3Q19 one of Qian et al. cited in Sec. 2; the body force is the
 * Guo, Zheng & Shi (2002) scheme, u = (j + F/2)/rho; bounce-back is the
 * halfway rule. The paper gives neither the force nor the bounce-back
 * variant; these are this library's readings.
 *
 * Conventions shared by every call:
 *   - Lattice of nx * ny * nz cells, all three axes periodic; walls are cells
 *     flagged solid. Canonical arrays are C-ordered [.. ][nz][ny][nx] (x
 *     fastest); N = nx * ny * nz.
 *   - Velocity set (19 directions, fixed order): rest; +x, -x, +y, -y, +z, -z;
 *     then (+1,+1,0), (+1,-1,0), (-1,+1,0), (-1,-1,0), (+1,0,+1), (+1,0,-1),
 *     (-1,0,+1), (-1,0,-1), (0,+1,+1), (0,+1,-1), (0,-1,+1), (0,-1,-1).
 *     Weights 1/3, 1/18 (axis), 1/36 (diagonal). lbm_lattice_table() returns it.
 *   - "real" is double when the context stores LBM_F64 and float otherwise:
 *     every canonical input and output array (density, velocity, force
 *     field, tape, adjoint gradients) has that element type.
 *   - Population state is exchanged as shifted deviations s_i = f_i - w_i,
 *     canonical layout [19][nz][ny][nx], in any of the four storage formats.
 *   - Pointers to canonical arrays may be device pointers or host pointers
 *     (pageable or pinned); the library tells them apart with
 *     cudaPointerGetAttributes. A call that reads a host array copies it in
 *     before returning; a call that writes a host array synchronizes the
 *     context's stream and the data is valid when it returns. Device arrays
 *     are read and written asynchronously on the context's stream.
 *   - The caller owns every array it passes; the context owns the lattices,
 *     its copies of flags and force field, the adjoint lattices and scratch.
 *   - Every call returns an lbm_status; no C++ exception crosses this
 *     interface. On error, lbm_last_error() describes the failure.
 *   - Kernel-side failures (a non-finite or non-positive density) set bits of
 *     a device status word which lbm_status_word() reads; they never trap.
 *     The calls that synchronize the context's stream on their own
 *     (lbm_synchronize, lbm_reduce, lbm_reduce_planes) return
 *     LBM_ERR_DIVERGED while the divergence bit is set; lbm_init_equilibrium
 *     and lbm_set_state clear the word, as they start a new run.
 */
#ifndef LBM_CAPI_H
#define LBM_CAPI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_Q 19

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,         /* invalid argument (size, tau, pointer, format) */
    LBM_ERR_OOM = 2,         /* device allocation failed or size would not fit */
    LBM_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    LBM_ERR_STATE = 4,       /* call out of order (e.g. adjoint step before seed) */
    LBM_ERR_DIVERGED = 5,    /* a kernel saw a non-finite or non-positive density: returned by
                                the calls that synchronize (lbm_synchronize, lbm_reduce,
                                lbm_reduce_planes) when the status word's divergence bit is
                                set; the results those calls return are still written */
                             /* (6 is not used) */
    LBM_ERR_UNSUPPORTED = 7  /* combination the library does not support */
} lbm_status;

/* Population storage formats. S = shifted: the stored value is f_i - w_i
 * (density deviation around rest, rho0 = 1); collision arithmetic is FP64 for
 * LBM_F64 and FP32 for the others. Narrow formats round to nearest even.
 *
 * M = moment split (this library's format; the paper stores SP or DP only,
 * Sec. 7): each cell keeps, for the 19 post-collision values P_i it holds,
 * their momentum J = sum_i P_i e_i and the remainders
 * g_i = (P_i - w_i) - 3 w_i (e_i . J), every one of them a 16-bit value (J
 * rounded first, and used rounded in g). A reader rebuilds
 * P_i = w_i + 3 w_i (e_i . J) + g_i in FP32, so a value is off by the rounding
 * of its remainder only, not of the whole deviation: the remainder is what the
 * linear equilibrium part leaves over (quadratic and non-equilibrium parts),
 * an order of magnitude or more smaller in flows at low Mach number. Per cell
 * and lattice: 19 remainders plus J in an 8-byte word (three values and an
 * unused one), 46 bytes, so 92 B per lattice update. The M formats run the
 * two-grid pull update only (no LBM_PATTERN_AA, no row staging, no halo
 * copies: those return LBM_ERR_UNSUPPORTED). Their canonical state arrays
 * (lbm_get_state, lbm_set_state) hold plain shifted deviations in the 16-bit
 * element type of the format. */
typedef enum {
    LBM_F64 = 0,   /* double, 304 B per lattice update  */
    LBM_F32 = 1,   /* float,  152 B per lattice update  */
    LBM_F16S = 2,  /* IEEE binary16, 76 B per lattice update */
    LBM_BF16S = 3, /* bfloat16,      76 B per lattice update */
    LBM_F16M = 4,  /* IEEE binary16 moment split, 92 B per lattice update */
    LBM_BF16M = 5  /* bfloat16 moment split,      92 B per lattice update */
} lbm_storage;

/* Bits of the device status word (bit 0x2 is not used). Kernels set them and
 * never trap; lbm_status_word() reads and clears them, and the synchronizing
 * calls report the divergence bit as LBM_ERR_DIVERGED. */
#define LBM_STATUS_DIVERGED 0x1u /* some fluid cell had rho <= 0 or non-finite rho */
#define LBM_STATUS_TIMEOUT  0x4u /* a kernel gave up waiting (about 1 s) for its asynchronous copies */

/* Streaming pattern: how the fused update moves populations through memory. */
typedef enum {
    LBM_PATTERN_PULL = 0, /* two lattices (Sec. 2, Sec. 6): each step gathers from the
                             neighbours in one lattice and stores at the cell in the other */
    LBM_PATTERN_AA = 1    /* one lattice updated in place, alternating a local step and a
                             neighbour step (the AA pattern of Bailey et al., 2009): the
                             same bytes per update, half the population memory */
} lbm_pattern;

/* Equilibrium of the collision (Sec. 2 cites Qian et al.; the paper calls its
 * solver incompressible and leaves the 1/rho out of its velocity moment). */
typedef enum {
    LBM_MODEL_QIAN = 0,           /* f_eq = w rho [1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u], u = (j + F/2)/rho */
    LBM_MODEL_INCOMPRESSIBLE = 1  /* He & Luo (1997): f_eq = w [rho + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u],
                                     u = j + F/2 (the momentum of the reference density 1) */
} lbm_model;

typedef struct {
    lbm_storage storage; /* default LBM_F32 */
    void *cuda_stream;   /* cudaStream_t used for every launch and copy; NULL = default stream */
    int row_align;       /* bytes each padded row starts on: 0 (default) = rows padded only
                            to a whole pair of cells (the kernels move pairs); otherwise a
                            power of two >= 2 elements of the storage format, e.g. 128 for
                            the paper's padding (Sec. 6), which measured 4-8% slower on GB300
                            for row lengths that are not multiples of it */
    lbm_pattern pattern; /* default LBM_PATTERN_PULL */
    lbm_model model;     /* default LBM_MODEL_QIAN; applies to every call (step, macros,
                            totals, init, adjoint) */
    int stage_rows;      /* 1: the two-grid step stages its source rows in shared memory with
                            TMA bulk copies where the rows allow it (FP32 and 16-bit storage,
                            rows a multiple of 16 bytes); 0 (default): it loads them directly,
                            which measured faster on walled lattices. Same bits either way. */
} lbm_options;

typedef struct {
    int nx, ny, nz;
    int pitch;                  /* padded row length in elements: nx rounded up to a whole pair
                                   of cells, or to lbm_options.row_align bytes when set */
    lbm_storage storage;
    int real_size;              /* bytes of "real": 8 (LBM_F64) or 4 */
    double tau;
    int64_t n_cells;            /* nx * ny * nz */
    int64_t n_fluid;            /* cells with flag 0 */
    size_t lattice_bytes;       /* bytes of one padded population lattice (19 arrays) */
    size_t tape_bytes_per_step; /* bytes lbm_step_record writes per step */
    int64_t steps_done;         /* time steps since the last init or set_state */
    lbm_pattern pattern;        /* streaming pattern (one lattice for LBM_PATTERN_AA, else two) */
    lbm_model model;            /* equilibrium */
} lbm_info;

/* Fill *opt with defaults (LBM_F32, default stream, rows padded only to a
 * pair of cells (row_align 0), LBM_PATTERN_PULL, LBM_MODEL_QIAN, no row
 * staging). */
lbm_status lbm_options_default(lbm_options *opt);

/* Create a context for an nx * ny * nz periodic lattice (Sec. 2: the uniform
 * grid of lattice nodes, two lattices for the stream-collide update, Sec. 6).
 *   tau   relaxation time of Eq. 1; must exceed 0.5 (viscosity (tau - 1/2)/3).
 *   flags nullable (= all fluid); uint8 [nz][ny][nx], 0 = fluid, 2 = wall
 *         moving with the velocity set by lbm_set_wall_velocity (the lid of
 *         the paper's lid-driven cavity, Sec. 7), any other nonzero value =
 *         solid at rest (obstacle, bounce-back per Sec. 2); host or device; copied.
 *   force nullable (= zero); host array of 3 doubles: uniform body-force
 *         density in lattice units.
 *   opt   nullable (= defaults).
 * Sizes: 1 <= nx, ny; 1 <= nz <= 65535; padded cells nz * ny * pitch < 2^31.
 * Returns LBM_ERR_OOM if the lattices (two; one with LBM_PATTERN_AA) do not
 * fit in free device memory, and LBM_ERR_UNSUPPORTED for 16-bit shifted
 * storage when one direction has more than 65535 * 1024 bounce-back links
 * (the link kernel's grid). The state is the rest state after creation. */
lbm_status lbm_create(lbm_ctx **out, int nx, int ny, int nz, double tau, const uint8_t *flags,
                      const double force[3], const lbm_options *opt);

/* Free everything the context owns. NULL-safe. Synchronizes its stream. */
void lbm_destroy(lbm_ctx *ctx);

lbm_status lbm_get_info(const lbm_ctx *ctx, lbm_info *info);

/* Replace the uniform body force (host array of 3 doubles; NULL = zero). */
lbm_status lbm_set_uniform_force(lbm_ctx *ctx, const double force[3]);

/* Velocity u_w of the cells flagged 2 (host array of 3 doubles; NULL = rest).
 * A population bounced back from such a wall gains 6 w_i (e_i . u_w), the
 * halfway bounce-back rule for a moving wall (Ladd) with the wall density
 * taken as the reference density 1. Applies from the next step on. */
lbm_status lbm_set_wall_velocity(lbm_ctx *ctx, const double u_w[3]);

/* Install a per-cell force field F: real [3][nz][ny][nx], host or device,
 * copied into the context. NULL removes the field (back to the uniform force). */
lbm_status lbm_set_force_field(lbm_ctx *ctx, const void *F);

/* Initialise the populations to the equilibrium f_eq(rho0, u0) at every fluid
 * cell (Sec. 2; equilibrium of Qian et al.).
 *   rho nullable (= 1): real [nz][ny][nx];  u: real [3][nz][ny][nx].
 * Resets steps_done to 0. */
lbm_status lbm_init_equilibrium(lbm_ctx *ctx, const void *rho, const void *u);

/* Enqueue n >= 0 fused stream-collide time steps (Sec. 2 steps 1-3 with
 * bounce-back; Sec. 6 pull-style update over two grids, or the in-place AA
 * update when the context was created with LBM_PATTERN_AA; both give the same
 * f^n sequence, and every other call sees the same state). Asynchronous. Whole
 * blocks of 32 steps, and a remaining 2 to 31, replay CUDA graphs of that many
 * steps (one launch each), captured on first use or by lbm_step_prepare and
 * dropped when the force or wall velocity changes; a single step is launched
 * on its own. A call that captures a graph should not be made while the
 * context's stream is being captured. */
lbm_status lbm_step(lbm_ctx *ctx, int n);

/* Capture the graphs that lbm_step(ctx, n) replays, from either starting
 * lattice, without running a step (host work only; nothing is enqueued), so
 * that a later lbm_step(n) does not capture them while the GPU waits. n >= 0;
 * a graph that cannot be captured leaves lbm_step launching step by step. */
lbm_status lbm_step_prepare(lbm_ctx *ctx, int n);

/* lbm_step(ctx, n) between two CUDA events recorded on the context's stream;
 * waits for the second and writes the device time between them to *ms
 * (milliseconds). Synchronizes, and like lbm_synchronize returns
 * LBM_ERR_DIVERGED if the status word's divergence bit is set. The time
 * includes any idle gap while the host enqueues, so a call that captures a
 * step graph (the first with a given n after create or a force change, unless
 * lbm_step_prepare(n) came first) reads longer than the ones after it. ms must
 * not be NULL (LBM_ERR_ARG). */
lbm_status lbm_step_timed(lbm_ctx *ctx, int n, float *ms);

/* Macroscopic fields of the current state (Sec. 2 step 1): rho = sum f_i,
 * u = (sum f_i e_i + F/2) / rho. rho nullable: real [nz][ny][nx];
 * u: real [3][nz][ny][nx]. Solid cells read 0. */
lbm_status lbm_macros(lbm_ctx *ctx, void *rho, void *u);

/* Totals over fluid cells of the current state, accumulated in FP64 in a
 * fixed order (deterministic): out = {sum rho, sum rho u_x, sum rho u_y,
 * sum rho u_z} with rho u = j + F/2. out is a host array; synchronizes.
 * Returns LBM_ERR_DIVERGED (out still written) if the status word's
 * divergence bit is set. */
lbm_status lbm_reduce(lbm_ctx *ctx, double out[4]);

/* Largest lattice, in cells (nx * ny * nz), that lbm_reduce_state_noalloc
 * accepts: its fixed scratch array holds one partial sum per 16384 cells. */
#define LBM_NOALLOC_MAX_CELLS 268435456LL

/* The totals of lbm_reduce, computed from a state the caller passes in,
 * without allocating any device memory. The paper has no counterpart; this
 * exists for callers that cannot call cudaMalloc where they need the totals:
 * code embedded in a framework whose caching allocator already holds the free
 * device memory, and pipelines that cannot afford cudaMalloc's implicit
 * device-wide synchronization between their launches.
 *   state   device array, shifted populations s_i = f_i - w_i in format fmt,
 *           canonical [19][nz][ny][nx] (as lbm_get_state writes it).
 *   flags   nullable (= all fluid): device uint8 [nz][ny][nx], nonzero = solid.
 *   force   nullable (= zero): host array of 3 doubles, the uniform body force
 *           that enters rho u = j + F/2.
 *   out     device array of 4 doubles: {sum rho, sum rho u_x, sum rho u_y,
 *           sum rho u_z} over fluid cells, accumulated in FP64 in a fixed order.
 *   cuda_stream  cudaStream_t to launch on (NULL = default stream).
 * Scratch: a file-scope device array of 512 KiB, which every GPU that loads
 * the library keeps until the process exits; each call overwrites the slots it
 * uses, so nothing has to be cleared. All calls share that one array: calls
 * whose kernels can overlap on the GPU (different streams, or different host
 * threads without ordering) race and may return wrong totals. Every call made
 * outside a stream capture looks up the array's device address
 * (cudaGetSymbolAddress with the calling thread's current device), so a
 * device reset in between leaves nothing stale; a call made while cuda_stream
 * is being captured reuses the address of the last call outside a capture on
 * that device, so make one call on each device before any stream capture (and
 * one again after a cudaDeviceReset).
 * Asynchronous on cuda_stream. Returns LBM_ERR_ARG for a null state or out, a
 * bad format or size, and when nx * ny * nz exceeds LBM_NOALLOC_MAX_CELLS;
 * LBM_ERR_CUDA if the address look-up or a launch fails. It calls no
 * cudaMalloc, cudaFree or allocating library routine. */
lbm_status lbm_reduce_state_noalloc(const void *state, lbm_storage fmt, int nx, int ny, int nz,
                                    const uint8_t *flags, const double force[3], double *out,
                                    void *cuda_stream);

/* The totals of lbm_reduce for the current state, then n >= 1 steps, with
 * the totals summed inside the first step from the moments it forms anyway
 * (no pass over the lattice of their own: the reduction fused into the step
 * as an epilogue). out: 4 doubles, host (the call synchronizes) or device
 * (asynchronous). The same totals as lbm_reduce up to the order of the FP64
 * sums; deterministic. Both streaming patterns fuse the sum into their
 * first step. */
lbm_status lbm_step_reduce(lbm_ctx *ctx, int n, double *out);

/* Copy the current state out as shifted populations s_i = f_i - w_i in format
 * fmt, canonical [19][nz][ny][nx] (element type double / float / binary16 /
 * bfloat16). Solid cells read 0. Host or device destination. */
lbm_status lbm_get_state(lbm_ctx *ctx, void *dst, lbm_storage fmt);

/* Load a state written by lbm_get_state (any format; converted to the
 * context's storage with round-to-nearest-even). Solid-cell values ignored.
 * Resets steps_done to 0. Round trip in the context's own format is exact. */
lbm_status lbm_set_state(lbm_ctx *ctx, const void *src, lbm_storage fmt);

/* z-slab halo exchange, the one exchange per step when a lattice is split
 * along z into slabs (a domain decomposition over GPUs; Sec. 2's pull update
 * makes each step read only the nearest planes). A slab is a context of its
 * own whose planes 0 and nz - 1 are ghosts: copies of the neighbouring slabs'
 * boundary planes, with the flags (and force field) of those planes passed to
 * lbm_create. The interior plane 1 reads from ghost plane 0 only the five
 * populations with e_z = +1, and plane nz - 2 reads from plane nz - 1 only
 * the five with e_z = -1. Before each lbm_step(ctx, 1) of every slab:
 *   lbm_halo_pack(slab k, 1, b)   then lbm_halo_unpack(slab k + 1, 0, b)
 *   lbm_halo_pack(slab k, 0, b')  then lbm_halo_unpack(slab k - 1, 1, b')
 * and the interior planes then evolve bit for bit as the same planes of the
 * unsplit lattice. The readers (lbm_get_state, lbm_macros, lbm_reduce) gather
 * each cell's populations from its pull sources, which for the boundary
 * planes lie in the ghosts: exchange before reading a slab.
 *
 * lbm_halo_bytes: size of one packed buffer, 5 * ny * pitch elements of the
 * storage type (0 for an invalid context).
 * lbm_halo_pack: copies from the current state the five outgoing populations
 * of an interior boundary plane, side 0: plane 1, e_z = -1; side 1: plane
 * nz - 2, e_z = +1. Layout [5][ny][pitch], directions in increasing index
 * order (lbm_lattice_table), padding columns included.
 * lbm_halo_unpack: writes such a buffer into a ghost plane, side 0: plane 0
 * (the e_z = +1 populations packed by the slab below), side 1: plane nz - 1
 * (the e_z = -1 ones packed by the slab above), at fluid cells only: a solid
 * ghost cell's slots hold the bounce-back values of this slab's own step.
 * buf: host or device, owned by the caller (a host buffer is staged and the
 * call synchronizes). Returns LBM_ERR_ARG for a null buffer, side not 0 or 1,
 * or nz < 3; LBM_ERR_UNSUPPORTED with LBM_PATTERN_AA (its layout alternates
 * between steps). Asynchronous on cuda_stream for device buffers. */
size_t lbm_halo_bytes(const lbm_ctx *ctx);
lbm_status lbm_halo_pack(lbm_ctx *ctx, int side, void *buf);
lbm_status lbm_halo_unpack(lbm_ctx *ctx, int side, const void *buf);

/* The totals of lbm_reduce over the fluid cells of planes z0 <= z < z1 only
 * (0 <= z0 <= z1 <= nz; z0 == z1 gives zeros), in the same fixed FP64 order.
 * For a slab, the interior planes 1 .. nz - 2 read after an exchange: the
 * totals of all slabs then add up to those of the unsplit lattice (to the
 * order of the FP64 sums), the mass/momentum check of a split run, summed
 * over ranks with an all-reduce. out is a host array; synchronizes. Returns
 * LBM_ERR_ARG for a null out or planes outside that range, LBM_ERR_DIVERGED
 * (out still written) if the status word's divergence bit is set. */
lbm_status lbm_reduce_planes(lbm_ctx *ctx, int z0, int z1, double out[4]);

/* The halo exchange of the adjoint of a z-slab run. The reverse step
 * (lbm_adjoint_step) reads lambda_i at x + e_i, so the adjoint populations
 * cross each face the other way: interior plane 1 reads from ghost plane 0
 * the five with e_z = -1, and plane nz - 2 reads from plane nz - 1 the five
 * with e_z = +1. Record the forward one step at a time (lbm_step_record with
 * n = 1, the forward exchange before each), exchange the forward halos before
 * lbm_adjoint_seed, and before each lbm_adjoint_step(ctx, 1, tape_k, ...):
 *   lbm_adjoint_halo_pack(slab k, 0, b)  then lbm_adjoint_halo_unpack(slab k - 1, 1, b)
 *   lbm_adjoint_halo_pack(slab k, 1, b') then lbm_adjoint_halo_unpack(slab k + 1, 0, b')
 * and lambda on the interior planes (and the gradients from it) is then bit
 * for bit that of the unsplit lattice.
 *
 * lbm_adjoint_halo_bytes: size of one packed buffer, 5 * ny * pitch elements
 * of real (0 for an invalid context).
 * lbm_adjoint_halo_pack: copies from the current adjoint lattice the five
 * outgoing populations of a boundary plane, side 0: plane 1, e_z = +1; side
 * 1: plane nz - 2, e_z = -1. Layout [5][ny][pitch], directions in increasing
 * index order.
 * lbm_adjoint_halo_unpack: writes such a buffer into a ghost plane, side 0:
 * plane 0 (the e_z = -1 populations packed by the slab below), side 1: plane
 * nz - 1 (the e_z = +1 ones packed by the slab above), at fluid cells only
 * (the reverse step reads a solid neighbour's link from the cell itself).
 * buf: host or device, owned by the caller, as for lbm_halo_pack. Returns
 * LBM_ERR_STATE before lbm_adjoint_seed, otherwise the errors of
 * lbm_halo_pack. Asynchronous on cuda_stream for device buffers. */
size_t lbm_adjoint_halo_bytes(const lbm_ctx *ctx);
lbm_status lbm_adjoint_halo_pack(lbm_ctx *ctx, int side, void *buf);
lbm_status lbm_adjoint_halo_unpack(lbm_ctx *ctx, int side, const void *buf);

/* One step of the cells of planes z0 <= z < z1 only (0 <= z0 <= z1 <= nz),
 * read from the current state and written to the next lattice; the current
 * state stays current until a call with last != 0, which runs what follows
 * the whole step (the link bounce in 16-bit storage with flags) and makes the
 * next lattice current. A step taken as several such calls, every plane in
 * exactly one of them and the last with last != 0, equals lbm_step(ctx, 1)
 * bit for bit. It lets a slab update its interior planes 2 .. nz - 3, which
 * read no ghost plane, while its halo exchange runs on another stream (see
 * lbm_set_stream), and then planes 1 and nz - 2; a slab's ghost planes need
 * no update, as the next exchange refills what its interior reads there.
 * out nullable: 4 doubles that receive the totals of lbm_reduce_planes(z0,
 * z1) for the current state, summed inside this call's step as
 * lbm_step_reduce does (the same totals up to the order of the FP64 sums):
 * host (the call synchronizes) or device (asynchronous). Returns LBM_ERR_ARG
 * for planes outside that range, LBM_ERR_UNSUPPORTED with LBM_PATTERN_AA.
 * Asynchronous on cuda_stream unless out is a host array. */
lbm_status lbm_step_planes(lbm_ctx *ctx, int z0, int z1, int last, double *out);

/* Make cuda_stream (a cudaStream_t; NULL = default stream) the stream every
 * later call of this context enqueues on. Work already enqueued on the
 * previous stream is not waited for: order the two streams with events. */
lbm_status lbm_set_stream(lbm_ctx *ctx, void *cuda_stream);

/* As lbm_step, and also record, for each of the n steps k, the moments the
 * adjoint needs: (rho, u_x, u_y, u_z) of the pre-collision state at step k,
 * u including the F/2 shift. tape: device array of n * tape_bytes_per_step
 * bytes (opaque layout). */
lbm_status lbm_step_record(lbm_ctx *ctx, int n, void *tape);

/* Start a discrete adjoint (not in the paper: the transpose of the update
 * above) at the current state f^T for a loss L(rho_T, u_T):
 *   dL_du   real [3][nz][ny][nx] (required), dL_drho nullable real [nz][ny][nx].
 *   grad_F  nullable real [3][nz][ny][nx], device: receives dL/dF from the
 *           explicit F/2 in u_T (accumulated: +=).
 * Sets the adjoint populations lambda^T = dL/df^T. */
lbm_status lbm_adjoint_seed(lbm_ctx *ctx, const void *dL_du, const void *dL_drho, void *grad_F);

/* n reverse steps of the adjoint: lambda^k = J_k^T G^T lambda^(k+1) for
 * k = n-1 .. 0, where G is the streaming/bounce-back permutation and J_k the
 * BGK + Guo collision Jacobian at the moments recorded in tape (written by
 * lbm_step_record for the same n steps from the matching state).
 * grad_F nullable, device real [3][nz][ny][nx]: dL/dF(x) is accumulated (+=). */
lbm_status lbm_adjoint_step(lbm_ctx *ctx, int n, const void *tape, void *grad_F);

/* Gradients with respect to the initial fields of lbm_init_equilibrium:
 * grad_u0 [3][nz][ny][nx] and grad_rho0 [nz][ny][nx] (nullable), both real,
 * device or host, overwritten, from lambda^0 and the same rho0 (nullable =
 * 1) and u0 that were passed to lbm_init_equilibrium. */
lbm_status lbm_adjoint_init_grad(lbm_ctx *ctx, const void *rho0, const void *u0, void *grad_u0,
                                 void *grad_rho0);

/* Read (and clear, if clear != 0) the device status word; synchronizes. */
lbm_status lbm_status_word(lbm_ctx *ctx, uint32_t *out, int clear);

/* Block the host until all work enqueued on the context's stream is done.
 * Returns LBM_ERR_DIVERGED if the status word's divergence bit is set (the
 * bit stays set until lbm_status_word clears it or a new initial state is
 * loaded), so a caller that synchronizes learns of a diverged run there. */
lbm_status lbm_synchronize(lbm_ctx *ctx);

/* Message of the last failed call on this context (empty if none). */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Name of a status code. */
const char *lbm_status_string(lbm_status s);

/* The velocity set the kernels were compiled with: e[19*3] (row i = e_i),
 * w[19], opp[19] (index of -e_i). Returns 19. Needs no GPU. */
int lbm_lattice_table(int *e, double *w, int *opp);

/* Host-side check of the index arithmetic of every kernel launch the library
 * makes for an nx * ny * nz lattice in format fmt with rows aligned to
 * row_align bytes (as in lbm_options; 0 = pairs only): walks every thread of each
 * launch configuration on the CPU and verifies that every address it forms
 * lies inside its buffer (two-grid and AA step kernels, reverse step,
 * per-cell kernels, reduction, halo copies). Returns the number of violations (0 = all in
 * bounds), or -1 for invalid sizes or alignment. Needs no GPU. */
int64_t lbm_check_launch_indices(int nx, int ny, int nz, lbm_storage fmt, int row_align);

#ifdef __cplusplus
}
#endif

#endif /* LBM_CAPI_H */
