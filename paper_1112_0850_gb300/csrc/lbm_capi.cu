// C-ABI of the D3Q19 BGK library (declared in include/lbm_capi.h): context
// management, argument checks, host/device pointer handling, and dispatch of
// each call to the kernels of its storage format.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbm_launch.h"

using namespace lbm;

// Steps per captured block graph (even, so a replay ends on the lattice it
// began on); a call's remaining 2 .. GRAPH_STEPS - 1 steps replay a graph of
// their own count.
constexpr int GRAPH_STEPS = 32;

struct lbm_ctx {
    Geom g;
    RowLaunch L;
    lbm_storage storage;
    double tau;
    double F[3];
    double u_wall[3];   // velocity of the cells flagged 2
    bool has_moving;    // some cell is flagged 2
    cudaStream_t stream;
    int device;
    lbm_pattern pattern;
    lbm_model model;
    bool stage_rows;
    int num_sms;
    void *lat[2];       // pull: lat[cur] holds the latest post-collision populations;
                        // AA: lat[0] is the one lattice, lat[1] is null
    int cur;            // pull: current lattice; AA: 0 = natural layout, 1 = swapped
    int box[4];         // y0, rows, z0, planes: the smallest y/z box holding every fluid cell
    uint8_t *flags_d;   // padded [qs], 1 = solid (padding included), or null
    uint32_t *mask_d;   // padded [qs] push masks for the step kernels, or null
    uint32_t *links_d;  // bounce-back links (fluid cell, solid cell), grouped by direction
    int link_off[20];
    int link_max;
    void *Ffield_d;     // padded [3][qs] of the arithmetic type, or null
    void *lam[2];       // adjoint lattices (allocated on first seed)
    int lcur;
    bool lam_valid;
    double *red_partials;  // RED_BLOCKS * 4 doubles
    double *red_out;       // 4 doubles
    double *step_partials; // 4 doubles per block of the step grid (fused reduction), on first use
    size_t step_partials_n;
    unsigned *status_d;
    void *staging;         // device buffer for host-side arrays
    size_t staging_bytes;
    int64_t n_fluid;
    int64_t steps_done;
    // CUDA graphs of n consecutive steps (graph[from][n], 2 <= n <= GRAPH_STEPS),
    // one per starting lattice (lat[0] or lat[1] as source), captured on first
    // use or by lbm_step_prepare; dropped when the step parameters change
    cudaGraphExec_t graph[2][GRAPH_STEPS + 1];
    bool graph_failed;
    std::string err;
};

namespace {

const char *status_names[] = {"LBM_OK",        "LBM_ERR_ARG",      "LBM_ERR_OOM",     "LBM_ERR_CUDA",
                              "LBM_ERR_STATE", "LBM_ERR_DIVERGED", "unknown status", "LBM_ERR_UNSUPPORTED"};

lbm_status fail(lbm_ctx *ctx, lbm_status s, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return s;
}

lbm_status cuda_fail(lbm_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// The status word v, read after a synchronization: LBM_ERR_DIVERGED while
// its divergence bit is set.
lbm_status diverged(lbm_ctx *ctx, unsigned v) {
    if (v & LBM_STATUS_DIVERGED) {
        char msg[160];
        snprintf(msg, sizeof msg,
                 "a fluid cell reached a non-finite or non-positive density (status word 0x%x); "
                 "lbm_status_word clears it", v);
        return fail(ctx, LBM_ERR_DIVERGED, msg);
    }
    return LBM_OK;
}

size_t real_size(lbm_storage s) { return s == LBM_F64 ? 8 : 4; }

bool valid_storage(int s) { return s >= LBM_F64 && s <= LBM_BF16M; }

// Elements per padded row so that each row starts on a row_align-byte
// boundary (0 = a whole pair of cells); -1 if row_align is not allowed.
int pitch_for(int nx, lbm_storage s, int row_align = 0) {
    const int eb = (int)storage_bytes(s);
    const int align = row_align ? row_align : 2 * eb;
    if (align < 2 * eb || (align & (align - 1)) || align > 4096) return -1;
    const int per = align / eb;
    return (nx + per - 1) / per * per;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

Dev make_dev(const lbm_ctx *ctx) {
    Dev d;
    d.g = ctx->g;
    d.L = ctx->L;
    d.P = pair_launch(ctx->g, ctx->box[0], ctx->box[1], ctx->box[2], ctx->box[3]);
    d.PF = flat_launch(d.P);
    d.flat_step = rows_leave_lanes_idle(d.P);
    d.flags = ctx->flags_d;
    d.mask = ctx->mask_d;
    d.Ffield = ctx->Ffield_d;
    d.F[0] = ctx->F[0];
    d.F[1] = ctx->F[1];
    d.F[2] = ctx->F[2];
    d.force_on = ctx->Ffield_d != nullptr || ctx->F[0] != 0.0 || ctx->F[1] != 0.0 || ctx->F[2] != 0.0;
    d.omega = 1.0 / ctx->tau;
    d.cs = ctx->tau - 0.5;
    d.omega_f = (float)d.omega;
    d.cs_f = (float)d.cs;
    for (int a = 0; a < 3; ++a) d.F_f[a] = (float)d.F[a];
    const double cF = 1.0 - 0.5 * d.omega;
    for (int p = 0; p < NPAIR; ++p) {
        const int i = pair_first(p);
        const double eF = ex(i) * ctx->F[0] + ey(i) * ctx->F[1] + ez(i) * ctx->F[2];
        d.gA[p] = 9.0 * cF * weight(i) * eF;
        d.gC[p] = 3.0 * cF * weight(i) * eF;
        d.gAf[p] = (float)d.gA[p];
        d.gCf[p] = (float)d.gC[p];
        d.gAtf[p] = (float)(9.0 * d.cs * weight(i) * eF);
        d.gCtf[p] = (float)(3.0 * d.cs * weight(i) * eF);
    }
    d.has_moving = ctx->has_moving;
    d.moving_on = ctx->has_moving && (ctx->u_wall[0] != 0.0 || ctx->u_wall[1] != 0.0 || ctx->u_wall[2] != 0.0);
    for (int i = 0; i < Q; ++i) {
        d.wc[i] = 6.0 * weight(i) * (ex(i) * ctx->u_wall[0] + ey(i) * ctx->u_wall[1] + ez(i) * ctx->u_wall[2]);
        d.wcf[i] = (float)d.wc[i];
    }
    d.links = ctx->links_d;
    for (int j = 0; j < 20; ++j) d.link_off[j] = ctx->link_off[j];
    d.link_max = ctx->link_max;
    d.status = ctx->status_d;
    d.stream = ctx->stream;
    d.n_cells = (long long)ctx->g.nx * ctx->g.ny * ctx->g.nz;
    d.layout = ctx->pattern == LBM_PATTERN_AA ? (ctx->cur ? LAYOUT_AA_SWAP : LAYOUT_AA_NAT) : LAYOUT_PULL;
    d.incomp = ctx->model == LBM_MODEL_INCOMPRESSIBLE;
    d.row_staging = ctx->stage_rows;
    d.num_sms = ctx->num_sms;
    d.jo = split_j_offset(ctx->g.qs);
    d.zrev = 0;
    return d;
}

// Host-pointer handling: each canonical array is either used in place (device)
// or staged through ctx->staging. Inputs are copied in (and the stream
// synchronized, so the caller may reuse its host buffer on return); outputs
// are copied back and the stream synchronized by finish().
struct Staged {
    struct Item {
        const void *user;
        void *dev;
        size_t bytes;
        bool output;
        bool host;
    };
    lbm_ctx *ctx;
    std::vector<Item> items;
    explicit Staged(lbm_ctx *c) : ctx(c) {}

    int add(const void *user, size_t bytes, bool output) {
        Item it{user, const_cast<void *>(user), bytes, output, user && !is_device_ptr(user)};
        items.push_back(it);
        return (int)items.size() - 1;
    }
    void *dev(int k) { return items[k].dev; }

    lbm_status prepare() {
        size_t need = 0;
        for (auto &it : items)
            if (it.host) need += (it.bytes + 255) / 256 * 256;
        if (need > ctx->staging_bytes) {
            if (ctx->staging) cudaFree(ctx->staging);
            ctx->staging = nullptr;
            ctx->staging_bytes = 0;
            cudaError_t e = cudaMalloc(&ctx->staging, need);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(ctx, LBM_ERR_OOM, "cannot allocate staging buffer for host arrays");
            }
            ctx->staging_bytes = need;
        }
        size_t off = 0;
        bool copied_in = false;
        for (auto &it : items) {
            if (!it.host) continue;
            it.dev = static_cast<char *>(ctx->staging) + off;
            off += (it.bytes + 255) / 256 * 256;
            if (!it.output) {
                cudaError_t e = cudaMemcpyAsync(it.dev, it.user, it.bytes, cudaMemcpyHostToDevice, ctx->stream);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "copy of a host input");
                copied_in = true;
            }
        }
        if (copied_in) {
            cudaError_t e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "copy of a host input");
        }
        return LBM_OK;
    }

    lbm_status finish() {
        bool any = false;
        for (auto &it : items) {
            if (!it.host || !it.output) continue;
            cudaError_t e = cudaMemcpyAsync(const_cast<void *>(it.user), it.dev, it.bytes, cudaMemcpyDeviceToHost,
                                            ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "copy of a host output");
            any = true;
        }
        if (any) {
            cudaError_t e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "copy of a host output");
        }
        return LBM_OK;
    }
};

#define LBM_DISPATCH(ctx, call)                                             \
    ((ctx)->storage == LBM_F64     ? Ops<LBM_F64>::call                     \
     : (ctx)->storage == LBM_F32   ? Ops<LBM_F32>::call                     \
     : (ctx)->storage == LBM_F16S  ? Ops<LBM_F16S>::call                    \
     : (ctx)->storage == LBM_BF16S ? Ops<LBM_BF16S>::call                   \
     : (ctx)->storage == LBM_F16M  ? Ops<LBM_F16M>::call                    \
                                   : Ops<LBM_BF16M>::call)
#define LBM_AA_DISPATCH(ctx, call)                                          \
    ((ctx)->storage == LBM_F64    ? AaOps<LBM_F64>::call                    \
     : (ctx)->storage == LBM_F32  ? AaOps<LBM_F32>::call                    \
     : (ctx)->storage == LBM_F16S ? AaOps<LBM_F16S>::call                   \
                                  : AaOps<LBM_BF16S>::call)

// The lattice holding the state f^n (in the layout make_dev reports).
void *state_lat(const lbm_ctx *ctx) { return ctx->pattern == LBM_PATTERN_AA ? ctx->lat[0] : ctx->lat[ctx->cur]; }

// One step from parity / lattice c (pull: lat[c] -> lat[c ^ 1]; AA: the even
// step for c = 0, the odd one for c = 1).
// Steps alternate the order of their planes (ascending from lattice 0 or for
// an even AA step, descending otherwise): each step starts on the planes the
// step before it wrote last, which are still in L2.
cudaError_t step_from(const lbm_ctx *ctx, const Dev &d, int c, void *tape) {
    Dev dc = d;
    dc.zrev = c;
    if (ctx->pattern == LBM_PATTERN_AA) return LBM_AA_DISPATCH(ctx, step(dc, ctx->lat[0], c, tape));
    return LBM_DISPATCH(ctx, step(dc, ctx->lat[c], ctx->lat[c ^ 1], tape));
}

lbm_status check_ctx(const lbm_ctx *ctx) {
    if (!ctx) return LBM_ERR_ARG;
    cudaSetDevice(ctx->device);
    return LBM_OK;
}

void drop_graphs(lbm_ctx *ctx) {
    for (int k = 0; k < 2; ++k)
        for (int n = 0; n <= GRAPH_STEPS; ++n) {
            if (ctx->graph[k][n]) cudaGraphExecDestroy(ctx->graph[k][n]);
            ctx->graph[k][n] = nullptr;
        }
}

void free_ctx(lbm_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    drop_graphs(ctx);
    void *ptrs[] = {ctx->lat[0], ctx->lat[1],  ctx->flags_d,     ctx->mask_d,   ctx->links_d,        ctx->Ffield_d,
                    ctx->lam[0], ctx->lam[1], ctx->red_partials, ctx->red_out, ctx->step_partials, ctx->status_d,
                    ctx->staging};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete ctx;
}

}  // namespace

extern "C" {

lbm_status lbm_options_default(lbm_options *opt) {
    if (!opt) return LBM_ERR_ARG;
    opt->storage = LBM_F32;
    opt->cuda_stream = nullptr;
    opt->row_align = 0;
    opt->pattern = LBM_PATTERN_PULL;
    opt->model = LBM_MODEL_QIAN;
    opt->stage_rows = 0;
    return LBM_OK;
}

lbm_status lbm_create(lbm_ctx **out, int nx, int ny, int nz, double tau, const uint8_t *flags,
                      const double force[3], const lbm_options *opt) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    lbm_options o;
    lbm_options_default(&o);
    if (opt) o = *opt;
    if (nx < 1 || ny < 1 || nz < 1 || nz > 65535 || !(tau > 0.5) || !valid_storage(o.storage) ||
        (o.pattern != LBM_PATTERN_PULL && o.pattern != LBM_PATTERN_AA) ||
        (o.model != LBM_MODEL_QIAN && o.model != LBM_MODEL_INCOMPRESSIBLE))
        return LBM_ERR_ARG;
    const bool aa = o.pattern == LBM_PATTERN_AA;
    if (is_split(o.storage) && (aa || o.stage_rows)) return LBM_ERR_UNSUPPORTED;
    const int pitch = pitch_for(nx, o.storage, o.row_align);
    if (pitch < 0) return LBM_ERR_ARG;
    const long long qs = (long long)nz * ny * pitch;
    if (qs >= (1LL << 31)) return LBM_ERR_ARG;
    const long long N = (long long)nx * ny * nz;

    lbm_ctx *ctx = new lbm_ctx();
    memset(&ctx->g, 0, sizeof(ctx->g));
    ctx->g.nx = nx;
    ctx->g.ny = ny;
    ctx->g.nz = nz;
    ctx->g.pitch = pitch;
    ctx->g.qs = qs;
    ctx->L = row_launch(ctx->g);
    ctx->storage = o.storage;
    ctx->pattern = o.pattern;
    ctx->model = o.model;
    ctx->stage_rows = o.stage_rows != 0;
    ctx->num_sms = 1;
    ctx->tau = tau;
    for (int a = 0; a < 3; ++a) ctx->F[a] = force ? force[a] : 0.0;
    for (int a = 0; a < 3; ++a) ctx->u_wall[a] = 0.0;
    ctx->has_moving = false;
    ctx->box[0] = 0;
    ctx->box[1] = ny;
    ctx->box[2] = 0;
    ctx->box[3] = nz;
    ctx->stream = static_cast<cudaStream_t>(o.cuda_stream);
    ctx->lat[0] = ctx->lat[1] = nullptr;
    ctx->cur = 0;
    ctx->flags_d = nullptr;
    ctx->mask_d = nullptr;
    ctx->links_d = nullptr;
    for (int j = 0; j < 20; ++j) ctx->link_off[j] = 0;
    ctx->link_max = 0;
    ctx->Ffield_d = nullptr;
    ctx->lam[0] = ctx->lam[1] = nullptr;
    ctx->lcur = 0;
    ctx->lam_valid = false;
    ctx->red_partials = ctx->red_out = nullptr;
    ctx->step_partials = nullptr;
    ctx->step_partials_n = 0;
    ctx->status_d = nullptr;
    ctx->staging = nullptr;
    ctx->staging_bytes = 0;
    ctx->steps_done = 0;
    for (int k = 0; k < 2; ++k)
        for (int n = 0; n <= GRAPH_STEPS; ++n) ctx->graph[k][n] = nullptr;
    ctx->graph_failed = false;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) {
        delete ctx;
        return LBM_ERR_CUDA;
    }

    const size_t lat_bytes = lattice_bytes_of(o.storage, qs);
    size_t free_b = 0, total_b = 0;
    e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) {
        delete ctx;
        return LBM_ERR_CUDA;
    }
    // lattices, flags and push masks, reduction scratch
    const size_t need = (aa ? 1 : 2) * lat_bytes + (flags ? 5 * (size_t)qs : 0) +
                        ((size_t)RED_BLOCKS * 4 + 8) * sizeof(double);
    if (need > free_b) {
        delete ctx;
        return LBM_ERR_OOM;
    }

    // Flags: padded copy (padding marked solid) and the fluid-cell count.
    std::vector<uint8_t> hflags;
    int64_t n_fluid = N;
    if (flags) {
        std::vector<uint8_t> canon;
        const uint8_t *hf = flags;
        if (is_device_ptr(flags)) {
            canon.resize((size_t)N);
            e = cudaMemcpy(canon.data(), flags, (size_t)N, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                delete ctx;
                return LBM_ERR_CUDA;
            }
            hf = canon.data();
        }
        hflags.assign((size_t)qs, 1);
        n_fluid = 0;
        long long ylo = ny, yhi = -1, zlo = nz, zhi = -1;  // box of the fluid cells
        for (long long z = 0; z < nz; ++z)
            for (long long y = 0; y < ny; ++y) {
                // one row, branch-free: 0 fluid, 2 moving wall, any other value solid (1)
                const uint8_t *src = hf + (size_t)(nx * (y + ny * z));
                uint8_t *dst = hflags.data() + (size_t)((z * ny + y) * pitch);
                long long fluid = 0;
                unsigned moving = 0;
                for (long long x = 0; x < nx; ++x) {
                    const uint8_t v = src[x];
                    const uint8_t f = (uint8_t)(v == 0 ? 0 : (v == 2 ? 2 : 1));
                    dst[x] = f;
                    fluid += f == 0;
                    moving |= f == 2;
                }
                if (moving) ctx->has_moving = true;
                if (!fluid) continue;
                n_fluid += fluid;
                if (y < ylo) ylo = y;
                if (y > yhi) yhi = y;
                if (z < zlo) zlo = z;
                if (z > zhi) zhi = z;
            }
        if (n_fluid > 0) {  // the step kernels update rows of this box only
            ctx->box[0] = (int)ylo;
            ctx->box[1] = (int)(yhi - ylo + 1);
            ctx->box[2] = (int)zlo;
            ctx->box[3] = (int)(zhi - zlo + 1);
        }
    }
    ctx->n_fluid = n_fluid;
    bool ok = cudaMalloc(&ctx->lat[0], lat_bytes) == cudaSuccess &&
              (aa || cudaMalloc(&ctx->lat[1], lat_bytes) == cudaSuccess) &&
              cudaMalloc((void **)&ctx->red_partials, (size_t)RED_BLOCKS * 4 * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void **)&ctx->red_out, 4 * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void **)&ctx->status_d, sizeof(unsigned)) == cudaSuccess;
    if (ok && flags) ok = cudaMalloc((void **)&ctx->flags_d, (size_t)qs) == cudaSuccess;
    if (ok && flags) ok = cudaMalloc((void **)&ctx->mask_d, (size_t)qs * sizeof(uint32_t)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_ctx(ctx);
        return LBM_ERR_OOM;
    }
    ok = cudaMemsetAsync(ctx->lat[0], 0, lat_bytes, ctx->stream) == cudaSuccess &&
         (aa || cudaMemsetAsync(ctx->lat[1], 0, lat_bytes, ctx->stream) == cudaSuccess) &&
         cudaMemsetAsync(ctx->status_d, 0, sizeof(unsigned), ctx->stream) == cudaSuccess;
    // (copies are ordered on the context's stream, ahead of the kernels that read them)
    if (ok && flags)
        ok = cudaMemcpyAsync(ctx->flags_d, hflags.data(), (size_t)qs, cudaMemcpyHostToDevice, ctx->stream) ==
             cudaSuccess;
    // push masks, built on the device from the padded flags
    if (ok && flags) ok = build_push_mask(ctx->g, ctx->flags_d, ctx->mask_d, ctx->stream) == cudaSuccess;
    if (ok && flags) {
        Dev d = make_dev(ctx);
        ok = LBM_DISPATCH(ctx, fill_solid(d, ctx->lat[0])) == cudaSuccess &&
             (aa || LBM_DISPATCH(ctx, fill_solid(d, ctx->lat[1])) == cudaSuccess);
    }
    // Bounce-back links of the separate-kernel form (16-bit storage): every
    // (fluid cell, solid neighbour x + e_j at rest), grouped by direction j,
    // cells in increasing order; read off the masks of the cells next to solids.
    if (ok && flags && !aa && bounce_mode(o.storage) == BB_LINKS) {
        std::vector<uint32_t> hmask((size_t)qs);
        ok = cudaMemcpyAsync(hmask.data(), ctx->mask_d, (size_t)qs * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                             ctx->stream) == cudaSuccess &&
             cudaStreamSynchronize(ctx->stream) == cudaSuccess;
        std::vector<std::vector<uint32_t>> per(Q);
        for (int z = 0; ok && z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const int c = cell_index(ctx->g, x, y, z);
                    const uint32_t m = hmask[(size_t)c];
                    if ((m & SOLID_BIT) || !m) continue;
                    for (int j = 1; j < Q; ++j)
                        if ((m >> j) & 1u) {
                            const int t = push_dst(ctx->g, x, y, z, j);
                            if (hflags[(size_t)t] == 2) continue;  // moving wall: written by the step
                            per[j].push_back((uint32_t)c);
                            per[j].push_back((uint32_t)t);
                        }
                }
        std::vector<uint32_t> hlinks;
        for (int j = 1; j < Q; ++j) {
            const int cnt = (int)(per[j].size() / 2);
            ctx->link_off[j + 1] = ctx->link_off[j] + cnt;
            if (cnt > ctx->link_max) ctx->link_max = cnt;
            hlinks.insert(hlinks.end(), per[j].begin(), per[j].end());
        }
        if ((long long)ctx->link_max > BOUNCE_MAX_LINKS) {  // more spans than k_bounce's grid holds
            free_ctx(ctx);
            return LBM_ERR_UNSUPPORTED;
        }
        if (ok && !hlinks.empty())
            ok = cudaMalloc((void **)&ctx->links_d, hlinks.size() * sizeof(uint32_t)) == cudaSuccess &&
                 cudaMemcpyAsync(ctx->links_d, hlinks.data(), hlinks.size() * sizeof(uint32_t),
                                 cudaMemcpyHostToDevice, ctx->stream) == cudaSuccess &&
                 cudaStreamSynchronize(ctx->stream) == cudaSuccess;
    }
    if (ok) ok = cudaStreamSynchronize(ctx->stream) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_ctx(ctx);
        return LBM_ERR_CUDA;
    }
    *out = ctx;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx *ctx) { free_ctx(ctx); }

lbm_status lbm_get_info(const lbm_ctx *ctx, lbm_info *info) {
    if (!ctx || !info) return LBM_ERR_ARG;
    info->nx = ctx->g.nx;
    info->ny = ctx->g.ny;
    info->nz = ctx->g.nz;
    info->pitch = ctx->g.pitch;
    info->storage = ctx->storage;
    info->real_size = (int)real_size(ctx->storage);
    info->tau = ctx->tau;
    info->n_cells = (int64_t)ctx->g.nx * ctx->g.ny * ctx->g.nz;
    info->n_fluid = ctx->n_fluid;
    info->lattice_bytes = lattice_bytes_of(ctx->storage, ctx->g.qs);
    info->tape_bytes_per_step = 4 * (size_t)ctx->g.qs * real_size(ctx->storage);
    info->steps_done = ctx->steps_done;
    info->pattern = ctx->pattern;
    info->model = ctx->model;
    return LBM_OK;
}

lbm_status lbm_set_uniform_force(lbm_ctx *ctx, const double force[3]) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    cudaStreamSynchronize(ctx->stream);
    drop_graphs(ctx);  // the force is a kernel argument baked into the graphs
    for (int a = 0; a < 3; ++a) ctx->F[a] = force ? force[a] : 0.0;
    return LBM_OK;
}

lbm_status lbm_set_wall_velocity(lbm_ctx *ctx, const double u_w[3]) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    cudaStreamSynchronize(ctx->stream);
    drop_graphs(ctx);  // the wall terms are kernel arguments baked into the graphs
    for (int a = 0; a < 3; ++a) ctx->u_wall[a] = u_w ? u_w[a] : 0.0;
    return LBM_OK;
}

lbm_status lbm_set_force_field(lbm_ctx *ctx, const void *F) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    if ((F != nullptr) != (ctx->Ffield_d != nullptr)) {  // the force mode is baked into the graphs
        cudaStreamSynchronize(ctx->stream);
        drop_graphs(ctx);
    }
    if (!F) {
        if (ctx->Ffield_d) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(ctx->Ffield_d);
        }
        ctx->Ffield_d = nullptr;
        return LBM_OK;
    }
    const size_t rs = real_size(ctx->storage);
    if (!ctx->Ffield_d) {
        cudaError_t e = cudaMalloc(&ctx->Ffield_d, 3 * (size_t)ctx->g.qs * rs);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->Ffield_d = nullptr;
            return fail(ctx, LBM_ERR_OOM, "cannot allocate the force field");
        }
        e = cudaMemsetAsync(ctx->Ffield_d, 0, 3 * (size_t)ctx->g.qs * rs, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "clear force field");
    }
    // canonical rows of nx reals -> padded rows of pitch reals
    cudaError_t e = cudaMemcpy2DAsync(ctx->Ffield_d, (size_t)ctx->g.pitch * rs, F, (size_t)ctx->g.nx * rs,
                                      (size_t)ctx->g.nx * rs, (size_t)3 * ctx->g.ny * ctx->g.nz, cudaMemcpyDefault,
                                      ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy of the force field");
    if (!is_device_ptr(F)) {
        e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "copy of the force field");
    }
    return LBM_OK;
}

lbm_status lbm_init_equilibrium(lbm_ctx *ctx, const void *rho, const void *u) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    if (!u) return fail(ctx, LBM_ERR_ARG, "u is required");
    const size_t N = (size_t)ctx->g.nx * ctx->g.ny * ctx->g.nz, rs = real_size(ctx->storage);
    Staged st(ctx);
    int ir = rho ? st.add(rho, N * rs, false) : -1;
    int iu = st.add(u, 3 * N * rs, false);
    lbm_status s = st.prepare();
    if (s) return s;
    if (ctx->pattern == LBM_PATTERN_AA) ctx->cur = 0;  // written in the natural layout
    Dev d = make_dev(ctx);
    cudaError_t e = LBM_DISPATCH(ctx, init_eq(d, state_lat(ctx), ir >= 0 ? st.dev(ir) : nullptr, st.dev(iu)));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "init_equilibrium launch");
    e = cudaMemsetAsync(ctx->status_d, 0, sizeof(unsigned), ctx->stream);  // a new run
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status word reset");
    ctx->steps_done = 0;
    ctx->lam_valid = false;
    return LBM_OK;
}

// Capture n steps starting from lattice `from` into ctx->graph[from][n] (on a
// private stream; the graph is then launched on the context's stream).
// Returns false, leaving no graph, if capture or instantiation fails.
static bool build_graph(lbm_ctx *ctx, int from, int n) {
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    Dev d = make_dev(ctx);
    d.stream = cs;
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    for (int k = 0; ok && k < n; ++k) {
        const int c = from ^ (k & 1);
        ok = step_from(ctx, d, c, nullptr) == cudaSuccess;
    }
    const bool ended = cudaStreamEndCapture(cs, &graph) == cudaSuccess;
    ok = ok && ended && graph && cudaGraphInstantiate(&ctx->graph[from][n], graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (!ok) {
        cudaGetLastError();
        ctx->graph[from][n] = nullptr;
    }
    return ok;
}

// The graph of n steps from lattice `from`, captured if missing; null if
// graphs failed on this context (the caller then launches step by step).
static cudaGraphExec_t graph_for(lbm_ctx *ctx, int from, int n) {
    if (ctx->graph_failed) return nullptr;
    if (!ctx->graph[from][n] && !build_graph(ctx, from, n)) ctx->graph_failed = true;
    return ctx->graph[from][n];
}

lbm_status lbm_step(lbm_ctx *ctx, int n) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    if (n < 0) return fail(ctx, LBM_ERR_ARG, "n must be >= 0");
    // whole blocks of GRAPH_STEPS steps, then a remainder of 2 or more, replay
    // captured graphs (one launch each); a single step, or every step where
    // graphs failed, is launched on its own
    while (n >= 2) {
        const int m = n >= GRAPH_STEPS ? GRAPH_STEPS : n;
        cudaGraphExec_t ge = graph_for(ctx, ctx->cur, m);
        if (!ge) break;
        cudaError_t e = cudaGraphLaunch(ge, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "stream-collide graph launch");
        n -= m;
        ctx->cur ^= m & 1;
        ctx->steps_done += m;
    }
    Dev d = make_dev(ctx);
    for (int k = 0; k < n; ++k) {
        cudaError_t e = step_from(ctx, d, ctx->cur, nullptr);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "stream-collide launch");
        ctx->cur ^= 1;
        ctx->steps_done++;
    }
    return LBM_OK;
}

lbm_status lbm_step_prepare(lbm_ctx *ctx, int n) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    if (n < 0) return fail(ctx, LBM_ERR_ARG, "n must be >= 0");
    const int r = n % GRAPH_STEPS;
    for (int from = 0; from < 2; ++from) {
        if (n >= GRAPH_STEPS) graph_for(ctx, from, GRAPH_STEPS);
        if (r >= 2) graph_for(ctx, from, r);
    }
    return LBM_OK;
}

lbm_status lbm_step_timed(lbm_ctx *ctx, int n, float *ms) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    if (!ms) return fail(ctx, LBM_ERR_ARG, "ms is required");
    if (n < 0) return fail(ctx, LBM_ERR_ARG, "n must be >= 0");
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], ctx->stream);
    lbm_status s = LBM_OK;
    if (e == cudaSuccess) {
        s = lbm_step(ctx, n);
        if (s == LBM_OK) {
            e = cudaEventRecord(ev[1], ctx->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(ms, ev[0], ev[1]);
        }
    }
    for (cudaEvent_t v : ev)
        if (v) cudaEventDestroy(v);
    if (s != LBM_OK) return s;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "timed steps");
    return lbm_synchronize(ctx);
}

lbm_status lbm_set_stream(lbm_ctx *ctx, void *cuda_stream) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    return LBM_OK;
}

lbm_status lbm_step_record(lbm_ctx *ctx, int n, void *tape) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    if (n < 0) return fail(ctx, LBM_ERR_ARG, "n must be >= 0");
    if (n > 0 && (!tape || !is_device_ptr(tape))) return fail(ctx, LBM_ERR_ARG, "tape must be a device array");
    const size_t per = 4 * (size_t)ctx->g.qs * real_size(ctx->storage);
    Dev d = make_dev(ctx);
    for (int k = 0; k < n; ++k) {
        void *tk = static_cast<char *>(tape) + per * (size_t)k;
        cudaError_t e = step_from(ctx, d, ctx->cur, tk);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "stream-collide (record) launch");
        ctx->cur ^= 1;
        ctx->steps_done++;
    }
    return LBM_OK;
}

lbm_status lbm_macros(lbm_ctx *ctx, void *rho, void *u) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    if (!u) return fail(ctx, LBM_ERR_ARG, "u is required");
    const size_t N = (size_t)ctx->g.nx * ctx->g.ny * ctx->g.nz, rs = real_size(ctx->storage);
    Staged st(ctx);
    int ir = rho ? st.add(rho, N * rs, true) : -1;
    int iu = st.add(u, 3 * N * rs, true);
    lbm_status s = st.prepare();
    if (s) return s;
    Dev d = make_dev(ctx);
    cudaError_t e = LBM_DISPATCH(ctx, macros(d, state_lat(ctx), ir >= 0 ? st.dev(ir) : nullptr, st.dev(iu)));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "macros launch");
    return st.finish();
}

lbm_status lbm_reduce_planes(lbm_ctx *ctx, int z0, int z1, double out[4]) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    if (!out) return fail(ctx, LBM_ERR_ARG, "out is required");
    if (z0 < 0 || z1 < z0 || z1 > ctx->g.nz) return fail(ctx, LBM_ERR_ARG, "planes must satisfy 0 <= z0 <= z1 <= nz");
    Dev d = make_dev(ctx);
    cudaError_t e = LBM_DISPATCH(ctx, reduce(d, state_lat(ctx), z0, z1, ctx->red_partials, ctx->red_out));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reduce launch");
    unsigned v = 0;
    e = cudaMemcpyAsync(out, ctx->red_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v, ctx->status_d, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reduce result copy");
    return diverged(ctx, v);
}

lbm_status lbm_reduce(lbm_ctx *ctx, double out[4]) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    return lbm_reduce_planes(ctx, 0, ctx->g.nz, out);
}

// Scratch of the fused step-reduce: one partial per block of either launch
// mapping of the whole step (a plane window's launch has fewer blocks).
static lbm_status ensure_step_partials(lbm_ctx *ctx, const Dev &d) {
    const size_t nb_rows = (size_t)d.P.nxb * d.P.nyb * d.P.nzr, nb_flat = (size_t)d.PF.nxb * d.PF.nyb * d.PF.nzr;
    const size_t nb = nb_rows > nb_flat ? nb_rows : nb_flat;
    if (ctx->step_partials_n >= nb) return LBM_OK;
    if (ctx->step_partials) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->step_partials);
    }
    ctx->step_partials = nullptr;
    ctx->step_partials_n = 0;
    cudaError_t e = cudaMalloc((void **)&ctx->step_partials, nb * 4 * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->step_partials = nullptr;
        return fail(ctx, LBM_ERR_OOM, "cannot allocate the fused-reduction partials");
    }
    ctx->step_partials_n = nb;
    return LBM_OK;
}

// The 4 totals in red_out to out: device (asynchronous) or host (synchronizes).
static lbm_status copy_totals(lbm_ctx *ctx, double *out) {
    const bool dev = is_device_ptr(out);
    cudaError_t e = cudaMemcpyAsync(out, ctx->red_out, 4 * sizeof(double),
                                    dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && !dev) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "totals copy");
    return LBM_OK;
}

lbm_status lbm_step_reduce(lbm_ctx *ctx, int n, double *out) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    if (n < 1 || !out) return fail(ctx, LBM_ERR_ARG, "n must be >= 1 and out is required");
    cudaError_t e;
    Dev d = make_dev(ctx);
    lbm_status s0 = ensure_step_partials(ctx, d);
    if (s0) return s0;
    if (ctx->pattern == LBM_PATTERN_AA)
        e = LBM_AA_DISPATCH(ctx, step_reduce(d, ctx->lat[0], ctx->cur, ctx->step_partials, ctx->red_out));
    else
        e = LBM_DISPATCH(ctx, step_reduce(d, ctx->lat[ctx->cur], ctx->lat[ctx->cur ^ 1], ctx->step_partials,
                                          ctx->red_out));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fused step-reduce launch");
    ctx->cur ^= 1;
    ctx->steps_done++;
    lbm_status s = lbm_step(ctx, n - 1);
    if (s) return s;
    return copy_totals(ctx, out);
}

// The rows of launch L that lie in planes z0 <= z < z1 (none: nzr = 0).
static void clip_planes(RowLaunch &L, int z0, int z1) {
    const int a = L.z0 > z0 ? L.z0 : z0, b = L.z0 + L.nzr < z1 ? L.z0 + L.nzr : z1;
    L.z0 = a;
    L.nzr = b > a ? b - a : 0;
}

lbm_status lbm_step_planes(lbm_ctx *ctx, int z0, int z1, int last, double *out) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    if (z0 < 0 || z1 < z0 || z1 > ctx->g.nz) return fail(ctx, LBM_ERR_ARG, "planes must satisfy 0 <= z0 <= z1 <= nz");
    if (ctx->pattern != LBM_PATTERN_PULL) return fail(ctx, LBM_ERR_UNSUPPORTED, "plane steps need the pull pattern");
    Dev d = make_dev(ctx);
    Dev part = d;
    clip_planes(part.P, z0, z1);
    clip_planes(part.PF, z0, z1);
    part.link_max = 0;  // the link bounce follows the whole step, below
    const bool any = part.P.nzr > 0 && part.PF.nzr > 0;
    cudaError_t e = cudaSuccess;
    if (out) {
        lbm_status s = ensure_step_partials(ctx, d);
        if (s) return s;
        if (any)
            e = LBM_DISPATCH(ctx, step_reduce(part, ctx->lat[ctx->cur], ctx->lat[ctx->cur ^ 1], ctx->step_partials,
                                              ctx->red_out));
        else
            e = cudaMemsetAsync(ctx->red_out, 0, 4 * sizeof(double), ctx->stream);
    } else if (any) {
        e = step_from(ctx, part, ctx->cur, nullptr);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream-collide (planes) launch");
    if (last) {
        e = LBM_DISPATCH(ctx, bounce(d, ctx->lat[ctx->cur ^ 1]));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "bounce launch");
        ctx->cur ^= 1;
        ctx->steps_done++;
    }
    return out ? copy_totals(ctx, out) : LBM_OK;
}

lbm_status lbm_get_state(lbm_ctx *ctx, void *dst, lbm_storage fmt) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    if (!dst || !valid_storage(fmt)) return fail(ctx, LBM_ERR_ARG, "bad destination or format");
    const size_t N = (size_t)ctx->g.nx * ctx->g.ny * ctx->g.nz;
    Staged st(ctx);
    int k = st.add(dst, (size_t)Q * N * storage_bytes(fmt), true);
    lbm_status s = st.prepare();
    if (s) return s;
    Dev d = make_dev(ctx);
    cudaError_t e = LBM_DISPATCH(ctx, get_state(d, state_lat(ctx), st.dev(k), (int)fmt));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "get_state launch");
    return st.finish();
}

lbm_status lbm_set_state(lbm_ctx *ctx, const void *src, lbm_storage fmt) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    if (!src || !valid_storage(fmt)) return fail(ctx, LBM_ERR_ARG, "bad source or format");
    const size_t N = (size_t)ctx->g.nx * ctx->g.ny * ctx->g.nz;
    Staged st(ctx);
    int k = st.add(src, (size_t)Q * N * storage_bytes(fmt), false);
    lbm_status s = st.prepare();
    if (s) return s;
    if (ctx->pattern == LBM_PATTERN_AA) ctx->cur = 0;  // written in the natural layout
    Dev d = make_dev(ctx);
    cudaError_t e = LBM_DISPATCH(ctx, set_state(d, state_lat(ctx), st.dev(k), (int)fmt));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set_state launch");
    e = cudaMemsetAsync(ctx->status_d, 0, sizeof(unsigned), ctx->stream);  // a new run
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status word reset");
    ctx->steps_done = 0;
    return LBM_OK;
}

size_t lbm_halo_bytes(const lbm_ctx *ctx) {
    if (check_ctx(ctx)) return 0;
    return (size_t)5 * ctx->g.ny * ctx->g.pitch * storage_bytes(ctx->storage);
}

size_t lbm_adjoint_halo_bytes(const lbm_ctx *ctx) {
    if (check_ctx(ctx)) return 0;
    return (size_t)5 * ctx->g.ny * ctx->g.pitch * real_size(ctx->storage);
}

// Pack copies the boundary interior plane's outgoing populations (side 0:
// plane 1, e_z = -1; side 1: plane nz - 2, e_z = +1); unpack writes the
// incoming ones into the ghost plane (side 0: plane 0, e_z = +1; side 1:
// plane nz - 1, e_z = -1) at fluid cells. The adjoint populations cross the
// other way (the reverse step reads lambda_i at x + e_i), so for them every
// e_z sign flips; they are copied from and into the current adjoint lattice.
static lbm_status halo_copy(lbm_ctx *ctx, int side, const void *buf, bool unpack, bool adjoint) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    if (!buf || (side != 0 && side != 1)) return fail(ctx, LBM_ERR_ARG, "bad halo buffer or side");
    if (ctx->g.nz < 3) return fail(ctx, LBM_ERR_ARG, "a slab needs nz >= 3: two ghost planes and an interior");
    if (ctx->pattern != LBM_PATTERN_PULL) return fail(ctx, LBM_ERR_UNSUPPORTED, "halo copies need the pull pattern");
    if (is_split(ctx->storage))
        return fail(ctx, LBM_ERR_UNSUPPORTED, "halo copies do not carry the momentum words of moment-split storage");
    if (adjoint && !ctx->lam_valid) return fail(ctx, LBM_ERR_STATE, "lbm_adjoint_seed must come first");
    Staged st(ctx);
    const int k = st.add(buf, adjoint ? lbm_adjoint_halo_bytes(ctx) : lbm_halo_bytes(ctx), !unpack);
    lbm_status s = st.prepare();
    if (s) return s;
    const int z = unpack ? (side == 0 ? 0 : ctx->g.nz - 1) : (side == 0 ? 1 : ctx->g.nz - 2);
    const int dir = ((side == 1) != unpack) != adjoint ? 1 : -1;
    void *lat = adjoint ? ctx->lam[ctx->lcur] : state_lat(ctx);
    const int elem = (int)(adjoint ? real_size(ctx->storage) : storage_bytes(ctx->storage));
    cudaError_t e = launch_halo(ctx->g, lat, elem, st.dev(k), z, dir, unpack, ctx->flags_d, ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, unpack ? "halo unpack launch" : "halo pack launch");
    return st.finish();
}

lbm_status lbm_halo_pack(lbm_ctx *ctx, int side, void *buf) { return halo_copy(ctx, side, buf, false, false); }

lbm_status lbm_halo_unpack(lbm_ctx *ctx, int side, const void *buf) { return halo_copy(ctx, side, buf, true, false); }

lbm_status lbm_adjoint_halo_pack(lbm_ctx *ctx, int side, void *buf) { return halo_copy(ctx, side, buf, false, true); }

lbm_status lbm_adjoint_halo_unpack(lbm_ctx *ctx, int side, const void *buf) {
    return halo_copy(ctx, side, buf, true, true);
}

static lbm_status ensure_lambda(lbm_ctx *ctx) {
    // the reverse step gathers with the push masks (built at create; kept
    // here for a context whose masks are missing)
    if (ctx->flags_d && !ctx->mask_d) {
        cudaError_t e = cudaMalloc((void **)&ctx->mask_d, (size_t)ctx->g.qs * sizeof(uint32_t));
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->mask_d = nullptr;
            return fail(ctx, LBM_ERR_OOM, "cannot allocate the push masks");
        }
        e = build_push_mask(ctx->g, ctx->flags_d, ctx->mask_d, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "push mask build");
    }
    const size_t bytes = (size_t)Q * (size_t)ctx->g.qs * real_size(ctx->storage);
    for (int k = 0; k < 2; ++k) {
        if (ctx->lam[k]) continue;
        cudaError_t e = cudaMalloc(&ctx->lam[k], bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->lam[k] = nullptr;
            return fail(ctx, LBM_ERR_OOM, "cannot allocate the adjoint lattices");
        }
    }
    return LBM_OK;
}

lbm_status lbm_adjoint_seed(lbm_ctx *ctx, const void *dL_du, const void *dL_drho, void *grad_F) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    if (!dL_du) return fail(ctx, LBM_ERR_ARG, "dL_du is required");
    if (grad_F && !is_device_ptr(grad_F)) return fail(ctx, LBM_ERR_ARG, "grad_F must be a device array");
    lbm_status s = ensure_lambda(ctx);
    if (s) return s;
    const size_t N = (size_t)ctx->g.nx * ctx->g.ny * ctx->g.nz, rs = real_size(ctx->storage);
    Staged st(ctx);
    int iu = st.add(dL_du, 3 * N * rs, false);
    int ir = dL_drho ? st.add(dL_drho, N * rs, false) : -1;
    s = st.prepare();
    if (s) return s;
    Dev d = make_dev(ctx);
    cudaError_t e = LBM_DISPATCH(ctx, adj_seed(d, state_lat(ctx), st.dev(iu), ir >= 0 ? st.dev(ir) : nullptr,
                                               ctx->lam[ctx->lcur], grad_F));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "adjoint seed launch");
    ctx->lam_valid = true;
    return LBM_OK;
}

lbm_status lbm_adjoint_step(lbm_ctx *ctx, int n, const void *tape, void *grad_F) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    if (n < 0) return fail(ctx, LBM_ERR_ARG, "n must be >= 0");
    if (!ctx->lam_valid) return fail(ctx, LBM_ERR_STATE, "lbm_adjoint_seed must come first");
    if (n > 0 && (!tape || !is_device_ptr(tape))) return fail(ctx, LBM_ERR_ARG, "tape must be a device array");
    if (grad_F && !is_device_ptr(grad_F)) return fail(ctx, LBM_ERR_ARG, "grad_F must be a device array");
    const size_t per = 4 * (size_t)ctx->g.qs * real_size(ctx->storage);
    Dev d = make_dev(ctx);
    for (int k = n - 1; k >= 0; --k) {
        const void *tk = static_cast<const char *>(tape) + per * (size_t)k;
        d.zrev = ctx->lcur;  // alternating plane order, as in the forward steps
        cudaError_t e = ctx->storage == LBM_F64
                            ? AdjOps<double>::step(d, ctx->lam[ctx->lcur], ctx->lam[ctx->lcur ^ 1], tk, grad_F)
                            : AdjOps<float>::step(d, ctx->lam[ctx->lcur], ctx->lam[ctx->lcur ^ 1], tk, grad_F);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "adjoint step launch");
        ctx->lcur ^= 1;
    }
    return LBM_OK;
}

lbm_status lbm_adjoint_init_grad(lbm_ctx *ctx, const void *rho0, const void *u0, void *grad_u0, void *grad_rho0) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    if (!u0 || !grad_u0) return fail(ctx, LBM_ERR_ARG, "u0 and grad_u0 are required");
    if (!ctx->lam_valid) return fail(ctx, LBM_ERR_STATE, "lbm_adjoint_seed must come first");
    const size_t N = (size_t)ctx->g.nx * ctx->g.ny * ctx->g.nz, rs = real_size(ctx->storage);
    Staged st(ctx);
    int ir = rho0 ? st.add(rho0, N * rs, false) : -1;
    int iu = st.add(u0, 3 * N * rs, false);
    int ig = st.add(grad_u0, 3 * N * rs, true);
    int igr = grad_rho0 ? st.add(grad_rho0, N * rs, true) : -1;
    lbm_status s = st.prepare();
    if (s) return s;
    Dev d = make_dev(ctx);
    const void *r = ir >= 0 ? st.dev(ir) : nullptr;
    void *gr = igr >= 0 ? st.dev(igr) : nullptr;
    cudaError_t e = ctx->storage == LBM_F64
                        ? AdjOps<double>::init_grad(d, ctx->lam[ctx->lcur], r, st.dev(iu), st.dev(ig), gr)
                        : AdjOps<float>::init_grad(d, ctx->lam[ctx->lcur], r, st.dev(iu), st.dev(ig), gr);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "adjoint init-grad launch");
    return st.finish();
}

lbm_status lbm_status_word(lbm_ctx *ctx, uint32_t *out, int clear) {
    if (check_ctx(ctx) || !out) return LBM_ERR_ARG;
    unsigned v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, ctx->status_d, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess && clear) e = cudaMemsetAsync(ctx->status_d, 0, sizeof(unsigned), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status word");
    *out = v;
    return LBM_OK;
}

lbm_status lbm_synchronize(lbm_ctx *ctx) {
    if (check_ctx(ctx)) return LBM_ERR_ARG;
    unsigned v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, ctx->status_d, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
    return diverged(ctx, v);
}

const char *lbm_last_error(const lbm_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

const char *lbm_status_string(lbm_status s) {
    return (s >= LBM_OK && s <= LBM_ERR_UNSUPPORTED) ? status_names[s] : "unknown status";
}

int lbm_lattice_table(int *e, double *w, int *o) {
    for (int i = 0; i < Q; ++i) {
        if (e) {
            e[3 * i] = ex(i);
            e[3 * i + 1] = ey(i);
            e[3 * i + 2] = ez(i);
        }
        if (w) w[i] = weight(i);
        if (o) o[i] = opp(i);
    }
    return Q;
}

// Walk every thread of the row launch (and the reduction's cell loop) on the
// host, forming the same addresses as the kernels with the same helpers.
int64_t lbm_check_launch_indices(int nx, int ny, int nz, lbm_storage fmt, int row_align) {
    if (nx < 1 || ny < 1 || nz < 1 || nz > 65535 || !valid_storage(fmt)) return -1;
    Geom g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.pitch = pitch_for(nx, fmt, row_align);
    if (g.pitch < 0) return -1;
    g.qs = (long long)nz * ny * g.pitch;
    if (g.qs >= (1LL << 31)) return -1;
    const RowLaunch L = row_launch(g);
    const long long N = (long long)nx * ny * nz;
    int64_t bad = 0;
    auto cell_ok = [&](int c) { return c >= 0 && c < g.qs && (c % g.pitch) < nx; };
    long long visited = 0;
    for (int bz = 0; bz < nz; ++bz)
        for (int bx = 0; bx < L.nxb * L.nyb; ++bx)
            for (int ty = 0; ty < L.by_threads; ++ty)
                for (int tx = 0; tx < L.bx_threads; ++tx) {
                    int x, y, z;
                    if (!row_cell(g, L.nxb, L.bx_threads, L.by_threads, bx, bz, tx, ty, x, y, z)) continue;
                    ++visited;
                    const int c = cell_index(g, x, y, z);
                    if (!cell_ok(c)) ++bad;
                    const long long cc = canon_index(g, x, y, z);
                    if (cc < 0 || cc >= N) ++bad;
                    for (int i = 0; i < Q; ++i) {
                        if (!cell_ok(pull_src(g, x, y, z, i))) ++bad;
                        if (!cell_ok(push_dst(g, x, y, z, i))) ++bad;
                        const long long cn = canon_index(g, wrap1(x + ex(i), nx), wrap1(y + ey(i), ny),
                                                         wrap1(z + ez(i), nz));
                        if (cn < 0 || cn >= N) ++bad;
                        if ((long long)opp(i) * g.qs + c >= (long long)Q * g.qs) ++bad;
                    }
                }
    if (visited != N) ++bad;  // every cell owned by exactly one thread
    // paired launch of the step kernels: every address k_step forms, which
    // covers the AA kernels too (the odd step loads at the pull sources and
    // stores at the reverse step's rows and columns; both touch the pair at c)
    const RowLaunch Prows = pair_launch(g);
    auto walk_pairs = [&](const RowLaunch &P, bool flat) {
    long long visited2 = 0;
    auto in_row = [&](int rowbase, int x) { return x >= 0 && x < g.pitch && rowbase + x < g.qs && rowbase >= 0; };
    for (int bz = 0; bz < nz; ++bz)
        for (int bx = 0; bx < P.nxb * P.nyb; ++bx)
            for (int ty = 0; ty < P.by_threads; ++ty)
                for (int tx = 0; tx < P.bx_threads; ++tx) {
                    int x0, y, z;
                    if (!(flat ? pair_cell<true>(g, P, P.bx_threads, P.by_threads, bx, bz, tx, ty, x0, y, z)
                             : pair_cell<false>(g, P, P.bx_threads, P.by_threads, bx, bz, tx, ty, x0, y, z))) continue;
                    const bool has1 = x0 + 1 < nx;
                    visited2 += has1 ? 2 : 1;
                    const int c = cell_index(g, x0, y, z);
                    if (c % 2 || !in_row(c - x0, x0) || !in_row(c - x0, x0 + 1)) ++bad;  // pair at c, c + 1
                    if ((nx & 1) && x0 == 0 && !in_row(c, nx)) ++bad;  // split formats' copy of cell 0 after an odd row
                    const int xa = wrap1(x0 - 1, nx), xb = wrap1(x0 + 1, nx), xc = has1 ? wrap1(x0 + 2, nx) : x0;
                    for (int j = 1; j < Q; ++j)  // store-side bounce-back targets
                        if (!cell_ok(push_dst(g, x0, y, z, j)) || (has1 && !cell_ok(push_dst(g, x0 + 1, y, z, j))))
                            ++bad;
                    for (int i = 0; i < Q; ++i) {
                        const int row = (wrap1(z - ez(i), nz) * ny + wrap1(y - ey(i), ny)) * g.pitch;
                        // reverse step: mu_i(x) = lambda_i(x + e_i)
                        const int rowp = (wrap1(z + ez(i), nz) * ny + wrap1(y + ey(i), ny)) * g.pitch;
                        if (ex(i) == 0) {
                            if (!in_row(row, x0) || !in_row(row, x0 + 1) || (row + x0) % 2) ++bad;
                            if (!in_row(rowp, x0) || !in_row(rowp, x0 + 1) || (rowp + x0) % 2) ++bad;
                        } else {
                            if (!in_row(row, ex(i) > 0 ? xa : xb) || !in_row(row, ex(i) > 0 ? x0 : xc)) ++bad;
                            if ((ex(i) > 0 ? xa : xb) >= nx || (has1 && (ex(i) > 0 ? x0 : xc) >= nx)) ++bad;
                            if (!in_row(rowp, ex(i) > 0 ? xb : xa) || !in_row(rowp, ex(i) > 0 ? xc : x0)) ++bad;
                            if ((ex(i) > 0 ? xb : xa) >= nx || (has1 && (ex(i) > 0 ? xc : x0) >= nx)) ++bad;
                        }
                    }
                }
    if (visited2 != N) ++bad;
    };
    walk_pairs(Prows, false);
    walk_pairs(flat_launch(Prows), true);  // the two-grid step's launch when rows leave lanes idle
    // the FP32 reverse step, one cell per thread over the box rows in order
    {
        long long visited1 = 0;
        const long long cells = (long long)Prows.nyr * nx, nblk = (cells + 255) / 256;
        for (int bz = 0; bz < Prows.nzr; ++bz)
            for (long long k = 0; k < nblk * 256; ++k) {
                const long long r = k / nx;
                if (r >= Prows.nyr) continue;
                ++visited1;
                const int x = (int)(k - r * nx), y = Prows.y0 + (int)r, z = Prows.z0 + bz;
                const int c = cell_index(g, x, y, z);
                if (!cell_ok(c) || canon_index(g, x, y, z) >= N) ++bad;
                for (int i = 0; i < Q; ++i)
                    if (!cell_ok(push_dst(g, x, y, z, i))) ++bad;
            }
        if (visited1 != N) ++bad;
    }
    const RowLaunch &P = Prows;
    if (P.bx_threads * P.by_threads > 256 || P.bx_threads % 32 || P.by_threads < 1) ++bad;
    if (L.bx_threads * L.by_threads != 256 || L.bx_threads % 32) ++bad;
    // z-slab halo copies (lbm_halo.cu): the ghost and boundary planes, five
    // directions each, buffer [5][ny][pitch]
    if (nz >= 3) {
        const long long plane = (long long)ny * g.pitch;
        const int zs[4] = {0, 1, nz - 2, nz - 1};
        for (int dir = -1; dir <= 1; dir += 2)
            for (int zi = 0; zi < 4; ++zi) {
                int k = 0;
                for (int i = 0; i < Q; ++i) {
                    if (ez(i) != dir) continue;
                    for (long long r = 0; r < plane; ++r) {
                        const long long at = (long long)i * g.qs + zs[zi] * plane + r;
                        if (at < 0 || at >= (long long)Q * g.qs || zs[zi] * plane + r >= g.qs) ++bad;
                        if (k * plane + r >= 5 * plane) ++bad;
                    }
                    ++k;
                }
                if (k != 5) ++bad;
            }
    }
    // reduction: canonical walk
    for (long long cc = 0; cc < N; ++cc) {
        const int x = (int)(cc % nx);
        const long long r = cc / nx;
        const int y = (int)(r % ny), z = (int)(r / ny);
        if (!cell_ok(cell_index(g, x, y, z))) ++bad;
    }
    return bad;
}

}  // extern "C"
