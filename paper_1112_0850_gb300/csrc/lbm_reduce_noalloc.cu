// Mass and momentum totals of a caller-provided state with no device
// allocation: the per-block partial sums live in a fixed, file-scope device
// array instead of memory obtained from cudaMalloc. This serves callers that
// cannot allocate device memory at the point they need the totals, e.g. code
// running inside a framework whose caching allocator already owns the free
// device memory, or a pipeline that must not pay cudaMalloc's device-wide
// synchronization between launches. See lbm_reduce_state_noalloc in
// include/lbm_capi.h.
#include <mutex>

#include "lbm_kernels.cuh"

namespace lbm {
namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_CELLS_PER_THREAD = 64;
constexpr int NA_CELLS_PER_BLOCK = NA_THREADS * NA_CELLS_PER_THREAD;  // 16384 cells per block
constexpr int NA_MAX_BLOCKS = 16384;
constexpr long long NA_MAX_CELLS = (long long)NA_MAX_BLOCKS * NA_CELLS_PER_BLOCK;  // 2^28 cells
static_assert(NA_MAX_CELLS == LBM_NOALLOC_MAX_CELLS, "header limit must match the scratch size");

// 4 partial sums per block: 16384 * 4 doubles = 512 KiB on every device that
// loads this library, held until the process exits. Shared by all calls.
static __device__ __align__(256) double g_noalloc_partials[NA_MAX_BLOCKS * 4];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
// device address of g_noalloc_partials per device, as last looked up outside
// a stream capture (used by calls made during one)
void *g_noalloc_addr[NA_MAX_DEVICES];

// Block b sums cells [b * 16384, (b + 1) * 16384): thread t takes cells
// b * 16384 + t + 256 k, k = 0..63 (coalesced), adds rho = 1 + sum s_i and
// rho u = sum s_i e_i + F/2 in FP64, then the block combines its threads in a
// fixed order. Every block overwrites its own 4 slots, so nothing in the
// scratch array needs clearing before a call.
template <int D>
__global__ void __launch_bounds__(NA_THREADS)
    k_sum_state(const typename IOFmt<D>::T *__restrict__ s, long long N, const uint8_t *__restrict__ flags,
                double Fx, double Fy, double Fz, double *__restrict__ partials) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const long long base = (long long)blockIdx.x * NA_CELLS_PER_BLOCK + threadIdx.x;
    for (int k = 0; k < NA_CELLS_PER_THREAD; ++k) {
        const long long c = base + (long long)k * NA_THREADS;
        if (c >= N || (flags && flags[c])) continue;
        double r = 1.0, jx = 0.5 * Fx, jy = 0.5 * Fy, jz = 0.5 * Fz;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double v = IOFmt<D>::get(s + (long long)i * N + c);
            r += v;
            jx += ex(i) * v;
            jy += ey(i) * v;
            jz += ez(i) * v;
        }
        acc[0] += r;
        acc[1] += jx;
        acc[2] += jy;
        acc[3] += jz;
    }
    __shared__ double sm[NA_THREADS / 32][4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sm[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < NA_THREADS / 32; ++w) t += sm[w][threadIdx.x];
        partials[blockIdx.x * 4 + threadIdx.x] = t;
    }
}

// Device address of the scratch array on the current device
// (cudaGetSymbolAddress with that device current). It is looked up afresh on
// every call made outside a stream capture, so a device reset (which unloads
// the module and may place the array elsewhere when it is loaded again) never
// leaves a stale address behind; a call made while `st` is being captured
// uses the address of the last call outside a capture on this device (the
// first call on a device therefore belongs before any capture).
cudaError_t noalloc_scratch(cudaStream_t st, double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();  // (the legacy stream while another stream captures): take it as captured
        cap = cudaStreamCaptureStatusActive;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (cap == cudaStreamCaptureStatusNone || !g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = static_cast<double *>(g_noalloc_addr[dev]);
    return cudaSuccess;
}

template <int D>
cudaError_t launch_sum(const void *state, long long N, const uint8_t *flags, const double F[3], double *scratch,
                       double *out, cudaStream_t st) {
    const int blocks = (int)((N + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK);
    k_sum_state<D><<<blocks, NA_THREADS, 0, st>>>(static_cast<const typename IOFmt<D>::T *>(state), N, flags, F[0],
                                                  F[1], F[2], scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, RED_THREADS, 0, st>>>(scratch, blocks, out);
    return cudaGetLastError();
}

}  // namespace
}  // namespace lbm

extern "C" lbm_status lbm_reduce_state_noalloc(const void *state, lbm_storage fmt, int nx, int ny, int nz,
                                               const uint8_t *flags, const double force[3], double *out,
                                               void *cuda_stream) {
    using namespace lbm;
    if (!state || !out || nx < 1 || ny < 1 || nz < 1 || fmt < LBM_F64 || fmt > LBM_BF16S) return LBM_ERR_ARG;
    const long long N = (long long)nx * ny * nz;
    if (N > NA_MAX_CELLS) return LBM_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    double *scratch = nullptr;
    cudaError_t e = noalloc_scratch(st, &scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    const double F[3] = {force ? force[0] : 0.0, force ? force[1] : 0.0, force ? force[2] : 0.0};
    switch (fmt) {
    case LBM_F64: e = launch_sum<LBM_F64>(state, N, flags, F, scratch, out, st); break;
    case LBM_F32: e = launch_sum<LBM_F32>(state, N, flags, F, scratch, out, st); break;
    case LBM_F16S: e = launch_sum<LBM_F16S>(state, N, flags, F, scratch, out, st); break;
    default: e = launch_sum<LBM_BF16S>(state, N, flags, F, scratch, out, st); break;
    }
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
