// One-time set-up kernels run by lbm_create.
#include "lbm_launch.h"

namespace lbm {

// Push mask of every padded cell c: bit j when the neighbour x + e_j is solid
// (periodic), MOVING_BIT when one of them is a moving wall (flag 2),
// SOLID_BIT on solid cells and on row padding.
__global__ void __launch_bounds__(256) k_build_mask(const Geom g, const uint8_t *__restrict__ flags,
                                                    uint32_t *__restrict__ mask) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.qs) return;
    const int x = (int)(c % g.pitch);
    const long long r = c / g.pitch;
    const int y = (int)(r % g.ny), z = (int)(r / g.ny);
    if (x >= g.nx || z >= g.nz) {
        mask[c] = SOLID_BIT;
        return;
    }
    uint32_t m = flags[c] ? SOLID_BIT : 0u;
#pragma unroll
    for (int j = 1; j < Q; ++j) {
        const uint8_t f = flags[push_dst(g, x, y, z, j)];
        if (f) m |= 1u << j;
        if (f == 2) m |= MOVING_BIT;
    }
    mask[c] = m;
}

cudaError_t build_push_mask(const Geom &g, const uint8_t *flags, uint32_t *mask, cudaStream_t st) {
    const long long blocks = (g.qs + 255) / 256;
    k_build_mask<<<(unsigned)blocks, 256, 0, st>>>(g, flags, mask);
    return cudaGetLastError();
}

}  // namespace lbm
