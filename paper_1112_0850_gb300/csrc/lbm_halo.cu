// z-slab halo copies: the one exchange per step of a lattice split along z
// into slabs (the domain decomposition of a multi-GPU run). A slab is a
// lattice of its own whose first and last planes are ghosts, copies of the
// neighbouring slabs' boundary planes. In the pull update (Sec. 2) interior
// plane z = 1 reads from ghost plane z = 0 only the five populations with
// e_z = +1, and plane nz - 2 reads from plane nz - 1 only those with e_z = -1,
// so these five are all that cross a face.
#include "lbm_launch.h"

namespace lbm {

// Direction indices with e_z = dir, in increasing order.
LBM_HD constexpr int zpop(int k, int dir) {
    return dir > 0 ? (k == 0 ? 5 : 9 + 2 * k) : (k == 0 ? 6 : 10 + 2 * k);
}
static_assert(ez(zpop(0, 1)) == 1 && ez(zpop(4, 1)) == 1 && ez(zpop(2, 1)) == 1, "e_z = +1 set");
static_assert(ez(zpop(0, -1)) == -1 && ez(zpop(4, -1)) == -1 && ez(zpop(2, -1)) == -1, "e_z = -1 set");
static_assert(zpop(1, 1) == 11 && zpop(3, 1) == 15 && zpop(1, -1) == 12 && zpop(3, -1) == 16, "direction order");

// Pack: buf[k][y][x] = P[zpop(k, dir)][z][y][x] over the whole plane (pitch
// columns included). Unpack: the reverse, at fluid cells only (flags null:
// all cells fluid), since a solid ghost cell's slots hold this slab's own
// bounce-back values. One thread per element, grid-stride.
template <class E, bool UNPACK>
__global__ void __launch_bounds__(256) k_halo(const Geom g, E *__restrict__ P, E *__restrict__ buf, int z, int dir,
                                                const uint8_t *__restrict__ flags) {
    const long long plane = (long long)g.ny * g.pitch;
    const long long n = 5 * plane;
    const long long base = (long long)z * plane;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t / plane);
        const long long r = t - k * plane;  // y * pitch + x
        const long long at = zpop(k, dir) * g.qs + base + r;
        if (UNPACK) {
            const int x = (int)(r % g.pitch);
            if (x < g.nx && (!flags || flags[base + r] == 0)) P[at] = buf[t];
        } else {
            buf[t] = P[at];
        }
    }
}

template <class E>
static cudaError_t launch_halo_t(const Geom &g, void *lat, void *buf, int z, int dir, bool unpack,
                                 const uint8_t *flags, int num_sms, cudaStream_t s) {
    const long long n = 5LL * g.ny * g.pitch;
    const long long want = (n + 255) / 256;
    const int blocks = (int)(want < 8LL * num_sms ? want : 8LL * num_sms);
    if (unpack)
        k_halo<E, true><<<blocks, 256, 0, s>>>(g, static_cast<E *>(lat), static_cast<E *>(buf), z, dir, flags);
    else
        k_halo<E, false><<<blocks, 256, 0, s>>>(g, static_cast<E *>(lat), static_cast<E *>(buf), z, dir, flags);
    return cudaGetLastError();
}

cudaError_t launch_halo(const Geom &g, void *lat, int elem_bytes, void *buf, int z, int dir, bool unpack,
                        const uint8_t *flags, int num_sms, cudaStream_t s) {
    switch (elem_bytes) {
    case 2: return launch_halo_t<uint16_t>(g, lat, buf, z, dir, unpack, flags, num_sms, s);
    case 4: return launch_halo_t<uint32_t>(g, lat, buf, z, dir, unpack, flags, num_sms, s);
    case 8: return launch_halo_t<unsigned long long>(g, lat, buf, z, dir, unpack, flags, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm
