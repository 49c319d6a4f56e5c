"""Seeded synthetic inputs for the D3Q19 lattice Boltzmann workloads.

This module holds input recipes only (initial velocity fields, flag
geometries, force fields); it contains none of the method's arithmetic. It is
shared by the tests, the benchmark and the smoke check, and feeds the same
arrays to the CUDA path and to the CPU oracle.

Layouts are canonical, x fastest: u[3][nz][ny][nx], flags[nz][ny][nx] (uint8,
0 = fluid, 1 = solid), F[3][nz][ny][nx]. Every generator draws from
numpy.random.default_rng(seed) (PCG64).

The paper's workloads are synthetic cubes and a lid-driven cavity (Sec. 6, 7);
these recipes stand in for the periodic box, the walled channel with
obstacles, the Taylor-Green vortex and the random solenoidal field used for
the adjoint.
"""
import numpy as np

SEED_BASE = 11120850


def seed_for(config_index: int) -> int:
    return SEED_BASE + int(config_index)


def shear_wave(n=32, amp=0.01, noise=1e-4, seed=SEED_BASE):
    """u_x = amp sin(2 pi y / n) plus i.i.d. U(-noise, noise) on every component."""
    rng = np.random.default_rng(seed)
    y = np.arange(n, dtype=np.float64)
    u = np.zeros((3, n, n, n))
    u[0] += amp * np.sin(2.0 * np.pi * y / n)[None, :, None]
    if noise:
        u += rng.uniform(-noise, noise, size=u.shape)
    return u


def channel_flags(nx, ny, nz, solid_frac, seed, rmin=3.0, rmax=6.0, walls=True):
    """Channel along x: solid walls at y in {0, ny-1} and z in {0, nz-1}, plus
    random spheres until obstacles cover `solid_frac` of the interior cells.

    Sphere centres: x uniform in [0, nx) (periodic minimum image in x), y and z
    uniform in [1 + r, n - 2 - r]; radius uniform in [rmin, rmax], capped at
    (min(ny, nz) - 3)/2 so a sphere fits between the walls; a cell is solid
    when its index lies within r of the centre; overlap allowed. Boxes too
    small to reach the fraction stop after 1000 spheres that add nothing.
    """
    rng = np.random.default_rng(seed)
    flags = np.zeros((nz, ny, nx), dtype=np.uint8)
    interior = np.ones((nz, ny, nx), dtype=bool)
    if walls:
        interior[:, 0, :] = interior[:, ny - 1, :] = False
        interior[0, :, :] = interior[nz - 1, :, :] = False
    n_interior = int(interior.sum())
    target = solid_frac * n_interior
    solid = 0
    # a sphere must fit between the walls: 1 + r <= n - 2 - r on y and z
    r_fit = (min(ny, nz) - 3.0) / 2.0
    idle = 0  # consecutive spheres that added no cell (tiny boxes may never reach the target)
    while solid < target and r_fit >= 0.5 and idle < 1000:
        r = min(rng.uniform(rmin, rmax), r_fit)
        cx = rng.uniform(0.0, nx)
        cy = rng.uniform(1.0 + r, ny - 2.0 - r)
        cz = rng.uniform(1.0 + r, nz - 2.0 - r)
        R = int(np.ceil(r))
        xs = np.arange(int(np.floor(cx)) - R, int(np.floor(cx)) + R + 2)
        ys = np.arange(max(int(np.floor(cy)) - R, 0), min(int(np.floor(cy)) + R + 2, ny))
        zs = np.arange(max(int(np.floor(cz)) - R, 0), min(int(np.floor(cz)) + R + 2, nz))
        dx = ((xs - cx + nx / 2.0) % nx) - nx / 2.0
        inside = (dx[None, None, :] ** 2 + (ys - cy)[None, :, None] ** 2
                  + (zs - cz)[:, None, None] ** 2) <= r * r
        xw = xs % nx
        sub = np.ix_(zs, ys, xw)
        newly = inside & (flags[sub] == 0) & interior[sub]
        added = int(newly.sum())
        solid += added
        idle = 0 if added else idle + 1
        block = flags[sub]
        block[inside & interior[sub]] = 1
        flags[sub] = block
    if walls:
        flags[~interior] = 1
    return flags


def random_flags(nx, ny, nz, solid_frac, seed):
    """I.i.d. solid cells with probability `solid_frac` (tiny parity boxes)."""
    rng = np.random.default_rng(seed)
    return (rng.random((nz, ny, nx)) < solid_frac).astype(np.uint8)


def taylor_green(n, U0=0.02, dtype=np.float64):
    """Taylor-Green vortex on a periodic n^3 box, k = 2 pi / n:
    u = U0 sin kx cos ky cos kz, v = -U0 cos kx sin ky cos kz, w = 0,
    rho = 1 + 3 p with p = (U0^2/16)(cos 2kx + cos 2ky)(cos 2kz + 2).
    Built by broadcasting 1-D factors (no meshgrid), in `dtype`."""
    c = np.arange(n, dtype=np.float64) * (2.0 * np.pi / n)
    sx, cx = np.sin(c)[None, None, :], np.cos(c)[None, None, :]
    sy, cy = np.sin(c)[None, :, None], np.cos(c)[None, :, None]
    cz = np.cos(c)[:, None, None]
    c2x, c2y = np.cos(2 * c)[None, None, :], np.cos(2 * c)[None, :, None]
    c2z = np.cos(2 * c)[:, None, None]
    u = np.zeros((3, n, n, n), dtype=dtype)
    u[0] = (U0 * cz * cy) * sx
    u[1] = (-U0 * cz * sy) * cx
    rho = np.empty((n, n, n), dtype=dtype)
    rho[...] = 1.0 + 3.0 * (U0 * U0 / 16.0) * (c2z + 2.0) * (c2x + c2y)
    return rho, u


def solenoidal_velocity(n, amp, seed, kmax=4):
    """Random divergence-free field u = curl A on a periodic n^3 box.

    A has i.i.d. normal Fourier coefficients for 0 < |k| <= kmax (integer wave
    numbers); the curl is taken spectrally; u is scaled so max |u| = amp.
    """
    rng = np.random.default_rng(seed)
    kk = np.fft.fftfreq(n, d=1.0 / n)
    kz, ky, kx = np.meshgrid(kk, kk, kk, indexing="ij")
    kmag = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    band = (kmag > 0) & (kmag <= kmax)
    A = []
    for _ in range(3):
        real = rng.standard_normal((n, n, n))
        Ak = np.fft.fftn(real)
        A.append(np.where(band, Ak, 0.0))
    ax, ay, az = A
    two_pi_i = 2j * np.pi / n
    ux = two_pi_i * (ky * az - kz * ay)
    uy = two_pi_i * (kz * ax - kx * az)
    uz = two_pi_i * (kx * ay - ky * ax)
    u = np.stack([np.fft.ifftn(c).real for c in (ux, uy, uz)])
    speed = np.sqrt((u ** 2).sum(0)).max()
    return u * (amp / speed)


def smooth_velocity(shape, amp, seed, kmax=2):
    """Random smooth velocity field on a periodic box of any shape [nz][ny][nx]:
    i.i.d. normal Fourier coefficients for every integer wave vector with
    0 < |k| <= kmax (each axis counted in its own box length), back-transformed
    and scaled so max |u| = amp. Returns u [3][nz][ny][nx]."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    kz, ky, kx = np.meshgrid(np.fft.fftfreq(nz, d=1.0 / nz), np.fft.fftfreq(ny, d=1.0 / ny),
                             np.fft.fftfreq(nx, d=1.0 / nx), indexing="ij")
    band = (kx ** 2 + ky ** 2 + kz ** 2 > 0) & (kx ** 2 + ky ** 2 + kz ** 2 <= kmax ** 2)
    u = np.stack([np.fft.ifftn(np.where(band, np.fft.fftn(rng.standard_normal(shape)), 0.0)).real
                  for _ in range(3)])
    return u * (amp / np.sqrt((u ** 2).sum(0)).max())


def force_field(shape, sigma, seed):
    """F[3][nz][ny][nx] with i.i.d. N(0, sigma^2) components."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, sigma, size=(3,) + tuple(shape))


def uniform_noise(shape, amp, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-amp, amp, size=shape)
