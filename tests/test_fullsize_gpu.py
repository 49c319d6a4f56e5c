"""Parity at full workload sizes, in the launch configuration the benchmark
times: the oracle recomputes one update at sampled cells, one by one, from the
GPU's own state; conservation properties are checked over whole lattices.

Workloads: the 256x128x128 walled channel with 10% spherical obstacles (FP32
and FP64), the 512^3 periodic Taylor-Green vortex (FP32, FP16 and BF16
shifted storage) and the 384x256x256 porous channel with 15% obstacles (FP16
shifted storage).
"""
import numpy as np
import pytest
import torch

import lbm_inputs
import oracle
from gpu_helpers import REAL, ensure_built

pytestmark = pytest.mark.gpu

_E, _W, _OPP = oracle.lattice()


def _lattice(storage, nx, ny, nz, tau, flags, F, u0, rho0=None):
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    lat = Lattice(nx, ny, nz, tau, flags=flags, force=F, storage=storage)
    real = REAL[storage]
    lat.init_equilibrium(torch.as_tensor(u0, dtype=real).cuda(),
                         None if rho0 is None else torch.as_tensor(rho0, dtype=real).cuda())
    return lat


def _sample_cells(flags, shape, k, seed):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    out = []
    while len(out) < k:
        z, y, x = rng.integers(0, nz), rng.integers(0, ny), rng.integers(0, nx)
        if flags is None or flags[z, y, x] == 0:
            out.append((z, y, x))
    # include the corners of the periodic box and the ragged end of a row
    for c in [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (0, ny - 1, nx - 1), (nz // 2, ny // 2, nx - 1)]:
        if flags is None or flags[c] == 0:
            out.append(c)
    return out


def _gather_states(st, cells, shape):
    """Values of state tensor st [19][nz][ny][nx] (device) at each cell and its 18 neighbours (FP64, host)."""
    nz, ny, nx = shape
    idx = []
    for (z, y, x) in cells:
        for i in range(19):
            idx.append(((z - _E[i][2]) % nz, (y - _E[i][1]) % ny, (x - _E[i][0]) % nx))
    zz = torch.tensor([a for a, _, _ in idx], device="cuda")
    yy = torch.tensor([b for _, b, _ in idx], device="cuda")
    xx = torch.tensor([c for _, _, c in idx], device="cuda")
    vals = st[:, zz, yy, xx].double().cpu().numpy()  # [19][len(idx)]
    return vals.T.reshape(len(cells), 19, 19), idx


def _expected_next(S, cells, idx, flags, tau, F):
    """f^{n+1}_i(x) = f*_i(x - e_i) if that cell is fluid, else f*_{opp(i)}(x);
    f* = oracle collision of f^n = w + S at that cell. Returns shifted values."""
    out = np.zeros((len(cells), 19))
    for k, (z, y, x) in enumerate(cells):
        own = oracle.collide_cell(S[k, 0] + _W, tau, F)  # S[k, 0]: state at x itself (i = 0: no shift)
        for i in range(19):
            sz, sy, sx = idx[19 * k + i]
            if flags is not None and flags[sz, sy, sx]:
                out[k, i] = own[_OPP[i]] - _W[i]
            else:
                out[k, i] = oracle.collide_cell(S[k, i] + _W, tau, F)[i] - _W[i]
    return out


def _ulp(v, storage):
    a = np.abs(v)
    if storage == "f16s":
        return np.spacing(a.astype(np.float16)).astype(np.float64)
    e = np.floor(np.log2(np.maximum(a, 1e-38)))
    return 2.0 ** (e - 7)  # bfloat16


def _check_one_step(storage, lat, shape, flags, tau, F, nsamp=200, seed=5):
    st0 = lat.get_state()
    cells = _sample_cells(flags, shape, nsamp, seed)
    S, idx = _gather_states(st0, cells, shape)
    del st0
    lat.step(1)
    st1 = lat.get_state()
    zz = torch.tensor([c[0] for c in cells], device="cuda")
    yy = torch.tensor([c[1] for c in cells], device="cuda")
    xx = torch.tensor([c[2] for c in cells], device="cuda")
    got = st1[:, zz, yy, xx].double().cpu().numpy().T
    del st1
    want = _expected_next(S, cells, idx, flags, tau, np.zeros(3) if F is None else np.asarray(F, np.float64))
    if storage == "f64":
        # shifted FP64 arithmetic against the oracle's unshifted FP64: a few ulp of |f| < 0.4
        assert np.abs(got - want).max() <= 1e-15
    elif storage == "f32":
        assert np.abs(got - want).max() <= 1e-7
    else:
        # one rounding of an FP32 result to the 16-bit format: at most one unit
        # in the last place of the exactly rounded value
        # (half a unit for the rounding, plus the FP32-vs-FP64 arithmetic difference
        # that can move a value across a rounding boundary)
        assert np.all(np.abs(got - want) <= _ulp(want, storage) * 1.01 + 1e-30)


@pytest.fixture(scope="module")
def channel_flags():
    return lbm_inputs.channel_flags(256, 128, 128, 0.10, lbm_inputs.seed_for(1))


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_channel_256x128x128_one_step_sampled(storage, channel_flags):
    nx, ny, nz = 256, 128, 128
    F = (1e-6, 0.0, 0.0)
    rng = np.random.default_rng(7)
    u0 = 0.01 * rng.standard_normal((3, nz, ny, nx)).astype(np.float32)
    lat = _lattice(storage, nx, ny, nz, 0.55, channel_flags, F, u0)
    lat.step(10)
    mass0 = lat.reduce()[0]
    _check_one_step(storage, lat, (nz, ny, nx), channel_flags, 0.55, F)
    lat.step(20)
    mass1 = lat.reduce()[0]
    assert abs(mass1 - mass0) <= (1e-13 if storage == "f64" else 1e-6) * mass0
    assert lat.status_word() == 0
    lat.close()


@pytest.mark.parametrize("storage", ["f32", "f16s", "bf16s"])
def test_taylor_green_512_one_step_sampled(storage):
    n = 512
    rho0, u0 = lbm_inputs.taylor_green(n, 0.02, dtype=np.float32)
    lat = _lattice(storage, n, n, n, 0.52, None, None, u0, rho0)
    del rho0, u0
    lat.step(3)
    s0 = lat.reduce()
    _check_one_step(storage, lat, (n, n, n), None, 0.52, None, nsamp=150)
    s1 = lat.reduce()
    tol = {"f32": 1e-6, "f16s": 1e-4, "bf16s": 1e-3}[storage]
    assert abs(s1[0] - s0[0]) <= tol * s0[0]
    assert lat.status_word() == 0
    lat.close()


def test_porous_channel_384x256x256_fp16_one_step_sampled():
    nx, ny, nz = 384, 256, 256
    flags = lbm_inputs.channel_flags(nx, ny, nz, 0.15, lbm_inputs.seed_for(4))
    F = (1e-6, 0.0, 0.0)
    rng = np.random.default_rng(9)
    u0 = (0.01 * rng.standard_normal((3, nz, ny, nx))).astype(np.float32)
    lat = _lattice("f16s", nx, ny, nz, 0.55, flags, F, u0)
    lat.step(5)
    _check_one_step("f16s", lat, (nz, ny, nx), flags, 0.55, F, nsamp=150)
    assert lat.status_word() == 0
    lat.close()
