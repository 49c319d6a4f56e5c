"""Moving walls (flag 2) on the GPU: the paper's lid-driven cavity (Sec. 7)
against the oracle in every storage format, plane Couette flow against its
exact linear profile, and the adjoint with a moving lid against the FP64
reference adjoint."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import REAL, STORAGES, TOL_U, as_input, ensure_built, fluid_mask, rel_l2
from oracle import adjoint as oadj

pytestmark = pytest.mark.gpu


def _cavity(n=14):
    flags = np.ones((n, n, n), np.uint8)
    flags[1:-1, 1:-1, 1:-1] = 0
    flags[1:-1, n - 1, 1:-1] = 2  # lid: the y = n - 1 face
    return flags


def _lattice(*a, **k):
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    return Lattice(*a, **k)


def _mass_bound(storage, f, flags, T):
    """Bound on |total mass (GPU) - total mass (oracle)| after T steps.

    f64: the oracle stores f unshifted, so each step each of its 19 N stored
    populations (all <= 1) rounds by up to 2^-53; T 19 N 2^-53 bounds that.
    f32: the bound that held for the walled channel, 1e-5.
    16-bit: each step rounds every stored s_i = f_i - w_i to the format's unit
    roundoff u (2^-11 FP16, 2^-8 BF16), errors of either sign, so the mass
    walks by about u rms|s| sqrt(19 N T / 3); 8 times that (rms|s| from the
    oracle's final state)."""
    fl = flags == 0
    n = int(fl.sum())
    if storage == "f64":
        return T * 19 * n * 2.0 ** -53
    if storage == "f32":
        return 1e-5
    u = {"f16s": 2.0 ** -11, "bf16s": 2.0 ** -8}[storage]
    s = f - oracle.lattice()[1][:, None, None, None]
    rms = float(np.sqrt((s[:, fl] ** 2).mean()))
    return 8 * u * rms * np.sqrt(19 * n * T / 3)


@pytest.mark.parametrize("storage", STORAGES)
def test_lid_driven_cavity_matches_oracle(storage):
    n, tau, T = 14, 0.6, 150
    uw = np.array([0.05, 0.0, 0.01])
    flags = _cavity(n)
    rng = np.random.default_rng(41)
    u0 = 0.005 * rng.standard_normal((3, n, n, n)) * (flags == 0)
    lat = _lattice(n, n, n, tau, flags=flags, storage=storage)
    lat.set_wall_velocity(uw)
    lat.init_equilibrium(torch.tensor(u0, dtype=REAL[storage]).cuda())
    lat.step(T)
    rho, u = lat.macros()
    mass = lat.reduce()[0]
    lat.close()
    f = oracle.run(oracle.init_equilibrium(as_input(u0, storage), flags=flags), tau, T, flags=flags,
                   u_wall=uw if storage == "f64" else np.float32(uw).astype(np.float64))
    rho_o, u_o = oracle.macros(f, flags=flags)
    m = fluid_mask(flags, (n, n, n))
    assert rel_l2(u.double().cpu().numpy(), u_o, m) <= TOL_U[storage]
    assert abs(mass - oracle.sums(f, flags=flags)[0]) <= _mass_bound(storage, f, flags, T)
    assert u_o[0, 1:-1, n - 2, 1:-1].mean() > 0.01  # the lid drives the flow


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_couette_profile_is_linear(storage):
    H, U, tau = 16, 0.01, 0.8
    ny = H + 2
    flags = np.zeros((2, ny, 4), np.uint8)
    flags[:, 0, :] = 1
    flags[:, ny - 1, :] = 2
    lat = _lattice(4, ny, 2, tau, flags=flags, storage=storage)
    lat.set_wall_velocity((U, 0.0, 0.0))
    lat.init_equilibrium(lat.zeros(3))
    lat.step(20000)
    _, u = lat.macros()
    lat.close()
    y = np.arange(1, ny - 1)
    got = u[0, :, 1:ny - 1, :].double().cpu().numpy()
    exact = U * (y - 0.5) / H
    assert np.abs(got - exact[None, :, None]).max() <= {"f64": 1e-10, "f32": 1e-5}[storage] * U


def test_adjoint_with_moving_lid_matches_reference():
    from paper_1112_0850_gb300.rollout import LBMRollout, velocity_loss
    n, tau, T = 7, 0.6, 10
    flags = _cavity(n)
    uw = np.array([0.04, 0.0, 0.0])
    rng = np.random.default_rng(42)
    m = flags == 0
    u0 = 0.01 * rng.standard_normal((3, n, n, n)) * m
    F = 1e-4 * rng.standard_normal((3, n, n, n)) * m
    ut = 0.01 * rng.standard_normal((3, n, n, n))
    lat = _lattice(n, n, n, tau, flags=flags, storage="f64")
    lat.set_wall_velocity(uw)
    u0t = torch.tensor(u0, device="cuda", requires_grad=True)
    Ft = torch.tensor(F, device="cuda", requires_grad=True)
    u = LBMRollout.apply(u0t, Ft, lat, T, 4, None)
    L = velocity_loss(u, torch.tensor(ut, device="cuda"), torch.tensor(m, device="cuda"))
    gu, gF = torch.autograd.grad(L, (u0t, Ft))
    lat.close()
    Lr, gur, gFr = oadj.gradients(u0, F, tau, T, ut, flags, uw)
    assert abs(L.item() - Lr) <= 1e-12 * Lr
    assert rel_l2(gu.cpu().numpy(), gur, m) <= 1e-10
    assert rel_l2(gF.cpu().numpy(), gFr, m) <= 1e-10


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_wall_velocity_change_rebuilds_step_graphs(storage):
    n = 10
    flags = _cavity(n)
    a = _lattice(n, n, n, 0.6, flags=flags, storage=storage)
    b = _lattice(n, n, n, 0.6, flags=flags, storage=storage)
    for lat in (a, b):
        lat.set_wall_velocity((0.03, 0.0, 0.0))
        lat.init_equilibrium(lat.zeros(3))
    a.step(40)
    for _ in range(40):
        b.step(1)
    for lat in (a, b):
        lat.set_wall_velocity((0.0, 0.0, -0.02))
    a.step(40)
    for _ in range(40):
        b.step(1)
    assert torch.equal(a.get_state(), b.get_state())
    a.close()
    b.close()


@pytest.mark.parametrize("pattern", ["pull", "aa"])
@pytest.mark.parametrize("storage", STORAGES)
def test_moving_wall_sharing_a_pair_with_fluid(storage, pattern):
    """A moving wall plane at odd x (each wall cell is paired with a fluid
    cell in the step kernels' two-cell threads) and a resting plane, walls
    sliding tangentially; against the oracle."""
    nx, ny, nz, tau, T = 9, 6, 5, 0.7, 40
    flags = np.zeros((nz, ny, nx), np.uint8)
    flags[:, :, 3] = 2
    flags[:, :, 7] = 1
    uw = np.array([0.0, 0.03, 0.01])
    rng = np.random.default_rng(44)
    u0 = 0.01 * rng.standard_normal((3, nz, ny, nx)) * (flags == 0)
    lat = _lattice(nx, ny, nz, tau, flags=flags, storage=storage, pattern=pattern)
    lat.set_wall_velocity(uw)
    lat.init_equilibrium(torch.tensor(u0, dtype=REAL[storage]).cuda())
    lat.step(T)
    _, u = lat.macros()
    lat.close()
    f = oracle.run(oracle.init_equilibrium(as_input(u0, storage), flags=flags), tau, T, flags=flags,
                   u_wall=uw if storage == "f64" else np.float32(uw).astype(np.float64))
    _, u_o = oracle.macros(f, flags=flags)
    m = fluid_mask(flags, (nz, ny, nx))
    assert rel_l2(u.double().cpu().numpy(), u_o, m) <= TOL_U[storage]
    assert np.abs(u_o[1][m]).max() > 1e-3  # the wall drives the flow
