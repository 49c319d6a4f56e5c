"""The AA pattern (one lattice updated in place, alternating a local and a
neighbour step) on the GPU.

The two-grid update and the AA update gather the same values and collide them
with the same code, so without moving walls the two give the same bits in
every storage format, after even and odd step counts (the AA lattice is then
in its natural or its swapped layout). With moving walls the two round the
wall term at different points, so they are held to the oracle instead.
"""
import numpy as np
import pytest
import torch

import lbm_inputs
from gpu_helpers import REAL, STORAGES, TOL_U, as_input, ensure_built, fluid_mask, oracle_run, rel_l2
from test_parity_gpu import CASES, _case

pytestmark = pytest.mark.gpu


def _lattice(*a, **k):
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    return Lattice(*a, **k)


def _run(pattern, storage, case, steps, flags_override=None):
    u0, rho0, tau, _, flags, F, Ffield = _case(case)
    if flags_override is not None:
        flags = flags_override
    nz, ny, nx = u0.shape[1:]
    real = REAL[storage]
    lat = _lattice(nx, ny, nz, tau, flags=flags, force=F, storage=storage, pattern=pattern)
    if Ffield is not None:
        lat.set_force_field(torch.as_tensor(Ffield, dtype=real).cuda())
    lat.init_equilibrium(torch.as_tensor(u0, dtype=real).cuda(),
                         None if rho0 is None else torch.as_tensor(rho0, dtype=real).cuda())
    lat.step(steps)
    state = lat.get_state()
    rho, u = lat.macros()
    sums = lat.reduce()
    torch.cuda.synchronize()
    lat.close()
    return state, rho, u, sums


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("case", CASES)
def test_aa_matches_two_grid_bitwise(storage, case):
    for steps in (7, 8):
        sa, ra, ua, ma = _run("aa", storage, case, steps)
        sp, rp, up, mp = _run("pull", storage, case, steps)
        assert torch.equal(sa, sp), (case, steps)
        assert torch.equal(ra, rp) and torch.equal(ua, up), (case, steps)
        assert np.array_equal(ma, mp), (case, steps)


@pytest.mark.parametrize("storage", STORAGES)
def test_aa_matches_oracle(storage):
    u0, rho0, tau, steps, flags, F, Ffield = _case("channel_64x20x18")
    steps = 21  # ends in the swapped layout
    _, rho, u, _ = _run("aa", storage, "channel_64x20x18", steps)
    rho_o, u_o, _ = oracle_run(as_input(u0, storage), tau, steps, flags, as_input(F, storage),
                               as_input(rho0, storage))
    m = fluid_mask(flags, u0.shape[1:])
    assert rel_l2(u.double().cpu().numpy(), u_o, m) <= TOL_U[storage]


def _cavity(n):
    flags = np.ones((n, n, n), np.uint8)
    flags[1:-1, 1:-1, 1:-1] = 0
    flags[1:-1, n - 1, 1:-1] = 2
    return flags


@pytest.mark.parametrize("storage", STORAGES)
def test_aa_lid_driven_cavity_matches_oracle(storage):
    import oracle
    n, tau, T = 12, 0.6, 61
    uw = np.array([0.05, 0.0, 0.01])
    flags = _cavity(n)
    rng = np.random.default_rng(43)
    u0 = 0.005 * rng.standard_normal((3, n, n, n)) * (flags == 0)
    real = REAL[storage]
    lat = _lattice(n, n, n, tau, flags=flags, storage=storage, pattern="aa")
    lat.set_wall_velocity(uw)
    lat.init_equilibrium(torch.tensor(u0, dtype=real).cuda())
    lat.step(T)
    _, u = lat.macros()
    lat.close()
    f = oracle.run(oracle.init_equilibrium(as_input(u0, storage), flags=flags), tau, T, flags=flags,
                   u_wall=uw if storage == "f64" else np.float32(uw).astype(np.float64))
    _, u_o = oracle.macros(f, flags=flags)
    assert rel_l2(u.double().cpu().numpy(), u_o, fluid_mask(flags, (n, n, n))) <= TOL_U[storage]


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s"])
def test_aa_state_round_trip_in_swapped_layout(storage):
    u0, rho0, tau, _, flags, F, _ = _case("flags_33x7x5")
    nz, ny, nx = u0.shape[1:]
    real = REAL[storage]
    a = _lattice(nx, ny, nz, tau, flags=flags, force=F, storage=storage, pattern="aa")
    a.init_equilibrium(torch.as_tensor(u0, dtype=real).cuda(), torch.as_tensor(rho0, dtype=real).cuda())
    a.step(5)  # odd: swapped layout
    s = a.get_state()
    b = _lattice(nx, ny, nz, tau, flags=flags, force=F, storage=storage, pattern="aa")
    b.set_state(s)
    assert torch.equal(b.get_state(), s)
    a.step(6)
    b.step(6)
    assert torch.equal(a.get_state(), b.get_state())
    a.close()
    b.close()


def test_aa_graph_replay_matches_single_launches():
    u0, rho0, tau, _, flags, F, _ = _case("channel_64x20x18")
    nz, ny, nx = u0.shape[1:]
    out = []
    for chunks in ([69], [1] * 69):
        lat = _lattice(nx, ny, nz, tau, flags=flags, force=F, storage="f32", pattern="aa")
        lat.init_equilibrium(torch.as_tensor(u0, dtype=torch.float32).cuda())
        for n in chunks:
            lat.step(n)
        out.append(lat.get_state())
        lat.close()
    assert torch.equal(out[0], out[1])


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_aa_adjoint_matches_two_grid(storage):
    from paper_1112_0850_gb300.rollout import LBMRollout, velocity_loss
    shape = (6, 7, 9)
    nz, ny, nx = shape
    rng = np.random.default_rng(51)
    flags = lbm_inputs.random_flags(nx, ny, nz, 0.15, 51)
    m = fluid_mask(flags, shape)
    u0 = 0.02 * rng.standard_normal((3,) + shape) * m
    F = 1e-4 * rng.standard_normal((3,) + shape) * m
    ut = 0.02 * rng.standard_normal((3,) + shape)
    real = REAL[storage]
    grads = []
    for pattern in ("pull", "aa"):
        lat = _lattice(nx, ny, nz, 0.6, flags=flags, storage=storage, pattern=pattern)
        u0t = torch.tensor(u0, dtype=real, device="cuda", requires_grad=True)
        Ft = torch.tensor(F, dtype=real, device="cuda", requires_grad=True)
        u = LBMRollout.apply(u0t, Ft, lat, 11, 4)
        L = velocity_loss(u, torch.tensor(ut, dtype=real, device="cuda"), torch.tensor(m, device="cuda"))
        grads.append(torch.autograd.grad(L, (u0t, Ft)))
        lat.close()
    assert torch.equal(grads[0][0], grads[1][0]) and torch.equal(grads[0][1], grads[1][1])


def test_aa_holds_one_lattice():
    n = 192
    torch.cuda.synchronize()
    used = {}
    for pattern in ("pull", "aa"):
        free0 = torch.cuda.mem_get_info()[0]
        lat = _lattice(n, n, n, 0.6, storage="f32", pattern=pattern)
        used[pattern] = free0 - torch.cuda.mem_get_info()[0]
        assert lat.info.pattern == (1 if pattern == "aa" else 0)
        lat.close()
    lattice = 19 * n * n * n * 4
    assert used["aa"] < 1.25 * lattice < 1.9 * lattice < used["pull"]
