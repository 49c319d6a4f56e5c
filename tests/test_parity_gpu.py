"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle,
element by element on the same seeded inputs, for every storage format.

Sizes span several x tiles with a ragged tail, random obstacle flags, uniform
and per-cell forces, and the degenerate lattices (1 cell, one-cell-thin axes).
Velocity tolerances are the method's targets: FP64 storage 1e-12, FP32 1e-5,
16-bit shifted storage 1e-3 (relative L2 over fluid cells).
"""
import zlib

import numpy as np
import pytest
import torch

import lbm_inputs
import oracle
from gpu_helpers import (EMUL, REAL, STORAGES, TOL_U, as_input, ensure_built, fluid_mask, gpu_run, oracle_run,
                         rel_l2, shifted)

pytestmark = pytest.mark.gpu

TOL_RHO = {"f64": 1e-13, "f32": 1e-6, "f16s": 1e-4, "bf16s": 1e-4}
TOL_STATE = {"f64": 1e-14, "f32": 1e-6, "f16s": 1e-3, "bf16s": 1e-3}


def _case(name):
    """(u0, rho0, tau, steps, flags, F, Ffield) for a named parity case."""
    S = lbm_inputs.seed_for(0)
    if name == "shear32":  # periodic 32^3 shear wave with noise, tau 0.6, 100 steps
        return lbm_inputs.shear_wave(32, seed=S), None, 0.6, 100, None, None, None
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    dims = {"flags_8x6x5": (8, 6, 5), "flags_33x7x5": (33, 7, 5), "ragged_300x5x4": (300, 5, 4),
            "channel_64x20x18": (64, 20, 18), "one_cell": (1, 1, 1), "thin_x": (1, 7, 5),
            "thin_y": (9, 1, 4), "thin_z": (40, 3, 1), "field_10x9x8": (10, 9, 8)}[name]
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    u0 = 0.02 * rng.standard_normal((3,) + shape)
    rho0 = 1.0 + 0.01 * rng.standard_normal(shape)
    flags = None
    if name.startswith("flags") or name in ("ragged_300x5x4", "field_10x9x8", "thin_x"):
        flags = lbm_inputs.random_flags(nx, ny, nz, 0.2, S + 7)
    if name == "channel_64x20x18":
        flags = lbm_inputs.channel_flags(nx, ny, nz, 0.1, S + 1)
    F = np.array([1e-5, -2e-5, 3e-5])
    Ffield = None
    if name == "field_10x9x8":
        F = None
        Ffield = lbm_inputs.force_field(shape, 1e-4, S + 3)
    return u0, rho0, 0.55, 20, flags, F, Ffield


CASES = ["shear32", "flags_8x6x5", "flags_33x7x5", "ragged_300x5x4", "channel_64x20x18", "one_cell", "thin_x",
         "thin_y", "thin_z", "field_10x9x8"]


@pytest.fixture(scope="module")
def oracle_results():
    cache = {}

    def get(name, storage):
        prec = "f64" if storage == "f64" else "f32"
        key = (name, prec)
        if key not in cache:
            u0, rho0, tau, steps, flags, F, Ff = _case(name)
            Fi = None if F is None else as_input(F, storage)
            cache[key] = oracle_run(as_input(u0, storage), tau, steps, flags, Fi, as_input(rho0, storage),
                                    as_input(Ff, storage))
        return cache[key]

    return get


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("name", CASES)
def test_velocity_density_state_match_oracle(name, storage, oracle_results):
    u0, rho0, tau, steps, flags, F, Ff = _case(name)
    rho, u, st, lat = gpu_run(storage, u0, tau, steps, flags, F, rho0, Ff)
    rho_o, u_o, f_o = oracle_results(name, storage)
    m = fluid_mask(flags, u0.shape[1:])
    err_u = rel_l2(u, u_o, m)
    assert err_u <= TOL_U[storage], (name, storage, err_u)
    assert np.abs(rho - rho_o)[m].max() <= TOL_RHO[storage]
    assert np.abs(st - shifted(f_o, flags))[:, m].max() <= TOL_STATE[storage]
    assert np.all(rho[~m] == 0) and np.all(u[:, ~m] == 0) and np.all(st[:, ~m] == 0)
    assert lat.status_word() == 0
    lat.close()


def _round_to(a, storage):
    if storage == "f32":
        return a.astype(np.float32).astype(np.float64)
    if storage == "f16s":
        return a.astype(np.float16).astype(np.float64)
    return torch.tensor(a.astype(np.float32)).to(torch.bfloat16).double().numpy()


@pytest.mark.parametrize("storage", ["f32", "f16s", "bf16s"])
@pytest.mark.parametrize("name", ["shear32", "flags_33x7x5", "field_10x9x8"])
def test_one_step_matches_rounding_emulation(name, storage):
    """From the same narrow-format state, one GPU step equals the oracle step
    followed by rounding to that format, up to one unit in the last place
    (FP32 against FP64 arithmetic before the final rounding). Over many steps
    the two accumulate independent rounding noise, so only one step is
    compared this tightly; the multi-step comparison is the tolerance test."""
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    u0, rho0, tau, steps, flags, F, Ff = _case(name)
    nz, ny, nx = u0.shape[1:]
    Fi = None if F is None else as_input(F, storage)
    Ffi = as_input(Ff, storage)
    # a state exactly representable in the format: the oracle's emulated run
    f_n = oracle.run(oracle.init_equilibrium(as_input(u0, storage), rho0=as_input(rho0, storage), flags=flags,
                                             fmt=EMUL[storage]), tau, 5, flags=flags, F=Ffi if Ffi is not None else Fi,
                     fmt=EMUL[storage])
    s_n = _round_to(shifted(f_n, flags), storage)  # exactly representable deviations
    _, w, _ = oracle.lattice()
    f_n = w[:, None, None, None] + s_n
    if flags is not None:
        f_n[:, flags != 0] = 0.0
    lat = Lattice(nx, ny, nz, tau, flags=flags, force=F, storage=storage)
    if Ff is not None:
        lat.set_force_field(torch.tensor(Ff, dtype=torch.float32).cuda())
    lat.set_state(torch.tensor(s_n).cuda())
    assert np.array_equal(lat.get_state("f64").cpu().numpy(), s_n)
    lat.step(1)
    got = lat.get_state("f64").cpu().numpy()
    want = shifted(oracle.run(f_n, tau, 1, flags=flags, F=Ffi if Ffi is not None else Fi, fmt=EMUL[storage]), flags)
    m = fluid_mask(flags, (nz, ny, nx))
    d = np.abs(got - want)[:, m]
    a = np.abs(want)[:, m]
    # FP32 collision arithmetic: sums of 19 terms no larger than the largest
    # deviation in the state, so its error stays below ~19 * 2^-24 of that
    arith = 2.0 ** -20 * np.abs(s_n).max()
    if storage == "f32":
        assert np.all(d <= arith), d.max() / arith
    else:
        if storage == "f16s":
            ulp = np.spacing(a.astype(np.float16)).astype(np.float64)
        else:
            ulp = 2.0 ** (np.floor(np.log2(np.maximum(a, 1e-38))) - 7)
        # one rounding to the format, possibly on the other side of a
        # rounding boundary because of the FP32 arithmetic before it
        assert np.all(d <= 1.01 * ulp + arith), (d / (ulp + arith)).max()
        assert (d == 0).mean() > 0.9  # nearly every value is rounded identically
    lat.close()


@pytest.mark.parametrize("storage", STORAGES)
def test_init_state_is_equilibrium(storage):
    u0, rho0, tau, steps, flags, F, Ff = _case("flags_33x7x5")
    _, _, st, lat = gpu_run(storage, u0, tau, 0, flags, F, rho0)
    f0 = oracle.init_equilibrium(as_input(u0, storage), rho0=as_input(rho0, storage), flags=flags)
    s0 = shifted(f0, flags)
    m = fluid_mask(flags, u0.shape[1:])
    # a few units in the last place of the stored format (|s| < 0.02); for
    # FP64 the oracle's own f - w near w_0 = 1/3 is exact only to ~ulp(1/3)
    tol = {"f64": 1e-16, "f32": 4e-9, "f16s": 1e-5, "bf16s": 1e-4}[storage]
    assert np.abs(st - s0)[:, m].max() <= tol
    lat.close()


@pytest.mark.parametrize("storage", STORAGES)
def test_reduction_matches_oracle_sums(storage, oracle_results):
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    for name in ("flags_33x7x5", "ragged_300x5x4", "field_10x9x8"):
        u0, rho0, tau, steps, flags, F, Ff = _case(name)
        _, _, st, lat = gpu_run(storage, u0, tau, steps, flags, F, rho0, Ff)
        got = lat.reduce()
        _, _, f_o = oracle_results(name, storage)
        want = oracle.sums(f_o, flags=flags, F=as_input(Ff if Ff is not None else F, storage))
        tol = {"f64": 1e-13, "f32": 1e-6, "f16s": 1e-4, "bf16s": 1e-4}[storage]
        assert abs(got[0] - want[0]) <= tol * abs(want[0])
        assert np.abs(got[1:] - want[1:]).max() <= tol * abs(want[0]) * 0.1 + 1e-12
        # deterministic: same bits on repeat
        assert np.array_equal(got, lat.reduce())
        lat.close()
    assert Lattice is not None


@pytest.mark.parametrize("storage", STORAGES)
def test_rest_state_stays_bitwise_zero_with_walls(storage):
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    nx, ny, nz = 40, 9, 7
    flags = lbm_inputs.channel_flags(nx, ny, nz, 0.1, 5)
    lat = Lattice(nx, ny, nz, 0.6, flags=flags, storage=storage)
    lat.init_equilibrium(lat.zeros(3))
    lat.step(50)
    st = lat.get_state()
    assert torch.count_nonzero(st.float()).item() == 0
    lat.close()


@pytest.mark.parametrize("storage", STORAGES)
def test_state_round_trip_and_conversion(storage):
    """get_state -> set_state is exact in the context's own format; loading an
    FP64 state into a narrow format rounds each deviation to nearest even."""
    u0, rho0, tau, steps, flags, F, Ff = _case("flags_33x7x5")
    _, _, _, lat = gpu_run(storage, u0, tau, 5, flags, F, rho0)
    a = lat.get_state()
    lat.set_state(a)
    b = lat.get_state()
    assert torch.equal(a, b)
    rng = np.random.default_rng(3)
    s = 0.01 * rng.standard_normal((19,) + u0.shape[1:])
    m = fluid_mask(flags, u0.shape[1:])
    s[:, ~m] = 0.0
    lat.set_state(torch.tensor(s, dtype=torch.float64).cuda())
    got = lat.get_state("f64").cpu().numpy()
    np_t = {"f64": np.float64, "f32": np.float32, "f16s": np.float16}.get(storage)
    if np_t is not None:
        want = s.astype(np_t).astype(np.float64)
    else:
        want = torch.tensor(s, dtype=torch.float64).to(torch.bfloat16).double().numpy()
        # torch rounds float64 -> bfloat16 directly or through float32; allow the
        # double-rounding corner on exact ties only
        diff = np.abs(got - want)[:, m]
        assert (diff > 0).mean() < 1e-3
        return lat.close()
    assert np.array_equal(got[:, m], want[:, m])
    lat.close()


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_host_buffers_give_same_result(storage):
    """Host (CPU) arrays through the same calls give the same bits as device arrays."""
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    u0, rho0, tau, steps, flags, F, Ff = _case("flags_8x6x5")
    nz, ny, nx = u0.shape[1:]
    real = REAL[storage]
    out = []
    for dev in ("cuda", "cpu"):
        lat = Lattice(nx, ny, nz, tau, flags=flags, force=F, storage=storage)
        lat.init_equilibrium(torch.tensor(u0, dtype=real, device=dev), torch.tensor(rho0, dtype=real, device=dev))
        lat.step(7)
        u = torch.zeros((3, nz, ny, nx), dtype=real, device=dev)
        rho = torch.zeros((nz, ny, nx), dtype=real, device=dev)
        lat.macros(rho, u)
        torch.cuda.synchronize()
        out.append((rho.cpu(), u.cpu()))
        lat.close()
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


@pytest.mark.parametrize("storage", STORAGES)
def test_tape_records_pre_collision_moments(storage):
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    u0, rho0, tau, steps, flags, F, Ff = _case("flags_33x7x5")
    nz, ny, nx = u0.shape[1:]
    real = REAL[storage]
    n = 4
    a = Lattice(nx, ny, nz, tau, flags=flags, force=F, storage=storage)
    b = Lattice(nx, ny, nz, tau, flags=flags, force=F, storage=storage)
    for lat in (a, b):
        lat.init_equilibrium(torch.tensor(u0, dtype=real).cuda(), torch.tensor(rho0, dtype=real).cuda())
    tape = a.new_tape(n)
    a.step_record(n, tape)
    pitch = a.info.pitch
    T = tape.view(real).view(n, 4, nz, ny, pitch)[..., :nx]
    m = torch.tensor(fluid_mask(flags, (nz, ny, nx))).cuda()
    for k in range(n):
        rho, u = b.macros()
        assert torch.equal(T[k, 0][m], rho[m])
        assert torch.equal(T[k, 1:][:, m], u[:, m])
        b.step(1)
    assert torch.equal(a.get_state(), b.get_state())
    a.close()
    b.close()


def test_status_word_flags_nonphysical_density():
    """A state with negative density sets the divergence bit; the kernels keep
    running in bounds (addresses never depend on data) and nothing traps."""
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    lat = Lattice(8, 6, 5, 0.6, storage="f32")
    e, w, _ = oracle.lattice()
    bad = torch.tensor(np.broadcast_to(-2.0 * w[:, None, None, None], (19, 5, 6, 8)).copy(),
                       dtype=torch.float32).cuda()
    lat.set_state(bad)
    assert lat.status_word() == 0
    lat.step(1)
    assert lat.status_word(clear=True) & 1
    assert lat.status_word() == 0
    lat.close()


def test_create_rejects_bad_arguments():
    from paper_1112_0850_gb300.capi import LBMError
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    for args in [(0, 4, 4, 0.6), (4, 4, 4, 0.5), (4, 4, 70000, 0.6)]:
        with pytest.raises(LBMError):
            Lattice(*args)
    with pytest.raises(LBMError):
        Lattice(4, 4, 4, 0.6, storage=7)
    for kw in [{"pattern": 2}, {"model": 5}, {"row_align": 3}, {"row_align": 8192}, {"row_align": 4, "storage": "f64"}]:
        with pytest.raises(LBMError):
            Lattice(4, 4, 4, 0.6, **kw)


@pytest.mark.parametrize("storage", STORAGES)
def test_padded_rows_match_oracle(storage, oracle_results):
    """Rows padded to 128 bytes (the paper's padding) give the same results as
    the default layout (rows padded only to a pair of cells)."""
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    name = "ragged_300x5x4"
    u0, rho0, tau, steps, flags, F, Ff = _case(name)
    nz, ny, nx = u0.shape[1:]
    real = REAL[storage]
    es = {"f64": 8, "f32": 4, "f16s": 2, "bf16s": 2}[storage]
    lat = Lattice(nx, ny, nz, tau, flags=flags, force=F, storage=storage, row_align=128)
    assert lat.info.pitch % (128 // es) == 0 and lat.info.pitch > nx
    lat.init_equilibrium(torch.tensor(u0, dtype=real).cuda(), torch.tensor(rho0, dtype=real).cuda())
    lat.step(steps)
    rho, u = lat.macros()
    _, u_o, _ = oracle_results(name, storage)
    m = fluid_mask(flags, u0.shape[1:])
    assert rel_l2(u.double().cpu().numpy(), u_o, m) <= TOL_U[storage]
    lat.close()


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_graph_replay_matches_single_launches(storage):
    """lbm_step(n) replays captured 32-step graphs; the result equals n single
    steps bit for bit, also after the uniform force changes (graphs rebuilt)."""
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    u0, rho0, tau, steps, flags, F, Ff = _case("flags_33x7x5")
    nz, ny, nx = u0.shape[1:]
    real = REAL[storage]
    lats = []
    for _ in range(2):
        lat = Lattice(nx, ny, nz, tau, flags=flags, force=F, storage=storage)
        lat.init_equilibrium(torch.tensor(u0, dtype=real).cuda(), torch.tensor(rho0, dtype=real).cuda())
        lats.append(lat)
    a, b = lats
    a.step(70)  # 2 graph replays + 6 single steps
    for _ in range(70):
        b.step(1)
    assert torch.equal(a.get_state(), b.get_state())
    F2 = (-3e-5, 1e-5, 2e-5)
    a.set_uniform_force(F2)
    b.set_uniform_force(F2)
    a.step(33)
    for _ in range(33):
        b.step(1)
    assert torch.equal(a.get_state(), b.get_state())
    a.close()
    b.close()


def test_step_timed_is_step_with_a_device_time():
    """lbm_step_timed(n) leaves the state lbm_step(n) leaves and returns a
    positive device time that grows with n; a missing output pointer and a
    negative count are refused."""
    import ctypes
    from paper_1112_0850_gb300 import capi
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    u0, rho0, tau, steps, flags, F, Ff = _case("channel_64x20x18")
    nz, ny, nx = u0.shape[1:]
    lats = []
    for _ in range(2):
        lat = Lattice(nx, ny, nz, tau, flags=flags, force=F, storage="f32")
        lat.init_equilibrium(torch.tensor(u0, dtype=torch.float32).cuda(),
                             torch.tensor(rho0, dtype=torch.float32).cuda())
        lats.append(lat)
    a, b = lats
    t_first = a.step_timed(64)  # captures the step graph
    t_short = a.step_timed(32)
    t_long = a.step_timed(320)
    b.step(64 + 32 + 320)
    assert torch.equal(a.get_state(), b.get_state())
    assert t_first > 0 and t_short > 0 and t_long > 2 * t_short, (t_first, t_short, t_long)
    assert a.step_timed(0) >= 0
    L = capi.lib()
    assert L.lbm_step_timed(a.handle, 4, None) == 1  # LBM_ERR_ARG
    ms = ctypes.c_float(0)
    assert L.lbm_step_timed(a.handle, -1, ctypes.byref(ms)) == 1
    a.close()
    b.close()


@pytest.mark.parametrize("storage,pattern", [("f32", "pull"), ("f16s", "pull"), ("bf16m", "pull"), ("f32", "aa"),
                                             ("f16s", "aa")])
def test_step_counts_replay_graphs_bit_for_bit(storage, pattern):
    """lbm_step(n) replays a graph of 32-step blocks and one of the remaining
    2..31 steps, each from either lattice, captured on first use or ahead by
    lbm_step_prepare; every count gives the bits of the same steps launched
    one by one."""
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    u0, rho0, tau, steps, flags, F, Ff = _case("flags_33x7x5")
    nz, ny, nx = u0.shape[1:]
    real = REAL[storage]
    lats = []
    for _ in range(2):
        lat = Lattice(nx, ny, nz, tau, flags=flags, force=F, storage=storage, pattern=pattern)
        lat.init_equilibrium(torch.tensor(u0, dtype=real).cuda(), torch.tensor(rho0, dtype=real).cuda())
        lats.append(lat)
    a, b = lats
    a.prepare_steps(5)
    a.prepare_steps(37)
    a.prepare_steps(0)
    counts = [2, 3, 5, 31, 33, 64, 7, 4, 37, 1]
    for n in counts:
        a.step(n)
    for _ in range(sum(counts)):
        b.step(1)
    assert torch.equal(a.get_state(), b.get_state())
    assert a.info.steps_done == b.info.steps_done == sum(counts)
    a.close()
    b.close()
