"""z-slab decomposition on one GPU: a lattice split into 1-4 slabs, each a
context with two ghost planes, exchanging the five crossing populations per
face through lbm_halo_pack / lbm_halo_unpack before every step. The interior
planes must evolve bit for bit as in the unsplit lattice, for every storage
format, with walls, obstacles, a uniform or per-cell force and moving walls
(solid ghost cells keep their own bounce-back values)."""
import numpy as np
import pytest
import torch

import lbm_inputs
from gpu_helpers import REAL, STORAGES, ensure_built

pytestmark = pytest.mark.gpu


def _fields(nx, ny, nz, seed, flags_kind):
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx)
    u0 = 0.02 * rng.standard_normal((3,) + shape)
    rho0 = 1.0 + 0.01 * rng.standard_normal(shape)
    flags = None
    if flags_kind == "channel":
        flags = lbm_inputs.channel_flags(nx, ny, nz, 0.1, seed)
    elif flags_kind == "random":
        flags = lbm_inputs.random_flags(nx, ny, nz, 0.2, seed)
    elif flags_kind == "moving":
        flags = lbm_inputs.random_flags(nx, ny, nz, 0.15, seed)
        flags[:, 0, :] = 1
        flags[:, ny - 1, :] = 2
        flags[3, :, :] = np.where(flags[3] == 0, 2, flags[3])  # a moving plane across z
    if flags is not None:
        u0 *= flags == 0
    return u0, rho0, flags


def _pair(storage, k, nx=21, ny=10, nz=14, flags_kind="channel", force="uniform", u_wall=None, steps=9, seed=5,
          totals=False, overlap=False):
    from paper_1112_0850_gb300.lattice import Lattice
    from paper_1112_0850_gb300.slabs import SlabSet
    ensure_built()
    u0, rho0, flags = _fields(nx, ny, nz, seed, flags_kind)
    real = REAL[storage]
    F = (2e-5, -1e-5, 3e-5) if force == "uniform" else None
    Ff = None
    if force == "field":
        Ff = torch.as_tensor(lbm_inputs.force_field((nz, ny, nx), 1e-4, seed + 1), dtype=real).cuda()
    tau = 0.56
    whole = Lattice(nx, ny, nz, tau, flags=flags, force=F, storage=storage)
    slabs = SlabSet(nx, ny, nz, tau, k, flags=flags, force=F, storage=storage, overlap=overlap)
    u0t, rho0t = torch.as_tensor(u0, dtype=real).cuda(), torch.as_tensor(rho0, dtype=real).cuda()
    for lat in (whole, slabs):
        if Ff is not None:
            lat.set_force_field(Ff)
        if u_wall is not None:
            lat.set_wall_velocity(u_wall)
        lat.init_equilibrium(u0t, rho0t)
    whole.step(steps)
    slabs.step(steps)
    a, b = whole.get_state(), slabs.get_state()
    sa, sb = whole.status_word(), slabs.status_word()
    ta, tb = (whole.reduce(), slabs.totals()) if totals else (None, None)
    whole.close()
    slabs.close()
    return (a, b, sa, sb, ta, tb) if totals else (a, b, sa, sb)


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_slabs_equal_unsplit_channel(storage, k):
    a, b, sa, sb = _pair(storage, k)
    assert torch.equal(a, b), (storage, k)
    assert sa == sb == 0


@pytest.mark.parametrize("storage", STORAGES)
def test_slabs_equal_unsplit_random_obstacles_force_field(storage):
    a, b, _, _ = _pair(storage, 3, nx=17, ny=9, nz=11, flags_kind="random", force="field")
    assert torch.equal(a, b)


@pytest.mark.parametrize("storage", STORAGES)
def test_slabs_equal_unsplit_periodic(storage):
    # no flags: every ghost cell is fluid and takes the neighbour's values
    a, b, _, _ = _pair(storage, 4, nx=16, ny=8, nz=12, flags_kind=None, force=None)
    assert torch.equal(a, b)


@pytest.mark.parametrize("storage", STORAGES)
def test_slabs_equal_unsplit_moving_walls(storage):
    a, b, _, _ = _pair(storage, 3, nx=19, ny=9, nz=12, flags_kind="moving", u_wall=(0.03, 0.0, -0.01))
    assert torch.equal(a, b)


def test_slab_of_one_interior_plane():
    # six slabs of one interior plane each: both ghosts border the same plane
    a, b, _, _ = _pair("f32", 6, nx=12, ny=7, nz=6)
    assert torch.equal(a, b)


def test_halo_pack_layout_and_host_buffer():
    """The packed buffer holds the five crossing populations of the boundary
    plane, [5][ny][pitch] in increasing direction order, and a host buffer
    (staged by the library) receives the same bytes. The slot P_i(x) is what
    cell x + e_i gathers, so where x and x + e_i are both fluid it equals the
    state read at x + e_i."""
    from paper_1112_0850_gb300.lattice import Lattice, lattice_table
    ensure_built()
    nx, ny, nz = 13, 6, 7
    u0, rho0, flags = _fields(nx, ny, nz, 9, "random")
    lat = Lattice(nx, ny, nz, 0.6, flags=flags, storage="f32")
    lat.init_equilibrium(torch.as_tensor(u0, dtype=torch.float32).cuda(),
                         torch.as_tensor(rho0, dtype=torch.float32).cuda())
    lat.step(3)
    state = lat.get_state()
    fluid = torch.as_tensor(flags == 0, device="cuda")
    e = np.asarray(lattice_table()[0])
    pitch = lat.info.pitch
    for side, z, ez in ((0, 1, -1), (1, nz - 2, 1)):
        buf = lat.new_halo()
        lat.halo_pack(side, buf)
        host = torch.empty_like(buf, device="cpu")
        lat.halo_pack(side, host)
        assert torch.equal(buf.cpu(), host)
        dirs = [i for i in range(19) if e[i][2] == ez]
        assert len(dirs) == 5
        got = buf.view(5, ny, pitch)[:, :, :nx]
        for k, i in enumerate(dirs):
            sh = (-int(e[i][1]), -int(e[i][0]))  # [y][x] -> value at (y + e_y, x + e_x)
            want = torch.roll(state[i, z + ez], shifts=sh, dims=(0, 1))
            m = fluid[z] & torch.roll(fluid[z + ez], shifts=sh, dims=(0, 1))
            assert int(m.sum()) > 0
            assert torch.equal(got[k][m], want[m]), (side, i)
    lat.close()


def test_halo_argument_errors():
    from paper_1112_0850_gb300.capi import LBMError
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    lat = Lattice(8, 5, 6, 0.6, storage="f32")
    buf = lat.new_halo()
    assert buf.numel() == 5 * 5 * lat.info.pitch
    with pytest.raises(LBMError):
        lat.halo_pack(2, buf)
    with pytest.raises(LBMError):
        lat.halo_unpack(-1, buf)
    lat.close()
    thin = Lattice(8, 5, 2, 0.6, storage="f32")
    with pytest.raises(LBMError):
        thin.halo_pack(0, thin.new_halo())
    thin.close()
    aa = Lattice(8, 5, 6, 0.6, storage="f32", pattern="aa")
    with pytest.raises(LBMError, match="UNSUPPORTED|pull"):
        aa.halo_pack(0, aa.new_halo())
    aa.close()


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("k,flags_kind,force", [(2, "channel", "uniform"), (3, "random", "field"),
                                                (4, None, None)])
def test_slab_totals_equal_unsplit(storage, k, flags_kind, force):
    """Mass and momentum of a split run: the slabs' interior-plane totals
    (lbm_reduce_planes) add up to the unsplit lattice's lbm_reduce totals, up
    to the order of the FP64 sums (the per-cell moments are the same, as the
    states are bit for bit equal)."""
    a, b, _, _, ta, tb = _pair(storage, k, nx=17, ny=9, nz=12, flags_kind=flags_kind, force=force, totals=True)
    assert torch.equal(a, b)
    assert np.allclose(tb, ta, rtol=0, atol=1e-12 * ta[0]), (tb, ta)


def test_reduce_planes_match_per_plane_macros():
    """FP64 storage: the totals over planes z0 <= z < z1 equal the FP64 sums of
    lbm_macros' rho and rho u over those planes, for ranges that cut the
    lattice anywhere; the ranges of a partition add up to lbm_reduce; an empty
    range gives zeros."""
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    nx, ny, nz = 13, 9, 11
    u0, rho0, flags = _fields(nx, ny, nz, 8, "random")
    lat = Lattice(nx, ny, nz, 0.61, flags=flags, force=(1e-5, 2e-5, -3e-5), storage="f64")
    lat.init_equilibrium(torch.as_tensor(u0).cuda(), torch.as_tensor(rho0).cuda())
    lat.step(5)
    rho, u = lat.macros()
    rho, u = rho.cpu().numpy(), u.cpu().numpy()
    fluid = flags == 0
    for z0, z1 in [(0, nz), (0, 1), (4, 7), (nz - 1, nz), (1, nz - 1)]:
        got = lat.reduce(z0, z1)
        r = np.where(fluid, rho, 0.0)[z0:z1]
        want = np.array([r.sum()] + [(r * u[a, z0:z1]).sum() for a in range(3)])
        assert np.allclose(got, want, rtol=0, atol=1e-12 * max(want[0], 1.0)), (z0, z1, got, want)
    parts = lat.reduce(0, 3) + lat.reduce(3, 8) + lat.reduce(8, nz)
    full = lat.reduce()
    assert np.allclose(parts, full, rtol=0, atol=1e-12 * full[0])
    assert np.array_equal(lat.reduce(5, 5), np.zeros(4))
    lat.close()


def test_reduce_planes_argument_errors():
    from paper_1112_0850_gb300.capi import LBMError
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    lat = Lattice(8, 5, 6, 0.6, storage="f32")
    for z0, z1 in [(-1, 3), (2, 7), (4, 3)]:
        with pytest.raises(LBMError):
            lat.reduce(z0, z1)
    lat.close()


def _adjoint_pair(storage, k, nx=15, ny=9, nz=12, flags_kind="channel", force="uniform", steps=7, seed=9):
    """dL/du0 and dL/dF of the unsplit lattice and of k slabs, for the loss
    sum(g_u . u_T + g_rho rho_T) with random g at the fluid cells."""
    from paper_1112_0850_gb300.lattice import Lattice
    from paper_1112_0850_gb300.slabs import SlabSet
    ensure_built()
    u0, rho0, flags = _fields(nx, ny, nz, seed, flags_kind)
    real = REAL[storage]
    rng = np.random.default_rng(seed + 2)
    fluid = np.ones((nz, ny, nx)) if flags is None else (flags == 0)
    g_u = torch.as_tensor(rng.standard_normal((3, nz, ny, nx)) * fluid, dtype=real).cuda()
    g_rho = torch.as_tensor(rng.standard_normal((nz, ny, nx)) * fluid, dtype=real).cuda()
    F = (2e-5, -1e-5, 3e-5) if force == "uniform" else None
    Ff = None
    if force == "field":
        Ff = torch.as_tensor(lbm_inputs.force_field((nz, ny, nx), 1e-4, seed + 1), dtype=real).cuda()
    u0t, rho0t = torch.as_tensor(u0, dtype=real).cuda(), torch.as_tensor(rho0, dtype=real).cuda()
    tau = 0.57
    whole = Lattice(nx, ny, nz, tau, flags=flags, force=F, storage=storage)
    slabs = SlabSet(nx, ny, nz, tau, k, flags=flags, force=F, storage=storage)
    for lat in (whole, slabs):
        if Ff is not None:
            lat.set_force_field(Ff)
        lat.init_equilibrium(u0t, rho0t)
    tape = whole.new_tape(steps)
    whole.step_record(steps, tape)
    gF = whole.zeros(3)
    whole.adjoint_seed(g_u, g_rho, gF)
    whole.adjoint_step(steps, tape, gF)
    gu = whole.adjoint_init_grad(u0t, rho0t)[0]
    tapes = slabs.new_tapes(steps)
    slabs.step_record(steps, tapes)
    slabs.adjoint_seed(g_u, g_rho)
    slabs.adjoint_step(steps, tapes)
    gu_s, gF_s = slabs.adjoint_init_grad(u0t, rho0t)
    whole.close()
    slabs.close()
    return gu, gF, gu_s, gF_s


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("k,flags_kind,force", [(2, "channel", "uniform"), (3, "random", "field"),
                                                (4, None, None), (6, "channel", "uniform")])
def test_slab_adjoint_equals_unsplit(storage, k, flags_kind, force):
    """The adjoint of a split run, with the reverse exchange (the e_z = +1
    adjoint populations of plane 1 down, the e_z = -1 ones of plane nz - 2
    up) before every reverse step, gives the unsplit lattice's dL/du0 and
    dL/dF bit for bit; six slabs of 12 planes are two interior planes each."""
    gu, gF, gu_s, gF_s = _adjoint_pair(storage, k, flags_kind=flags_kind, force=force)
    assert float(gu.abs().max()) > 0
    assert torch.equal(gu, gu_s)
    assert torch.equal(gF, gF_s)


def test_slab_adjoint_exchange_is_needed():
    """Without the reverse exchange the boundary planes' gradients differ (the
    test above is not passing by accident)."""
    from paper_1112_0850_gb300 import slabs as sl
    saved = sl.SlabSet.adjoint_exchange
    sl.SlabSet.adjoint_exchange = lambda self: None
    try:
        gu, _, gu_s, _ = _adjoint_pair("f64", 2)
    finally:
        sl.SlabSet.adjoint_exchange = saved
    assert not torch.equal(gu, gu_s)


def test_adjoint_halo_needs_a_seed():
    from paper_1112_0850_gb300.capi import LBMError
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    lat = Lattice(8, 5, 6, 0.6, storage="f32")
    buf = lat.new_adjoint_halo()
    assert buf.numel() == 5 * 5 * lat.info.pitch and buf.dtype == torch.float32
    with pytest.raises(LBMError, match="STATE|seed"):
        lat.adjoint_halo_pack(0, buf)
    lat.close()


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("k,nz,flags_kind,force", [(2, 14, "channel", "uniform"), (3, 11, "random", "field"),
                                                   (4, 12, None, None), (6, 12, "channel", "uniform"),
                                                   (5, 5, "channel", "uniform")])
def test_slabs_overlapped_exchange_equal_unsplit(storage, k, nz, flags_kind, force):
    """The exchange on a second stream while the interior planes update, then
    planes 1 and nz - 2: still the unsplit lattice bit for bit, down to slabs
    of two and of one interior plane."""
    a, b, sa, sb = _pair(storage, k, nx=17, ny=9, nz=nz, flags_kind=flags_kind, force=force, overlap=True)
    assert torch.equal(a, b), (storage, k)
    assert sa == sb == 0


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("flags_kind", ["channel", "random", None])
def test_step_planes_equal_step(storage, flags_kind):
    """A step taken as plane windows (any order, an empty window, windows
    outside the fluid box of a walled channel) equals lbm_step bit for bit."""
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    nx, ny, nz = 19, 10, 13
    u0, rho0, flags = _fields(nx, ny, nz, 4, flags_kind)
    if flags is not None:
        flags[:2] = 1  # two solid planes: a window there is empty after clipping to the fluid box
    u0 = u0 * (flags == 0) if flags is not None else u0
    real = REAL[storage]
    F = (1e-5, -2e-5, 3e-5)
    lats = [Lattice(nx, ny, nz, 0.58, flags=flags, force=F, storage=storage) for _ in range(2)]
    for lat in lats:
        lat.init_equilibrium(torch.as_tensor(u0, dtype=real).cuda(), torch.as_tensor(rho0, dtype=real).cuda())
    windows = [[(0, 2), (7, 13), (2, 5), (5, 5), (5, 7)], [(0, 13)], [(12, 13), (0, 12)]]
    for step in range(6):
        lats[0].step(1)
        w = windows[step % len(windows)]
        for j, (z0, z1) in enumerate(w):
            lats[1].step_planes(z0, z1, j == len(w) - 1)
    a, b = lats[0].get_state(), lats[1].get_state()
    assert torch.equal(a, b)
    for lat in lats:
        lat.close()


def test_step_planes_argument_errors():
    from paper_1112_0850_gb300.capi import LBMError
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    lat = Lattice(8, 5, 6, 0.6, storage="f32")
    for z0, z1 in [(-1, 3), (2, 7), (4, 3)]:
        with pytest.raises(LBMError):
            lat.step_planes(z0, z1, True)
    lat.close()
    aa = Lattice(8, 5, 6, 0.6, storage="f32", pattern="aa")
    with pytest.raises(LBMError, match="UNSUPPORTED|pull"):
        aa.step_planes(0, 6, True)
    aa.close()


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("flags_kind", ["channel", None])
def test_step_planes_fused_totals(storage, flags_kind):
    """Totals summed inside a plane window's step equal lbm_reduce_planes over
    the same planes taken before it (to the order of the FP64 sums), on the
    host and into a device array; an empty window gives zeros; the stepped
    state still equals lbm_step's bit for bit."""
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    nx, ny, nz = 17, 9, 12
    u0, rho0, flags = _fields(nx, ny, nz, 6, flags_kind)
    real = REAL[storage]
    lats = [Lattice(nx, ny, nz, 0.6, flags=flags, force=(2e-5, 0.0, -1e-5), storage=storage) for _ in range(2)]
    for lat in lats:
        lat.init_equilibrium(torch.as_tensor(u0, dtype=real).cuda(), torch.as_tensor(rho0, dtype=real).cuda())
    dev_out = torch.zeros(4, dtype=torch.float64, device="cuda")
    for step, windows in enumerate([[(0, 5), (5, 12)], [(3, 3), (0, 3), (3, 12)], [(1, 11), (0, 1), (11, 12)]]):
        lats[0].step(1)
        for j, (z0, z1) in enumerate(windows):
            want = lats[1].reduce(z0, z1)
            last = j == len(windows) - 1
            if j % 2:
                got = lats[1].step_planes(z0, z1, last, out=dev_out).cpu().numpy()
            else:
                got = lats[1].step_planes(z0, z1, last, totals=True)
            if z0 == z1:
                assert np.array_equal(got, np.zeros(4))
            else:
                assert np.allclose(got, want, rtol=0, atol=1e-12 * max(want[0], 1.0)), (step, z0, z1, got, want)
    assert torch.equal(lats[0].get_state(), lats[1].get_state())
    for lat in lats:
        lat.close()


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("k", [2, 3])
def test_slab_step_reduce_equals_unsplit(storage, k):
    """SlabSet.step_reduce: the totals of the split lattice summed inside the
    first step (interior planes only) equal the unsplit lbm_step_reduce
    totals, and the states after the steps are equal bit for bit."""
    from paper_1112_0850_gb300.lattice import Lattice
    from paper_1112_0850_gb300.slabs import SlabSet
    ensure_built()
    nx, ny, nz = 17, 9, 12
    u0, rho0, flags = _fields(nx, ny, nz, 7, "channel")
    real = REAL[storage]
    F = (2e-5, -1e-5, 3e-5)
    whole = Lattice(nx, ny, nz, 0.57, flags=flags, force=F, storage=storage)
    slabs = SlabSet(nx, ny, nz, 0.57, k, flags=flags, force=F, storage=storage)
    u0t, rho0t = torch.as_tensor(u0, dtype=real).cuda(), torch.as_tensor(rho0, dtype=real).cuda()
    for lat in (whole, slabs):
        lat.init_equilibrium(u0t, rho0t)
    whole.step(3)
    slabs.step(3)
    ta = whole.step_reduce(4)
    tb = slabs.step_reduce(4)
    assert np.allclose(tb, ta, rtol=0, atol=1e-12 * ta[0]), (tb, ta)
    assert torch.equal(whole.get_state(), slabs.get_state())
    whole.close()
    slabs.close()


@pytest.mark.parametrize("storage", STORAGES)
def test_rank_slab_on_one_rank_equals_unsplit(storage):
    """The rank driver (RankSlab: one z-slab per rank of a torch.distributed
    group, exchange then step) on a single rank, whose exchange is the
    periodic copy of its own faces: the slab's interior equals the unsplit
    lattice bit for bit, and its all-reduced totals equal lbm_reduce's to the
    order of the FP64 sums."""
    import datetime
    import socket
    import torch.distributed as dist
    from paper_1112_0850_gb300.lattice import Lattice
    from paper_1112_0850_gb300.slabs import RankSlab
    ensure_built()
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=0, world_size=1,
                            timeout=datetime.timedelta(seconds=60))
    try:
        nx, ny, nz = 21, 10, 14
        u0, rho0, flags = _fields(nx, ny, nz, 5, "channel")
        real = REAL[storage]
        F = (2e-5, -1e-5, 3e-5)
        u0t, rho0t = torch.as_tensor(u0, dtype=real).cuda(), torch.as_tensor(rho0, dtype=real).cuda()
        whole = Lattice(nx, ny, nz, 0.56, flags=flags, force=F, storage=storage)
        rank = RankSlab(nx, ny, nz, 0.56, flags=flags, force=F, storage=storage)
        assert (rank.z0, rank.z1) == (0, nz)
        for lat in (whole, rank):
            lat.init_equilibrium(u0t, rho0t)
            lat.step(9)
        assert torch.equal(whole.get_state(), rank.interior_state())
        want, got = whole.reduce(), rank.totals()
        assert abs(got[0] - want[0]) <= 1e-12 * want[0] and np.abs(got[1:] - want[1:]).max() <= 1e-12 * want[0]
        whole.close()
        rank.close()
    finally:
        dist.destroy_process_group()
