"""z-slab decomposition on the host: the plane bookkeeping of
paper_1112_0850_gb300.slabs, and its rank-to-rank exchange run on gloo ranks
on the CPU, each rank advancing one slab with the FP64 oracle. The oracle's
state is pre-collision and a step pushes, so its slabs exchange whole planes
(all 19 populations) before every step; after T steps the joined interiors
must equal the unsplit oracle run bit for bit. A rank that stops sending makes
its neighbour's exchange return EXCHANGE_FAILED within the bounded wait
instead of blocking."""
import datetime
import os
import socket
import sys
import time

import numpy as np
import pytest

import lbm_inputs
from paper_1112_0850_gb300 import slabs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NX, NY, NZ, TAU, T = 9, 7, 10, 0.58, 6


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem():
    flags = lbm_inputs.channel_flags(NX, NY, NZ, 0.15, 41)
    rng = np.random.default_rng(41)
    u0 = 0.03 * rng.standard_normal((3, NZ, NY, NX)) * (flags == 0)
    rho0 = 1.0 + 0.02 * rng.standard_normal((NZ, NY, NX))
    F = np.array([3e-5, 1e-5, -2e-5])
    return flags, u0, rho0, F


def test_split_planes_cover_and_balance():
    for nz in (1, 2, 7, 10, 64):
        for k in range(1, min(nz, 6) + 1):
            b = slabs.split_planes(nz, k)
            assert b[0][0] == 0 and b[-1][1] == nz
            assert all(b[j][1] == b[j + 1][0] for j in range(k - 1))
            sizes = [z1 - z0 for z0, z1 in b]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slabs.split_planes(3, 4)
    with pytest.raises(ValueError):
        slabs.split_planes(3, 0)


def test_with_ghosts_wraps_periodically():
    import torch
    a = np.arange(2 * 5 * 3 * 4).reshape(2, 5, 3, 4)
    g = slabs.with_ghosts(a, 0, 2)
    assert g.shape == (2, 4, 3, 4)
    assert np.array_equal(g[:, 0], a[:, 4]) and np.array_equal(g[:, 1:3], a[:, 0:2])
    assert np.array_equal(g[:, 3], a[:, 2])
    g = slabs.with_ghosts(a, 3, 5)
    assert np.array_equal(g[:, 0], a[:, 2]) and np.array_equal(g[:, 3], a[:, 0])
    t = slabs.with_ghosts(torch.from_numpy(a), 3, 5)
    assert np.array_equal(t.numpy(), g) and t.is_contiguous()
    f = np.arange(5 * 3 * 4).reshape(5, 3, 4)  # a scalar field: z is axis 0 = -3
    assert np.array_equal(slabs.with_ghosts(f, 1, 4), f[[0, 1, 2, 3, 4]])
    assert slabs.ghost_planes(5, 0, 5) == [4, 0, 1, 2, 3, 4, 0]


@pytest.mark.parametrize("nz", [3, 4, 5, 6, 7, 12, 258])
def test_overlap_windows_cover_interior_once_and_spare_the_ghosts(nz):
    interior, boundary = slabs.overlap_windows(nz)
    planes = [z for z0, z1 in interior + boundary for z in range(z0, z1)]
    assert sorted(planes) == list(range(1, nz - 1))  # every interior plane once, no ghost
    for z0, z1 in interior:
        # pull: plane z reads planes z - 1 .. z + 1, none of them a ghost
        assert z0 - 1 >= 1 and z1 <= nz - 2
    for z0, z1 in boundary:
        assert z1 - z0 == 1 and z0 in (1, nz - 2)
    assert boundary  # the step completes after the exchange


def test_overlap_windows_need_a_slab():
    with pytest.raises(ValueError):
        slabs.overlap_windows(2)


def _rank_worker(rank, world, port, q, stop_at, skip_reduce):
    """One slab per rank: exchange whole planes, then one oracle step; at the
    end the totals of the rank's interior planes, summed over the ranks."""
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1112_0850_gb300 import slabs as sl
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    flags, u0, rho0, F = _problem()
    z0, z1 = sl.split_planes(NZ, world)[rank]
    fl = sl.with_ghosts(flags, z0, z1)
    f = oracle.init_equilibrium(sl.with_ghosts(u0, z0, z1), rho0=sl.with_ghosts(rho0, z0, z1), flags=fl)
    plane = f[:, 0].shape
    below, above = torch.zeros(plane, dtype=torch.float64), torch.zeros(plane, dtype=torch.float64)
    status, msg, t_fail = sl.EXCHANGE_OK, "", 0.0
    for step in range(T):
        if rank == 1 and step == stop_at:
            time.sleep(4.0)  # this rank stops sending (a dropped message), then leaves
            break
        t0 = time.time()
        status, msg = sl.exchange_ranks(torch.from_numpy(np.ascontiguousarray(f[:, 1])),
                                        torch.from_numpy(np.ascontiguousarray(f[:, -2])), below, above,
                                        timeout=datetime.timedelta(seconds=1.5))
        if status != sl.EXCHANGE_OK:
            t_fail = time.time() - t0
            break
        f[:, 0] = below.numpy()
        f[:, -1] = above.numpy()
        f = oracle.run(f, TAU, 1, flags=fl, F=F, threads=1)
    tot, rstatus, rmsg = None, sl.EXCHANGE_FAILED, "not reached"
    if status == sl.EXCHANGE_OK:
        if rank == 1 and skip_reduce:
            time.sleep(4.0)  # this rank never joins the all-reduce, then leaves
        else:
            tot = torch.from_numpy(np.array(oracle.sums(f[:, 1:-1], flags=fl[1:-1], F=F), dtype=np.float64))
            t0 = time.time()
            rstatus, rmsg = sl.reduce_ranks(tot, timeout=datetime.timedelta(seconds=1.5))
            t_fail = time.time() - t0
            tot = tot.numpy()
    q.put((rank, status, msg, t_fail, f[:, 1:-1] if status == sl.EXCHANGE_OK else None, tot, rstatus, rmsg))
    q.close()
    q.join_thread()  # flush the result before leaving
    os._exit(0)  # no collective teardown: a failed rank's peer may be gone


def _run_ranks(world, stop_at=-1, skip_reduce=False):
    import torch.multiprocessing as mp
    import oracle
    oracle.default()  # build once before the ranks start
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_worker, args=(r, world, port, q, stop_at, skip_reduce)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
    return res


@pytest.mark.parametrize("world", [2, 3])
def test_oracle_slabs_over_gloo_ranks_equal_unsplit(world):
    import oracle
    flags, u0, rho0, F = _problem()
    ref = oracle.run(oracle.init_equilibrium(u0, rho0=rho0, flags=flags), TAU, T, flags=flags, F=F, threads=1)
    res = _run_ranks(world)
    assert all(r[1] == slabs.EXCHANGE_OK for r in res), [r[2] for r in res]
    joined = np.concatenate([r[4] for r in res], axis=1)
    assert joined.shape == ref.shape
    assert np.array_equal(joined, ref)
    # mass and momentum: every rank holds the all-reduced sum of the slabs'
    # interior totals, equal to the unsplit totals up to the order of the sums
    want = np.array(oracle.sums(ref, flags=flags, F=F))
    assert all(r[6] == slabs.EXCHANGE_OK for r in res), [r[7] for r in res]
    for r in res:
        assert np.allclose(r[5], want, rtol=0, atol=1e-12 * want[0]), (r[5], want)
    assert all(np.array_equal(r[5], res[0][5]) for r in res)


def test_rank_that_stops_sending_fails_the_exchange_in_bounded_time():
    res = _run_ranks(2, stop_at=2)
    r0 = res[0]
    assert r0[1] == slabs.EXCHANGE_FAILED, r0[2]
    assert "rank 1" in r0[2]
    assert r0[3] < 10.0  # the 1.5 s bound, not the 60 s process-group timeout


def test_rank_that_skips_the_totals_all_reduce_fails_it_in_bounded_time():
    res = _run_ranks(2, skip_reduce=True)
    r0 = res[0]
    assert r0[1] == slabs.EXCHANGE_OK, r0[2]
    assert r0[6] == slabs.EXCHANGE_FAILED and "all-reduce" in r0[7], r0[7]
    assert r0[3] < 10.0  # the 1.5 s bound, not the 60 s process-group timeout


class _OracleSlab:
    """A rank's slab for slabs.run_ranks on the CPU: the FP64 oracle on the
    slab's planes with their ghosts. The oracle's state is pre-collision and a
    step pushes, so a face is a whole plane (all 19 populations): plane 1 goes
    down, plane nz - 2 up, into the neighbours' ghost planes."""

    def __init__(self, rank, world):
        import oracle
        from paper_1112_0850_gb300 import slabs as sl
        self.oracle = oracle
        flags, u0, rho0, self.F = _problem()
        z0, z1 = sl.split_planes(NZ, world)[rank]
        self.flags = sl.with_ghosts(flags, z0, z1)
        self.f = oracle.init_equilibrium(sl.with_ghosts(u0, z0, z1), rho0=sl.with_ghosts(rho0, z0, z1),
                                         flags=self.flags)

    def new_halo(self):
        import torch
        return torch.zeros(self.f[:, 0].shape, dtype=torch.float64)

    def halo_pack(self, side, buf):
        import torch
        buf.copy_(torch.from_numpy(np.ascontiguousarray(self.f[:, 1 if side == 0 else -2])))

    def halo_unpack(self, side, buf):
        self.f[:, 0 if side == 0 else -1] = buf.numpy()

    def step(self, n):
        self.f = self.oracle.run(self.f, TAU, n, flags=self.flags, F=self.F, threads=1)


def _driver_worker(rank, world, port, q, stop_after):
    """slabs.run_ranks, the library's rank driver, with an oracle slab per
    rank; with stop_after >= 0 rank 1 leaves after that many steps."""
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1112_0850_gb300 import slabs as sl
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    slab = _OracleSlab(rank, world)
    bufs = tuple(slab.new_halo() for _ in range(4))
    steps = stop_after if (rank == 1 and stop_after >= 0) else T
    t0 = time.time()
    status, msg = sl.run_ranks(slab, bufs, steps, timeout=datetime.timedelta(seconds=1.5))
    if rank == 1 and stop_after >= 0:
        time.sleep(4.0)  # stopped: sends nothing more, then leaves
    q.put((rank, status, msg, time.time() - t0, slab.f[:, 1:-1]))
    q.close()
    q.join_thread()
    os._exit(0)


def _run_driver(world, stop_after=-1):
    import torch.multiprocessing as mp
    import oracle
    oracle.default()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_driver_worker, args=(r, world, port, q, stop_after)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
    return res


@pytest.mark.parametrize("world", [2, 3])
def test_rank_driver_over_gloo_equals_unsplit(world):
    """The decomposed driver (exchange_halos, then a step, every step, as RankSlab runs
    it on GPUs) on gloo ranks: the joined interiors equal the unsplit oracle
    run bit for bit."""
    import oracle
    flags, u0, rho0, F = _problem()
    ref = oracle.run(oracle.init_equilibrium(u0, rho0=rho0, flags=flags), TAU, T, flags=flags, F=F, threads=1)
    res = _run_driver(world)
    assert all(r[1] == slabs.EXCHANGE_OK for r in res), [r[2] for r in res]
    assert np.array_equal(np.concatenate([r[4] for r in res], axis=1), ref)


def test_rank_driver_stops_when_a_neighbour_leaves():
    res = _run_driver(2, stop_after=2)
    assert res[0][1] == slabs.EXCHANGE_FAILED and "rank 1" in res[0][2], res[0][2]
    assert res[0][3] < 10.0  # the 1.5 s bound per wait, not the 60 s process-group timeout


def test_reduce_ranks_wants_float64():
    import torch
    with pytest.raises(TypeError):
        slabs.reduce_ranks(torch.zeros(4, dtype=torch.float32))


class _FakeLattice:
    """Stands in for Lattice in SlabSet's host wiring: a pack writes (slab,
    side, kind) into the buffer, an unpack records what it received."""
    count = 0

    def __init__(self, nx, ny, nz, tau, flags=None, force=None, **kw):
        import torch
        self.id = _FakeLattice.count
        _FakeLattice.count += 1
        self.shape = (nz, ny, nx)
        self.stream = None
        self.got = {}
        self._t = torch

    def new_halo(self):
        return self._t.zeros(3)

    new_adjoint_halo = new_halo

    def _pack(self, kind, side, buf):
        buf[:] = self._t.tensor([self.id, side, kind], dtype=buf.dtype)

    def halo_pack(self, side, buf):
        self._pack(0, side, buf)

    def adjoint_halo_pack(self, side, buf):
        self._pack(1, side, buf)

    def halo_unpack(self, side, buf):
        self.got[("f", side)] = tuple(int(v) for v in buf)

    def adjoint_halo_unpack(self, side, buf):
        self.got[("a", side)] = tuple(int(v) for v in buf)

    def close(self):
        pass


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_slab_exchange_wiring(monkeypatch, k):
    """Forward: ghost plane 0 of slab j gets the plane nz - 2 pack (side 1) of
    slab j - 1, ghost plane nz - 1 the plane 1 pack (side 0) of slab j + 1.
    Adjoint, the reverse: ghost plane nz - 1 gets slab j + 1's side-0 pack
    (its e_z = +1 populations of plane 1), ghost plane 0 slab j - 1's side-1
    pack. Periodic in z."""
    from paper_1112_0850_gb300 import lattice
    monkeypatch.setattr(lattice, "Lattice", _FakeLattice)
    _FakeLattice.count = 0
    s = slabs.SlabSet(4, 3, 4 * k, 0.6, k)
    s._lam_ex = [(lat.new_adjoint_halo(), lat.new_adjoint_halo()) for lat in s.slabs]
    s.exchange()
    s.adjoint_exchange()
    for j, lat in enumerate(s.slabs):
        below, above = (j - 1) % k, (j + 1) % k
        assert lat.got[("f", 0)] == (below, 1, 0)
        assert lat.got[("f", 1)] == (above, 0, 0)
        assert lat.got[("a", 1)] == (above, 0, 1)
        assert lat.got[("a", 0)] == (below, 1, 1)
    s.close()
