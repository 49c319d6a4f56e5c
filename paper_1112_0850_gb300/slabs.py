"""z-slab domain decomposition of a lattice: the method's one exchange per step.

The pull update (Sec. 2) reads only nearest neighbours, so a lattice split
along z into slabs needs, before each step, one plane from each neighbouring
slab, and of that plane only the five populations that cross the face. Each
slab is a lattice of its own whose first and last planes are ghosts; the
library's halo calls (lbm_halo_pack / lbm_halo_unpack) move the crossing
populations between a slab's boundary planes and packed buffers.

- `split_planes`, `with_ghosts`: which planes each slab holds (host logic).
- `SlabSet`: k slabs of one lattice on one device, exchanged through device
  buffers; the interior planes evolve bit for bit as in the unsplit lattice.
- `exchange_ranks`: the same exchange between processes, one slab per rank,
  over torch.distributed point-to-point calls with bounded waits. It moves
  whatever tensors it is given (packed halos, or whole planes).
- `SlabSet.step_record`, `adjoint_seed`, `adjoint_step`, `adjoint_init_grad`:
  the discrete adjoint of a split run. The reverse step reads lambda_i at
  x + e_i, so its exchange (lbm_adjoint_halo_pack / _unpack) moves the five
  populations of each face the other way, before every reverse step.
- `SlabSet.totals`, `SlabSet.step_reduce`, `reduce_ranks`: the FP64 mass and
  momentum totals of a split lattice, each slab summing its interior planes
  (lbm_reduce_planes, or inside the step with lbm_step_planes) and the slabs'
  sums added on the host, or over ranks by an all-reduce.
- `exchange_halos`, `run_ranks`, `RankSlab`: one slab per rank of a
  torch.distributed group (NCCL between GPUs; gloo on CPU ranks in the tests):
  each step packs the slab's two faces, exchanges them with the neighbouring
  ranks (`exchange_ranks`) and unpacks them into the ghosts before the slab's
  step.
"""
import datetime

import numpy as np
import torch


def split_planes(nz, k):
    """Interior planes [z0, z1) of k slabs covering planes 0 .. nz - 1, sizes
    differing by at most one."""
    if not 1 <= k <= nz:
        raise ValueError("cannot split %d planes into %d slabs" % (nz, k))
    b = [nz * i // k for i in range(k + 1)]
    return [(b[i], b[i + 1]) for i in range(k)]


def ghost_planes(nz, z0, z1):
    """Global plane indices of a slab with its ghosts: z0 - 1, z0 .. z1 - 1, z1
    (periodic in z)."""
    return [(z0 - 1) % nz] + list(range(z0, z1)) + [z1 % nz]


def overlap_windows(nz):
    """The plane windows of one overlapped step of a slab of nz planes (ghosts
    0 and nz - 1): (interior, boundary). The interior windows read no ghost
    plane (planes 2 .. nz - 3 gather from planes 1 .. nz - 2), so they run
    while the exchange fills the ghosts; the boundary windows (planes 1 and
    nz - 2) follow it, the last of them completing the step. Together they
    cover planes 1 .. nz - 2 once each."""
    if nz < 3:
        raise ValueError("a slab needs nz >= 3")
    interior = [(2, nz - 2)] if nz - 2 > 2 else []
    boundary = [(1, 2), (nz - 2, nz - 1)] if nz - 2 > 1 else [(1, 2)]
    return interior, boundary


def with_ghosts(a, z0, z1, axis=-3):
    """Planes z0 - 1 .. z1 of field `a` along `axis` (z of [..][nz][ny][nx]),
    periodic; numpy array or torch tensor, returned contiguous."""
    nz = a.shape[axis]
    idx = ghost_planes(nz, z0, z1)
    if torch.is_tensor(a):
        return a.index_select(axis % a.dim(), torch.tensor(idx, device=a.device)).contiguous()
    return np.ascontiguousarray(np.take(a, idx, axis=axis))


class SlabSet:
    """k z-slabs of an nx x ny x nz lattice on the current device.

    Slab j is a `Lattice` of nz_j + 2 planes: the interior planes of
    `split_planes(nz, k)[j]` between two ghost planes, created with the flags
    of those planes. `step` exchanges the halos, then steps every slab once;
    with overlap=True the exchange runs on a second stream while each slab
    updates its interior planes 2 .. nz - 3 (which read no ghost plane), and
    planes 1 and nz - 2 follow it (lbm_step_planes). Keyword arguments go to
    `Lattice` (storage, model, ...; pull pattern)."""

    def __init__(self, nx, ny, nz, tau, k, flags=None, force=None, overlap=False, **kw):
        from .lattice import Lattice
        self.shape = (nz, ny, nx)
        self.overlap = bool(overlap)
        self._side = None
        self.bounds = split_planes(nz, k)
        self.slabs = []
        try:
            for z0, z1 in self.bounds:
                fl = None if flags is None else with_ghosts(np.asarray(flags, dtype=np.uint8), z0, z1)
                self.slabs.append(Lattice(nx, ny, z1 - z0 + 2, tau, flags=fl, force=force, **kw))
        except Exception:
            self.close()
            raise
        self.stream = self.slabs[0].stream
        self.up = [lat.new_halo() for lat in self.slabs]    # side-1 packs, for the slab above
        self.down = [lat.new_halo() for lat in self.slabs]  # side-0 packs, for the slab below

    def set_force_field(self, F):
        """Per-cell force [3][nz][ny][nx] (device tensor of the arithmetic type)."""
        for lat, (z0, z1) in zip(self.slabs, self.bounds):
            lat.set_force_field(with_ghosts(F, z0, z1))

    def set_wall_velocity(self, u_w):
        for lat in self.slabs:
            lat.set_wall_velocity(u_w)

    def init_equilibrium(self, u0, rho0=None):
        """u0 [3][nz][ny][nx], rho0 [nz][ny][nx] or None, as for `Lattice`."""
        for lat, (z0, z1) in zip(self.slabs, self.bounds):
            lat.init_equilibrium(with_ghosts(u0, z0, z1), None if rho0 is None else with_ghosts(rho0, z0, z1))

    def exchange(self):
        """Fill every ghost plane from the neighbouring slab (periodic in z)."""
        k = len(self.slabs)
        for j, lat in enumerate(self.slabs):
            lat.halo_pack(1, self.up[j])
            lat.halo_pack(0, self.down[j])
        for j, lat in enumerate(self.slabs):
            lat.halo_unpack(0, self.up[(j - 1) % k])
            lat.halo_unpack(1, self.down[(j + 1) % k])

    def step(self, n=1):
        if self.overlap:
            return self._step_overlapped(n)
        for _ in range(int(n)):
            self.exchange()
            for lat in self.slabs:
                lat.step(1)

    def _step_overlapped(self, n):
        main = self.stream
        if self._side is None:
            self._side = torch.cuda.Stream(device=main.device)
            self._ready, self._halo_done = torch.cuda.Event(), torch.cuda.Event()
        side = self._side
        for _ in range(int(n)):
            self._ready.record(main)  # the current state is complete
            for lat in self.slabs:
                for z0, z1 in overlap_windows(lat.shape[0])[0]:
                    lat.step_planes(z0, z1, False)
            # the exchange reads planes 1 and nz - 2 of the current state and
            # writes its ghost planes, neither of which the interior writes
            side.wait_event(self._ready)
            for lat in self.slabs:
                lat.set_stream(side)
            try:
                self.exchange()
            finally:
                for lat in self.slabs:
                    lat.set_stream(main)
            self._halo_done.record(side)
            main.wait_event(self._halo_done)
            for lat in self.slabs:
                boundary = overlap_windows(lat.shape[0])[1]
                for j, (z0, z1) in enumerate(boundary):
                    lat.step_planes(z0, z1, j == len(boundary) - 1)

    def get_state(self, fmt=None):
        """The interior planes of all slabs joined: [19][nz][ny][nx]. The
        state is read by gathering each cell's populations from its pull
        sources, which for the boundary planes lie in the ghosts, so the
        ghosts are refreshed first."""
        self.exchange()
        return torch.cat([lat.get_state(fmt)[:, 1:-1] for lat in self.slabs], dim=1)

    # -- the adjoint: one step at a time, with an exchange before each -------
    def new_tapes(self, n):
        """Per slab, a tape for n recorded steps."""
        return [lat.new_tape(n) for lat in self.slabs]

    def step_record(self, n, tapes):
        """n steps, recording each slab's moments for the adjoint."""
        for k in range(int(n)):
            self.exchange()
            for lat, tape in zip(self.slabs, tapes):
                per = lat.info.tape_bytes_per_step
                lat.step_record(1, tape[k * per:(k + 1) * per])

    def _split(self, a):
        """Per slab, the planes z0 - 1 .. z1 of a [..][nz][ny][nx] device tensor
        (None stays None)."""
        return [None if a is None else with_ghosts(a, z0, z1) for z0, z1 in self.bounds]

    def adjoint_seed(self, dL_du, dL_drho=None):
        """Start the adjoint at the current state for dL/du (and dL/drho) of
        the whole lattice. The seed reads each cell's moments, so the forward
        halos are exchanged first; the slabs' ghost cells get no seed of their
        own (their entries are overwritten by each reverse exchange)."""
        self.exchange()
        self._lam_ex = [(lat.new_adjoint_halo(), lat.new_adjoint_halo()) for lat in self.slabs]
        self._grad_F = [lat.zeros(3) for lat in self.slabs]
        for lat, du, dr, gF in zip(self.slabs, self._split(dL_du), self._split(dL_drho), self._grad_F):
            du[..., 0, :, :] = 0
            du[..., -1, :, :] = 0
            if dr is not None:
                dr[0] = 0
                dr[-1] = 0
            lat.adjoint_seed(du, dr, gF)

    def adjoint_exchange(self):
        """Fill every ghost plane of the adjoint lattices from the neighbouring
        slab: the e_z = +1 populations of plane 1 go to the slab below, the
        e_z = -1 ones of plane nz - 2 to the slab above."""
        k = len(self.slabs)
        for lat, (down, up) in zip(self.slabs, self._lam_ex):
            lat.adjoint_halo_pack(0, down)
            lat.adjoint_halo_pack(1, up)
        for j, lat in enumerate(self.slabs):
            lat.adjoint_halo_unpack(1, self._lam_ex[(j + 1) % k][0])
            lat.adjoint_halo_unpack(0, self._lam_ex[(j - 1) % k][1])

    def adjoint_step(self, n, tapes):
        """n reverse steps, from the last recorded step back: each an adjoint
        exchange, then one reverse step of every slab with its tape."""
        for k in range(int(n) - 1, -1, -1):
            self.adjoint_exchange()
            for lat, tape, gF in zip(self.slabs, tapes, self._grad_F):
                per = lat.info.tape_bytes_per_step
                lat.adjoint_step(1, tape[k * per:(k + 1) * per], gF)

    def adjoint_init_grad(self, u0, rho0=None):
        """dL/du0 [3][nz][ny][nx] and dL/dF [3][nz][ny][nx] of the whole
        lattice (the interior planes of every slab joined), for the u0 and
        rho0 given to init_equilibrium."""
        gu = [lat.adjoint_init_grad(u, r)[0]
              for lat, u, r in zip(self.slabs, self._split(u0), self._split(rho0))]
        join = lambda parts: torch.cat([p[:, 1:-1] for p in parts], dim=1)
        return join(gu), join(self._grad_F)

    def step_reduce(self, n=1):
        """The totals of `totals()` for the current state, then n >= 1 steps:
        after an exchange, each slab's first step covers its interior planes
        only and sums their totals inside the step (lbm_step_planes with out);
        the slabs' sums are added on the host in slab order."""
        if int(n) < 1:
            raise ValueError("n must be >= 1")
        self.exchange()
        out = np.zeros(4)
        for lat in self.slabs:
            out += lat.step_planes(1, lat.shape[0] - 1, True, totals=True)
        self.step(int(n) - 1)
        return out

    def totals(self):
        """{sum rho, sum rho u_x, sum rho u_y, sum rho u_z} over the fluid
        cells of the whole lattice: each slab's interior planes summed on the
        device in FP64 (after an exchange, as the readers need), the slabs'
        sums added in slab order, so the result is deterministic."""
        self.exchange()
        out = np.zeros(4)
        for lat in self.slabs:
            out += lat.reduce(1, lat.shape[0] - 1)
        return out

    def status_word(self, clear=False):
        w = 0
        for lat in self.slabs:
            w |= lat.status_word(clear)
        return w

    def close(self):
        for lat in self.slabs:
            lat.close()
        self.slabs = []


# Status of `exchange_ranks`: done, or a wait that ran out or lost its peer.
EXCHANGE_OK = 0
EXCHANGE_FAILED = 1


def exchange_ranks(send_down, send_up, recv_below, recv_above, timeout=datetime.timedelta(seconds=10), group=None):
    """One step's halo exchange between ranks that each hold one slab, the
    slabs in rank order and periodic: `send_up` goes to rank + 1 (its
    `recv_below`), `send_down` to rank - 1 (its `recv_above`). Every wait is
    bounded by `timeout`; a wait that runs out, or whose peer has gone, returns
    (EXCHANGE_FAILED, which wait and why) instead of blocking, so that the
    caller can stop before its next step. Returns (EXCHANGE_OK, "") otherwise."""
    import torch.distributed as dist
    r, n = dist.get_rank(group), dist.get_world_size(group)
    if n == 1:
        recv_below.copy_(send_up)
        recv_above.copy_(send_down)
        return EXCHANGE_OK, ""
    lo, hi = (r - 1) % n, (r + 1) % n
    # One batch of the four point-to-point operations, posted in the same order
    # on every rank: NCCL then runs them as one group (individual sends and
    # receives, each rank posting its receives first, would wait on each
    # other), gloo as four operations. With two ranks lo == hi: the order (and,
    # for gloo, the tag) tells the two messages between them apart.
    names = ["receive from rank %d (below)" % lo, "receive from rank %d (above)" % hi,
             "send to rank %d (above)" % hi, "send to rank %d (below)" % lo]
    ops = [dist.P2POp(dist.irecv, recv_below, lo, group, 1), dist.P2POp(dist.irecv, recv_above, hi, group, 2),
           dist.P2POp(dist.isend, send_up, hi, group, 1), dist.P2POp(dist.isend, send_down, lo, group, 2)]
    try:
        reqs = dist.batch_isend_irecv(ops)
    except RuntimeError as e:
        return EXCHANGE_FAILED, "posting the exchange: %s" % str(e).splitlines()[0][:200]
    if len(reqs) != len(names):  # coalesced into one request
        names = ["exchange with ranks %d and %d" % (lo, hi)] * len(reqs)
    for what, w in zip(names, reqs):
        try:
            w.wait(timeout=timeout)
        except RuntimeError as e:
            return EXCHANGE_FAILED, "%s: %s" % (what, str(e).splitlines()[0][:200])
    return EXCHANGE_OK, ""


def reduce_ranks(totals, timeout=datetime.timedelta(seconds=10), group=None):
    """Sum a rank's FP64 totals (any float64 tensor, e.g. the 4 of
    `Lattice.reduce(1, nz - 1)` over its slab's interior planes) over all
    ranks, in place, with an all-reduce whose wait is bounded by `timeout`.
    Returns (EXCHANGE_OK, "") or, when the wait runs out or a rank has gone,
    (EXCHANGE_FAILED, why); the tensor's contents are then undefined."""
    import torch.distributed as dist
    if totals.dtype != torch.float64:
        raise TypeError("totals are summed in float64")
    if dist.get_world_size(group) == 1:
        return EXCHANGE_OK, ""
    w = dist.all_reduce(totals, op=dist.ReduceOp.SUM, group=group, async_op=True)
    try:
        w.wait(timeout=timeout)
    except RuntimeError as e:
        return EXCHANGE_FAILED, "all-reduce of totals: %s" % str(e).splitlines()[0][:200]
    return EXCHANGE_OK, ""


def exchange_halos(slab, bufs, timeout=datetime.timedelta(seconds=10), group=None):
    """One step's halo exchange of this rank's slab with the ranks below and
    above. `slab` is any object with halo_pack(side, buf) and
    halo_unpack(side, buf) (a `Lattice` slab on the GPU, moving the five
    populations that cross each face; a test slab on the CPU, moving whole
    planes); `bufs` = (send_down, send_up, recv_below, recv_above), tensors of
    one packed halo each, on the device the group's backend moves. Side 0 of
    the slab is its bottom face (plane 1 out, ghost plane 0 in), side 1 its
    top face (plane nz - 2 out, ghost plane nz - 1 in). Returns the status of
    `exchange_ranks`; on EXCHANGE_FAILED the ghosts are left as they were."""
    send_down, send_up, recv_below, recv_above = bufs
    slab.halo_pack(0, send_down)
    slab.halo_pack(1, send_up)
    st, why = exchange_ranks(send_down, send_up, recv_below, recv_above, timeout, group)
    if st != EXCHANGE_OK:
        return st, why
    slab.halo_unpack(0, recv_below)
    slab.halo_unpack(1, recv_above)
    return EXCHANGE_OK, ""


def run_ranks(slab, bufs, steps, timeout=datetime.timedelta(seconds=10), group=None):
    """`steps` steps of a lattice decomposed over the ranks of `group`, one
    z-slab per rank in rank order (periodic in z): before each step of the
    slab, the exchange of `exchange_halos`. Stops at the first exchange that
    fails and returns its status (no step is taken after it), else
    (EXCHANGE_OK, "")."""
    for _ in range(int(steps)):
        st, why = exchange_halos(slab, bufs, timeout, group)
        if st != EXCHANGE_OK:
            return st, why
        slab.step(1)
    return EXCHANGE_OK, ""


class RankSlab:
    """This rank's z-slab of an nx x ny x nz lattice decomposed over the ranks
    of a torch.distributed group: the planes `split_planes(nz, ranks)[rank]`
    between two ghost planes, as one `Lattice` on the current device, created
    with the flags of those planes. Each step exchanges the halos with the
    neighbouring ranks (point-to-point sends and receives into this rank's
    own buffers, every wait bounded) and then steps the slab; on a single rank
    the exchange is the periodic copy of the slab's own faces, and the slab's
    interior evolves bit for bit as the unsplit lattice. With NCCL the halo
    buffers are device tensors and the library's stream must be torch's
    current stream (the `Lattice` default). Keyword arguments go to `Lattice`
    (storage, model, ...; pull pattern, shifted or FP32/FP64 storage)."""

    def __init__(self, nx, ny, nz, tau, flags=None, force=None, group=None,
                 timeout=datetime.timedelta(seconds=10), **kw):
        import torch.distributed as dist
        from .lattice import Lattice
        self.group = group
        self.timeout = timeout
        self.rank, self.ranks = dist.get_rank(group), dist.get_world_size(group)
        self.z0, self.z1 = split_planes(nz, self.ranks)[self.rank]
        self.shape = (nz, ny, nx)
        fl = None if flags is None else with_ghosts(np.asarray(flags, dtype=np.uint8), self.z0, self.z1)
        self.lat = Lattice(nx, ny, self.z1 - self.z0 + 2, tau, flags=fl, force=force, **kw)
        self.stream = self.lat.stream
        self.bufs = tuple(self.lat.new_halo() for _ in range(4))

    def init_equilibrium(self, u0, rho0=None):
        """u0 [3][nz][ny][nx] (and rho0 [nz][ny][nx]) of the whole lattice."""
        self.lat.init_equilibrium(with_ghosts(u0, self.z0, self.z1),
                                  None if rho0 is None else with_ghosts(rho0, self.z0, self.z1))

    def set_force_field(self, F):
        self.lat.set_force_field(with_ghosts(F, self.z0, self.z1))

    def step(self, n=1):
        """n exchange-then-step rounds; raises RuntimeError naming the wait if
        an exchange fails (a neighbour that stopped, a wait that ran out)."""
        st, why = run_ranks(self.lat, self.bufs, n, self.timeout, self.group)
        if st != EXCHANGE_OK:
            raise RuntimeError("z-slab exchange failed: " + why)

    def interior_state(self, fmt=None):
        """This rank's interior planes of the state, [19][z1 - z0][ny][nx],
        read after an exchange (the readers gather from the ghosts)."""
        st, why = exchange_halos(self.lat, self.bufs, self.timeout, self.group)
        if st != EXCHANGE_OK:
            raise RuntimeError("z-slab exchange failed: " + why)
        return self.lat.get_state(fmt)[:, 1:-1]

    def totals(self):
        """{sum rho, sum rho u} over the fluid cells of the whole lattice: this
        rank's interior planes (after an exchange) in FP64, all-reduced over
        the ranks with a bounded wait."""
        st, why = exchange_halos(self.lat, self.bufs, self.timeout, self.group)
        if st != EXCHANGE_OK:
            raise RuntimeError("z-slab exchange failed: " + why)
        t = torch.tensor(self.lat.reduce(1, self.lat.shape[0] - 1), dtype=torch.float64,
                         device=self.bufs[0].device)
        st, why = reduce_ranks(t, self.timeout, self.group)
        if st != EXCHANGE_OK:
            raise RuntimeError("totals all-reduce failed: " + why)
        return t.cpu().numpy()

    def close(self):
        self.lat.close()
