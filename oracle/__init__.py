"""FP64 CPU oracle for the D3Q19 BGK update (ctypes front end of lbm_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this package; the product path never does. It
shares no code with the CUDA library.

Arrays are numpy float64 in canonical layout: populations f[19][nz][ny][nx],
velocity u[3][nz][ny][nx], x fastest; flags uint8 [nz][ny][nx] with 0 = fluid,
1 = solid. The state f is the pre-collision populations f^n (push form).

Every function follows Sec. 2 of the paper (moments, equilibrium after Qian et
al., BGK relaxation of Eq. 1, streaming, bounce-back after Ziegler), with the
Guo body force and halfway bounce-back as the readings stated in the C source.
`model` selects the equilibrium: "qian" (default) or "incompressible" (He &
Luo: velocity terms with the reference density 1, u = j + F/2).
"""
import ctypes

import numpy as np

from . import build as _build

Q = 19
FMT = {None: 0, "f64": 0, "f32": 1, "f16": 2, "bf16": 3, "f16m": 4, "bf16m": 5}
MODEL = {None: 0, "qian": 0, "incompressible": 1}

class Oracle:
    """The oracle's functions bound to one build of lbm_oracle.c (ctypes)."""

    def __init__(self, path):
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        vp = ctypes.c_void_p
        ci = ctypes.c_int
        L.oracle_lattice.argtypes = [ip, dp, ip]
        L.oracle_equilibrium.argtypes = [ctypes.c_double, dp, dp]
        L.oracle_equilibrium_incompressible.argtypes = [ctypes.c_double, dp, dp]
        L.oracle_moments.argtypes = [dp, dp, dp, dp]
        L.oracle_moments_incompressible.argtypes = [dp, dp, dp, dp]
        L.oracle_collide_cell.argtypes = [dp, ctypes.c_double, dp, dp]
        L.oracle_collide_cell_model.argtypes = [ci, dp, ctypes.c_double, dp, dp]
        L.oracle_round.argtypes = [ctypes.c_double, ci]
        L.oracle_round.restype = ctypes.c_double
        L.oracle_init.argtypes = [ci] * 3 + [vp, vp, vp, vp, ci, ci]
        L.oracle_init.restype = ci
        L.oracle_split_round.argtypes = [dp, ci]
        L.oracle_store.argtypes = [ci] * 3 + [vp, vp, ci]
        L.oracle_store.restype = ci
        L.oracle_run.argtypes = [ci] * 3 + [ctypes.c_double, vp, vp, ci, vp, vp, ci, ci, ci, ci]
        L.oracle_run.restype = ci
        L.oracle_macros.argtypes = [ci] * 3 + [vp, vp, ci, vp, vp, vp, ci]
        L.oracle_sums.argtypes = [ci] * 3 + [vp, vp, ci, vp, vp, ci]
        L.oracle_max_threads.restype = ci
        self.lib = L
        self.path = path

    def lattice(self):
        """Return (e [19,3] int, w [19] float64, opp [19] int) of the oracle's D3Q19 table."""
        e = np.zeros((Q, 3), dtype=np.int32)
        w = np.zeros(Q)
        opp = np.zeros(Q, dtype=np.int32)
        ip = ctypes.POINTER(ctypes.c_int)
        self.lib.oracle_lattice(e.ctypes.data_as(ip), _dp(w), opp.ctypes.data_as(ip))
        return e, w, opp

    def equilibrium(self, rho, u, model=None):
        """f_eq(rho, u) for one cell (Qian et al., cited in Sec. 2; or He & Luo)."""
        u = _f64(u)
        out = np.zeros(Q)
        fn = self.lib.oracle_equilibrium_incompressible if MODEL[model] else self.lib.oracle_equilibrium
        fn(float(rho), _dp(u), _dp(out))
        return out

    def moments(self, f, F=(0.0, 0.0, 0.0), model=None):
        """(rho, u) of one cell, u = (j + F/2)/rho (Sec. 2 step 1 with the Guo
        shift), or u = j + F/2 for the incompressible model."""
        f, F = _f64(f), _f64(F)
        rho = np.zeros(1)
        u = np.zeros(3)
        fn = self.lib.oracle_moments_incompressible if MODEL[model] else self.lib.oracle_moments
        fn(_dp(f), _dp(F), _dp(rho), _dp(u))
        return rho[0], u

    def collide_cell(self, f, tau, F=(0.0, 0.0, 0.0), model=None):
        """Post-collision populations of one cell (Eq. 1 plus the Guo source)."""
        f, F = _f64(f), _f64(F)
        out = np.zeros(Q)
        self.lib.oracle_collide_cell_model(MODEL[model], _dp(f), float(tau), _dp(F), _dp(out))
        return out

    def round_storage_value(self, v, fmt):
        """Round one FP64 value to 'f32' | 'f16' | 'bf16' (ties to even)."""
        return self.lib.oracle_round(float(v), FMT[fmt])

    def split_round(self, P, fmt):
        """One cell's 19 values through the moment-split format 'f16m' | 'bf16m':
        J = sum P_i e_i and g_i = (P_i - w_i) - 3 w_i e_i.J~ rounded, rebuilt
        as w_i + 3 w_i e_i.J~ + g~_i. Returns the rebuilt values."""
        out = np.array(P, dtype=np.float64, copy=True)
        assert out.shape == (Q,)
        self.lib.oracle_split_round(_dp(out), FMT[fmt])
        return out

    def store_state(self, f, flags=None, fmt=None):
        """State f [19][nz][ny][nx] as storage format fmt holds it once written
        (elementwise rounding of f - w, or the moment-split storage of the
        values each cell holds for its neighbours to pull); returns a new array."""
        f = np.array(f, dtype=np.float64, order="C", copy=True)
        shape = f.shape[1:]
        nz, ny, nx = shape
        fl = _flags(flags, shape)
        if self.lib.oracle_store(nx, ny, nz, _vp(fl), _vp(f), FMT[fmt]) != 0:
            raise MemoryError("oracle_store could not allocate its scratch")
        return f

    def init_equilibrium(self, u0, rho0=None, flags=None, fmt=None, model=None):
        """f^0 = f_eq(rho0, u0) per fluid cell; u0 [3][nz][ny][nx]; returns f [19][nz][ny][nx]."""
        u0 = _f64(u0)
        shape = u0.shape[1:]
        nz, ny, nx = shape
        fl = _flags(flags, shape)
        r0 = None if rho0 is None else _f64(rho0)
        f = np.zeros((Q,) + shape)
        if self.lib.oracle_init(nx, ny, nz, _vp(fl), _vp(r0), _vp(u0), _vp(f), FMT[fmt], MODEL[model]) != 0:
            raise MemoryError("oracle_init could not allocate its scratch")
        return f

    def run(self, f, tau, steps, flags=None, F=None, fmt=None, threads=None, u_wall=None, model=None):
        """Advance state f by `steps` collide-and-stream steps; returns a new array.

        Cells flagged 2 are walls moving with velocity u_wall (3,)."""
        f = np.array(f, dtype=np.float64, order="C", copy=True)
        shape = f.shape[1:]
        nz, ny, nx = shape
        fl = _flags(flags, shape)
        Fa, per_cell = _force(F, shape)
        uw = None if u_wall is None else _f64(u_wall)
        nt = threads if threads else self.lib.oracle_max_threads()
        rc = self.lib.oracle_run(nx, ny, nz, float(tau), _vp(fl), _vp(Fa), per_cell, _vp(uw), _vp(f),
                                 int(steps), FMT[fmt], int(nt), MODEL[model])
        if rc != 0:
            raise MemoryError("oracle_run could not allocate its second lattice")
        return f

    def macros(self, f, flags=None, F=None, model=None):
        """(rho [nz][ny][nx], u [3][nz][ny][nx]) of state f; zeros at solid cells."""
        f = _f64(f)
        shape = f.shape[1:]
        nz, ny, nx = shape
        fl = _flags(flags, shape)
        Fa, per_cell = _force(F, shape)
        rho = np.zeros(shape)
        u = np.zeros((3,) + shape)
        self.lib.oracle_macros(nx, ny, nz, _vp(fl), _vp(Fa), per_cell, _vp(f), _vp(rho), _vp(u), MODEL[model])
        return rho, u

    def sums(self, f, flags=None, F=None, model=None):
        """[sum rho, and the sum of the momentum j + F/2] over fluid cells."""
        f = _f64(f)
        shape = f.shape[1:]
        nz, ny, nx = shape
        fl = _flags(flags, shape)
        Fa, per_cell = _force(F, shape)
        out = np.zeros(4)
        self.lib.oracle_sums(nx, ny, nz, _vp(fl), _vp(Fa), per_cell, _vp(f), _vp(out), MODEL[model])
        return out

    def max_threads(self):
        return self.lib.oracle_max_threads()


_default = None


def default():
    """The oracle built from oracle/lbm_oracle.c (compiled on first use)."""
    global _default
    if _default is None:
        _default = Oracle(_build.build())
    return _default


def load(path):
    """An Oracle bound to another build of the same C source (used by mutation tests)."""
    return Oracle(path)


def lattice():
    return default().lattice()


def equilibrium(rho, u, model=None):
    return default().equilibrium(rho, u, model)


def moments(f, F=(0.0, 0.0, 0.0), model=None):
    return default().moments(f, F, model)


def collide_cell(f, tau, F=(0.0, 0.0, 0.0), model=None):
    return default().collide_cell(f, tau, F, model)


def round_storage_value(v, fmt):
    return default().round_storage_value(v, fmt)


def split_round(P, fmt):
    return default().split_round(P, fmt)


def store_state(f, flags=None, fmt=None):
    return default().store_state(f, flags, fmt)


def init_equilibrium(u0, rho0=None, flags=None, fmt=None, model=None):
    return default().init_equilibrium(u0, rho0, flags, fmt, model)


def run(f, tau, steps, flags=None, F=None, fmt=None, threads=None, u_wall=None, model=None):
    return default().run(f, tau, steps, flags, F, fmt, threads, u_wall, model)


def macros(f, flags=None, F=None, model=None):
    return default().macros(f, flags, F, model)


def sums(f, flags=None, F=None, model=None):
    return default().sums(f, flags, F, model)


def max_threads():
    return default().max_threads()


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vp(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _flags(flags, shape):
    if flags is None:
        return None
    fl = np.ascontiguousarray(flags, dtype=np.uint8)
    assert fl.shape == shape, (fl.shape, shape)
    return fl


def _force(F, shape):
    """Return (array or None, per_cell flag) for a uniform [3] or field [3][nz][ny][nx] force."""
    if F is None:
        return None, 0
    F = _f64(F)
    if F.shape == (3,):
        return F, 0
    assert F.shape == (3,) + shape, F.shape
    return F, 1


__all__ = ["Q", "Oracle", "default", "load", "lattice", "equilibrium", "moments", "collide_cell", "round_storage_value",
           "split_round", "store_state", "init_equilibrium", "run", "macros", "sums", "max_threads"]
