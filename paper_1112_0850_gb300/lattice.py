"""Python front end of the D3Q19 BGK library: one `Lattice` per context.

Argument marshalling only: device memory comes from torch, pointers go to
the C-ABI (capi.py), and every step of the computation runs in the CUDA
library. Arrays are canonical, x fastest: u[3][nz][ny][nx], rho[nz][ny][nx];
"real" is float64 for storage "f64" and float32 otherwise.
"""
import ctypes

import numpy as np
import torch

from . import capi


def _real_dtype(storage):
    return torch.float64 if storage == capi.LBM_F64 else torch.float32


# element type of the canonical state arrays of each format (the moment-split
# formats exchange plain shifted deviations in their 16-bit element type)
_FMT_DTYPE = {capi.LBM_F64: torch.float64, capi.LBM_F32: torch.float32, capi.LBM_F16S: torch.float16,
              capi.LBM_BF16S: torch.bfloat16, capi.LBM_F16M: torch.float16, capi.LBM_BF16M: torch.bfloat16}
_DTYPE_FMT = {torch.float64: capi.LBM_F64, torch.float32: capi.LBM_F32, torch.float16: capi.LBM_F16S,
              torch.bfloat16: capi.LBM_BF16S}


def _storage_code(s):
    return capi.STORAGE[s] if isinstance(s, str) else int(s)


class Lattice:
    """A periodic nx * ny * nz D3Q19 lattice on the current CUDA device.

    flags: optional uint8 array [nz][ny][nx] (0 fluid, 2 moving wall, other nonzero solid);
    force: optional uniform body force (3,); storage: "f64" | "f32" | "f16s" |
    "bf16s" | "f16m" | "bf16m" (16-bit moment split: momentum plus remainders).
    Work is enqueued on `stream` (default: torch's current stream at
    construction). row_align: bytes each padded row starts on (0 = pairs only,
    128 = the paper's padding).
    pattern: "pull" (two lattices) or "aa" (one lattice updated in place).
    model: "qian" (default) or "incompressible" (He & Luo equilibrium).
    stage_rows: True makes the two-grid step stage its source rows in shared
    memory with TMA bulk copies where possible (same results; off by default).
    """

    def __init__(self, nx, ny, nz, tau, flags=None, force=None, storage="f32", stream=None, row_align=0,
                 pattern="pull", model="qian", stage_rows=False):
        L = capi.lib()
        self.storage = _storage_code(storage)
        self.pattern = capi.PATTERN[pattern] if isinstance(pattern, str) else int(pattern)
        self.shape = (nz, ny, nx)
        self.real = _real_dtype(self.storage)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.model = capi.MODEL[model] if isinstance(model, str) else int(model)
        opt = capi.lbm_options(self.storage, ctypes.c_void_p(self.stream.cuda_stream), int(row_align),
                               self.pattern, self.model, 1 if stage_rows else 0)
        fl = None
        if flags is not None:
            fl = np.ascontiguousarray(np.asarray(flags.cpu() if torch.is_tensor(flags) else flags), dtype=np.uint8)
            assert fl.shape == self.shape, (fl.shape, self.shape)
        self._flags_host = fl
        F = None if force is None else (ctypes.c_double * 3)(*[float(v) for v in force])
        h = ctypes.c_void_p()
        st = L.lbm_create(ctypes.byref(h), int(nx), int(ny), int(nz), float(tau),
                          None if fl is None else fl.ctypes.data, F, ctypes.byref(opt))
        capi.check(st, None, "lbm_create(%d, %d, %d)" % (nx, ny, nz))
        self._h = h
        self.tau = float(tau)

    # -- plumbing -----------------------------------------------------------
    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("lattice is closed")
        return self._h

    def _call(self, name, *args):
        capi.check(getattr(capi.lib(), name)(self.handle, *args), self.handle, name)

    def _ptr(self, t, dtype, shape, device_only=False):
        """Pointer of tensor t after checking dtype, shape and contiguity."""
        if t is None:
            return None
        assert t.dtype == dtype, (t.dtype, dtype)
        assert tuple(t.shape) == tuple(shape), (tuple(t.shape), shape)
        assert t.is_contiguous()
        if device_only:
            assert t.is_cuda
        return t.data_ptr()

    def close(self):
        if getattr(self, "_h", None) is not None:
            capi.lib().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def info(self):
        inf = capi.lbm_info()
        self._call("lbm_get_info", ctypes.byref(inf))
        return inf

    @property
    def n_fluid(self):
        return self.info.n_fluid

    def zeros(self, *lead, dtype=None, device="cuda"):
        return torch.zeros(*lead, *self.shape, dtype=dtype or self.real, device=device)

    # -- the calls of include/lbm_capi.h ------------------------------------
    def set_uniform_force(self, force):
        F = None if force is None else (ctypes.c_double * 3)(*[float(v) for v in force])
        self._call("lbm_set_uniform_force", F)

    def set_wall_velocity(self, u_w):
        U = None if u_w is None else (ctypes.c_double * 3)(*[float(v) for v in u_w])
        self._call("lbm_set_wall_velocity", U)

    def set_force_field(self, F):
        self._call("lbm_set_force_field", self._ptr(F, self.real, (3,) + self.shape))

    def init_equilibrium(self, u, rho=None):
        self._call("lbm_init_equilibrium", self._ptr(rho, self.real, self.shape),
                   self._ptr(u, self.real, (3,) + self.shape))

    def step(self, n=1):
        self._call("lbm_step", int(n))

    def prepare_steps(self, n):
        """Capture the step graphs that step(n) replays, running nothing."""
        self._call("lbm_step_prepare", int(n))

    def step_timed(self, n=1):
        """n steps between two CUDA events on the context's stream; returns
        their device time in milliseconds (synchronizes)."""
        ms = ctypes.c_float(0.0)
        self._call("lbm_step_timed", int(n), ctypes.byref(ms))
        return ms.value

    def macros(self, rho=None, u=None, with_rho=True):
        if u is None:
            u = self.zeros(3)
        if rho is None and with_rho:
            rho = self.zeros()
        self._call("lbm_macros", self._ptr(rho, self.real, self.shape), self._ptr(u, self.real, (3,) + self.shape))
        return rho, u

    def step_planes(self, z0, z1, last, totals=False, out=None):
        """One step of planes z0 <= z < z1 only; last=True completes the step
        (every plane in exactly one call per step). With totals=True (host
        numpy result) or a device float64 tensor `out` (asynchronous), also
        the totals of reduce(z0, z1) for the current state, summed inside the
        step."""
        if out is not None:
            assert out.is_cuda and out.dtype == torch.float64 and out.numel() >= 4
            self._call("lbm_step_planes", int(z0), int(z1), 1 if last else 0, ctypes.c_void_p(out.data_ptr()))
            return out
        if totals:
            res = (ctypes.c_double * 4)()
            self._call("lbm_step_planes", int(z0), int(z1), 1 if last else 0, res)
            return np.array(res[:])
        self._call("lbm_step_planes", int(z0), int(z1), 1 if last else 0, None)

    def set_stream(self, stream):
        """Enqueue every later call on `stream` (a torch.cuda.Stream); order it
        against the previous stream with events."""
        self._call("lbm_set_stream", ctypes.c_void_p(stream.cuda_stream))
        self.stream = stream

    def reduce(self, z0=None, z1=None):
        """{sum rho, sum rho u} over the fluid cells, in FP64; with z0, z1 over
        planes z0 <= z < z1 only (a slab's interior planes: 1, nz - 1)."""
        out = (ctypes.c_double * 4)()
        if z0 is None and z1 is None:
            self._call("lbm_reduce", out)
        else:
            z0 = 0 if z0 is None else int(z0)
            z1 = self.shape[0] if z1 is None else int(z1)
            self._call("lbm_reduce_planes", z0, z1, out)
        return np.array(out[:])

    def step_reduce(self, n=1, out=None):
        """Totals of the current state (as reduce()), then n steps, the totals
        summed inside the first step. out: optional device float64 tensor [4]
        (asynchronous); otherwise a host numpy array is returned."""
        if out is not None:
            assert out.is_cuda and out.dtype == torch.float64 and out.numel() >= 4
            self._call("lbm_step_reduce", int(n), out.data_ptr())
            return out
        res = (ctypes.c_double * 4)()
        self._call("lbm_step_reduce", int(n), res)
        return np.array(res[:])

    def get_state(self, fmt=None, out=None):
        fmt = self.storage if fmt is None else _storage_code(fmt)
        if out is None:
            out = torch.empty((capi.Q,) + self.shape, dtype=_FMT_DTYPE[fmt], device="cuda")
        self._call("lbm_get_state", self._ptr(out, _FMT_DTYPE[fmt], (capi.Q,) + self.shape), fmt)
        return out

    def set_state(self, state):
        fmt = _DTYPE_FMT[state.dtype]
        self._call("lbm_set_state", self._ptr(state, state.dtype, (capi.Q,) + self.shape), fmt)

    def new_halo(self):
        """A device buffer for one packed halo: [5][ny][pitch] of the storage type."""
        dt = _FMT_DTYPE[self.storage]
        n = capi.lib().lbm_halo_bytes(self.handle) // torch.empty(0, dtype=dt).element_size()
        return torch.empty(n, dtype=dt, device="cuda")

    def halo_pack(self, side, buf):
        """Outgoing populations of interior plane 1 (side 0) or nz - 2 (side 1)."""
        assert buf.dtype == _FMT_DTYPE[self.storage] and buf.is_contiguous()
        assert buf.numel() * buf.element_size() >= capi.lib().lbm_halo_bytes(self.handle)
        self._call("lbm_halo_pack", int(side), buf.data_ptr())

    def halo_unpack(self, side, buf):
        """Incoming populations into ghost plane 0 (side 0) or nz - 1 (side 1), fluid cells."""
        assert buf.dtype == _FMT_DTYPE[self.storage] and buf.is_contiguous()
        assert buf.numel() * buf.element_size() >= capi.lib().lbm_halo_bytes(self.handle)
        self._call("lbm_halo_unpack", int(side), buf.data_ptr())

    def new_adjoint_halo(self):
        """A device buffer for one packed adjoint halo: [5][ny][pitch] of real."""
        n = capi.lib().lbm_adjoint_halo_bytes(self.handle) // torch.empty(0, dtype=self.real).element_size()
        return torch.empty(n, dtype=self.real, device="cuda")

    def adjoint_halo_pack(self, side, buf):
        """Outgoing adjoint populations of plane 1 (side 0, e_z = +1) or nz - 2 (side 1, e_z = -1)."""
        assert buf.dtype == self.real and buf.is_contiguous()
        assert buf.numel() * buf.element_size() >= capi.lib().lbm_adjoint_halo_bytes(self.handle)
        self._call("lbm_adjoint_halo_pack", int(side), buf.data_ptr())

    def adjoint_halo_unpack(self, side, buf):
        """Incoming adjoint populations into ghost plane 0 (side 0) or nz - 1 (side 1), fluid cells."""
        assert buf.dtype == self.real and buf.is_contiguous()
        assert buf.numel() * buf.element_size() >= capi.lib().lbm_adjoint_halo_bytes(self.handle)
        self._call("lbm_adjoint_halo_unpack", int(side), buf.data_ptr())

    def new_tape(self, n):
        return torch.empty(int(n) * self.info.tape_bytes_per_step, dtype=torch.uint8, device="cuda")

    def step_record(self, n, tape):
        assert tape.is_cuda and tape.numel() >= n * self.info.tape_bytes_per_step
        self._call("lbm_step_record", int(n), tape.data_ptr())

    def adjoint_seed(self, dL_du, dL_drho=None, grad_F=None):
        self._call("lbm_adjoint_seed", self._ptr(dL_du, self.real, (3,) + self.shape),
                   self._ptr(dL_drho, self.real, self.shape),
                   self._ptr(grad_F, self.real, (3,) + self.shape, device_only=True))

    def adjoint_step(self, n, tape, grad_F=None):
        assert tape.is_cuda and tape.numel() >= n * self.info.tape_bytes_per_step
        self._call("lbm_adjoint_step", int(n), tape.data_ptr(),
                   self._ptr(grad_F, self.real, (3,) + self.shape, device_only=True))

    def adjoint_init_grad(self, u0, rho0=None, grad_u0=None, grad_rho0=None, with_rho=False):
        if grad_u0 is None:
            grad_u0 = self.zeros(3)
        if grad_rho0 is None and with_rho:
            grad_rho0 = self.zeros()
        self._call("lbm_adjoint_init_grad", self._ptr(rho0, self.real, self.shape),
                   self._ptr(u0, self.real, (3,) + self.shape), self._ptr(grad_u0, self.real, (3,) + self.shape),
                   self._ptr(grad_rho0, self.real, self.shape))
        return grad_u0, grad_rho0

    def status_word(self, clear=False):
        v = ctypes.c_uint32()
        self._call("lbm_status_word", ctypes.byref(v), 1 if clear else 0)
        return v.value

    def synchronize(self):
        self._call("lbm_synchronize")


def lattice_table():
    """(e [19,3], w [19], opp [19]) as compiled into the library."""
    e = (ctypes.c_int * 57)()
    w = (ctypes.c_double * 19)()
    o = (ctypes.c_int * 19)()
    capi.lib().lbm_lattice_table(e, w, o)
    return np.array(e[:]).reshape(19, 3), np.array(w[:]), np.array(o[:])
