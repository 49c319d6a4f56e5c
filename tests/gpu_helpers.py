"""Helpers shared by the GPU parity tests: run the CUDA path through the
C-ABI (Lattice) and the FP64 oracle on the same seeded inputs, and compare."""
import numpy as np
import torch

import oracle
from paper_1112_0850_gb300 import build
from paper_1112_0850_gb300.lattice import Lattice

# Velocity tolerances (relative L2 over fluid cells against the FP64 oracle)
# stated by the method's accuracy targets: FP64 storage 1e-12, FP32 1e-5,
# 16-bit shifted storage 1e-3. bfloat16 keeps 8 significant bits: one
# rounding of a deviation w_i (3 e.u) ~ 3e-3 costs ~2^-9 of it per step, and
# over the parity runs (20-100 steps) that leaves 2.2e-3 to 5.3e-3 relative
# error in u, the same in the oracle's own emulation of the rounding (the
# format's floor). BF16 shifted storage therefore misses the 1e-3 target; it is
# held to that measured floor plus a margin (the moment-split bfloat16 format,
# tests/test_split_gpu.py, is the one that meets it on smooth flows).
TOL_U = {"f64": 1e-12, "f32": 1e-5, "f16s": 1e-3, "bf16s": 7e-3}
STORAGES = ["f64", "f32", "f16s", "bf16s"]
REAL = {"f64": torch.float64, "f32": torch.float32, "f16s": torch.float32, "bf16s": torch.float32,
        "f16m": torch.float32, "bf16m": torch.float32}
EMUL = {"f64": None, "f32": "f32", "f16s": "f16", "bf16s": "bf16", "f16m": "f16m", "bf16m": "bf16m"}

_built = False


def ensure_built():
    global _built
    if not _built:
        build.build()
        _built = True


def fluid_mask(flags, shape):
    return np.ones(shape, bool) if flags is None else np.asarray(flags) == 0


def rel_l2(a, b, mask):
    a = np.asarray(a, dtype=np.float64)[..., mask] if mask is not None else np.asarray(a, np.float64)
    b = np.asarray(b, dtype=np.float64)[..., mask] if mask is not None else np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def gpu_run(storage, u0, tau, steps, flags=None, F=None, rho0=None, Ffield=None):
    """Create, init, step on the GPU; return (rho, u, state, lattice) as float64 numpy + the Lattice."""
    ensure_built()
    nz, ny, nx = u0.shape[1:]
    lat = Lattice(nx, ny, nz, tau, flags=flags, force=F, storage=storage)
    real = REAL[storage]
    u = torch.as_tensor(u0, dtype=real).cuda().contiguous()
    r = None if rho0 is None else torch.as_tensor(rho0, dtype=real).cuda().contiguous()
    if Ffield is not None:
        lat.set_force_field(torch.as_tensor(Ffield, dtype=real).cuda().contiguous())
    lat.init_equilibrium(u, r)
    lat.step(steps)
    rho, uu = lat.macros()
    st = lat.get_state("f64")
    torch.cuda.synchronize()
    return rho.double().cpu().numpy(), uu.double().cpu().numpy(), st.cpu().numpy(), lat


def as_input(x, storage):
    """The values the GPU actually receives: canonical inputs are FP64 for
    storage f64 and FP32 otherwise, so the oracle is fed the same rounding."""
    if x is None or storage == "f64":
        return x
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def oracle_run(u0, tau, steps, flags=None, F=None, rho0=None, Ffield=None, fmt=None):
    Fo = Ffield if Ffield is not None else (None if F is None else np.asarray(F, np.float64))
    f = oracle.init_equilibrium(u0, rho0=rho0, flags=flags, fmt=fmt)
    f = oracle.run(f, tau, steps, flags=flags, F=Fo, fmt=fmt)
    rho, u = oracle.macros(f, flags=flags, F=Fo)
    return rho, u, f


def shifted(f, flags=None):
    """Oracle state f -> shifted deviations f - w (0 at solid cells)."""
    _, w, _ = oracle.lattice()
    s = f - w[:, None, None, None]
    if flags is not None:
        s[:, np.asarray(flags) != 0] = 0.0
    return s
