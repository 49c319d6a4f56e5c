"""GB300-native D3Q19 BGK lattice Boltzmann hot path (Habich et al., arXiv 1112.0850).

The computation lives in liblbm_gb300.so (CUDA, sm_103a) behind the C-ABI of
include/lbm_capi.h; this package is its thin Python binding:
  capi     ctypes prototypes, same names as the C functions
  lattice  Lattice: one context (create, init, step, macros, reduce, state, adjoint)
  rollout  LBMRollout: torch.autograd.Function over the adjoint kernels
  build    compiles the library in-tree for sm_103a
"""
from . import capi  # noqa: F401
from .capi import LBMError  # noqa: F401


def __getattr__(name):
    # torch-dependent pieces are imported on first use
    if name in ("Lattice", "lattice_table"):
        from . import lattice
        return getattr(lattice, name)
    if name in ("LBMRollout", "velocity_loss"):
        from . import rollout
        return getattr(rollout, name)
    raise AttributeError(name)
