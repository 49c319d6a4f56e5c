"""ctypes binding of include/lbm_capi.h (argument marshalling only).

Every function keeps its C name and signature; pointers are passed as
integers (a torch tensor's data_ptr() or a host address). The library is
loaded on first use; if it is missing or cannot be loaded, the call raises:
there is no fallback implementation.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm_gb300.so")

LBM_F64, LBM_F32, LBM_F16S, LBM_BF16S, LBM_F16M, LBM_BF16M = 0, 1, 2, 3, 4, 5
STORAGE = {"f64": LBM_F64, "f32": LBM_F32, "f16s": LBM_F16S, "bf16s": LBM_BF16S, "f16m": LBM_F16M,
           "bf16m": LBM_BF16M}
STORAGE_NAME = {v: k for k, v in STORAGE.items()}
# bytes of one stored population value (a remainder, for the moment-split formats)
STORAGE_BYTES = {LBM_F64: 8, LBM_F32: 4, LBM_F16S: 2, LBM_BF16S: 2, LBM_F16M: 2, LBM_BF16M: 2}
STATUS_DIVERGED = 0x1
STATUS_TIMEOUT = 0x4
NOALLOC_MAX_CELLS = 268435456
Q = 19


LBM_PATTERN_PULL, LBM_PATTERN_AA = 0, 1
PATTERN = {"pull": LBM_PATTERN_PULL, "aa": LBM_PATTERN_AA}
LBM_MODEL_QIAN, LBM_MODEL_INCOMPRESSIBLE = 0, 1
MODEL = {"qian": LBM_MODEL_QIAN, "incompressible": LBM_MODEL_INCOMPRESSIBLE}


class lbm_options(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("row_align", ctypes.c_int),
                ("pattern", ctypes.c_int), ("model", ctypes.c_int), ("stage_rows", ctypes.c_int)]


class lbm_info(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("pitch", ctypes.c_int),
                ("storage", ctypes.c_int), ("real_size", ctypes.c_int), ("tau", ctypes.c_double),
                ("n_cells", ctypes.c_int64), ("n_fluid", ctypes.c_int64), ("lattice_bytes", ctypes.c_size_t),
                ("tape_bytes_per_step", ctypes.c_size_t), ("steps_done", ctypes.c_int64), ("pattern", ctypes.c_int),
                ("model", ctypes.c_int)]


_vp = ctypes.c_void_p
_i = ctypes.c_int
_st = ctypes.c_int  # lbm_status

# name -> (restype, argtypes), in the order of include/lbm_capi.h
PROTOTYPES = {
    "lbm_options_default": (_st, [ctypes.POINTER(lbm_options)]),
    "lbm_create": (_st, [ctypes.POINTER(_vp), _i, _i, _i, ctypes.c_double, _vp, _vp, ctypes.POINTER(lbm_options)]),
    "lbm_destroy": (None, [_vp]),
    "lbm_get_info": (_st, [_vp, ctypes.POINTER(lbm_info)]),
    "lbm_set_uniform_force": (_st, [_vp, _vp]),
    "lbm_set_wall_velocity": (_st, [_vp, _vp]),
    "lbm_set_force_field": (_st, [_vp, _vp]),
    "lbm_init_equilibrium": (_st, [_vp, _vp, _vp]),
    "lbm_step": (_st, [_vp, _i]),
    "lbm_step_prepare": (_st, [_vp, _i]),
    "lbm_step_timed": (_st, [_vp, _i, ctypes.POINTER(ctypes.c_float)]),
    "lbm_macros": (_st, [_vp, _vp, _vp]),
    "lbm_reduce": (_st, [_vp, _vp]),
    "lbm_step_reduce": (_st, [_vp, _i, _vp]),
    "lbm_reduce_state_noalloc": (_st, [_vp, _i, _i, _i, _i, _vp, _vp, _vp, _vp]),
    "lbm_get_state": (_st, [_vp, _vp, _i]),
    "lbm_set_state": (_st, [_vp, _vp, _i]),
    "lbm_halo_bytes": (ctypes.c_size_t, [_vp]),
    "lbm_halo_pack": (_st, [_vp, _i, _vp]),
    "lbm_halo_unpack": (_st, [_vp, _i, _vp]),
    "lbm_reduce_planes": (_st, [_vp, _i, _i, _vp]),
    "lbm_step_planes": (_st, [_vp, _i, _i, _i, _vp]),
    "lbm_set_stream": (_st, [_vp, _vp]),
    "lbm_adjoint_halo_bytes": (ctypes.c_size_t, [_vp]),
    "lbm_adjoint_halo_pack": (_st, [_vp, _i, _vp]),
    "lbm_adjoint_halo_unpack": (_st, [_vp, _i, _vp]),
    "lbm_step_record": (_st, [_vp, _i, _vp]),
    "lbm_adjoint_seed": (_st, [_vp, _vp, _vp, _vp]),
    "lbm_adjoint_step": (_st, [_vp, _i, _vp, _vp]),
    "lbm_adjoint_init_grad": (_st, [_vp, _vp, _vp, _vp, _vp]),
    "lbm_status_word": (_st, [_vp, ctypes.POINTER(ctypes.c_uint32), _i]),
    "lbm_synchronize": (_st, [_vp]),
    "lbm_last_error": (ctypes.c_char_p, [_vp]),
    "lbm_status_string": (ctypes.c_char_p, [_i]),
    "lbm_lattice_table": (_i, [_vp, _vp, _vp]),
    "lbm_check_launch_indices": (ctypes.c_int64, [_i, _i, _i, _i, _i]),
}

_lib = None


def lib():
    """The loaded library (raises if it is missing: build it with paper_1112_0850_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("liblbm_gb300.so is not built (%s); run paper_1112_0850_gb300.build.build()"
                               % LIB_PATH)
        try:
            import torch  # noqa: F401  (load torch's CUDA runtime first so both share it)
        except ImportError:
            pass
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class LBMError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        super().__init__("%s: %s" % (status_string(status), message))


def status_string(s):
    return lib().lbm_status_string(int(s)).decode()


def check(status, ctx=None, what=""):
    if status != 0:
        msg = lib().lbm_last_error(ctx).decode() if ctx else ""
        raise LBMError(status, (what + ": " if what else "") + msg)


def __getattr__(name):
    if name in PROTOTYPES:
        return getattr(lib(), name)
    raise AttributeError(name)
