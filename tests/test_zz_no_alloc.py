"""lbm_reduce_state_noalloc: the mass/momentum totals for callers that cannot
allocate device memory (its scratch is a fixed device array inside the
library). Called through the C-ABI and checked against lbm_reduce, which uses
memory the context allocated, on two calls in a row (the shared scratch keeps
the previous call's contents, which must not leak into the next result).

This file is collected last so that a run stopping at the first failure has
already run every other test; it passes alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest
import torch

import lbm_inputs
from gpu_helpers import REAL, ensure_built

pytestmark = pytest.mark.gpu

# Both paths read the same stored values; lbm_reduce forms each cell's
# moments in the context's arithmetic (FP32 for every format but FP64) and the
# entry point in FP64, and the two sum in different orders. Per cell that is a
# relative difference of a few 2^-24 in FP32, so the totals may differ by
# ~1e-7 of the mass and, for the momentum, by ~1e-5 absolute over these 25k
# fluid cells (the momentum total is ~1e-1 .. 1; a wrong F/2 term would move it
# by 0.5 |F| N ~ 0.25).
TOL_MASS = {"f64": 1e-13, "f32": 1e-7, "f16s": 1e-7, "bf16s": 1e-7}
TOL_MOM = {"f64": 1e-11, "f32": 1e-5, "f16s": 1e-5, "bf16s": 1e-5}


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s", "bf16s"])
def test_noalloc_totals_match_lbm_reduce_on_two_calls(storage):
    """Two calls in a row on two different states (the second sees a scratch
    array still holding the first call's partials), each against lbm_reduce;
    between the two calls nothing else allocates, and the device's free
    memory is the same after the second call as after the first."""
    from paper_1112_0850_gb300 import capi
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    nx, ny, nz = 70, 21, 19  # 27930 cells: two scratch blocks, the second one ragged
    flags = lbm_inputs.channel_flags(nx, ny, nz, 0.1, lbm_inputs.seed_for(1))
    F = (2e-5, -1e-5, 5e-6)
    rng = np.random.default_rng(11)
    u0 = 0.02 * rng.standard_normal((3, nz, ny, nx))
    lat = Lattice(nx, ny, nz, 0.57, flags=flags, force=F, storage=storage)
    lat.init_equilibrium(torch.tensor(u0, dtype=REAL[storage], device="cuda"))
    lat.step(6)
    fl = torch.tensor(flags, device="cuda")
    Fc = (ctypes.c_double * 3)(*F)
    stream = ctypes.c_void_p(lat.stream.cuda_stream)
    # everything the two calls read and write exists before the first one
    refs, states = [], []
    for _ in range(2):
        refs.append(lat.reduce())
        states.append(lat.get_state())
        lat.step(9)  # the second call sees a different state
    outs = [torch.full((4,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    free = []
    for call in range(2):
        rc = capi.lib().lbm_reduce_state_noalloc(states[call].data_ptr(), lat.storage, nx, ny, nz, fl.data_ptr(),
                                                 Fc, outs[call].data_ptr(), stream)
        assert rc == 0, capi.status_string(rc)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    assert free[1] == free[0], free
    for call in range(2):
        got, ref = outs[call].cpu().numpy(), refs[call]
        assert abs(got[0] - ref[0]) <= TOL_MASS[storage] * abs(ref[0]), (call, got, ref)
        assert np.abs(got[1:] - ref[1:]).max() <= TOL_MOM[storage], (call, got, ref)
    assert not np.array_equal(outs[0].cpu().numpy(), outs[1].cpu().numpy())
    lat.close()


def test_noalloc_rejects_lattices_beyond_its_scratch():
    from paper_1112_0850_gb300 import capi
    ensure_built()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(1, dtype=torch.float32, device="cuda")
    # 1024^3 cells exceed LBM_NOALLOC_MAX_CELLS: refused on the host, nothing launched
    rc = capi.lib().lbm_reduce_state_noalloc(dummy.data_ptr(), capi.LBM_F32, 1024, 1024, 1024, None, None,
                                             out.data_ptr(), None)
    assert rc == 1  # LBM_ERR_ARG
    assert 1024 ** 3 > capi.NOALLOC_MAX_CELLS
    rc = capi.lib().lbm_reduce_state_noalloc(None, capi.LBM_F32, 4, 4, 4, None, None, out.data_ptr(), None)
    assert rc == 1
