"""Failure paths of the C-ABI on the GPU, none of which faults the GPU:

- a deliberately unstable run (tau = 0.5001 with |u| up to 0.3, far beyond
  the stable range of BGK) drives densities negative and then non-finite; the
  kernels only set the divergence bit of the status word (every address is
  independent of the data), the synchronizing calls report LBM_ERR_DIVERGED,
  and the context stays usable once a new state is loaded;
- a lattice whose two lattices cannot fit in device memory is refused with
  LBM_ERR_OOM before anything is allocated.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import ensure_built

pytestmark = pytest.mark.gpu


def _lattice(*a, **k):
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    return Lattice(*a, **k)


@pytest.mark.parametrize("storage", ["f32", "f16s", "bf16m"])
def test_unstable_run_is_reported_not_trapped(storage):
    from paper_1112_0850_gb300 import capi
    n = 16
    rng = np.random.default_rng(7)
    u = torch.tensor(0.3 * rng.uniform(-1.0, 1.0, (3, n, n, n)), dtype=torch.float32).cuda()
    lat = _lattice(n, n, n, 0.5001, storage=storage)
    lat.init_equilibrium(u)
    lat.synchronize()  # a fresh state: no divergence yet
    lat.step(200)  # the FP64 oracle reaches negative densities within 40 steps
    with pytest.raises(capi.LBMError) as ex:
        lat.synchronize()
    assert ex.value.status == 5 and "LBM_ERR_DIVERGED" in str(ex.value)
    with pytest.raises(capi.LBMError) as ex:
        lat.reduce()
    assert ex.value.status == 5
    assert lat.status_word(clear=True) & capi.STATUS_DIVERGED
    # the context is still usable: a new state clears the word and runs cleanly
    lat.step(3)
    lat.init_equilibrium(torch.zeros_like(u))
    lat.step(10)
    lat.synchronize()
    tot = lat.reduce()
    assert abs(tot[0] - n ** 3) <= 1e-9 * n ** 3 and np.abs(tot[1:]).max() == 0.0
    lat.close()


def test_oom_refused_before_any_allocation():
    from paper_1112_0850_gb300 import capi
    ensure_built()
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info()
    # 1280 x 1280 x 1300 cells (just under 2^31 padded cells) in FP64: two
    # lattices of 19 x 8 B per cell need about 650 GB
    for storage in ("f64", "f32"):
        with pytest.raises(capi.LBMError) as ex:
            _lattice(1280, 1280, 1300, 0.6, storage=storage)
        assert ex.value.status == 2, str(ex.value)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
