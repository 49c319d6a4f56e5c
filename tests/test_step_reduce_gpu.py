"""lbm_step_reduce: the totals of the current state summed inside the next
step. They equal lbm_reduce's totals up to the order of the FP64 sums, and
the steps themselves are the same steps (same bits as lbm_step)."""
import numpy as np
import pytest
import torch

from gpu_helpers import REAL, STORAGES, ensure_built
from test_parity_gpu import _case

pytestmark = pytest.mark.gpu


def _pair(storage, case, pattern="pull", model="qian"):
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    u0, rho0, tau, _, flags, F, Ffield = _case(case)
    nz, ny, nx = u0.shape[1:]
    real = REAL[storage]
    lats = []
    for _ in range(2):
        lat = Lattice(nx, ny, nz, tau, flags=flags, force=F, storage=storage, pattern=pattern, model=model)
        if Ffield is not None:
            lat.set_force_field(torch.as_tensor(Ffield, dtype=real).cuda())
        lat.init_equilibrium(torch.as_tensor(u0, dtype=real).cuda(),
                             None if rho0 is None else torch.as_tensor(rho0, dtype=real).cuda())
        lat.step(3)
        lats.append(lat)
    return lats


def _close(a, b):
    scale = max(abs(a[0]), 1.0)
    return abs(a[0] - b[0]) <= 1e-13 * scale and np.abs(a[1:] - b[1:]).max() <= 1e-13 * scale


@pytest.mark.parametrize("pattern", ["pull", "aa"])
@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("case", ["channel_64x20x18", "shear32", "field_10x9x8", "ragged_300x5x4"])
def test_step_reduce_equals_reduce_then_step(case, storage, pattern):
    a, b = _pair(storage, case, pattern)
    want = b.reduce()
    b.step(5)
    got = a.step_reduce(5)
    assert _close(got, want), (got, want)
    assert torch.equal(a.get_state(), b.get_state())
    # and the totals after the steps, through the device output
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    a.step_reduce(1, out)
    assert _close(out.cpu().numpy(), b.reduce())
    a.close()
    b.close()


def test_step_reduce_incompressible_momentum():
    a, b = _pair("f32", "channel_64x20x18", model="incompressible")
    want = b.reduce()
    got = a.step_reduce(2)
    assert _close(got, want)
    a.close()
    b.close()
