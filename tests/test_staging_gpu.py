"""The two-grid step with TMA row staging (opt-in, FP32 and 16-bit storage)
against the same step with direct loads (the default): the gathered values, the
arithmetic and the stores are the same, so states, tapes and statuses must
agree bit for bit, across the parity cases (ragged rows, one-cell axes,
obstacles, uniform and per-cell forces) and with moving walls."""
import numpy as np
import pytest
import torch

from gpu_helpers import REAL, ensure_built
from test_parity_gpu import CASES, _case

pytestmark = pytest.mark.gpu


def _run(storage, case, staged, steps=9, record=False, u_wall=None, flags_override=None):
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    u0, rho0, tau, _, flags, F, Ffield = _case(case)
    if flags_override is not None:
        flags = flags_override
    nz, ny, nx = u0.shape[1:]
    real = REAL[storage]
    # 128-byte rows, so that every case is eligible for the staged kernel
    lat = Lattice(nx, ny, nz, tau, flags=flags, force=F, storage=storage, stage_rows=staged, row_align=128)
    if Ffield is not None:
        lat.set_force_field(torch.as_tensor(Ffield, dtype=real).cuda())
    if u_wall is not None:
        lat.set_wall_velocity(u_wall)
    lat.init_equilibrium(torch.as_tensor(u0, dtype=real).cuda(),
                         None if rho0 is None else torch.as_tensor(rho0, dtype=real).cuda())
    tape = None
    if record:
        tape = lat.new_tape(steps)
        lat.step_record(steps, tape)
    else:
        lat.step(steps)
    out = (lat.get_state(), tape, lat.status_word())
    lat.close()
    return out


@pytest.mark.parametrize("storage", ["f32", "f16s", "bf16s"])
@pytest.mark.parametrize("case", CASES)
def test_staged_step_equals_direct_loads(storage, case):
    a = _run(storage, case, False)
    b = _run(storage, case, True)
    assert torch.equal(a[0], b[0]), case
    assert a[2] == b[2] == 0


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_staged_record_equals_direct_loads(storage):
    a = _run(storage, "channel_64x20x18", False, steps=5, record=True)
    b = _run(storage, "channel_64x20x18", True, steps=5, record=True)
    assert torch.equal(a[0], b[0])
    # the tape at fluid cells (solid cells' entries are never read, and rows of
    # solid cells outside the fluid box are not written)
    u0, _, _, _, flags, _, _ = _case("channel_64x20x18")
    nz, ny, nx = u0.shape[1:]
    ta = a[1].view(REAL[storage]).view(5, 4, nz, ny, -1)[..., :nx]
    tb = b[1].view(REAL[storage]).view(5, 4, nz, ny, -1)[..., :nx]
    m = torch.tensor(flags == 0, device=ta.device)
    assert torch.equal(ta[:, :, m], tb[:, :, m])


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_staged_moving_walls_equal_direct_loads(storage):
    u0, _, _, _, _, _, _ = _case("flags_33x7x5")
    nz, ny, nx = u0.shape[1:]
    flags = np.zeros((nz, ny, nx), np.uint8)
    flags[:, 0, :] = 1
    flags[:, ny - 1, :] = 2
    flags[:, :, 5] = 2
    a = _run(storage, "flags_33x7x5", False, steps=12, u_wall=(0.02, 0.0, 0.01), flags_override=flags)
    b = _run(storage, "flags_33x7x5", True, steps=12, u_wall=(0.02, 0.0, 0.01), flags_override=flags)
    assert torch.equal(a[0], b[0])
