"""The FP32 step with flags addresses its lattice with 32-bit offsets while
all 19 padded population arrays span fewer than 2^32 elements, and the FP32
reverse step while they (and the 3 gradient components) span fewer than
2^31; past that both take 64-bit offsets. Rows padded to 4096 bytes (1024
FP32 values) make such lattices from few cells, so the same cells can be run
in both forms: the padded lattice must evolve, and give the force gradient,
bit for bit as the unpadded one (the arithmetic per cell does not depend on
the layout, and the 32-bit forms are checked against the oracle in the
parity and adjoint tests).

Device memory: about 36 GB for the forward case, 58 GB for the reverse one.
"""
import numpy as np
import pytest
import torch

import lbm_inputs
from gpu_helpers import ensure_built

pytestmark = pytest.mark.gpu

Q = 19
PAD = 4096  # bytes per padded row


def _pair(n, F):
    from paper_1112_0850_gb300.lattice import Lattice
    ensure_built()
    flags = lbm_inputs.channel_flags(8, n, n, 0.1, lbm_inputs.seed_for(1))
    wide = Lattice(8, n, n, 0.55, flags=flags, force=F, storage="f32", row_align=PAD)
    narrow = Lattice(8, n, n, 0.55, flags=flags, force=F, storage="f32")
    assert wide.info.pitch == PAD // 4 and narrow.info.pitch == 8
    rng = np.random.default_rng(5)
    u0 = torch.tensor(0.02 * rng.standard_normal((3, n, n, 8)) * (flags == 0), dtype=torch.float32, device="cuda")
    for lat in (wide, narrow):
        lat.init_equilibrium(u0)
    return flags, wide, narrow


def test_step_past_32bit_offsets_matches_unpadded_bit_for_bit():
    n = 470  # padded: 19 x 470 x 470 x 1024 = 4.298e9 elements > 2^32
    assert Q * n * n * (PAD // 4) >= 2 ** 32
    _, wide, narrow = _pair(n, (1e-5, -2e-6, 3e-6))
    for lat in (wide, narrow):
        lat.step(1)   # one launch
        lat.step(11)  # a replayed graph of 11 steps
    a, b = wide.get_state(), narrow.get_state()
    torch.cuda.synchronize()
    assert wide.status_word() == 0 and narrow.status_word() == 0
    assert torch.count_nonzero(b).item() > 0
    assert torch.equal(a, b)
    wide.close()
    narrow.close()


def test_reverse_step_past_31bit_offsets_matches_unpadded_bit_for_bit():
    n = 336  # padded: 19 x 336 x 336 x 1024 = 2.197e9 elements > 2^31 (and < 2^32: the forward step is 32-bit)
    assert 2 ** 31 <= Q * n * n * (PAD // 4) < 2 ** 32
    flags, wide, narrow = _pair(n, (1e-5, -2e-6, 3e-6))
    K = 3
    rng = np.random.default_rng(9)
    seed = torch.tensor(1e-3 * rng.standard_normal((3, n, n, 8)) * (flags == 0), dtype=torch.float32,
                        device="cuda")
    grads = []
    for lat in (wide, narrow):
        lat.step(2)
        tape = lat.new_tape(K)
        lat.step_record(K, tape)
        gF = lat.zeros(3)
        lat.adjoint_seed(seed, None, gF)
        lat.adjoint_step(K, tape, gF)
        torch.cuda.synchronize()
        assert lat.status_word() == 0
        grads.append(gF)
        del tape
    assert torch.count_nonzero(grads[1]).item() > 0
    assert torch.equal(grads[0], grads[1])
    wide.close()
    narrow.close()
