"""Differentiable rollout: u(T) = LBM^T(u0, F) with a hand-written discrete adjoint.

`LBMRollout.apply(u0, F, lattice, steps, ckpt_every, ckpt_fmt)` runs
`steps` fused stream-collide updates from f^0 = f_eq(1, u0) under the
per-cell body force F and returns the final velocity u(T) (real
[3][nz][ny][nx]). Its backward pass gives dL/du0 and dL/dF through the
library's adjoint kernels (lbm_adjoint_seed / lbm_adjoint_step /
lbm_adjoint_init_grad), with uniform checkpointing: the forward pass keeps the
state every `ckpt_every` steps (in format `ckpt_fmt`), the backward pass
restores each checkpoint, recomputes its segment while recording the moments
the adjoint needs (lbm_step_record), and then runs the segment's adjoint
steps in reverse. Memory: one checkpoint per segment plus one segment's tape.
Checkpoints default to the lattice's own storage format; a moment-split
lattice (whose canonical state has no exact 16-bit form) keeps FP32 ones.
"""
import torch

from . import capi


class LBMRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, F, lattice, steps, ckpt_every, ckpt_fmt=None):
        lat = lattice
        own = capi.LBM_F32 if lat.storage in (capi.LBM_F16M, capi.LBM_BF16M) else lat.storage
        fmt = own if ckpt_fmt is None else (capi.STORAGE[ckpt_fmt] if isinstance(ckpt_fmt, str) else int(ckpt_fmt))
        u0 = u0.detach().contiguous()
        F = F.detach().contiguous()
        lat.set_force_field(F)
        lat.init_equilibrium(u0)
        K = max(1, int(ckpt_every))
        ckpts = []
        done = 0
        while done < steps:
            n = min(K, steps - done)
            ckpts.append((lat.get_state(fmt), n))
            lat.step(n)
            done += n
        final = lat.get_state(own)
        _, u = lat.macros(with_rho=False)
        ctx.lat = lat
        ctx.ckpts = ckpts
        ctx.final = final
        ctx.K = K
        ctx.save_for_backward(u0, F)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        lat = ctx.lat
        u0, F = ctx.saved_tensors
        lat.set_force_field(F)
        lat.set_state(ctx.final)
        grad_F = torch.zeros_like(F)
        lat.adjoint_seed(grad_u.contiguous().to(lat.real), None, grad_F)
        tape = lat.new_tape(ctx.K)
        for state, n in reversed(ctx.ckpts):
            lat.set_state(state)
            lat.step_record(n, tape)
            lat.adjoint_step(n, tape, grad_F)
        grad_u0, _ = lat.adjoint_init_grad(u0)
        return grad_u0, grad_F, None, None, None, None


def velocity_loss(u, u_target, fluid_mask=None):
    """L = 1/2 sum over fluid cells of |u - u_target|^2."""
    r = u - u_target
    if fluid_mask is not None:
        r = r * fluid_mask
    return 0.5 * (r * r).sum()
