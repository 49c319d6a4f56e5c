"""The FP64 reference adjoint (autograd over an independent PyTorch restatement
of the update) against the C oracle's forward and against central finite
differences of the C oracle (CPU only)."""
import numpy as np
import pytest
import torch

import lbm_inputs
import oracle
from oracle import adjoint as oadj


def _case(n=(5, 6, 7), flags_frac=0.15, seed=21):
    nz, ny, nx = n
    rng = np.random.default_rng(seed)
    flags = lbm_inputs.random_flags(nx, ny, nz, flags_frac, seed) if flags_frac else None
    u0 = 0.02 * rng.standard_normal((3,) + n)
    F = 1e-4 * rng.standard_normal((3,) + n)
    ut = 0.02 * rng.standard_normal((3,) + n)
    return flags, u0, F, ut


def _loss_c(u0, F, tau, steps, ut, flags):
    f = oracle.init_equilibrium(u0, flags=flags)
    f = oracle.run(f, tau, steps, flags=flags, F=F, threads=1)
    _, u = oracle.macros(f, flags=flags, F=F)
    fluid = np.ones(u0.shape[1:], bool) if flags is None else flags == 0
    r = (u - ut) * fluid
    return 0.5 * float((r * r).sum())


@pytest.mark.parametrize("with_flags", [False, True])
def test_torch_forward_matches_c_oracle(with_flags):
    flags, u0, F, _ = _case(flags_frac=0.2 if with_flags else 0.0)
    rho_t, u_t, f_t = oadj.forward(torch.tensor(u0), torch.tensor(F), 0.57, 9, flags)
    f_c = oracle.run(oracle.init_equilibrium(u0, flags=flags), 0.57, 9, flags=flags, F=F)
    rho_c, u_c = oracle.macros(f_c, flags=flags, F=F)
    # same arithmetic, different operation order: a few ulp apart after 9 steps
    assert np.abs(f_t.numpy() - f_c).max() < 4e-15
    assert np.abs(u_t.numpy() - u_c).max() < 2e-15
    assert np.abs(rho_t.numpy() - rho_c).max() < 8e-15


@pytest.mark.parametrize("with_flags", [False, True])
def test_reference_gradient_matches_central_differences(with_flags):
    flags, u0, F, ut = _case(flags_frac=0.2 if with_flags else 0.0, seed=22)
    tau, steps = 0.6, 12
    L, gu, gF = oadj.gradients(u0, F, tau, steps, ut, flags)
    assert abs(L - _loss_c(u0, F, tau, steps, ut, flags)) < 1e-15 * max(1.0, L) * 10
    rng = np.random.default_rng(23)
    fluid = np.ones(u0.shape[1:], bool) if flags is None else flags == 0
    for _ in range(3):
        vu = rng.standard_normal(u0.shape) * fluid
        vF = rng.standard_normal(F.shape) * fluid
        eu = 1e-5 * np.linalg.norm(u0) / np.linalg.norm(vu)
        eF = 1e-5 * np.linalg.norm(F) / np.linalg.norm(vF)
        fd_u = (_loss_c(u0 + eu * vu, F, tau, steps, ut, flags)
                - _loss_c(u0 - eu * vu, F, tau, steps, ut, flags)) / (2 * eu)
        fd_F = (_loss_c(u0, F + eF * vF, tau, steps, ut, flags)
                - _loss_c(u0, F - eF * vF, tau, steps, ut, flags)) / (2 * eF)
        assert abs(fd_u - (gu * vu).sum()) <= 1e-6 * abs(fd_u), (fd_u, (gu * vu).sum())
        assert abs(fd_F - (gF * vF).sum()) <= 1e-6 * abs(fd_F), (fd_F, (gF * vF).sum())


def test_reference_vjp_is_linear_in_cotangent():
    flags, u0, F, _ = _case(seed=24)
    rng = np.random.default_rng(25)
    g1, g2 = rng.standard_normal(u0.shape), rng.standard_normal(u0.shape)
    a = oadj.vjp_of_velocity(u0, F, 0.6, 4, g1, flags)
    b = oadj.vjp_of_velocity(u0, F, 0.6, 4, g2, flags)
    c = oadj.vjp_of_velocity(u0, F, 0.6, 4, 2.0 * g1 - g2, flags)
    for k in range(2):
        assert np.abs(c[k] - (2 * a[k] - b[k])).max() < 1e-12 * np.abs(c[k]).max()


def test_torch_forward_matches_c_oracle_with_moving_lid():
    n = 7
    flags = np.ones((n, n, n), np.uint8)
    flags[1:-1, 1:-1, 1:-1] = 0
    flags[1:-1, n - 1, 1:-1] = 2
    rng = np.random.default_rng(31)
    u0 = 0.01 * rng.standard_normal((3, n, n, n)) * (flags == 0)
    F = np.zeros((3, n, n, n))
    uw = np.array([0.05, 0.0, 0.02])
    _, u_t, f_t = oadj.forward(torch.tensor(u0), torch.tensor(F), 0.6, 12, flags, u_wall=uw)
    f_c = oracle.run(oracle.init_equilibrium(u0, flags=flags), 0.6, 12, flags=flags, F=F, u_wall=uw)
    assert np.abs(f_t.numpy() - f_c).max() < 4e-15


def _loss_c_model(u0, F, tau, steps, ut, flags, model):
    f = oracle.init_equilibrium(u0, flags=flags, model=model)
    f = oracle.run(f, tau, steps, flags=flags, F=F, threads=1, model=model)
    _, u = oracle.macros(f, flags=flags, F=F, model=model)
    fluid = np.ones(u0.shape[1:], bool) if flags is None else flags == 0
    r = (u - ut) * fluid
    return 0.5 * float((r * r).sum())


def test_incompressible_torch_forward_matches_c_oracle():
    flags, u0, F, _ = _case(flags_frac=0.2, seed=26)
    inc = "incompressible"
    rho0 = 1.0 + 0.05 * np.random.default_rng(27).standard_normal(u0.shape[1:])
    _, u_t, f_t = oadj.forward(torch.tensor(u0), torch.tensor(F), 0.57, 9, flags, rho0=torch.tensor(rho0),
                               model=inc)
    f_c = oracle.run(oracle.init_equilibrium(u0, rho0=rho0, flags=flags, model=inc), 0.57, 9, flags=flags, F=F,
                     model=inc)
    _, u_c = oracle.macros(f_c, flags=flags, F=F, model=inc)
    assert np.abs(f_t.numpy() - f_c).max() < 4e-15
    assert np.abs(u_t.numpy() - u_c).max() < 2e-15
    # and it is not the Qian update
    f_q = oracle.run(oracle.init_equilibrium(u0, rho0=rho0, flags=flags), 0.57, 9, flags=flags, F=F)
    assert np.abs(f_q - f_c).max() > 1e-5


def test_incompressible_reference_gradient_matches_central_differences():
    flags, u0, F, ut = _case(flags_frac=0.2, seed=28)
    tau, steps, inc = 0.6, 10, "incompressible"
    L, gu, gF = oadj.gradients(u0, F, tau, steps, ut, flags, model=inc)
    assert abs(L - _loss_c_model(u0, F, tau, steps, ut, flags, inc)) < 1e-14 * max(1.0, L)
    rng = np.random.default_rng(29)
    fluid = flags == 0
    for _ in range(2):
        vu = rng.standard_normal(u0.shape) * fluid
        vF = rng.standard_normal(F.shape) * fluid
        eu = 1e-5 * np.linalg.norm(u0) / np.linalg.norm(vu)
        eF = 1e-5 * np.linalg.norm(F) / np.linalg.norm(vF)
        fd_u = (_loss_c_model(u0 + eu * vu, F, tau, steps, ut, flags, inc)
                - _loss_c_model(u0 - eu * vu, F, tau, steps, ut, flags, inc)) / (2 * eu)
        fd_F = (_loss_c_model(u0, F + eF * vF, tau, steps, ut, flags, inc)
                - _loss_c_model(u0, F - eF * vF, tau, steps, ut, flags, inc)) / (2 * eF)
        assert abs(fd_u - (gu * vu).sum()) <= 1e-6 * abs(fd_u), (fd_u, (gu * vu).sum())
        assert abs(fd_F - (gF * vF).sum()) <= 1e-6 * abs(fd_F), (fd_F, (gF * vF).sum())
