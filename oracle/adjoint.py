"""FP64 reference adjoint of the D3Q19 BGK update, by reverse-mode autograd.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). This file restates the
forward update of Sec. 2 (moments, Qian equilibrium, BGK relaxation of Eq. 1,
streaming, bounce-back after Ziegler) with the Guo body force, as whole-array
PyTorch CPU operations in float64, written independently of lbm_oracle.c; the
tests check the two forward codes against each other. The gradient of a
final-time loss is then torch.autograd's exact reverse of those operations,
so no adjoint formula is written out by hand here.

Canonical layout as in the C oracle: f[19][nz][ny][nx], u[3][nz][ny][nx],
flags uint8 [nz][ny][nx] (0 fluid, 1 solid), all axes periodic. `model`
"incompressible" selects the He & Luo equilibrium (velocity terms with the
reference density 1, u = j + F/2) instead of the Qian one.
"""
import torch

# D3Q19 (Qian et al., cited in Sec. 2): rest, +x,-x,+y,-y,+z,-z, then the edge
# diagonals (+-1,+-1,0), (+-1,0,+-1), (0,+-1,+-1), + before -.
_E = [(0, 0, 0),
      (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
      (1, 1, 0), (1, -1, 0), (-1, 1, 0), (-1, -1, 0),
      (1, 0, 1), (1, 0, -1), (-1, 0, 1), (-1, 0, -1),
      (0, 1, 1), (0, 1, -1), (0, -1, 1), (0, -1, -1)]
_W = [1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12
_OPP = [_E.index((-a, -b, -c)) for (a, b, c) in _E]


def _fluid_mask(flags, shape):
    if flags is None:
        return torch.ones(shape, dtype=torch.bool)
    return torch.as_tensor(flags) == 0


def equilibrium(rho, u, model=None):
    """f_eq_i = w_i rho [1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u] (Qian), or
    w_i [rho + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u] (He & Luo), stacked over i."""
    uu = (u * u).sum(0)
    out = []
    for (ex, ey, ez), w in zip(_E, _W):
        eu = ex * u[0] + ey * u[1] + ez * u[2]
        if model == "incompressible":
            out.append(w * (rho + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu))
        else:
            out.append(w * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu))
    return torch.stack(out)


def moments(f, F, fluid, model=None):
    """rho = sum f_i, u = (sum f_i e_i + F/2)/rho (Qian) or sum f_i e_i + F/2
    (He & Luo); rho set to 1 on solid cells."""
    rho = f.sum(0)
    rho = torch.where(fluid, rho, torch.ones_like(rho))
    j = [sum(e[a] * f[i] for i, e in enumerate(_E)) for a in range(3)]
    if model == "incompressible":
        u = torch.stack([j[a] + 0.5 * F[a] for a in range(3)])
    else:
        u = torch.stack([(j[a] + 0.5 * F[a]) / rho for a in range(3)])
    return rho, u


def step(f, tau, fluid, F, moving=None, u_wall=None, model=None):
    """One collide-and-push step (Sec. 2 steps 1-3 and the bounce-back rule).

    moving: bool mask of walls moving with u_wall; a population reflected off
    one loses 6 w_i (e_i . u_wall) (halfway bounce-back for a moving wall)."""
    rho, u = moments(f, F, fluid, model)
    feq = equilibrium(rho, u, model)
    uF = (u * F).sum(0)
    c = 1.0 - 1.0 / (2.0 * tau)
    new = [torch.zeros_like(f[0]) for _ in _E]
    for i, ((ex, ey, ez), w) in enumerate(zip(_E, _W)):
        eu = ex * u[0] + ey * u[1] + ez * u[2]
        eF = ex * F[0] + ey * F[1] + ez * F[2]
        S = c * w * (3.0 * (eF - uF) + 9.0 * eu * eF)
        fstar = f[i] - (f[i] - feq[i]) / tau + S
        # fluid(x + e_i) seen from x
        dest_fluid = torch.roll(fluid, shifts=(-ez, -ey, -ex), dims=(0, 1, 2))
        pushed = torch.where(fluid & dest_fluid, fstar, torch.zeros_like(fstar))
        new[i] = new[i] + torch.roll(pushed, shifts=(ez, ey, ex), dims=(0, 1, 2))
        refl = fstar
        if moving is not None and u_wall is not None:
            dest_moving = torch.roll(moving, shifts=(-ez, -ey, -ex), dims=(0, 1, 2))
            eu_w = ex * float(u_wall[0]) + ey * float(u_wall[1]) + ez * float(u_wall[2])
            refl = fstar - 6.0 * w * eu_w * dest_moving.to(fstar.dtype)
        bounced = torch.where(fluid & ~dest_fluid, refl, torch.zeros_like(fstar))
        new[_OPP[i]] = new[_OPP[i]] + bounced
    return torch.stack(new)


def forward(u0, F, tau, steps, flags=None, rho0=None, u_wall=None, model=None):
    """f^0 = f_eq(rho0, u0) at fluid cells, then `steps` updates; returns (rho_T, u_T, f_T).
    Cells flagged 2 are walls moving with u_wall."""
    shape = u0.shape[1:]
    fluid = _fluid_mask(flags, shape)
    moving = None if flags is None else torch.as_tensor(flags) == 2
    rho_init = torch.ones(shape, dtype=u0.dtype) if rho0 is None else rho0
    f = equilibrium(rho_init, u0, model) * fluid
    for _ in range(steps):
        f = step(f, tau, fluid, F, moving, u_wall, model)
    rho, u = moments(f, F, fluid, model)
    return rho * fluid, u * fluid, f


def velocity_loss(u0, F, tau, steps, u_target, flags=None, u_wall=None, model=None):
    """L = 1/2 sum over fluid cells of |u(T) - u_target|^2."""
    shape = u0.shape[1:]
    fluid = _fluid_mask(flags, shape)
    _, u, _ = forward(u0, F, tau, steps, flags, u_wall=u_wall, model=model)
    r = (u - u_target) * fluid
    return 0.5 * (r * r).sum()


def gradients(u0, F, tau, steps, u_target, flags=None, u_wall=None, model=None):
    """(L, dL/du0 [3][nz][ny][nx], dL/dF [3][nz][ny][nx]) in float64 by autograd.

    u0, F and u_target are numpy or torch arrays; F is a per-cell force field.
    """
    u0 = torch.as_tensor(u0, dtype=torch.float64).clone().requires_grad_(True)
    F = torch.as_tensor(F, dtype=torch.float64).clone().requires_grad_(True)
    ut = torch.as_tensor(u_target, dtype=torch.float64)
    L = velocity_loss(u0, F, tau, steps, ut, flags, u_wall, model)
    gu, gF = torch.autograd.grad(L, (u0, F))
    fluid = _fluid_mask(flags, u0.shape[1:])
    return L.item(), (gu * fluid).numpy(), (gF * fluid).numpy()


def vjp_of_velocity(u0, F, tau, steps, g, flags=None):
    """(d<g, u_T>/du0, d<g, u_T>/dF) for an arbitrary cotangent g [3][nz][ny][nx]."""
    u0 = torch.as_tensor(u0, dtype=torch.float64).clone().requires_grad_(True)
    F = torch.as_tensor(F, dtype=torch.float64).clone().requires_grad_(True)
    g = torch.as_tensor(g, dtype=torch.float64)
    _, u, _ = forward(u0, F, tau, steps, flags)
    gu, gF = torch.autograd.grad((u * g).sum(), (u0, F))
    return gu.numpy(), gF.numpy()
