"""dJ/dU0 through rollouts of REXI steps: finite differences, the oracle's adjoint,
checkpointing, and the dot-product identity on the GPU."""
import numpy as np
import pytest

from oracle import rexi_coeffs as rc
from oracle import step as ostep
from oracle.swe import Consts
from paper_1812_03431_gb300 import inputs

pytestmark = pytest.mark.gpu
C = Consts()


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1812_03431_gb300 import autograd, rexi
    rexi.load()
    return torch, rexi, autograd


def misfit(torch, autograd, plan, x0, y, nsteps, every):
    u = autograd.rollout(plan, x0, nsteps, checkpoint_every=every)
    return ((u - y) ** 2).sum()


@pytest.mark.parametrize("arith", ["fp64", "fp32x2"])
def test_gradient_matches_oracle_adjoint(env, arith):
    torch, rexi, autograd = env
    N, nlat, nlon, M, tau, steps = 31, 48, 96, 32, 3600.0, 3
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    gs = ostep.GridStep(N, nlat, nlon, al, be, tau, C)
    x0 = gs.synthesise(inputs.random_spectral(N, 1, 61))
    y = gs.synthesise(inputs.random_spectral(N, 1, 62))
    plan = rexi.Plan(N, nlat, nlon, tau=tau, alpha=al, beta=be, solve_arith=arith)
    X = torch.from_numpy(x0).cuda().requires_grad_(True)
    J = misfit(torch, autograd, plan, X, torch.from_numpy(y).cuda(), steps, 0)
    J.backward()
    # oracle: forward states, then the transposed steps applied to 2 (u - y)
    u = x0
    for _ in range(steps):
        u = gs(u)
    g = 2 * (u - y)
    for _ in range(steps):
        g = gs.adjoint(g)
    got = X.grad.cpu().numpy()
    assert np.linalg.norm(got - g) / np.linalg.norm(g) < 1e-10


@pytest.mark.parametrize("arith", ["fp64", "fp32x2"])
def test_c4_rollout_fd_and_checkpointing(env, arith):
    """T170 on 512x256, K=256, 8 steps of 3600 s, J = ||U(T) - y||^2, checkpoint every 2."""
    torch, rexi, autograd = env
    N, nlat, nlon, tau, steps = 170, 256, 512, 3600.0, 8
    plan = rexi.Plan(N, nlat, nlon, M=256, tau=tau, solve_arith=arith)
    S0 = torch.from_numpy(inputs.random_spectral(N, 1, 1003)).cuda()
    x0 = plan.synthesize(S0)
    yS = torch.from_numpy(inputs.random_spectral(N, 1, 1013)).cuda()
    y = plan.synthesize(S0 + 0.1 * yS)  # seeded perturbed state as the target
    X = x0.clone().requires_grad_(True)
    J = misfit(torch, autograd, plan, X, y, steps, 2)
    J.backward()
    gck = X.grad.clone()
    X2 = x0.clone().requires_grad_(True)
    misfit(torch, autograd, plan, X2, y, steps, 0).backward()
    assert torch.equal(gck, X2.grad)  # checkpointing changes nothing (linear, deterministic steps)
    d = plan.synthesize(torch.from_numpy(inputs.random_spectral(N, 1, 1023)).cuda())
    eps = 1e-6 * float(x0.norm() / d.norm())
    with torch.no_grad():
        jp = float(misfit(torch, autograd, plan, x0 + eps * d, y, steps, 0))
        jm = float(misfit(torch, autograd, plan, x0 - eps * d, y, steps, 0))
    fd = (jp - jm) / (2 * eps)
    an = float((gck * d).sum())
    assert abs(fd - an) <= 1e-6 * abs(an)


# float-float solves carry 32x binary64's unit roundoff (2^-48 against 2^-53)
DOT_TOL = {"fp64": 1e-13, "fp32x2": 3e-12}


@pytest.mark.parametrize("arith", ["fp64", "fp32x2"])
def test_dot_product_identity_gpu(env, arith):
    torch, rexi, _ = env
    for layout in ("grid", "spectral"):
        N, nlat, nlon = 63, 96, 192
        plan = rexi.Plan(N, nlat, nlon, M=64, tau=3600.0, max_batch=2, layout=layout, solve_arith=arith)
        if layout == "grid":
            x = torch.from_numpy(inputs.random_grid(2, nlat, nlon, 71)).cuda()
            y = torch.from_numpy(inputs.random_grid(2, nlat, nlon, 72)).cuda()
            lhs = float((plan.step(x) * y).sum())
            rhs = float((plan.step_adjoint(y) * x).sum())
            scale = float(plan.step(x).norm() * y.norm())
        else:
            x = torch.from_numpy(inputs.random_spectral(N, 2, 71)).cuda()
            y = torch.from_numpy(inputs.random_spectral(N, 2, 72)).cuda()
            lhs = float(torch.vdot(y.flatten(), plan.step(x).flatten()).real)
            rhs = float(torch.vdot(plan.step_adjoint(y).flatten(), x.flatten()).real)
            scale = float(plan.step(x).norm() * y.norm())
        assert abs(lhs - rhs) < DOT_TOL[arith] * scale
        plan.close()
