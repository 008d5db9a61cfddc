"""Mixed-precision form (3xTF32 tensor-core Legendre transforms, FP64 solves) vs the FP64 oracle.

Stated tolerance: relative L2 error <= 1e-5 per field.  The 3xTF32 products carry
~2^-22 relative error each and accumulate in FP32; measured on GB300 the largest
error is ~3.4e-6 (vorticity/divergence analysis at T127), the full step ~1e-6.
"""
import numpy as np
import pytest

from oracle import rexi_coeffs as rc
from oracle import step as ostep
from oracle.swe import Consts
from paper_1812_03431_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-5
C = Consts()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1812_03431_gb300 import rexi
    rexi.load()
    return torch, rexi


@pytest.mark.parametrize("N,nlat,nlon,M,B", [(1, 2, 4, 2, 1), (31, 48, 96, 32, 2), (63, 96, 192, 64, 3),
                                             (127, 192, 384, 64, 17), (20, 30, 90, 16, 18)])
def test_mixed_transforms_step_adjoint(env, N, nlat, nlon, M, B):
    torch, rexi = env
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    gs = ostep.GridStep(N, nlat, nlon, al, be, 3600.0, C)
    plan = rexi.Plan(N, nlat, nlon, tau=3600.0, max_batch=B, alpha=al, beta=be, precision="mixed")
    S = inputs.random_spectral(N, B, 23)
    x = gs.synthesise(S)
    X = torch.from_numpy(x).cuda()
    got_syn = plan.synthesize(torch.from_numpy(S).cuda()).cpu().numpy()
    got_ana = plan.analyze(X).cpu().numpy()
    ref_ana = gs.analyse(x)
    got = plan.step(X).cpu().numpy()
    ref = gs(x)
    got_adj = plan.step_adjoint(X).cpu().numpy()
    ref_adj = gs.adjoint(x)
    plan.check_device()  # no bounded tensor-core wait expired
    for f in range(3):
        assert rel(got_syn[:, f], x[:, f]) < TOL_MIXED
        assert rel(got_ana[:, f], ref_ana[:, f]) < TOL_MIXED
        assert rel(got[:, f], ref[:, f]) < TOL_MIXED
        assert rel(got_adj[:, f], ref_adj[:, f]) < TOL_MIXED
    plan.close()


def test_mixed_balanced_flow_stays_steady(env):
    torch, rexi = env
    N, nlat, nlon = 63, 96, 192
    from oracle.sphere import gauss_legendre
    mu, _ = gauss_legendre(nlat)
    x = inputs.balanced_grid(mu, nlon)[None]
    plan = rexi.Plan(N, nlat, nlon, M=128, tau=3600.0, precision="mixed")
    y = plan.step(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, x) < TOL_MIXED
    plan.close()


def test_c2_batched_mixed_vs_fp64(env):
    """T127 on 384x192, K=256 (P=535), 64 seeded states, tau=7200 s: the batched plain vs
    mixed-precision configuration.  The FP64 form matches the oracle (two states, 1e-10);
    the mixed form, with binary64 and with float-float solves, matches the FP64 form state
    by state within the stated 1e-5, and the two solve arithmetics agree to 1e-11."""
    torch, rexi = env
    N, nlat, nlon, M, B, tau = 127, 192, 384, 256, 64, 7200.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    gs = ostep.GridStep(N, nlat, nlon, al, be, tau, C)
    x = gs.synthesise(inputs.random_spectral(N, B, 1001))
    X = torch.from_numpy(x).cuda()
    out = {}
    for prec, arith in (("fp64", "fp64"), ("mixed", "fp64"), ("mixed", "fp32x2")):
        plan = rexi.Plan(N, nlat, nlon, tau=tau, max_batch=B, alpha=al, beta=be, precision=prec,
                         solve_arith=arith)
        plan.tune(B)
        out[prec, arith] = plan.step(X).cpu().numpy()
        plan.check_device()
        plan.close()
    ref = gs(x[:2])
    for f in range(3):
        assert rel(out["fp64", "fp64"][:2, f], ref[:, f]) < 1e-10
    for arith in ("fp64", "fp32x2"):
        worst = max(rel(out["mixed", arith][b, f], out["fp64", "fp64"][b, f]) for b in range(B) for f in range(3))
        assert worst < TOL_MIXED
    assert rel(out["mixed", "fp32x2"], out["mixed", "fp64"]) < 1e-11


def test_mixed_synthesis_staged_by_class_matches_oracle(env):
    """The tcgen05 synthesis stages one accumulator class per degree block (two CTAs per SM)
    for groups of up to 8 states on grids of at least three CTAs per SM, else both classes
    per block.  T255 (512 work tiles): 2 states take the first way, 12 the second; both
    against the oracle's synthesis, and against each other (the same products in the same
    order per state)."""
    torch, rexi = env
    N, nlat, nlon, B = 255, 384, 768, 12
    gs = ostep.GridStep(N, nlat, nlon, np.ones(1, complex), np.ones(1, complex), 1.0, C)
    plan = rexi.Plan(N, nlat, nlon, M=8, max_batch=B, precision="mixed")
    S = inputs.random_spectral(N, B, 31)
    ref = gs.synthesise(S)
    x2 = plan.synthesize(torch.from_numpy(S[:2]).cuda()).cpu().numpy()
    x12 = plan.synthesize(torch.from_numpy(S).cuda()).cpu().numpy()
    plan.check_device()
    plan.close()
    for f in range(3):
        for b in range(2):
            assert rel(x2[b, f], ref[b, f]) < TOL_MIXED
        for b in range(B):
            assert rel(x12[b, f], ref[b, f]) < TOL_MIXED
    assert rel(x2, x12[:2]) < 1e-6
