"""Large single state: T1279 on a 3840 x 1920 Gaussian grid, K = 512 (P = 1047), tau = 21600 s.

tau max|omega| ~ 1360 is far outside the poles' valid range h (M - 10) ~ 100, so the
REXI result is not exp(tau L) U for high degrees (the paper needs M ~ 4096 for such
steps); parity with the oracle, which computes the same rational function, is exact.
"""
import numpy as np
import pytest

from oracle import rexi_coeffs as rc
from oracle import step as ostep
from oracle.sphere import idx
from oracle.swe import Consts
from paper_1812_03431_gb300 import inputs

pytestmark = pytest.mark.gpu
N, NLAT, NLON, M, TAU = 1279, 1920, 3840, 512, 21600.0


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("arith", ["fp64", "fp32x2"])
def test_t1279_spectral_step_sampled_orders(arith):
    import torch
    from paper_1812_03431_gb300 import rexi
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    plan = rexi.Plan(N, NLAT, NLON, tau=TAU, layout="spectral", alpha=al, beta=be, solve_arith=arith)
    S = inputs.random_spectral(N, 1, 1004)
    got = plan.step(torch.from_numpy(S).cuda()).cpu().numpy()
    plan.close()
    ms = [0, 1, 640, 1278, 1279]
    ref = ostep.rexi_step_spectral(S, N, al, be, TAU, Consts(), ms=ms)
    sel = np.concatenate([np.arange(idx(m, m, N), idx(m, N, N) + 1) for m in ms])
    for f in range(3):
        assert rel(got[0, f, sel], ref[0, f, sel]) < 1e-10


def test_t1279_mixed_vs_fp64_grid_step():
    """T1279 on 3840x1920, K=512: 3xTF32 Legendre + FP32 FFTs (with binary64 and with
    float-float solves) vs all-FP64, same poles, one state."""
    import torch
    from paper_1812_03431_gb300 import rexi
    S = torch.from_numpy(inputs.random_spectral(N, 1, 1004)).cuda()
    out = {}
    for prec, arith in (("fp64", "fp64"), ("mixed", "fp64"), ("mixed", "fp32x2")):
        plan = rexi.Plan(N, NLAT, NLON, M=M, tau=TAU, precision=prec, solve_arith=arith)
        x = plan.synthesize(S) if prec == "fp64" else x
        out[prec, arith] = plan.step(x).cpu().numpy()
        plan.check_device()
        plan.close()
        torch.cuda.empty_cache()
    err = rel(out["mixed", "fp64"], out["fp64", "fp64"])
    err2 = rel(out["mixed", "fp32x2"], out["fp64", "fp64"])
    d = rel(out["mixed", "fp32x2"], out["mixed", "fp64"])
    print("T1279 vs FP64, relative L2: mixed %.3e, mixed with float-float solves %.3e (%.1e from binary64 solves)"
          % (err, err2, d))
    assert err < 1e-5 and err2 < 1e-5 and d < 1e-10
