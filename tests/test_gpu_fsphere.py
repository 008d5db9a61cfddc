"""f-sphere plans (constant f = 2 Omega, Sec. 4): the closed-form per-degree solve
path against the oracle's banded solves of the same operator."""
import numpy as np
import pytest

from oracle import rexi_coeffs as rc
from oracle import step as ostep
from oracle.swe import Consts
from paper_1812_03431_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-10
C = Consts()


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def fieldwise(got, ref, axis_f=-2):
    return max(relerr(np.take(got, f, axis=axis_f), np.take(ref, f, axis=axis_f)) for f in range(3))


@pytest.mark.parametrize("N,M,B,tau", [(2, 4, 1, 600.0), (31, 32, 3, 3600.0), (63, 128, 5, 7200.0)])
def test_fsphere_spectral_step(N, M, B, tau):
    import torch
    from paper_1812_03431_gb300 import rexi
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = inputs.random_spectral(N, B, 200 + N)
    plan = rexi.Plan(N, 2 * N + 2, 4 * N + 4, tau=tau, max_batch=B, layout="spectral", alpha=al, beta=be,
                     fsphere=True)
    x = torch.from_numpy(S).cuda()
    got = plan.step(x).cpu().numpy()
    assert fieldwise(got, ostep.rexi_step_spectral(S, N, al, be, tau, C, fsphere=True)) < TOL
    assert np.all(got[:, 1:, 0] == 0) and np.all(got[:, :, : N + 1].imag == 0)
    # adjoint, one pole, the allocation-free entry point, the tuner
    adj = plan.step_adjoint(x).cpu().numpy()
    assert fieldwise(adj, ostep.rexi_step_spectral(S, N, al, be, tau, C, adjoint=True, fsphere=True)) < TOL
    k = len(al) // 3
    one = plan.solve_pole(k, x).cpu().numpy()
    ref1 = ostep.rexi_step_spectral(S, N, al[k:k + 1], np.ones(1, complex), tau, C, real_m0=False, fsphere=True)
    assert fieldwise(one, ref1) < TOL
    np.testing.assert_array_equal(plan.step_static(x).cpu().numpy(), got)
    assert plan.tune(B) == 0
    plan.close()


def test_fsphere_grid_step():
    import torch
    from paper_1812_03431_gb300 import rexi
    N, nlat, nlon, M, B, tau = 42, 64, 128, 48, 2, 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    gs = ostep.GridStep(N, nlat, nlon, al, be, tau, C, fsphere=True)
    x = gs.synthesise(inputs.random_spectral(N, B, 77)) + 0.01 * inputs.random_grid(B, nlat, nlon, 78)
    plan = rexi.Plan(N, nlat, nlon, tau=tau, max_batch=B, alpha=al, beta=be, fsphere=True)
    got = plan.step(torch.from_numpy(x).cuda()).cpu().numpy()
    assert fieldwise(got, gs(x), axis_f=-3) < TOL
    plan.close()


def test_ragged_rejects_fsphere_plan():
    from paper_1812_03431_gb300 import rexi
    plan = rexi.Plan(15, 16, 32, M=8, layout="spectral", fsphere=True)
    with pytest.raises(rexi.RexiError):
        rexi.Ragged([plan], 2)
    plan.close()
