"""Pole sharding (Sec. 6.4: the REXI terms split evenly over ranks, then one reduction):
plans holding a contiguous share of the poles return partial steps whose sum is the full
step.  One GPU runs every share here; the multi-rank path (NCCL allreduce in bench.py)
adds nothing but the sum."""
import numpy as np
import pytest

from oracle import rexi_coeffs as rc
from paper_1812_03431_gb300 import inputs

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("layout,precision,world,tol,B", [("spectral", "fp64", 2, 1e-13, 3),
                                                          ("spectral", "fp64", 3, 1e-13, 3),
                                                          ("spectral", "fp64", 2, 1e-13, 1),  # fused solve
                                                          ("grid", "fp64", 2, 1e-12, 3), ("grid", "mixed", 4, 1e-5, 3)])
def test_shards_add_up_to_the_full_step(layout, precision, world, tol, B):
    import torch
    from paper_1812_03431_gb300 import rexi
    N, M, tau = 31, 32, 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    P = al.size
    kw = dict(tau=tau, max_batch=B, layout=layout, precision=precision, alpha=al, beta=be)
    full = rexi.Plan(N, 48, 96, **kw)
    S = torch.from_numpy(inputs.random_spectral(N, B, 41)).cuda()
    x = S if layout == "spectral" else full.synthesize(S)
    ref = full.step(x).cpu().numpy()
    total = np.zeros_like(ref)
    for r in range(world):
        b, e = rexi.pole_shard(P, r, world)
        plan = rexi.Plan(N, 48, 96, poles=(b, e), **kw)
        a2, b2 = plan.coefficients()
        np.testing.assert_array_equal(a2, al[b:e])  # the shard's own poles, in order
        np.testing.assert_array_equal(b2, be[b:e])
        total += plan.step(x).cpu().numpy()
        plan.close()
    full.close()
    assert relerr(total, ref) < tol


def test_shard_adjoint_adds_up():
    import torch
    from paper_1812_03431_gb300 import rexi
    N, M, B = 23, 16, 2
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    G = torch.from_numpy(inputs.random_spectral(N, B, 43)).cuda()
    kw = dict(tau=1800.0, max_batch=B, layout="spectral", alpha=al, beta=be)
    full = rexi.Plan(N, 48, 96, **kw)
    ref = full.step_adjoint(G).cpu().numpy()
    full.close()
    total = 0
    for r in range(2):
        plan = rexi.Plan(N, 48, 96, poles=rexi.pole_shard(al.size, r, 2), **kw)
        total = total + plan.step_adjoint(G).cpu().numpy()
        plan.close()
    assert relerr(total, ref) < 1e-13


def test_library_poles_shard_keeps_full_normalisation():
    # library-computed poles: each shard keeps its slice of the set renormalised over all poles
    import torch
    from paper_1812_03431_gb300 import rexi
    N, M = 15, 16
    full = rexi.Plan(N, 16, 32, M=M, layout="spectral")
    al, be = full.coefficients()
    S = torch.from_numpy(inputs.random_spectral(N, 1, 44)).cuda()
    ref = full.step(S).cpu().numpy()
    full.close()
    total = 0
    for r in range(2):
        b, e = rexi.pole_shard(al.size, r, 2)
        plan = rexi.Plan(N, 16, 32, M=M, layout="spectral", poles=(b, e))
        a2, b2 = plan.coefficients()
        np.testing.assert_array_equal(b2, be[b:e])
        total = total + plan.step(S).cpu().numpy()
        plan.close()
    assert relerr(total, ref) < 1e-13
    with pytest.raises(rexi.RexiError):
        rexi.Plan(N, 16, 32, M=M, layout="spectral", poles=(10, 10))
