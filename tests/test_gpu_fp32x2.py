"""Float-float solves (solve_arith="fp32x2") through the C-ABI vs the CPU oracle.

The banded solves and the beta-weighted pole sum run on the FP32 pipes with pairs of
binary32 numbers (48-bit significands, unit roundoff u ~ 2^-48 = 3.6e-15, against
2^-53 = 1.1e-16 for binary64).  The pole sum barely cancels (sum |beta_k x_k| is
about four times |sum beta_k x_k| for the poles of Sec. 4.1), and each row of a sweep
takes a few dozen operations, so the step's relative error stays near 1e-13: the
tests hold it to the FP64 form's bound, relative L2 <= 1e-10 per field, and the
mixed form (3xTF32 transforms) to its 1e-5.
"""
import ctypes

import numpy as np
import pytest

from oracle import rexi_coeffs as rc
from oracle import step as ostep
from oracle.swe import Consts
from paper_1812_03431_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-10
C = Consts()


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


@pytest.fixture(scope="module")
def rexi():
    from paper_1812_03431_gb300 import rexi as r
    r.load()
    return r


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def fieldwise(got, ref, axis_f=-2):
    return max(relerr(np.take(got, f, axis=axis_f), np.take(ref, f, axis=axis_f)) for f in range(3))


@pytest.mark.parametrize("N,M,B,tau", [(1, 2, 1, 600.0), (2, 4, 1, 600.0), (15, 16, 3, 3600.0), (31, 32, 5, 7200.0),
                                       (63, 128, 1, 3600.0), (63, 64, 17, 1800.0), (23, 16, 33, 900.0)])
def test_spectral_step_matches_oracle(torch, rexi, N, M, B, tau):
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = inputs.random_spectral(N, B, 100 + N)
    plan = rexi.Plan(N, 2 * N + 2, 4 * N + 4, tau=tau, max_batch=B, layout="spectral", alpha=al, beta=be,
                     solve_arith="fp32x2")
    got = plan.step(torch.from_numpy(S).cuda()).cpu().numpy()
    plan.close()
    ref = ostep.rexi_step_spectral(S, N, al, be, tau, C)
    err = fieldwise(got, ref)
    print("fp32x2 spectral N=%d M=%d B=%d: rel L2 %.2e" % (N, M, B, err))
    assert err < TOL
    assert np.all(got[:, 1:, 0] == 0)
    assert np.all(got[:, :, : N + 1].imag == 0)


@pytest.mark.parametrize("N,nlat,nlon,M,B", [(1, 2, 4, 2, 1), (31, 48, 96, 32, 2), (42, 64, 160, 48, 1),
                                             (20, 30, 90, 16, 18)])
def test_grid_step_matches_oracle(torch, rexi, N, nlat, nlon, M, B):
    tau = 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    gs = ostep.GridStep(N, nlat, nlon, al, be, tau, C)
    x = gs.synthesise(inputs.random_spectral(N, B, 7 + N)) + 0.01 * inputs.random_grid(B, nlat, nlon, 3)
    plan = rexi.Plan(N, nlat, nlon, tau=tau, max_batch=B, alpha=al, beta=be, solve_arith="fp32x2")
    got = plan.step(torch.from_numpy(x).cuda()).cpu().numpy()
    plan.close()
    assert fieldwise(got, gs(x), axis_f=-3) < TOL


def test_mixed_form_matches_oracle_and_fp64_solves(torch, rexi):
    """3xTF32 transforms with float-float solves: within the mixed form's 1e-5 of the
    oracle, and within 1e-11 of the same transforms with binary64 solves (the solve
    arithmetic adds nothing visible to the transforms' error)."""
    N, nlat, nlon, M, B, tau = 63, 96, 192, 128, 3, 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    gs = ostep.GridStep(N, nlat, nlon, al, be, tau, C)
    x = gs.synthesise(inputs.random_spectral(N, B, 63))
    xd = torch.from_numpy(x).cuda()
    outs = {}
    for arith in ("fp64", "fp32x2"):
        plan = rexi.Plan(N, nlat, nlon, tau=tau, max_batch=B, alpha=al, beta=be, precision="mixed",
                         solve_arith=arith)
        outs[arith] = plan.step(xd).cpu().numpy()
        plan.close()
    assert fieldwise(outs["fp32x2"], gs(x), axis_f=-3) < 1e-5
    d = fieldwise(outs["fp32x2"], outs["fp64"], axis_f=-3)
    print("mixed form, fp32x2 vs fp64 solves: rel L2 %.2e" % d)
    assert d < 1e-11


def test_spectral_adjoint_matches_oracle(torch, rexi):
    N, M, B, tau = 31, 32, 3, 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = inputs.random_spectral(N, B, 31)
    plan = rexi.Plan(N, 64, 128, tau=tau, max_batch=B, layout="spectral", alpha=al, beta=be, solve_arith="fp32x2")
    got = plan.step_adjoint(torch.from_numpy(S).cuda()).cpu().numpy()
    plan.close()
    assert fieldwise(got, ostep.rexi_step_spectral(S, N, al, be, tau, C, adjoint=True)) < TOL


def test_grid_adjoint_matches_oracle(torch, rexi):
    N, nlat, nlon, M, B, tau = 31, 48, 96, 32, 2, 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    gs = ostep.GridStep(N, nlat, nlon, al, be, tau, C)
    y = inputs.random_grid(B, nlat, nlon, 8)
    plan = rexi.Plan(N, nlat, nlon, tau=tau, max_batch=B, alpha=al, beta=be, solve_arith="fp32x2")
    got = plan.step_adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    plan.close()
    assert fieldwise(got, gs.adjoint(y), axis_f=-3) < TOL


@pytest.mark.parametrize("k", [0, 40, 86])
def test_single_pole_solve(torch, rexi, k):
    N, M, tau = 24, 32, 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = inputs.random_spectral(N, 2, 9)
    plan = rexi.Plan(N, 50, 100, tau=tau, max_batch=2, layout="spectral", alpha=al, beta=be, solve_arith="fp32x2")
    got = plan.solve_pole(k, torch.from_numpy(S).cuda()).cpu().numpy()
    plan.close()
    ref = ostep.rexi_step_spectral(S, N, al[k:k + 1], np.ones(1, complex), tau, C, real_m0=False)
    assert fieldwise(got, ref) < TOL


@pytest.mark.parametrize("N,M,B,slots,shape", [(63, 64, 4, 0, 0), (63, 64, 4, 8, 1), (31, 64, 1, 128, 0),
                                               (31, 64, 1, 151, 1)])
def test_layouts_deterministic_and_match_oracle(torch, rexi, N, M, B, slots, shape):
    """Every pole-slot layout, including the warp-per-output reduction (slots >= 128 with
    few outputs): bit-reproducible run to run, and within the bound of the oracle."""
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = inputs.random_spectral(N, B, 41)
    Sd = torch.from_numpy(S).cuda()
    plan = rexi.Plan(N, 2 * N + 2, 4 * N + 4, tau=3600.0, max_batch=B, layout="spectral", alpha=al, beta=be,
                     solve_arith="fp32x2")
    if slots:
        plan.set_pole_slots(B, slots, shape)
    a = plan.step(Sd).cpu().numpy()
    np.testing.assert_array_equal(a, plan.step(Sd).cpu().numpy())
    plan.close()
    assert fieldwise(a, ostep.rexi_step_spectral(S, N, al, be, 3600.0, C)) < TOL


def test_integrate_equals_repeated_steps(torch, rexi):
    N, M, B = 31, 32, 2
    plan = rexi.Plan(N, 48, 96, M=M, tau=3600.0, max_batch=B, layout="spectral", solve_arith="fp32x2")
    x = torch.from_numpy(inputs.random_spectral(N, B, 12)).cuda()
    y = x
    for _ in range(5):
        y = plan.step(y)
    z = plan.integrate(x, 5)
    np.testing.assert_array_equal(z.cpu().numpy(), y.cpu().numpy())
    plan.close()


def test_static_step_matches_rexi_step(torch, rexi):
    lib = rexi.load()
    N, M, B = 63, 64, 3
    plan = rexi.Plan(N, 96, 192, M=M, tau=3600.0, max_batch=B, layout="spectral", solve_arith="fp32x2")
    x = torch.from_numpy(inputs.random_spectral(N, B, 77)).cuda()
    ref = plan.step(x).cpu().numpy()
    out = torch.full_like(x, float("nan"))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.rexi_step_static(plan._h, x.data_ptr(), out.data_ptr(), B, stream) == rexi.REXI_OK
    assert fieldwise(out.cpu().numpy(), ref) < 1e-13
    plan.close()


@pytest.mark.parametrize("B", [1, 3, 9, 16])
def test_interleaved_plan_with_smaller_batches(torch, rexi, B):
    """A plan for 16 states keeps its factors interleaved (a warp's lanes share poles); calls
    with fewer states put different poles in a warp's lanes and stay within the bound."""
    N, M = 31, 32
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = inputs.random_spectral(N, B, 60 + B)
    plan = rexi.Plan(N, 64, 128, tau=3600.0, max_batch=16, layout="spectral", alpha=al, beta=be,
                     solve_arith="fp32x2")
    got = plan.step(torch.from_numpy(S).cuda()).cpu().numpy()
    plan.close()
    assert fieldwise(got, ostep.rexi_step_spectral(S, N, al, be, 3600.0, C)) < TOL


def test_ragged_fp32x2_matches_per_plan_steps(torch, rexi):
    # max_batch 2 (pole-fastest factors) and 8 (interleaved factors) in one launch
    plans = [rexi.Plan(N, 2 * N + 2, 4 * N + 4, M=M, tau=1200.0, max_batch=mb, layout="spectral",
                       solve_arith="fp32x2") for N, M, mb in ((31, 32, 2), (63, 64, 8))]
    state_plan = [0, 1, 1, 0]
    states = [torch.from_numpy(inputs.random_spectral(31 if p == 0 else 63, 1, 500 + s)[0]).cuda()
              for s, p in enumerate(state_plan)]
    outs = [torch.empty_like(x) for x in states]
    rg = rexi.Ragged(plans, 4)
    rg.step(states, outs, state_plan)
    torch.cuda.synchronize()
    for p, plan in enumerate(plans):
        idx = [s for s in range(4) if state_plan[s] == p]
        Y = plan.step(torch.stack([states[s] for s in idx])).cpu().numpy()
        for r, s in enumerate(idx):
            assert relerr(outs[s].cpu().numpy(), Y[r]) < 1e-13
    for s_, p, N in ((0, 0, 31), (1, 1, 63)):  # one state of each layout against the oracle
        al, be = plans[p].coefficients()
        ref = ostep.rexi_step_spectral(states[s_].cpu().numpy()[None], N, al, be, 1200.0, C)
        assert fieldwise(outs[s_].cpu().numpy()[None], ref) < TOL
    other = rexi.Plan(31, 64, 128, M=32, tau=1200.0, max_batch=2, layout="spectral")
    with pytest.raises(rexi.RexiError):
        rexi.Ragged([plans[0], other], 4)  # one solve arithmetic per ragged batch
    for p in plans + [other]:
        p.close()


def test_rejected_combinations(torch, rexi):
    with pytest.raises(rexi.RexiError):
        rexi.Plan(15, 16, 32, M=8, layout="spectral", fsphere=True, solve_arith="fp32x2")


def test_full_size_sampled_orders(torch, rexi):
    """T341, K=256 (P=535), tau=1200 s, batch 16, tuned layout (the bench's launch):
    sampled zonal orders against the oracle, and every coefficient against the binary64
    solves."""
    N, M, B, tau = 341, 256, 16, 1200.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = inputs.random_spectral(N, B, 1005)
    Sd = torch.from_numpy(S).cuda()
    outs = {}
    for arith in ("fp64", "fp32x2"):
        plan = rexi.Plan(N, 512, 1024, tau=tau, max_batch=B, layout="spectral", alpha=al, beta=be,
                         solve_arith=arith)
        plan.tune(B)
        outs[arith] = plan.step(Sd).cpu().numpy()
        plan.close()
    got = outs["fp32x2"]
    d = fieldwise(got, outs["fp64"])
    print("T341 B=16, fp32x2 vs fp64 solves: rel L2 %.2e" % d)
    assert d < TOL
    ms = [0, 1, 170, 340, 341]
    ref = ostep.rexi_step_spectral(S[:2], N, al, be, tau, C, ms=ms)
    from oracle.sphere import idx
    sel = np.concatenate([np.arange(idx(m, m, N), idx(m, N, N) + 1) for m in ms])
    assert fieldwise(got[:2][..., sel], ref[..., sel]) < TOL


@pytest.mark.parametrize("solver", ["delta", "phi"])
def test_range_errors_reported(torch, rexi, solver):
    """Float-float holds binary32's exponent range only.  A finite state value beyond it
    (here 1e39) is reported by rexi_check_device as REXI_ERANGE (once: the flag is
    cleared), and factors beyond it (a pole at 1e-45) fail plan creation with
    REXI_ERANGE; binary64 solves take both."""
    N, B = 15, 2
    S = inputs.random_spectral(N, B, 5)
    S_big = S.copy()
    S_big[1, 0, 3] = 1e39
    plan = rexi.Plan(N, 16, 32, M=8, max_batch=B, layout="spectral", solver=solver, solve_arith="fp32x2")
    plan.step(torch.from_numpy(S).cuda())
    plan.check_device()
    plan.step(torch.from_numpy(S_big).cuda())
    with pytest.raises(rexi.RexiError) as err:
        plan.check_device()
    assert err.value.status == rexi.REXI_ERANGE
    plan.check_device()  # reported once
    plan.close()
    p64 = rexi.Plan(N, 16, 32, M=8, max_batch=B, layout="spectral", solver=solver)
    y = p64.step(torch.from_numpy(S_big).cuda()).cpu().numpy()
    p64.check_device()
    assert np.all(np.isfinite(y))
    p64.close()
    al, be = np.array([1e-45 + 0j]), np.array([1.0 + 0j])
    with pytest.raises(rexi.RexiError) as err:
        rexi.Plan(N, 16, 32, layout="spectral", alpha=al, beta=be, solver=solver, solve_arith="fp32x2")
    assert err.value.status == rexi.REXI_ERANGE
    rexi.Plan(N, 16, 32, layout="spectral", alpha=al, beta=be, solver=solver).close()
