"""The paper's geopotential-only solver (REXI_SOLVER_PHI, Sec. 4.3 and 5) on the GPU against
the oracle's restatement of it (oracle/phi_solver.py), with binary64 and with float-float
solves (the same bound of 1e-10 for both).

Two oracle recoveries of zeta and delta serve as references.  ``recover="physical"`` is
the paper's own: the velocities V = A^{-1} (V0 + tau grad Phi) pointwise on the latitudes,
then their curl and divergence projected back (Sec. 5).  ``recover="spectral"`` takes
zeta and delta from the Phi and zeta rows of the system in spectral space, as the GPU
does.  The two are different discretisations at the truncation edge, so the physical
recovery is compared where truncation does not act: without rotation over every degree,
and in the degrees of a band-limited state on the rotating sphere."""
import numpy as np
import pytest

from oracle import phi_solver
from oracle import rexi_coeffs as rc
from oracle import step as ostep
from oracle.sphere import idx
from oracle.swe import Consts
from paper_1812_03431_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-10
C = Consts()


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def fieldwise(got, ref, axis_f=-2):
    return max(relerr(np.take(got, f, axis=axis_f), np.take(ref, f, axis=axis_f)) for f in range(3))


@pytest.mark.parametrize("arith", ["fp64", "fp32x2"])
@pytest.mark.parametrize("N,M,B,tau", [(2, 4, 1, 600.0), (15, 16, 3, 3600.0), (21, 32, 2, 1200.0),
                                       (42, 64, 5, 7200.0)])
def test_phi_spectral_step_matches_oracle(N, M, B, tau, arith):
    import torch
    from paper_1812_03431_gb300 import rexi
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = inputs.random_spectral(N, B, 300 + N)
    nlon = next(n for n in range(2 * N + 2, 8 * N + 16, 2) if rexi._smooth(n))
    plan = rexi.Plan(N, 2 * N + 2, nlon, tau=tau, max_batch=B, layout="spectral", alpha=al, beta=be,
                     solver="phi", solve_arith=arith)
    got = plan.step(torch.from_numpy(S).cuda()).cpu().numpy()
    plan.close()
    nlat = N + 4 + (N % 2)
    ref = phi_solver.rexi_step_phi(S, N, nlat, al, be, tau, C, recover="spectral")
    assert fieldwise(got, ref) < TOL
    assert np.all(got[:, 1:, 0] == 0) and np.all(got[:, :, : N + 1].imag == 0)


@pytest.mark.parametrize("arith", ["fp64", "fp32x2"])
def test_phi_grid_step_matches_oracle(arith):
    import torch
    from paper_1812_03431_gb300 import rexi
    N, nlat, nlon, M, B, tau = 31, 48, 96, 32, 2, 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    gs = ostep.GridStep(N, nlat, nlon, al, be, tau, C)
    x = gs.synthesise(inputs.random_spectral(N, B, 17)) + 0.01 * inputs.random_grid(B, nlat, nlon, 18)
    plan = rexi.Plan(N, nlat, nlon, tau=tau, max_batch=B, alpha=al, beta=be, solver="phi", solve_arith=arith)
    got = plan.step(torch.from_numpy(x).cuda()).cpu().numpy()
    plan.close()
    ref = gs.synthesise(phi_solver.rexi_step_phi(gs.analyse(x), N, nlat, al, be, tau, C, recover="spectral"))
    assert fieldwise(got, ref, axis_f=-3) < TOL


def test_phi_grid_step_mixed_precision():
    # the Phi-only solve behind the mixed form's tcgen05 Legendre transforms
    import torch
    from paper_1812_03431_gb300 import rexi
    N, nlat, nlon, M, B, tau = 63, 96, 192, 64, 3, 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    gs = ostep.GridStep(N, nlat, nlon, al, be, tau, C)
    x = gs.synthesise(inputs.random_spectral(N, B, 19))
    plan = rexi.Plan(N, nlat, nlon, tau=tau, max_batch=B, alpha=al, beta=be, solver="phi", precision="mixed")
    got = plan.step(torch.from_numpy(x).cuda()).cpu().numpy()
    plan.check_device()
    plan.close()
    ref = gs.synthesise(phi_solver.rexi_step_phi(gs.analyse(x), N, nlat, al, be, tau, C, recover="spectral"))
    assert fieldwise(got, ref, axis_f=-3) < 1e-5


def test_phi_and_delta_solvers_agree_in_low_degrees():
    # a state band-limited to n <= 12 at T63: both discretisations have converged in the
    # low degrees, where they agree to rounding; at the truncation edge they do not
    import torch
    from paper_1812_03431_gb300 import rexi
    L, N, M, tau = 12, 63, 64, 3600.0
    S0 = inputs.random_spectral(L, 2, 31)
    S = np.zeros((2, 3, (N + 1) * (N + 2) // 2), complex)
    for m in range(L + 1):
        for n in range(m, L + 1):
            S[..., idx(m, n, N)] = S0[..., idx(m, n, L)]
    x = torch.from_numpy(S).cuda()
    out = {}
    for solver in ("delta", "phi"):
        plan = rexi.Plan(N, 96, 192, M=M, tau=tau, max_batch=2, layout="spectral", solver=solver)
        out[solver] = plan.step(x).cpu().numpy()
        plan.close()
    low = [idx(m, n, N) for m in range(L + 1) for n in range(m, L + 1)]
    assert fieldwise(out["phi"][..., low], out["delta"][..., low]) < 1e-12


def _band_limited(L, N, B, seed):
    S0 = inputs.random_spectral(L, B, seed)
    S = np.zeros((B, 3, (N + 1) * (N + 2) // 2), complex)
    for m in range(L + 1):
        for n in range(m, L + 1):
            S[..., idx(m, n, N)] = S0[..., idx(m, n, L)]
    return S


@pytest.mark.parametrize("arith", ["fp64", "fp32x2"])
def test_phi_matches_physical_recovery_without_rotation(arith):
    # Omega = 0: D = alpha^2 is a constant, multiplying through by it commutes with
    # truncation, and the paper's pointwise velocity recovery is exact in every degree
    import torch
    from paper_1812_03431_gb300 import rexi
    N, M, B, tau, nlat = 31, 32, 2, 3600.0, 48
    c0 = Consts(omega=0.0)
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = inputs.random_spectral(N, B, 311)
    plan = rexi.Plan(N, nlat, 96, tau=tau, max_batch=B, layout="spectral", alpha=al, beta=be, solver="phi",
                     omega=0.0, solve_arith=arith)
    got = plan.step(torch.from_numpy(S).cuda()).cpu().numpy()
    plan.close()
    ref = phi_solver.rexi_step_phi(S, N, nlat, al, be, tau, c0, recover="physical")
    assert fieldwise(got, ref) < TOL


@pytest.mark.parametrize("arith", ["fp64", "fp32x2"])
@pytest.mark.parametrize("L,N,nlat", [(10, 21, 30), (12, 63, 96)])
def test_phi_matches_physical_recovery_in_band_limited_degrees(L, N, nlat, arith):
    # rotating sphere: for a state band-limited to n <= L both discretisations have
    # converged in those degrees (the oracle pins them to 1e-13 of each other), so the
    # GPU's spectral recovery meets the paper's physical one there
    import torch
    from paper_1812_03431_gb300 import rexi
    M, B, tau = 16 if N < 40 else 64, 2, 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = _band_limited(L, N, B, 320 + N)
    plan = rexi.Plan(N, nlat, 2 * nlat, tau=tau, max_batch=B, layout="spectral", alpha=al, beta=be, solver="phi",
                     solve_arith=arith)
    got = plan.step(torch.from_numpy(S).cuda()).cpu().numpy()
    plan.close()
    ref = phi_solver.rexi_step_phi(S, N, nlat, al, be, tau, C, recover="physical")
    low = [idx(m, n, N) for m in range(L + 1) for n in range(m, L + 1)]
    assert fieldwise(got[..., low], ref[..., low]) < TOL


@pytest.mark.parametrize("arith", ["fp64", "fp32x2"])
def test_phi_sampled_orders_t170(arith):
    import torch
    from paper_1812_03431_gb300 import rexi
    N, M, B, tau = 170, 256, 4, 1200.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = inputs.random_spectral(N, B, 1004)
    plan = rexi.Plan(N, 256, 512, tau=tau, max_batch=B, layout="spectral", alpha=al, beta=be, solver="phi",
                     solve_arith=arith)
    plan.tune(B)
    got = plan.step(torch.from_numpy(S).cuda()).cpu().numpy()
    plan.close()
    ms = [0, 85, 170]
    ref = phi_solver.rexi_step_phi(S[:1], N, 176, al, be, tau, C, ms=ms, recover="spectral")
    sel = np.concatenate([np.arange(idx(m, m, N), idx(m, N, N) + 1) for m in ms])
    assert fieldwise(got[:1][..., sel], ref[..., sel]) < TOL


def test_phi_unsupported_calls():
    import torch
    from paper_1812_03431_gb300 import rexi
    plan = rexi.Plan(15, 16, 32, M=8, max_batch=2, layout="spectral", solver="phi")
    S = torch.zeros((2, 3, plan.nspec), dtype=torch.complex128, device="cuda")
    for call in (lambda: plan.step_adjoint(S), lambda: plan.step_static(S), lambda: plan.solve_pole(0, S),
                 lambda: rexi.Ragged([plan], 2)):
        with pytest.raises(rexi.RexiError):
            call()
    plan.close()
    with pytest.raises(rexi.RexiError):
        rexi.Plan(15, 16, 32, M=8, layout="spectral", solver="phi", fsphere=True)


# Float-float carries a unit roundoff 32 times binary64's (2^-48 against 2^-53).  At this
# step the multiplied-through Phi system is badly conditioned (its coefficients span
# alpha^5 ~ 4e14 down to tau^4 F^4 alpha), so rounding is amplified: measured, binary64
# lands at 3.7e-13 and float-float at 1.6e-10.  Float-float is held to the binary64 bound
# scaled by the roundoff ratio, 1e-10 x 32, rounded down to 1e-9.
LONG_TOL = {"fp64": TOL, "fp32x2": 1e-9}


@pytest.mark.parametrize("arith", ["fp64", "fp32x2"])
def test_phi_long_step_matches_oracle(arith):
    """A 1.5-day step at T128 (tau omega up to ~820, the Gaussian-bump setting) with a
    spread of the M = 4116 poles, from the smallest |alpha| to the largest: the
    pentadiagonal LU without pivoting against the oracle's pivoted dense solves."""
    import torch
    from paper_1812_03431_gb300 import rexi
    N, tau = 128, 129600.0
    al, be, _ = rc.rexi_coefficients(4116, 0.2)
    pick = np.unique(np.concatenate([np.arange(0, al.size, 400), np.argsort(np.abs(al))[:8]]))
    al, be = al[pick], be[pick]
    S = inputs.random_spectral(N, 2, 77)
    plan = rexi.Plan(N, 192, 384, tau=tau, max_batch=2, layout="spectral", alpha=al, beta=be, solver="phi",
                     solve_arith=arith)
    got = plan.step(torch.from_numpy(S).cuda()).cpu().numpy()
    plan.close()
    ms = [0, 1, 64, 127, 128]
    ref = phi_solver.rexi_step_phi(S, N, 134, al, be, tau, C, ms=ms, recover="spectral")
    sel = np.concatenate([np.arange(idx(m, m, N), idx(m, N, N) + 1) for m in ms])
    err = fieldwise(got[..., sel], ref[..., sel])
    print("Phi-only solver, 1.5-day step, %s solves: rel L2 %.2e" % (arith, err))
    assert err < LONG_TOL[arith]
