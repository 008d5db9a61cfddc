"""CUDA path (librexi through its C-ABI) vs the CPU oracle, element by element.

FP64 tolerance: relative L2 error <= 1e-10 per field (the stated bound for the
plain FP64 form; rounding differences come from the pole-sum order, the
delta-eliminated vs full banded solves and the FFT algorithm).
"""
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


def spectral_state(N, B, seed):
    S = inputs.random_spectral(N, B, seed)
    return S


@pytest.mark.parametrize("N,M,B,tau", [(1, 2, 1, 600.0), (2, 4, 1, 600.0), (15, 16, 3, 3600.0), (31, 32, 5, 7200.0),
                                       (63, 128, 1, 3600.0), (63, 64, 17, 1800.0), (23, 16, 33, 900.0)])
def test_spectral_step_matches_oracle(torch, rexi, N, M, B, tau):
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = spectral_state(N, B, 100 + N)
    plan = rexi.Plan(N, 2 * N + 2, 4 * N + 4, tau=tau, max_batch=B, layout="spectral", alpha=al, beta=be)
    got = plan.step(torch.from_numpy(S).cuda()).cpu().numpy()
    ref = ostep.rexi_step_spectral(S, N, al, be, tau, C)
    assert fieldwise(got, ref) < TOL
    # conventions: zeta_0^0 = delta_0^0 = 0, m = 0 coefficients real
    assert np.all(got[:, 1:, 0] == 0)
    assert np.all(got[:, :, : N + 1].imag == 0)
    # coefficient readback is bit-exact and in the given order
    a2, b2 = plan.coefficients()
    np.testing.assert_array_equal(a2, al)
    np.testing.assert_array_equal(b2, be)


def test_library_default_poles(torch, rexi):
    N, M = 31, 32
    plan = rexi.Plan(N, 48, 96, M=M, tau=3600.0, layout="spectral")
    al, be = plan.coefficients()
    al0, be0, _ = rexi.rexi_coefficients(M, 0.2)
    np.testing.assert_array_equal(al, al0)
    np.testing.assert_array_equal(be, be0)
    S = spectral_state(N, 1, 5)
    got = plan.step(torch.from_numpy(S).cuda()).cpu().numpy()
    assert fieldwise(got, ostep.rexi_step_spectral(S, N, al, be, 3600.0, C)) < TOL


@pytest.mark.parametrize("k", [0, 17, 40, 86])
def test_single_pole_solve(torch, rexi, k):
    N, M, tau = 24, 32, 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = spectral_state(N, 2, 9)
    plan = rexi.Plan(N, 50, 100, tau=tau, max_batch=2, layout="spectral", alpha=al, beta=be)
    got = plan.solve_pole(k, torch.from_numpy(S).cuda()).cpu().numpy()
    ref = ostep.rexi_step_spectral(S, N, al[k:k + 1], np.ones(1, complex), tau, C, real_m0=False)
    assert fieldwise(got, ref) < TOL


@pytest.mark.parametrize("N,nlat,nlon,M,B", [(1, 2, 4, 2, 1), (31, 48, 96, 32, 2), (63, 96, 192, 128, 3),
                                             (42, 64, 160, 48, 1), (20, 30, 90, 16, 18)])
def test_grid_step_matches_oracle(torch, rexi, N, nlat, nlon, M, B):
    tau = 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    gs = ostep.GridStep(N, nlat, nlon, al, be, tau, C)
    x = gs.synthesise(spectral_state(N, B, 7 + N)) + 0.01 * inputs.random_grid(B, nlat, nlon, 3)
    plan = rexi.Plan(N, nlat, nlon, tau=tau, max_batch=B, alpha=al, beta=be)
    got = plan.step(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = gs(x)
    assert fieldwise(got, ref, axis_f=-3) < TOL


def test_transforms_match_oracle(torch, rexi):
    N, nlat, nlon, B = 63, 96, 192, 2
    gs = ostep.GridStep(N, nlat, nlon, np.ones(1, complex), np.ones(1, complex), 1.0, C)
    plan = rexi.Plan(N, nlat, nlon, M=8, max_batch=B)
    S = spectral_state(N, B, 21)
    x = plan.synthesize(torch.from_numpy(S).cuda()).cpu().numpy()
    assert fieldwise(x, gs.synthesise(S), axis_f=-3) < TOL
    g = inputs.random_grid(B, nlat, nlon, 4)
    s2 = plan.analyze(torch.from_numpy(g).cuda()).cpu().numpy()
    ref = gs.analyse(g)
    for f in range(3):
        assert relerr(s2[:, f], ref[:, f]) < TOL


def test_spectral_adjoint_matches_oracle(torch, rexi):
    N, M, B, tau = 31, 32, 3, 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = spectral_state(N, B, 31)
    plan = rexi.Plan(N, 64, 128, tau=tau, max_batch=B, layout="spectral", alpha=al, beta=be)
    got = plan.step_adjoint(torch.from_numpy(S).cuda()).cpu().numpy()
    ref = ostep.rexi_step_spectral(S, N, al, be, tau, C, adjoint=True)
    assert fieldwise(got, ref) < TOL


def test_grid_adjoint_matches_oracle(torch, rexi):
    N, nlat, nlon, M, B, tau = 31, 48, 96, 32, 2, 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    gs = ostep.GridStep(N, nlat, nlon, al, be, tau, C)
    y = inputs.random_grid(B, nlat, nlon, 8)
    plan = rexi.Plan(N, nlat, nlon, tau=tau, max_batch=B, alpha=al, beta=be)
    got = plan.step_adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    ref = gs.adjoint(y)
    assert fieldwise(got, ref, axis_f=-3) < TOL


def test_deterministic_and_slot_invariant(torch, rexi):
    N, M, B = 63, 64, 4
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = torch.from_numpy(spectral_state(N, B, 41)).cuda()
    outs = []
    for slots in (0, 1, 8, 64):
        plan = rexi.Plan(N, 96, 192, tau=3600.0, max_batch=B, layout="spectral", alpha=al, beta=be,
                         pole_slots=slots)
        a = plan.step(S).cpu().numpy()
        b = plan.step(S).cpu().numpy()
        np.testing.assert_array_equal(a, b)  # bit-reproducible run to run
        outs.append(a)
        plan.close()
    for o in outs[1:]:
        assert fieldwise(o, outs[0]) < 1e-13


def test_geostrophic_balance_grid(torch, rexi):
    # the balanced zonal flow without noise: the normalised REXI step keeps it steady (Sec. 6.1)
    N, nlat, nlon = 63, 96, 192
    plan = rexi.Plan(N, nlat, nlon, M=128, tau=3600.0)
    from oracle.sphere import gauss_legendre
    mu, _ = gauss_legendre(nlat)
    x = inputs.balanced_grid(mu, nlon)[None]
    y = plan.step(torch.from_numpy(x).cuda()).cpu().numpy()
    assert relerr(y, x) < 1e-12


def test_invalid_calls(torch, rexi):
    plan = rexi.Plan(15, 16, 32, M=4, max_batch=2, layout="spectral")
    S = torch.zeros((3, 3, plan.nspec), dtype=torch.complex128, device="cuda")
    with pytest.raises(rexi.RexiError):
        plan.step(S)  # batch 3 > max_batch 2
    S = torch.zeros((2, 3, plan.nspec), dtype=torch.complex128, device="cuda")
    import ctypes
    st = rexi.load().rexi_step(plan._h, S.data_ptr(), S.data_ptr(), 2, None)
    assert st == rexi.REXI_EINVAL  # in == out
    with pytest.raises(rexi.RexiError):
        plan.solve_pole(plan.info()["P"], S)
    out = torch.empty_like(S)
    assert rexi.load().rexi_step(plan._h, S.data_ptr(), out.data_ptr(), 0, None) == rexi.REXI_EINVAL  # empty batch
    assert rexi.load().rexi_step(plan._h, S.data_ptr() + 8, out.data_ptr(), 1, None) == rexi.REXI_EINVAL  # misaligned


def test_full_size_sampled_orders(torch, rexi):
    """T341, K=256 (P=535), tau=1200 s, batch 16: the bench's launch, checked on sampled m."""
    N, M, B, tau = 341, 256, 16, 1200.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = spectral_state(N, B, 1005)
    plan = rexi.Plan(N, 512, 1024, tau=tau, max_batch=B, layout="spectral", alpha=al, beta=be)
    got = plan.step(torch.from_numpy(S).cuda()).cpu().numpy()
    ms = [0, 1, 170, 340, 341]
    ref = ostep.rexi_step_spectral(S, N, al, be, tau, C, ms=ms)  # every state of the batch
    from oracle.sphere import idx
    sel = np.concatenate([np.arange(idx(m, m, N), idx(m, N, N) + 1) for m in ms])
    for b in range(B):
        assert fieldwise(got[b:b + 1][..., sel], ref[b:b + 1][..., sel]) < TOL, b


@pytest.fixture(scope="module")
def full_size_case():
    """Inputs and the oracle's grid-layout step of state 0 at the bench's workload."""
    N, nlat, nlon, M, B, tau = 341, 512, 1024, 256, 16, 1200.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    gs = ostep.GridStep(N, nlat, nlon, al, be, tau, C)
    x0 = gs.synthesise(spectral_state(N, 1, 1005))
    x = np.concatenate([x0, inputs.random_grid(B - 1, nlat, nlon, 5)])
    return dict(N=N, nlat=nlat, nlon=nlon, B=B, tau=tau, al=al, be=be, x=x, ref=gs(x0))


@pytest.mark.parametrize("precision,arith,tol", [("fp64", "fp64", TOL), ("mixed", "fp64", 1e-5),
                                                ("mixed", "fp32x2", 1e-5)])
def test_full_size_grid_step_bench_launch(torch, rexi, full_size_case, precision, arith, tol):
    """The bench's launches: T341, 1024x512, K=256, tau=1200 s, batch 16, grid layout, in each
    of its forms (mixed transforms with binary64 solves is the chosen one; float-float
    solves the extension).  The oracle computes the whole grid-layout step for state 0."""
    c = full_size_case
    plan = rexi.Plan(c["N"], c["nlat"], c["nlon"], tau=c["tau"], max_batch=c["B"], alpha=c["al"], beta=c["be"],
                     precision=precision, solve_arith=arith)
    plan.tune(c["B"])  # the layout the bench times
    got = plan.step(torch.from_numpy(c["x"]).cuda()).cpu().numpy()
    plan.close()
    assert fieldwise(got[:1], c["ref"], axis_f=-3) < tol


@pytest.mark.parametrize("precision,tol", [("fp64", TOL), ("mixed", 1e-5)])
def test_full_size_every_state_of_the_bench_launch(torch, rexi, precision, tol):
    """All 16 states of the bench's launch (T341, 1024x512, K=256, tau=1200 s, tuned layout,
    seeded n^-3 spectra): the oracle analyses the GPU's grid output and, on sampled zonal
    orders, compares it with its own spectral step of every state (the oracle's banded
    solves take the 16 states as right-hand sides of one solve per pole and order)."""
    from oracle.sphere import idx
    N, nlat, nlon, M, B, tau = 341, 512, 1024, 256, 16, 1200.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = spectral_state(N, B, 1005)
    gs = ostep.GridStep(N, nlat, nlon, al, be, tau, C)
    x = gs.synthesise(S)
    plan = rexi.Plan(N, nlat, nlon, tau=tau, max_batch=B, alpha=al, beta=be, precision=precision)
    plan.tune(B)
    y = plan.step(torch.from_numpy(x).cuda()).cpu().numpy()
    plan.close()
    got = gs.analyse(y)  # exact for the band-limited result of a grid step
    ms = [0, 1, 2, 85, 170, 255, 340, 341]
    ref = ostep.rexi_step_spectral(S, N, al, be, tau, C, ms=ms)
    sel = np.concatenate([np.arange(idx(m, m, N), idx(m, N, N) + 1) for m in ms])
    if precision == "fp64":
        for b in range(B):
            assert fieldwise(got[b:b + 1][..., sel], ref[b:b + 1][..., sel]) < tol, b
    # in the norm the error is stated in (h' and the wind on the grid): the sampled orders
    # of the difference and of the reference, synthesised (vorticity and divergence
    # coefficients weigh small scales by n, so FP32 rounding of the winds shows more there)
    E = np.zeros_like(ref)
    R = np.zeros_like(ref)
    E[..., sel] = got[..., sel] - ref[..., sel]
    R[..., sel] = ref[..., sel]
    e, r = gs.synthesise(E), gs.synthesise(R)
    for b in range(B):
        eh = np.linalg.norm(e[b, 0]) / np.linalg.norm(r[b, 0])
        ew = np.linalg.norm(e[b, 1:]) / np.linalg.norm(r[b, 1:])
        assert eh < tol and ew < tol, (b, eh, ew)


def test_tune_cache_and_set_pole_slots(torch, rexi, tmp_path):
    N, M, B = 63, 64, 4
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = torch.from_numpy(spectral_state(N, B, 51)).cuda()
    cache = str(tmp_path / "tune.json")
    plan = rexi.Plan(N, 96, 192, tau=3600.0, max_batch=B, layout="spectral", alpha=al, beta=be)
    s1 = plan.tune(B, cache=cache)          # miss: tunes and records
    y1 = plan.step(S).cpu().numpy()
    plan.close()
    plan = rexi.Plan(N, 96, 192, tau=3600.0, max_batch=B, layout="spectral", alpha=al, beta=be)
    s2 = plan.tune(B, cache=cache)          # hit: same layout without timing
    y2 = plan.step(S).cpu().numpy()
    assert s2 == s1
    np.testing.assert_array_equal(y1, y2)   # same layout, same bits
    for slots, shape in ((3, 0), (16, 1), (1, 1), (0, 2)):  # any layout is valid; only the sum order changes
        assert plan.set_pole_slots(B, slots, shape) >= (1 if shape < 2 else 0)
        ya = plan.step(S).cpu().numpy()
        np.testing.assert_array_equal(ya, plan.step(S).cpu().numpy())
        assert fieldwise(ya, y1) < 1e-13
    plan.close()


@pytest.mark.parametrize("M,h", [(128, 0.2), (128, 0.15)])
def test_stationary_mode_drift_without_renormalisation(torch, rexi, M, h):
    """Sec. 6.1: the balanced zonal flow is a zero-frequency mode, on which one step
    multiplies by the REXI response at x = 0, 1 - eps.  Without the renormalisation of
    the beta, K steps change it by (1 - eps)^K - 1 (the paper's error-growth estimate);
    with it the state stays put to rounding."""
    N, K, tau = 63, 4000, 3600.0
    al, be, eps = rc.rexi_coefficients(M, h, normalize=False)
    U = inputs.balanced_zonal_flow(N)[None]
    x = torch.from_numpy(U).cuda()
    plan = rexi.Plan(N, 96, 192, tau=tau, layout="spectral", alpha=al, beta=be)
    y = plan.integrate(x, K).cpu().numpy()
    plan.close()
    growth = (1.0 - eps) ** K - 1.0
    assert abs(growth) > 1e-9  # far above the rounding of the steps
    sel = np.abs(U[0, 0]) > 1e-3 * np.abs(U[0, 0]).max()  # Phi coefficients of the flow
    ratio = (y[0, 0][sel] - U[0, 0][sel]) / U[0, 0][sel]
    np.testing.assert_allclose(ratio.real, growth.real, rtol=0.02)
    al2, be2, _ = rc.rexi_coefficients(M, h)
    plan = rexi.Plan(N, 96, 192, tau=tau, layout="spectral", alpha=al2, beta=be2)
    y2 = plan.integrate(x, K).cpu().numpy()
    plan.close()
    assert relerr(y2, U) < 1e-3 * abs(growth)


def test_integrate_equals_repeated_steps(torch, rexi):
    N, M, B, K = 31, 32, 3, 7
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = torch.from_numpy(spectral_state(N, B, 61)).cuda()
    plan = rexi.Plan(N, 48, 96, tau=3600.0, max_batch=B, layout="spectral", alpha=al, beta=be)
    y = S
    for _ in range(K):
        y = plan.step(y)
    np.testing.assert_array_equal(plan.integrate(S, K).cpu().numpy(), y.cpu().numpy())  # bit for bit
    plan.close()
    plan = rexi.Plan(N, 48, 96, tau=3600.0, max_batch=B, alpha=al, beta=be)  # grid layout
    x = plan.synthesize(S)
    y = x
    for _ in range(K):
        y = plan.step(y)
    got = plan.integrate(x, K).cpu().numpy()
    assert fieldwise(got, y.cpu().numpy(), axis_f=-3) < 1e-12  # only the skipped transforms' rounding
    plan.close()
