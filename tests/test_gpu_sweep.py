"""Seeded sweep over plan configurations (truncation, grid, poles, batch, layout, precision,
solver, f-sphere, solve arithmetic) against the oracle, to catch indexing slips that fixed
cases miss."""
import numpy as np
import pytest

from oracle import phi_solver
from oracle import rexi_coeffs as rc
from oracle import step as ostep
from oracle.swe import Consts
from paper_1812_03431_gb300 import inputs

pytestmark = pytest.mark.gpu
C = Consts()


def smooth(n):
    for q in (2, 3, 5):
        while n % q == 0:
            n //= q
    return n == 1


def configs(count=48, seed=4242):
    rng = np.random.default_rng(seed)
    rng_arith = np.random.default_rng(seed + 1)  # a separate stream: the other draws stay as they were
    out = []
    while len(out) < count:
        N = int(rng.integers(1, 48))
        nlat = int(rng.integers(N + 1, 2 * N + 8))
        nlat += nlat % 2
        nlon = int(rng.integers(2 * N + 2, 4 * N + 16))
        nlon += nlon % 2
        while not smooth(nlon):
            nlon += 2
        M = int(rng.choice([2, 4, 8, 16, 32, 64]))
        B = int(rng.integers(1, 21))
        layout = str(rng.choice(["grid", "spectral"]))
        precision = str(rng.choice(["fp64", "mixed"])) if layout == "grid" else "fp64"
        kind = str(rng.choice(["delta", "delta", "phi", "fsphere"]))
        tau = float(rng.choice([600.0, 1800.0, 3600.0, 7200.0]))
        arith = str(rng_arith.choice(["fp64", "fp32x2"]))
        if kind == "fsphere":
            arith = "fp64"  # float-float solves serve the banded solvers on the rotating sphere
        out.append((N, nlat, nlon, M, B, layout, precision, kind, tau, arith))
    return out


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("cfg", configs(), ids=lambda c: "N%d_%dx%d_M%d_B%d_%s_%s_%s_%s" % (
    c[0], c[2], c[1], c[3], c[4], c[5], c[6], c[7], c[9]))
def test_sweep(cfg):
    import torch
    from paper_1812_03431_gb300 import rexi
    N, nlat, nlon, M, B, layout, precision, kind, tau, arith = cfg
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = inputs.random_spectral(N, B, 900 + N + B)
    plan = rexi.Plan(N, nlat, nlon, tau=tau, max_batch=B, layout=layout, precision=precision, alpha=al, beta=be,
                     solver="phi" if kind == "phi" else "delta", fsphere=kind == "fsphere", solve_arith=arith)

    def spectral_ref(X):
        if kind == "phi":
            return phi_solver.rexi_step_phi(X, N, N + 4 + N % 2, al, be, tau, C, recover="spectral")
        return ostep.rexi_step_spectral(X, N, al, be, tau, C, fsphere=kind == "fsphere")

    if layout == "spectral":
        got = plan.step(torch.from_numpy(S).cuda()).cpu().numpy()
        ref = spectral_ref(S)
        axis = -2
    else:
        gs = ostep.GridStep(N, nlat, nlon, al, be, tau, C)
        x = gs.synthesise(S)
        got = plan.step(torch.from_numpy(x).cuda()).cpu().numpy()
        ref = gs.synthesise(spectral_ref(gs.analyse(x)))
        axis = -3
    plan.check_device()
    plan.close()
    tol = 1e-5 if precision == "mixed" else 1e-10
    err = max(relerr(np.take(got, f, axis=axis), np.take(ref, f, axis=axis)) for f in range(3))
    assert err < tol, err
