"""Pins for oracle.rexi_coeffs (paper Sec. 4.1, Sec. 6.1)."""
import numpy as np
import pytest

from oracle import rexi_coeffs as rc


def test_gaussian_fit_near_double_precision(golden):
    # Sec. 4.1: K = 11 rational terms keep the error close to double precision.
    assert rc.K_GAUSS == int(golden["gauss_terms_K"])
    mu, a, err = rc.gaussian_fit()
    assert mu < 0  # all poles i y = -(mu + i l) on one side of the real axis
    y = np.linspace(-200.0, 200.0, 80001) + 0.00123  # not the fit samples
    e = np.abs(rc.gaussian_rational(y, mu, a).real - rc.psi(y)).max()
    assert e < 1e-12 and err < 1e-12
    np.testing.assert_allclose(a[::-1], np.conj(a), rtol=0, atol=1e-15 * np.abs(a).max())


@pytest.mark.parametrize("M,h", [(16, 0.2), (128, 0.2), (256, 0.2), (128, 0.15)])
def test_real_part_is_cosine(M, h):
    al, be, eps = rc.rexi_coefficients(M, h, normalize=False)
    assert al.size == 2 * (M + rc.K_GAUSS) + 1
    x = np.linspace(-h * (M - 10), h * (M - 10), 20001)
    f = rc.response(al, be, x)
    assert np.abs(f.real - np.cos(x)).max() < 1e-10


@pytest.mark.parametrize("M,h", [(128, 0.2), (256, 0.2), (512, 0.15)])
def test_imag_part_within_truncation_bound(M, h):
    al, be, _ = rc.rexi_coefficients(M, h, normalize=False)
    x = np.linspace(-h * M / 2, h * M / 2, 4001)
    f = rc.response(al, be, x)
    err = np.abs(f.imag - np.sin(x))
    assert np.all(err <= rc.imag_tail_bound(x, M, h) + 1e-10)
    # and the bound is not vacuous: the error is really of that size away from 0
    assert err.max() > 0.05 * rc.imag_tail_bound(x, M, h).max()


def test_x0_residual_has_printed_order(golden):
    # Sec. 6.1 prints eps = 1 - sum beta/alpha = -1.559352647e-11 at M = 128 (Haut's table,
    # h = 0.15).  The refitted table pins the order of magnitude only.
    printed = golden["eps_x0_M128"]
    _, _, eps = rc.rexi_coefficients(128, golden["h_paper"], normalize=False)
    assert abs(eps.imag) < 1e-15
    assert 1e-3 * abs(printed) < abs(eps.real) < 10 * abs(printed)
    # the other merges of the real and imaginary sets are far off at x = 0, which is what
    # selects beta = beta^Re as the reading of "merged"
    al, bre, bim = rc.rexi_parts(128, golden["h_paper"])
    for beta in (0.5 * (bre + 1j * bim), bre + 1j * bim):
        assert abs(1 - np.sum(beta / al)) > 1e-4


def test_normalisation_exact_at_zero():
    al, be, eps = rc.rexi_coefficients(256, 0.2, normalize=True)
    assert abs(1 - np.sum(be / al)) < 1e-15
    al2, be2, _ = rc.rexi_coefficients(256, 0.2, normalize=False)
    np.testing.assert_allclose(be, be2 / (1 - eps), rtol=1e-15)


def test_conjugate_symmetric_poles():
    al, be, _ = rc.rexi_coefficients(128, 0.2)
    np.testing.assert_array_equal(al[::-1], np.conj(al))
    np.testing.assert_allclose(be[::-1], np.conj(be), rtol=0, atol=1e-15 * np.abs(be).max())
    assert np.all(al.real < 0)


def test_printed_drift_estimate(golden):
    # Sec. 6.1: with the printed x = 0 residual the stationary modes drift by
    # (1 - eps)^N - 1; the number of steps to a drift of 1e-6 is "about 60000"
    eps = golden["eps_x0_M128"]
    n = np.log(1.0 + 1e-6) / abs(np.log(1.0 - eps))
    assert abs(n - golden["drift_steps_to_1e-6"]) < 0.1 * golden["drift_steps_to_1e-6"]
    assert abs(((1.0 - eps) ** n - 1.0) - 1e-6) < 1e-12
