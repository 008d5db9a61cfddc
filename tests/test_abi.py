"""The C-ABI library builds, loads and exports every symbol include/*.h declares (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT


def header_functions():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rexi_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1812_03431_gb300 import build, rexi
    if not os.path.exists(rexi.LIB_PATH):
        build.build()
    return rexi.load()


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_1812_03431_gb300 import rexi
    assert sorted(rexi.SIGNATURES) == header_functions()


def test_params_default(lib):
    from paper_1812_03431_gb300 import rexi
    p = rexi.rexi_params_default()
    assert (p.ntrunc, p.nlat, p.nlon, p.M, p.max_batch) == (63, 96, 192, 128, 1)
    assert p.radius == 6.37122e6 and p.omega == 7.292e-5 and p.gravity == 9.80616 and p.mean_depth == 1e4
    assert p.h == 0.2 and p.normalize == 1 and p.precision == rexi.REXI_FP64


def test_invalid_plan_rejected_before_any_cuda_call(lib):
    from paper_1812_03431_gb300 import rexi
    p = rexi.rexi_params_default()
    p.nlon = 7 * 32  # not a 2-3-5 product
    h = ctypes.c_void_p()
    st = lib.rexi_plan_create(ctypes.byref(p), ctypes.byref(h))
    assert st == rexi.REXI_EINVAL and not h.value
    assert b"nlon" in lib.rexi_last_error()
    p = rexi.rexi_params_default()
    p.nlat = 95
    assert lib.rexi_plan_create(ctypes.byref(p), ctypes.byref(h)) == rexi.REXI_EINVAL
    p = rexi.rexi_params_default()
    p.max_batch = 0
    assert lib.rexi_plan_create(ctypes.byref(p), ctypes.byref(h)) == rexi.REXI_EINVAL
    assert lib.rexi_plan_create(None, ctypes.byref(h)) == rexi.REXI_EINVAL
    lib.rexi_destroy(None)  # NULL-safe


@pytest.mark.parametrize("M,h", [(16, 0.2), (128, 0.2), (256, 0.2)])
def test_library_poles_match_oracle_response(lib, M, h):
    # two independent refits of the Gaussian approximation: same pole indexing and count,
    # responses equal to the fit level, real part equal to cos(x) (Sec. 4.1)
    from oracle import rexi_coeffs as rc
    from paper_1812_03431_gb300 import rexi
    al, be, eps = rexi.rexi_coefficients(M, h, normalize=False)
    al2, be2, eps2 = rc.rexi_coefficients(M, h, normalize=False)
    assert al.shape == al2.shape == (2 * (M + 11) + 1,)
    np.testing.assert_array_equal(al.imag, al2.imag)  # i h n, n ascending
    x = np.linspace(-h * (M - 10), h * (M - 10), 4001)
    f, f2 = rc.response(al, be, x), rc.response(al2, be2, x)
    assert np.abs(f - f2).max() < 1e-11
    assert np.abs(f.real - np.cos(x)).max() < 1e-10
    assert abs(eps) < 1e-10 and abs(eps - eps2.real) < 1e-11
    al3, be3, _ = rexi.rexi_coefficients(M, h, normalize=True)
    assert abs(1 - np.sum(be3 / al3)) < 1e-15


def test_coefficients_reject_bad_args(lib):
    from paper_1812_03431_gb300 import rexi
    with pytest.raises(rexi.RexiError):
        rexi.rexi_coefficients(0, 0.2)


def test_params_struct_matches_library():
    import ctypes
    from paper_1812_03431_gb300 import rexi
    lib = rexi.load()
    assert lib.rexi_params_size() == ctypes.sizeof(rexi.rexi_params)
    p = rexi.rexi_params_default()
    # the fields appended last keep their defaults: rotating sphere, delta elimination
    assert (p.fsphere, p.solver, p.max_batch, p.M) == (0, 0, 1, 128)


def test_missing_library_fails_loudly(monkeypatch):
    # no CPU fallback: without the built library every entry point raises
    from paper_1812_03431_gb300 import rexi
    monkeypatch.setattr(rexi, "_lib", None)
    monkeypatch.setattr(rexi, "LIB_PATH", "/nonexistent/librexi.so")
    with pytest.raises(RuntimeError, match="librexi.so not found"):
        rexi.load()
    with pytest.raises(RuntimeError):
        rexi.Plan(15, 16, 32, M=4)
