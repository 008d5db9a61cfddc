"""Device-side error reporting (rexi_check_device) without a device fault.

The tensor-core kernels wait on mbarriers with an iteration limit; a wait that runs
out sets a bit in the plan's device error word, skips its outputs and returns.  Making
a kernel actually wait out that limit would mean stalling a GPU on purpose, so the
reporting path is tested from the host instead: rexi_inject_device_error sets the bit
as the kernel would, and rexi_check_device must report it once and clear it.  The
device-side expiry itself is not exercised on a GPU."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture()
def plan():
    from paper_1812_03431_gb300 import rexi
    p = rexi.Plan(15, 16, 32, M=8, precision="mixed")
    yield p
    p.close()


def test_expired_wait_is_reported_once(plan):
    import torch
    from paper_1812_03431_gb300 import rexi
    x = torch.zeros((1, 3, 16, 32), dtype=torch.float64, device="cuda")
    plan.step(x)
    plan.check_device()  # a clean step reports nothing
    plan.inject_device_error(1)
    with pytest.raises(rexi.RexiError) as ei:
        plan.check_device()
    assert ei.value.status == rexi.REXI_ETIMEOUT
    assert "bounded device-side wait" in str(ei.value)
    plan.check_device()  # the bit was cleared by the report


def test_range_error_is_reported(plan):
    from paper_1812_03431_gb300 import rexi
    plan.inject_device_error(2)
    with pytest.raises(rexi.RexiError) as ei:
        plan.check_device()
    assert ei.value.status == rexi.REXI_ERANGE
    plan.check_device()


def test_both_bits_report_the_timeout_first(plan):
    from paper_1812_03431_gb300 import rexi
    plan.inject_device_error(3)
    with pytest.raises(rexi.RexiError) as ei:
        plan.check_device()
    assert ei.value.status == rexi.REXI_ETIMEOUT
    plan.check_device()  # one check clears the whole word


def test_injection_rejects_unknown_bits(plan):
    from paper_1812_03431_gb300 import rexi
    for bits in (0, 4, -1):
        with pytest.raises(rexi.RexiError) as ei:
            plan.inject_device_error(bits)
        assert ei.value.status == rexi.REXI_EINVAL
