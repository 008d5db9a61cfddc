"""rexi_step_static: the spectral step for callers that cannot allocate device memory
while they step.  Its per-call scratch lives in the library's fixed 64 MiB device
array; its result must equal rexi_step's on the same plan and input.

Collected last on purpose (file name), so that a run stopping at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL = 1e-10  # relative L2 per field, as in the other FP64 parity tests


def _call_static(lib, rexi, plan, x, out, torch):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.rexi_step_static(plan._h, x.data_ptr(), out.data_ptr(), x.shape[0], stream)


def test_static_step_matches_rexi_step_on_two_calls():
    import torch
    from paper_1812_03431_gb300 import inputs, rexi
    lib = rexi.load()
    N, M, B = 63, 64, 3
    plan = rexi.Plan(N, 96, 192, M=M, tau=3600.0, max_batch=B, layout="spectral")
    for call, seed in enumerate((77, 78)):  # two calls in a row, different inputs
        x = torch.from_numpy(inputs.random_spectral(N, B, seed)).cuda()
        ref = plan.step(x).cpu().numpy()
        out = torch.full_like(x, float("nan"))
        st = _call_static(lib, rexi, plan, x, out, torch)
        assert st == rexi.REXI_OK, (call, lib.rexi_last_error())
        got = out.cpu().numpy()
        for f in range(3):
            err = np.linalg.norm(got[:, f] - ref[:, f]) / np.linalg.norm(ref[:, f])
            assert err < TOL, (call, f, err)
    plan.close()


def test_static_step_rejects_sizes_above_its_limit():
    import torch
    from paper_1812_03431_gb300 import rexi
    lib = rexi.load()
    N, B = 255, 16
    plan = rexi.Plan(N, 256, 768, M=8, tau=600.0, max_batch=B, layout="spectral")
    x = torch.zeros((B, 3, plan.nspec), dtype=torch.complex128, device="cuda")
    out = torch.empty_like(x)
    assert _call_static(lib, rexi, plan, x, out, torch) == rexi.REXI_EINVAL
    assert b"64 MiB" in lib.rexi_last_error()
    plan.close()
