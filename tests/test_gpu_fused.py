"""The fused solve (the beta-weighted pole sum kept on chip, Sec. 5 / Algorithm 1) against the
oracle and against the pole-slot solve with its separate reduction, over every CTA shape
it takes: tiles of 1, 2, 4, 8 and 16 states (warps split over poles or states), CTAs of
eight, four and two warps, ragged
state tiles, pole counts below and above a warp's pole lanes, truncations up to the
largest whose running sums fit in shared memory."""
import numpy as np
import pytest

from oracle import rexi_coeffs as rc
from oracle import step as ostep
from oracle.swe import Consts
from paper_1812_03431_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-10
C = Consts()


def grid(N):
    from paper_1812_03431_gb300 import rexi
    return 2 * N + 2, next(n for n in range(2 * N + 2, 8 * N + 16, 2) if rexi._smooth(n))


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def fieldwise(got, ref):
    return max(relerr(got[:, f], ref[:, f]) for f in range(3))


@pytest.mark.parametrize("N,M,B,tau", [(7, 1, 1, 600.0), (15, 16, 1, 3600.0), (21, 8, 2, 1800.0),
                                       (23, 16, 3, 900.0), (31, 32, 4, 7200.0), (40, 16, 5, 3600.0),
                                       (33, 32, 9, 1200.0), (24, 16, 16, 2400.0), (19, 8, 17, 3600.0)])
def test_fused_step_matches_oracle_and_slot_solve(N, M, B, tau):
    import torch
    from paper_1812_03431_gb300 import rexi
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = inputs.random_spectral(N, B, 500 + N + B)
    x = torch.from_numpy(S).cuda()
    plan = rexi.Plan(N, *grid(N), tau=tau, max_batch=B, layout="spectral", alpha=al, beta=be)
    used = plan.set_pole_slots(B, 0, 2, groups=1)  # the default CTA tile, one CTA per tile
    tile = used % 256
    assert used // 256 == 1 and tile >= min(B, 32) and tile & (tile - 1) == 0
    fused = plan.step(x).cpu().numpy()
    np.testing.assert_array_equal(plan.step(x).cpu().numpy(), fused)  # bit-reproducible
    if B > 2:  # a smaller tile: more, shorter work items; the order of the pole sum changes
        # where the tile's poles are split over warp groups or a warp holds another number
        # of states (the last round of a pass splits its poles by the rows it lacks)
        assert plan.set_pole_slots(B, tile // 2, 2, groups=1) == tile // 2 + 256
        half = plan.step(x).cpu().numpy()
        np.testing.assert_array_equal(plan.step(x).cpu().numpy(), half)
        assert fieldwise(half, fused) < 1e-13
    # each tile's poles over several CTAs (the default count, then fixed ones, capped at
    # the passes); whichever CTA finishes last adds the groups in the same order
    for groups in (0, 2, 3):
        used = plan.set_pole_slots(B, tile, 2, groups=groups)
        assert used % 256 == tile and used // 256 >= 1 and (groups == 0 or used // 256 <= groups)
        split = plan.step(x).cpu().numpy()
        for _ in range(2):
            np.testing.assert_array_equal(plan.step(x).cpu().numpy(), split)
        assert fieldwise(split, fused) < 1e-13
    # the lean form (three or four CTAs of four warps per SM, prefetching into the caches)
    lt = plan.set_pole_slots(B, tile, 3, groups=1) % 256  # at most two states per warp: tiles of 8 or less
    assert 1 <= lt <= min(tile, 8)
    lean = plan.step(x).cpu().numpy()
    np.testing.assert_array_equal(plan.step(x).cpu().numpy(), lean)
    assert fieldwise(lean, fused) < 1e-13
    plan.set_pole_slots(B, lt, 3, groups=2)
    lean2 = plan.step(x).cpu().numpy()
    assert fieldwise(lean2, fused) < 1e-13
    # the lean form on CTAs of two warps (seven or eight per SM): a tile of two states or
    # fewer has no pole split over warps; larger tiles hold two states per warp
    for groups in (1, 3):
        lw = plan.set_pole_slots(B, tile, 4, groups=groups) % 256
        assert 1 <= lw <= min(tile, 4)
        two = plan.step(x).cpu().numpy()
        np.testing.assert_array_equal(plan.step(x).cpu().numpy(), two)
        assert fieldwise(two, fused) < 1e-13
    plan.set_pole_slots(B, 8, 0)  # the pole-slot solve and its reduction
    slot = plan.step(x).cpu().numpy()
    plan.close()
    ref = ostep.rexi_step_spectral(S, N, al, be, tau, C)
    assert fieldwise(fused, ref) < TOL
    assert fieldwise(fused, slot) < 1e-13  # the same sums in another order
    assert np.all(fused[:, 1:, 0] == 0) and np.all(fused[:, :, : N + 1].imag == 0)


@pytest.mark.parametrize("B", [1, 2])
def test_pole_groups_single_state_match_oracle(B):
    # Sec. 6.1's single state (T63, M = 128: 279 poles): every split of a tile's poles over
    # 1 ... 9 CTAs against the oracle; the default for one state splits them (128 systems
    # alone would leave most schedulers idle), and a split result is the same on every run
    import torch
    from paper_1812_03431_gb300 import rexi
    N, M, tau = 63, 128, 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = inputs.noisy_balanced(N, 1000) if B == 1 else inputs.random_spectral(N, B, 64)
    S = S.reshape(B, 3, -1)
    x = torch.from_numpy(S).cuda()
    plan = rexi.Plan(N, 96, 192, tau=tau, max_batch=B, layout="spectral", alpha=al, beta=be)
    ref = ostep.rexi_step_spectral(S, N, al, be, tau, C)
    ref_adj = ostep.rexi_step_spectral(S, N, al, be, tau, C, adjoint=True)
    default = plan.set_pole_slots(B, 0, 2) // 256
    if B == 1:
        assert default > 1
    seen = set()
    for groups in range(1, 10):
        ng = plan.set_pole_slots(B, 0, 2, groups=groups) // 256
        if ng in seen:
            continue
        seen.add(ng)
        got = plan.step(x).cpu().numpy()
        for _ in range(3):
            np.testing.assert_array_equal(plan.step(x).cpu().numpy(), got)
        assert fieldwise(got, ref) < TOL
        adj = plan.step_adjoint(x).cpu().numpy()
        assert fieldwise(adj, ref_adj) < TOL
    assert len(seen) >= 3
    plan.close()


def test_fused_is_the_small_batch_default_and_drops_the_reduction():
    import torch
    from paper_1812_03431_gb300 import rexi
    N, B = 31, 4
    plan = rexi.Plan(N, 48, 96, M=32, max_batch=B, layout="spectral")
    x = torch.from_numpy(inputs.random_spectral(N, B, 9)).cuda()
    plan.profile_enable(1)
    plan.step(x)
    st, n = plan.profile_read()
    assert n == 1 and st["solve"] > 0 and st["reduce"] == 0.0
    assert plan.info()["pole_slots"] == 0
    plan.close()
    # an explicit pole_slots at plan creation selects the slot solve, as does a larger batch
    plan = rexi.Plan(N, 48, 96, M=32, max_batch=B, layout="spectral", pole_slots=8)
    plan.profile_enable(1)
    plan.step(x)
    st, _ = plan.profile_read()
    assert st["reduce"] > 0
    plan.close()
    plan = rexi.Plan(N, 48, 96, M=32, max_batch=8, layout="spectral")
    plan.profile_enable(1)
    plan.step(torch.from_numpy(inputs.random_spectral(N, 8, 9)).cuda())
    st, _ = plan.profile_read()
    assert st["reduce"] > 0
    plan.close()


def test_fused_not_offered_where_it_does_not_apply():
    from paper_1812_03431_gb300 import rexi
    for kw in (dict(solve_arith="fp32x2"), dict(solver="phi"), dict(fsphere=True)):
        plan = rexi.Plan(15, 16, 32, M=8, max_batch=2, layout="spectral", **kw)
        with pytest.raises(rexi.RexiError):
            plan.set_pole_slots(2, 0, 2)
        plan.close()


@pytest.mark.parametrize("shape", [2, 3, 4])
def test_fused_adjoint_matches_oracle(shape):
    import torch
    from paper_1812_03431_gb300 import rexi
    N, M, B, tau = 27, 32, 3, 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    G = inputs.random_spectral(N, B, 77)
    plan = rexi.Plan(N, *grid(N), tau=tau, max_batch=B, layout="spectral", alpha=al, beta=be)
    plan.set_pole_slots(B, 0, shape)  # the fused solve (shape 3: its lean form)
    plan.profile_enable(1)
    got = plan.step_adjoint(torch.from_numpy(G).cuda()).cpu().numpy()
    st, _ = plan.profile_read()
    assert st["reduce"] == 0.0  # no slot reduction ran
    plan.close()
    ref = ostep.rexi_step_spectral(G, N, al, be, tau, C, adjoint=True)
    assert fieldwise(got, ref) < TOL


@pytest.mark.parametrize("shape", [2, 3, 4])
def test_fused_grid_mixed_step_matches_oracle(shape):
    # the chosen form's arithmetic (tcgen05 Legendre transforms, binary64 solves) with the
    # fused solve, against the oracle's grid step
    import torch
    from paper_1812_03431_gb300 import rexi
    N, nlat, nlon, M, B, tau = 63, 96, 192, 64, 5, 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    gs = ostep.GridStep(N, nlat, nlon, al, be, tau, C)
    x = gs.synthesise(inputs.random_spectral(N, B, 63))
    plan = rexi.Plan(N, nlat, nlon, tau=tau, max_batch=B, alpha=al, beta=be, precision="mixed")
    plan.set_pole_slots(B, 0, shape)
    got = plan.step(torch.from_numpy(x).cuda()).cpu().numpy()
    plan.check_device()
    plan.close()
    ref = gs(x)
    for b in range(B):
        assert relerr(got[b, 0], ref[b, 0]) < 1e-5 and relerr(got[b, 1:], ref[b, 1:]) < 1e-5


def test_fused_large_truncation_smaller_tiles():
    # T447 with 16 states: a 16-state tile's running sums (16 x 224 rows x 64 B) exceed
    # shared memory, so the layout takes 8-state tiles; sampled orders against the oracle
    import torch
    from paper_1812_03431_gb300 import rexi
    from oracle.sphere import idx
    N, M, B, tau = 447, 32, 16, 600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = inputs.random_spectral(N, B, 447)
    x = torch.from_numpy(S).cuda()
    plan = rexi.Plan(N, 450, 900, tau=tau, max_batch=B, layout="spectral", alpha=al, beta=be)
    got = plan.step(x).cpu().numpy()
    plan.set_pole_slots(B, 16, 0)
    slot = plan.step(x).cpu().numpy()
    plan.close()
    assert fieldwise(got, slot) < 1e-13
    ms = [0, 1, 224, 446, 447]
    ref = ostep.rexi_step_spectral(S[:2], N, al, be, tau, C, ms=ms)
    sel = np.concatenate([np.arange(idx(m, m, N), idx(m, N, N) + 1) for m in ms])
    assert fieldwise(got[:2][..., sel], ref[..., sel]) < TOL
