"""Ragged batches in one persistent launch, CUDA-graph capture, and the autotuner."""
import numpy as np
import pytest

from oracle import rexi_coeffs as rc
from oracle import step as ostep
from oracle.swe import Consts
from paper_1812_03431_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-10
C = Consts()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1812_03431_gb300 import rexi
    rexi.load()
    return torch, rexi


def grid_of(N):
    return {63: (96, 192), 127: (192, 384), 170: (256, 512), 255: (384, 768), 341: (512, 1024)}[N]


def test_ragged_c3_matches_per_plan_steps_and_graph_replay(env):
    """48 states, truncations drawn from {63,127,170,255,341}, K in {128,256} (seeded)."""
    torch, rexi = env
    rng = np.random.default_rng(1002)
    Ns = rng.choice([63, 127, 170, 255, 341], size=48)
    Ks = rng.choice([128, 256], size=48)
    kinds = sorted(set(zip(Ns.tolist(), Ks.tolist())))
    counts = {k: 0 for k in kinds}
    for k in zip(Ns.tolist(), Ks.tolist()):
        counts[k] += 1
    plans = [rexi.Plan(N, *grid_of(N), M=K, tau=1200.0, max_batch=counts[(N, K)], layout="spectral")
             for (N, K) in kinds]
    state_plan = [kinds.index(k) for k in zip(Ns.tolist(), Ks.tolist())]
    states = [torch.from_numpy(inputs.random_spectral(int(N), 1, 2000 + s)[0]).cuda()
              for s, N in enumerate(Ns)]
    outs = [torch.empty_like(x) for x in states]
    rg = rexi.Ragged(plans, 48)
    rg.step(states, outs, state_plan)
    torch.cuda.synchronize()
    # reference: each plan's own batched step
    for p, plan in enumerate(plans):
        idx = [s for s in range(48) if state_plan[s] == p]
        X = torch.stack([states[s] for s in idx])
        Y = plan.step(X).cpu().numpy()
        for r, s in enumerate(idx):
            assert rel(outs[s].cpu().numpy(), Y[r]) < 1e-13
    # one small state against the oracle as well
    s63 = [s for s in range(48) if Ns[s] == 63]
    if s63:
        s = s63[0]
        al, be = plans[state_plan[s]].coefficients()
        ref = ostep.rexi_step_spectral(states[s].cpu().numpy()[None], 63, al, be, 1200.0, C)[0]
        assert max(rel(outs[s].cpu().numpy()[f], ref[f]) for f in range(3)) < TOL
    # capture the ragged step in a CUDA graph and replay it
    eager = [o.clone() for o in outs]
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        rg.step(states, outs, state_plan)
    torch.cuda.current_stream().wait_stream(side)
    with torch.cuda.graph(g):
        rg.step(states, outs, state_plan)
    for o in outs:
        o.zero_()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(outs, eager):
        assert torch.equal(a, b)
    rg.close()
    for plan in plans:
        plan.close()


def test_ragged_rebuilds_after_a_plan_is_retuned(env):
    # the ragged object caches views of each plan's slot layout; re-tuning a plan (or
    # setting another slot count) replaces that layout, and the next ragged step must
    # rebuild its work list rather than read the freed one
    torch, rexi = env
    plans = [rexi.Plan(N, *grid_of(N), M=K, tau=1200.0, max_batch=3, layout="spectral")
             for N, K in ((63, 128), (127, 256))]
    state_plan = [0, 1, 1, 0, 1]
    states = [torch.from_numpy(inputs.random_spectral(63 if p == 0 else 127, 1, 3000 + s)[0]).cuda()
              for s, p in enumerate(state_plan)]
    outs = [torch.empty_like(x) for x in states]
    rg = rexi.Ragged(plans, 5)

    def check():
        rg.step(states, outs, state_plan)
        torch.cuda.synchronize()
        for p, plan in enumerate(plans):
            idx = [s for s in range(5) if state_plan[s] == p]
            Y = plan.step(torch.stack([states[s] for s in idx])).cpu().numpy()
            for r, s in enumerate(idx):
                assert rel(outs[s].cpu().numpy(), Y[r]) < 1e-13

    check()
    plans[1].set_pole_slots(3, 256, 1)  # another slot layout for the 3 states of plan 1
    check()
    plans[0].tune(2)
    plans[1].tune(3)
    check()
    rg.close()
    for plan in plans:
        plan.close()


def test_ragged_with_a_plan_left_out_and_odd_counts(env):
    # a call in which one plan has no states, then one with odd counts (the last tile of
    # each plan half empty), against each plan's own step and the oracle
    torch, rexi = env
    plans = [rexi.Plan(N, *grid_of(N), M=K, tau=1200.0, max_batch=5, layout="spectral")
             for N, K in ((63, 128), (127, 128), (63, 256))]
    rg = rexi.Ragged(plans, 8)
    for state_plan in ([2, 2, 0], [0, 1, 1, 1, 2, 0, 1, 2]):
        Ns = [63 if p != 1 else 127 for p in state_plan]
        states = [torch.from_numpy(inputs.random_spectral(N, 1, 4000 + s)[0]).cuda() for s, N in enumerate(Ns)]
        outs = [torch.empty_like(x) for x in states]
        rg.step(states, outs, state_plan)
        torch.cuda.synchronize()
        for p, plan in enumerate(plans):
            idx = [s for s in range(len(state_plan)) if state_plan[s] == p]
            if not idx:
                continue
            Y = plan.step(torch.stack([states[s] for s in idx])).cpu().numpy()
            for r, s in enumerate(idx):
                assert rel(outs[s].cpu().numpy(), Y[r]) < 1e-13
        s = state_plan.index(0)
        al, be = plans[0].coefficients()
        ref = ostep.rexi_step_spectral(states[s].cpu().numpy()[None], 63, al, be, 1200.0, C)[0]
        assert max(rel(outs[s].cpu().numpy()[f], ref[f]) for f in range(3)) < TOL
    rg.close()
    for plan in plans:
        plan.close()


@pytest.mark.parametrize("shape,precision,groups", [(None, "fp64", 0), (2, "fp64", 1), (3, "mixed", 0),
                                                    (0, "mixed", 0), (2, "fp64", 3)])
def test_step_in_cuda_graph(env, shape, precision, groups):
    # the default (slot) solve, the fused solve in both forms, a fixed slot layout, and the
    # fused solve with each tile's poles over three CTAs (the arrival counts are reset by
    # a memset inside the graph)
    torch, rexi = env
    N, nlat, nlon, B = 127, 192, 384, 4
    plan = rexi.Plan(N, nlat, nlon, M=128, tau=1200.0, max_batch=B, precision=precision)
    if shape is not None:
        used = plan.set_pole_slots(B, 16 if shape == 0 else 0, shape, groups=groups)
        if groups:
            assert used // 256 == groups
    x = plan.synthesize(torch.from_numpy(inputs.random_spectral(N, B, 5)).cuda())
    y = torch.empty_like(x)
    plan.step(x, out=y)  # first call with this batch builds the work list
    eager = y.clone()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.step(x, out=y)
    torch.cuda.current_stream().wait_stream(side)
    with torch.cuda.graph(g):
        plan.step(x, out=y)
    y.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, eager)
    plan.close()


def test_autotuner_keeps_results(env):
    torch, rexi = env
    N, B = 127, 16
    al, be, _ = rc.rexi_coefficients(64, 0.2)
    plan = rexi.Plan(N, 192, 384, tau=1200.0, max_batch=B, layout="spectral", alpha=al, beta=be)
    S = torch.from_numpy(inputs.random_spectral(N, B, 9)).cuda()
    before = plan.step(S).cpu().numpy()
    slots = plan.tune(B)
    assert slots >= 1
    after = plan.step(S).cpu().numpy()
    assert rel(after, before) < 1e-13
    ref = ostep.rexi_step_spectral(S.cpu().numpy()[:1], N, al, be, 1200.0, C, ms=[0, 5, 64, 127])
    from oracle.sphere import idx
    sel = np.concatenate([np.arange(idx(m, m, N), idx(m, N, N) + 1) for m in [0, 5, 64, 127]])
    assert max(rel(after[0, f, sel], ref[0, f, sel]) for f in range(3)) < TOL
    plan.close()
