#!/usr/bin/env python
"""REXI steps/s at T341, K=256 poles on one GB300 (or N replicas).

Workload: one T-REXI step (Algorithm 1) of the linear SWE for a batch of 16
seeded states (complex-normal n^-3 spectra, h' std 50 m, u,v std 5 m/s),
truncation T341 on a 1024 x 512 Gaussian grid, M = 256 Gaussian basis functions
per side (P = 535 poles), h = 0.2, tau = 1200 s, grid layout in and out (h', u, v
float64).  A step = longitude FFTs, Legendre analysis, the 535 x 342 x 2 banded
solves with the beta-weighted pole sum, Legendre synthesis, inverse FFTs.
Inputs (201 MB) and factors (4.5 GB) are larger than L2, so no flush is done.

The chosen form (its time is `value`): 3xTF32 tensor-core Legendre transforms with
FP32 accumulation, FP32 FFTs, and the banded solves and the beta-weighted pole sum in
binary64.  The plain FP64 form and a float-float-solve variant are timed beside it,
and every form's result for state 0 is compared with the CPU oracle's.

`python bench.py [--gpus N --steps K --warmup W] [--impl reference]` prints
one JSON line.  For N > 1 (torchrun) every rank runs an independent replica
by default (weak scaling: value is the sum over ranks); with `--shard poles` the
ranks split the poles of one batch evenly and every step ends with an NCCL
allreduce of the partial results (Sec. 6.4; strong scaling).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# The metric's workload (the default) and the specification's other single-GPU workloads,
# timed with --workload: T127 with 64 states, and a single T1279 state.  Seeds follow the
# input recipe (1000 + the workload's place in the specification; the metric's run 1005).
WORKLOADS = {
    "t341_b16": dict(N=341, nlat=512, nlon=1024, M=256, h=0.2, tau=1200.0, batch=16, seed=1005),
    "t127_b64": dict(N=127, nlat=192, nlon=384, M=256, h=0.2, tau=7200.0, batch=64, seed=1001),
    "t1279_b1": dict(N=1279, nlat=1920, nlon=3840, M=512, h=0.2, tau=21600.0, batch=1, seed=1004),
    # Sec. 6.1's single state: the balanced zonal flow plus n^-3 noise of std 1e-3
    "t63_c1": dict(N=63, nlat=96, nlon=192, M=128, h=0.2, tau=3600.0, batch=1, seed=1000, state="noisy_balanced"),
}
# the oracle's whole grid step for one state finishes in seconds up to T341; at T1279 it
# would take hours, so that workload reports no error against it
ORACLE_MAX_N = 341
WORK = dict(WORKLOADS["t341_b16"])
METRIC = "REXI steps/s at T341, K=256 poles: chosen vs plain FP64 form at stated error"
# (name, transforms, solve arithmetic); the first is the chosen form.  mixed: 3xTF32 Legendre
# and FP32 FFTs, binary64 banded solves and pole sum; fp64: every stage in binary64 (the
# plain form); ff_solve: the mixed transforms with the solves and the pole sum in
# float-float arithmetic on the FP32 pipes (48-bit significands), an extension timed for
# comparison only: it does not keep the solves in binary64.
FORMS = [("mixed", "mixed", "fp64"), ("fp64", "fp64", "fp64"), ("ff_solve", "mixed", "fp32x2")]
FLOPS_PER_ROW = 72  # FP64 flops per (state, pole, row) of the fused solve: 36 FMAs
# FP32 operations per (state, pole, row) of the float-float solve: the same 36 real
# multiply-adds, each an error-free product and sum of 12 FP32 operations (1 mul, 3 FMA,
# 8 add); stored values stay unnormalised pairs, so there is no renormalisation
FF_OPS_PER_ROW = 36 * 12
# DRAM bytes (read + write) of one solve launch from ncu captures (K=256, batch 16), keyed by
# (truncation, pole slots or, for the fused solve, states per CTA tile, layout shape):
# shape 0/1 the slot kernel, 2/3/4 the fused solve's register form, lean form, lean form on
# two-warp CTAs, with one pole group.
# A workload without its own capture takes the nearest layout captured at T170, scaled by
# rows (traffic per row is constant).  Re-captured after each change of the solve kernels.
SOLVE_TRAFFIC = {(341, 64, 0): 48.82e9, (341, 2, 3): 18.60e9, (341, 2, 4): 27.86e9,
                 (170, 32, 0): 12.64e9, (170, 32, 1): 12.58e9, (170, 64, 0): 11.63e9,
                 (170, 2, 2): 1.64e9, (170, 2, 3): 4.92e9}
SOLVE_FF_TRAFFIC_T170 = {(32, 0): 11.64e9}  # the float-float kernel (solve_kernel<true>)


def rows_of(N):
    return (N + 1) * (N + 2) // 2 - 1  # every (m, n) except (0, 0)


def fp64_peak_tflops(sm_mhz):
    # GB300: 152 SMs x 2 FP64 FMA/clk/SM (nominal 1.25 TFLOP/s at 2070 MHz); only a
    # fallback: the bench measures the rate (rexi_measure_fp64_fma) and divides by that
    return 152 * 4 * sm_mhz * 1e6 / 1e12


def fp32_peak_tops(sm_mhz):
    # GB300: 152 SMs x 128 FP32 lanes, one add, multiply or FMA per lane and clock
    return 152 * 128 * sm_mhz * 1e6 / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, "fallback"


def solve_layout(r):
    """The tuned solve layout of a form's record: pole slots and shape, or for the fused
    solve (shapes 2 to 4) its form, CTA tile and the CTAs that split each tile's poles."""
    if r["shape"] in (2, 3, 4):
        return {"fused": {2: "register", 3: "lean", 4: "lean, two-warp CTAs"}[r["shape"]],
                "tile": r["slots"] % 256, "pole_groups": r["slots"] // 256, "layout_shape": r["shape"]}
    return {"pole_slots": r["slots"], "layout_shape": r["shape"]}


def kernel_rooflines(form, stages, slots, sm_mhz, solve_arith="fp64", fp64_peak=None):
    """Every stage of the grid step against its own bound: algorithmic bytes (HBM-bound
    stages) or flops (ALU-bound stages) per launch / its live CUDA-event time.
    fp64_peak: the measured FP64 FMA rate in TFLOP/s (else derived from the clock)."""
    W = WORK
    N, B, nlat, nlon = W["N"], W["batch"], W["nlat"], W["nlon"]
    P = 2 * (W["M"] + 11) + 1
    ns = (N + 1) * (N + 2) // 2
    hbm, bf16, src = measured_peaks()
    fp64 = fp64_peak if fp64_peak else fp64_peak_tflops(sm_mhz)
    fp64_src = "measured FP64 FMA rate" if fp64_peak else "derived FP64"
    grid_b = B * 3 * nlat * nlon * 8
    four_b = nlat * (N + 1) * 3 * B * (8 if form == "mixed" else 16)  # complex FP32 / FP64
    spec_b = 3 * ns * B * 16
    out = {}

    def put(name, bound, amount, unit, peak, peak_src):
        ms = stages.get(name)
        if not ms:
            return
        ach = amount / (ms * 1e-3) / (1e9 if unit == "GB/s" else 1e12)
        out[name] = {"ms": ms, "bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                     "algorithmic": amount, "peak_source": peak_src}

    # FFTs: read the grid once, write the Fourier coefficients once (and back)
    if form == "mixed":
        put("fft_fwd", "hbm", grid_b + four_b, "GB/s", hbm, src + " HBM copy")
        put("fft_inv", "hbm", grid_b + four_b, "GB/s", hbm, src + " HBM copy")
        # tcgen05 Legendre: TF32 hi/lo tables P and H (2 x 2 x 4 B per (n, lat pair)),
        # Fourier data in, spectral coefficients out
        leg_b = 16 * ns * (nlat // 2) + four_b + spec_b
        put("leg_ana", "hbm", leg_b, "GB/s", hbm, src + " HBM copy")
        put("leg_syn", "hbm", leg_b, "GB/s", hbm, src + " HBM copy")
    else:
        # FP64 FFT: 5 n log2 n flops per half-length complex transform of each real row
        import math
        half = nlon // 2
        fl = 5.0 * half * math.log2(half) * B * 3 * nlat
        put("fft_fwd", "alu", fl, "TFLOP/s", fp64, fp64_src)
        put("fft_inv", "alu", fl, "TFLOP/s", fp64, fp64_src)
        # FP64 Legendre: 10 FMAs per (n, lat pair, state) each way
        fl = 20.0 * ns * (nlat // 2) * B
        put("leg_ana", "alu", fl, "TFLOP/s", fp64, fp64_src)
        put("leg_syn", "alu", fl, "TFLOP/s", fp64, fp64_src)
    if solve_arith == "fp32x2":
        put("solve", "alu", FF_OPS_PER_ROW * B * P * rows_of(N), "Tops/s", fp32_peak_tops(sm_mhz),
            "derived FP32 (ops = adds, multiplies and FMAs)")
        # float-float reduction: reads every slot's partials once, writes the result
        put("reduce", "hbm", (slots + 2) * 3 * ns * B * 16, "GB/s", hbm, src + " HBM copy")
    else:
        put("solve", "alu", FLOPS_PER_ROW * B * P * rows_of(N), "TFLOP/s", fp64, fp64_src)
        # reduction: one FP64 complex add per slot and output coefficient; the kernel is bound
        # by the FP64 issue rate (ncu: FP64 pipe 82 %, DRAM 47 %), where an add costs an FMA's slot
        put("reduce", "alu", 2.0 * slots * 3 * ns * B, "TFLOP/s", fp64 / 2, fp64_src + " (adds: half)")
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        note = None
        if not sms:
            # a timed region shorter than the sampling period: one reading right after it
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=10).stdout
                parts = [p.strip() for p in out.strip().split(",")]
                if len(parts) >= 9:
                    sms.append(float(parts[1]))
                    mx = float(parts[2])
                    for n, v in zip(names, parts[5:9]):
                        if v.lower() == "active":
                            reasons.add(n)
                    note = "timed region shorter than the 200 ms sampling period: one reading right after it"
            except (OSError, ValueError, subprocess.TimeoutExpired):
                pass
        if not sms:
            return None
        rec = {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons),
               "samples": len(sms) if note is None else 0}
        if note:
            rec["note"] = note
        return rec


def host_threads():
    """Threads the oracle's numpy/scipy calls may use on this host (BLAS pools)."""
    try:
        from threadpoolctl import threadpool_info
        return max([1] + [i.get("num_threads", 1) for i in threadpool_info()])
    except Exception:
        return 1


def make_states():
    """The workload's seeded spectral states [B, 3, nspec] (input recipe)."""
    from paper_1812_03431_gb300 import inputs
    W = WORK
    if W.get("state") == "noisy_balanced":
        return np.concatenate([inputs.noisy_balanced(W["N"], W["seed"] + b) for b in range(W["batch"])])
    return inputs.random_spectral(W["N"], W["batch"], W["seed"])


def oracle_grid_step(x0):
    """The oracle's whole grid-layout step (Algorithm 1 with its own poles, transforms and
    banded solves) for one state x0 [3, nlat, nlon]; returns (result, seconds)."""
    from oracle import rexi_coeffs
    from oracle import step as ostep
    W = WORK
    al, be, _ = rexi_coeffs.rexi_coefficients(W["M"], W["h"])
    gs = ostep.GridStep(W["N"], W["nlat"], W["nlon"], al, be, W["tau"])
    t0 = time.perf_counter()
    y = gs(x0[None])
    return y[0], time.perf_counter() - t0


def _oracle_solves(task):
    """Worker: the oracle's banded solves for a subset of zonal orders (one state)."""
    S, al, be, ms = task
    from oracle import step as ostep
    t0 = time.perf_counter()
    ostep.rexi_step_spectral(S, WORK["N"], al, be, WORK["tau"], ms=ms)
    return time.perf_counter() - t0


def cpu_baseline_all_cores(S0):
    """The oracle's banded solves for one state with its zonal orders spread over every host
    core (one process each, started by spawn); the oracle's code is unchanged."""
    import multiprocessing as mp
    from oracle import rexi_coeffs
    N, B = WORK["N"], WORK["batch"]
    al, be, _ = rexi_coeffs.rexi_coefficients(WORK["M"], WORK["h"])
    ms = list(range(N + 1))
    n = max(1, min(os.cpu_count() or 1, len(ms)))
    chunks = [ms[i::n] for i in range(n)]  # interleaved: the row counts fall with m
    with mp.get_context("spawn").Pool(n) as pool:
        pool.map(_oracle_solves, [(S0, al, be, [N]) for _ in range(n)], chunksize=1)  # start-up and imports
        t0 = time.perf_counter()
        pool.map(_oracle_solves, [(S0, al, be, c) for c in chunks], chunksize=1)
        wall = time.perf_counter() - t0
    return {"value": 1.0 / (B * wall), "unit": "steps/s", "cores": n, "sample_seconds": wall,
            "sample": "state 0 of %d: the banded solves of all %d zonal orders (every pole) on %d processes; "
                      "transforms not included; a step is %d such states" % (B, N + 1, n, B)}


def reference_arm(args, rank):
    """The oracle as it stands, on the host cores, on this workload: each timed step runs the
    oracle's banded solves for two zonal orders of state 0 with every pole (a bounded sample),
    and value extrapolates by the sampled fraction of the step's rows and states."""
    if rank != 0:
        return
    from oracle import rexi_coeffs
    from oracle import step as ostep
    W = WORK
    N, B = W["N"], W["batch"]
    al, be, _ = rexi_coeffs.rexi_coefficients(W["M"], W["h"])
    S0 = make_states()[:1]
    per, fracs = [], []
    for i in range(args.warmup + args.steps):
        m0 = (37 * i) % (N + 1)
        ms = sorted({m0, (m0 + (N + 1) // 2) % (N + 1)})
        t0 = time.perf_counter()
        ostep.rexi_step_spectral(S0, N, al, be, W["tau"], ms=ms)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            per.append(dt)
            fracs.append(sum(N - m + 1 for m in ms) / ((N + 1) * (N + 2) / 2) / B)
    ms_step = 1e3 * statistics.mean(per)  # measured: what one timed (sampled) step took
    frac = statistics.mean(fracs)
    v = frac * 1e3 / ms_step            # full steps per second, extrapolated by the sampled fraction
    cores = 1                            # the banded solves are scipy LAPACK calls on one thread
    sample = ("per timed step: state 0 of %d, the banded solves of 2 of the %d zonal orders with all %d poles "
              "(%.4f of a step's solves); transforms not included" % (B, N + 1, len(al), frac))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(), "extrapolated": True, "sample_fraction": frac,
            "ms_per_full_step_extrapolated": ms_step / frac,
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def shard_allreduce(y, dist):
    """The one reduction of Sec. 6.4 when the poles are split over ranks: every rank's
    partial step is summed in place (NCCL on the GPU, gloo on the CPU)."""
    if dist is not None:
        import torch
        dist.all_reduce(torch.view_as_real(y) if y.is_complex() else y, op=dist.ReduceOp.SUM)
    return y


def replica_max_ms(ms, dist):
    """Max of a per-rank time over all ranks (the slowest replica sets the job's time)."""
    if dist is None:
        return ms
    import torch
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_config():
    W = WORK
    P = 2 * (W["M"] + 11) + 1
    grid_mb = W["batch"] * 3 * W["nlat"] * W["nlon"] * 8 / 1e6
    fac_gb = 9 * rows_of(W["N"]) * P * 16 / 1e9
    state = ("the balanced zonal flow of Sec. 6.1 plus n^-3 noise of std 1e-3" if W.get("state") == "noisy_balanced"
             else "seeded n^-3 spectra")
    return {"workload": "T-REXI step, linear SWE on the sphere: T%d, %dx%d Gaussian grid, K=M=%d (P=%d poles), "
                        "h=%g, tau=%g s, %d state%s (%s), grid layout"
                        % (W["N"], W["nlon"], W["nlat"], W["M"], P, W["h"], W["tau"], W["batch"],
                           "s" if W["batch"] > 1 else "", state),
            "global_batch": W["batch"], "truncation": W["N"], "grid": [W["nlat"], W["nlon"]],
            "poles": P, "parallelism": "replicas",
            "l2": "inputs (%.0f MB) and factors (%.1f GB) larger than L2, no flush" % (grid_mb, fac_gb)
            if grid_mb * 1e6 > 129e6 or fac_gb * 1e9 > 129e6 else "inputs and factors fit in L2"}


def relerr_fields(got, ref):
    """Relative L2 errors of one grid state: h', the wind (u, v) as one vector field, and
    the components u and v on their own."""
    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    return {"h": rel(got[0], ref[0]), "wind": rel(got[1:], ref[1:]), "u": rel(got[1], ref[1]), "v": rel(got[2], ref[2])}


def time_form(rexi, torch, name, prec, arith, x, args, dist, local, stream, solver="delta"):
    """Plan, tune, warm up and time one form of the step; returns its record (and the e2e run
    for the chosen form).  With --shard poles each rank's plan holds its share of the poles
    and a step ends with the allreduce of the partial results."""
    W = WORK
    B = W["batch"]
    poles, sdist = None, None
    if args.shard == "poles" and dist is not None:
        P = 2 * (W["M"] + 11) + 1
        poles, sdist = rexi.pole_shard(P, dist.get_rank(), dist.get_world_size()), dist
    plan = rexi.Plan(W["N"], W["nlat"], W["nlon"], M=W["M"], h=W["h"], tau=W["tau"], max_batch=B,
                     precision=prec, solve_arith=arith, solver=solver, poles=poles)
    slots = plan.tune(B)  # the library's autotuner picks the pole-slot count for this batch
    y = torch.empty_like(x)

    def step(xx, yy, stream=None):
        plan.step(xx, out=yy, stream=stream)
        if sdist is not None:
            with torch.cuda.stream(stream or torch.cuda.current_stream()):
                shard_allreduce(yy, sdist)

    for _ in range(args.warmup):
        step(x, y)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    plan.profile_enable(args.steps)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    stages, ncalls = plan.profile_read()
    plan.profile_enable(0)
    ck = clocks.stop()
    ms = replica_max_ms(ms, dist)
    rec = dict(ms=ms, stages={k: v / max(ncalls, 1) for k, v in stages.items()}, clocks=ck, y=y,
               bytes=x.numel() * 8, info=plan.info(), slots=slots, shape=plan.layout_shape.get(B, 0),
               precision=prec, solve_arith=arith, plan=plan, step=step, poles=poles)
    return rec


def e2e_run(torch, step, x, y, args, dist):
    """End to end through the public API: every step copies its input from pinned host memory
    and its result back inside the timed region.  The copies run on their own streams with two
    device buffer pairs, so step i's result goes back and step i+1's input comes in while step
    i+1 / i computes (what a user's pipelined rollout does)."""
    xh = x.cpu().pin_memory()
    yh = torch.empty(y.shape, dtype=y.dtype).pin_memory()
    xd = [torch.empty_like(x) for _ in range(2)]
    yd = [torch.empty_like(y) for _ in range(2)]
    # a compute stream of its own and two copy streams, none of them the legacy default
    # stream (which would serialise with the others)
    cs, h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()

    def e2e_steps(n, start_event):
        computed, copied_back = [None, None], [None, None]
        h2d.wait_event(start_event)
        last = None
        for i in range(n):
            k = i % 2
            with torch.cuda.stream(h2d):
                if computed[k] is not None:
                    h2d.wait_event(computed[k])  # step i-2 has finished reading xd[k]
                xd[k].copy_(xh, non_blocking=True)
                loaded = torch.cuda.Event()
                loaded.record(h2d)
            cs.wait_event(loaded)
            if copied_back[k] is not None:
                cs.wait_event(copied_back[k])  # yd[k] of step i-2 is on the host
            step(xd[k], yd[k], stream=cs)
            computed[k] = torch.cuda.Event()
            computed[k].record(cs)
            with torch.cuda.stream(d2h):
                d2h.wait_event(computed[k])
                yh.copy_(yd[k], non_blocking=True)
                copied_back[k] = torch.cuda.Event()
                copied_back[k].record(d2h)
            last = copied_back[k]
        cs.wait_event(last)

    torch.cuda.synchronize()
    w0 = torch.cuda.Event()
    w0.record(cs)
    e2e_steps(2, w0)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(cs)
    e2e_steps(args.steps, f0)
    f1.record(cs)
    torch.cuda.synchronize()
    ms_e2e = replica_max_ms(f0.elapsed_time(f1) / args.steps, dist)
    same = bool(torch.equal(yh, y.cpu()))  # the copied-back result is the device step's, bit for bit
    return ms_e2e, same


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="auto", choices=["auto"] + [f[0] for f in FORMS],
                    help="auto: time every form, the first (chosen) one gives value")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle's step of state 0 (error vs oracle)")
    ap.add_argument("--no-fp64-peak", action="store_true",
                    help="skip measuring the FP64 FMA rate (the roofline then divides by the derived rate)")
    ap.add_argument("--no-phi-solver", action="store_true",
                    help="skip timing the paper's geopotential-only solver next to the default one")
    ap.add_argument("--shard", default="replicas", choices=["replicas", "poles"],
                    help="N > 1: replicas (every rank steps its own batch, weak scaling) or poles (the ranks "
                         "split the poles of one batch and allreduce the partial steps, strong scaling)")
    ap.add_argument("--workload", default="t341_b16", choices=sorted(WORKLOADS),
                    help="t341_b16: the metric's workload; the others time further workloads of the "
                         "specification (no CPU baseline, no Phi-only solver, no traffic figure)")
    args = ap.parse_args()
    WORK.clear()
    WORK.update(WORKLOADS[args.workload])
    default_workload = args.workload == "t341_b16"
    if not default_workload:
        args.no_cpu_baseline = True
        args.no_phi_solver = True
    if WORK["N"] > ORACLE_MAX_N:
        args.no_oracle = True
    if args.shard == "poles":  # one form, the chosen one, split over the ranks
        args.form = FORMS[0][0]
        args.no_phi_solver = True

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1812_03431_gb300 import rexi

    W = WORK
    B = W["batch"]
    forms = [f for f in FORMS if args.form in ("auto", f[0])]
    S = make_states()
    # one grid input for every form: synthesised once in FP64 (a plan with few poles, only
    # its transforms are used)
    with rexi.Plan(W["N"], W["nlat"], W["nlon"], M=1, h=W["h"], tau=W["tau"], max_batch=B) as sp:
        x = sp.synthesize(torch.from_numpy(S).cuda())
    torch.cuda.synchronize()
    results = {}
    stream = torch.cuda.current_stream()
    for i, (name, prec, arith) in enumerate(forms):
        r = time_form(rexi, torch, name, prec, arith, x, args, dist, local, stream)
        if i == 0:
            r["ms_e2e"], r["e2e_same"] = e2e_run(torch, r["step"], x, r["y"], args, dist)
        r["plan"].close()
        r["y0"] = r["y"][0].cpu().numpy()
        results[name] = r

    # the paper's geopotential-only solver on the same workload, for comparison: in the
    # plain FP64 form and with the chosen form's mixed transforms
    phi = {}
    for name, prec, arith in [("fp64", "fp64", "fp64"), ("mixed", "mixed", "fp64")] if not args.no_phi_solver else []:
        if name not in results:
            continue
        pr = time_form(rexi, torch, name, prec, arith, x, args, dist, local, stream, solver="phi")
        pr["plan"].close()
        f = results[name]["y"]
        phi[name] = {"value": world * 1e3 / pr["ms"], "ms_per_step": pr["ms"], "pole_slots": pr["slots"],
                     "stage_ms": pr["stages"], "difference_vs_delta_form": float((pr["y"] - f).norm() / f.norm()),
                     "y0": pr["y"][0].cpu().numpy(),
                     "note": "REXI_SOLVER_PHI: the paper's Phi-only system (Sec. 4.3, 5), pentadiagonal per "
                             "(pole, m, parity); a different truncation, so it differs from the delta "
                             "elimination at the highest degrees; compared with the %s form" % name}

    # the measured FP64 FMA rate: the solve's roofline divides by it
    fp64_tf, fp64_ms, fp64_clocks = None, None, None
    if not args.no_fp64_peak:
        clocks = ClockSampler(local)
        clocks.start()
        fp64_tf, fp64_ms = rexi.rexi_measure_fp64_fma(5)
        fp64_clocks = clocks.stop()

    chosen = forms[0][0]
    r = results[chosen]
    P = 2 * (W["M"] + 11) + 1
    solve_ms = r["stages"]["solve"]
    sm_mhz = (r["clocks"] or {}).get("sm_max_mhz") or 2070.0
    if r["solve_arith"] == "fp32x2":
        amount, peak = FF_OPS_PER_ROW * B * P * rows_of(W["N"]), fp32_peak_tops(sm_mhz)
        traffic_tab = {(170,) + k: v for k, v in SOLVE_FF_TRAFFIC_T170.items()}
        kname = "solve_kernel<true> (float-float banded solves + pole sum)"
        roof_unit, peak_source = "Tops/s", "derived: 152 SMs x 128 FP32 lanes x sm_max_mhz (ops = adds, mults, FMAs)"
    else:
        amount, peak = FLOPS_PER_ROW * B * P * rows_of(W["N"]), fp64_tf or fp64_peak_tflops(sm_mhz)
        traffic_tab, kname = SOLVE_TRAFFIC, "solve_kernel<false> (FP64 banded solves + pole sum)"
        roof_unit = "TFLOP/s"
        peak_source = ("measured: rexi_measure_fp64_fma, best of 5 per shape (FP64 FMA chains)" if fp64_tf else
                       "derived: 152 SMs x 2 FP64 FMA/clk x sm_max_mhz")
    achieved = amount / (solve_ms * 1e-3) / 1e12
    fused = r["shape"] in (2, 3, 4)
    # the fused solve's slot count packs its CTA tile and pole groups (tile + 256 x groups)
    tile_or_slots, groups = (r["slots"] % 256, r["slots"] // 256) if fused else (r["slots"], 1)
    tkey, traffic = None, None
    if (W["N"], tile_or_slots, r["shape"]) in traffic_tab:
        tkey = (W["N"], tile_or_slots, r["shape"])
        traffic = traffic_tab[tkey]
    else:
        near = [k for k in traffic_tab if k[0] == 170 and k[2] == r["shape"]]
        if near:
            tkey = min(near, key=lambda k: abs(k[1] - tile_or_slots))
            traffic = traffic_tab[tkey] * rows_of(W["N"]) / rows_of(170)
    if traffic and groups > 1:
        # the captures hold one pole group; NG groups add their partial sums, written once
        # and read once: B x NG x rows x 4 streams x 16 bytes each way
        traffic += 2 * B * groups * rows_of(W["N"]) * 64
    if fused:
        kname = "solve_fused_kernel (FP64 banded solves, beta-weighted pole sum on chip)"
    dtypes = {"mixed": "f64 solves + pole sum; 3xtf32 legendre; f32 fft", "fp64": "f64",
              "ff_solve": "f64 i/o; float-float (2 x f32) solves + pole sum; 3xtf32 legendre; f32 fft"}
    metric = METRIC if default_workload else "REXI steps/s at T%d, K=%d poles, %d state%s: chosen vs plain FP64 " \
        "form at stated error" % (W["N"], W["M"], B, "s" if B > 1 else "")
    if not default_workload:
        traffic = None  # the captured traffic is for 16 states; it does not scale by rows alone
    # one kernel per timed stage, plus the float-float solve's state split
    launches = sum(1 for v in r["stages"].values() if v > 0) + (1 if r["solve_arith"] == "fp32x2" else 0)
    sharded = args.shard == "poles" and world > 1
    jobs = 1 if sharded else world  # replicas each step a batch; shards step one batch together
    cfg = workload_config()
    if sharded:
        cfg["parallelism"] = "poles split over %d ranks (Sec. 6.4), NCCL allreduce of the grid result" % world
    line = {
        "metric": metric, "value": jobs * 1e3 / r["ms"], "unit": "steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True,
        "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": dtypes[chosen],
        "data": "synthetic", "config": cfg,
        "form": chosen, "solve_layout": solve_layout(r),
        "roofline": {"bound": "alu", "kernel": kname,
                     "achieved": achieved, "peak": peak, "unit": roof_unit, "frac": achieved / peak,
                     "traffic": traffic,
                     "traffic_source": ("ncu dram bytes at T%d/K256/B16, %d pole slots (fused: states per tile), "
                                        "layout shape %d (shapes 2 to 4 = fused; the bench's layout: %d, shape %d, "
                                        "%d pole group(s))%s" % (tkey[0], tkey[1], tkey[2], tile_or_slots, r["shape"],
                                                                 groups, "" if tkey[0] == W["N"] else
                                                                 ", scaled by rows to T%d" % W["N"]))
                     if default_workload and traffic else "not captured for this workload or kernel",
                     "dram_gbs": traffic / (solve_ms * 1e-3) / 1e9 if traffic else None,
                     "peak_source": peak_source, "algorithmic_per_launch": amount, "launch_ms": solve_ms},
        # the whole S4 stage (banded solves and the complete pole sum): the fused solve's time
        # alone, or the slot kernel's plus its reduction -- the two paths compared like for like
        "solve_stage": {"ms": solve_ms + r["stages"].get("reduce", 0.0),
                        "achieved": amount / ((solve_ms + r["stages"].get("reduce", 0.0)) * 1e-3) / 1e12,
                        "frac": amount / ((solve_ms + r["stages"].get("reduce", 0.0)) * 1e-3) / 1e12 / peak,
                        "unit": roof_unit, "kernels": "solve_fused_kernel" if fused else "solve_kernel + reduce_kernel"},
        "fp64_peak": {"tflops": fp64_tf, "ms": fp64_ms, "clocks": fp64_clocks,
                      "derived_tflops_at_max_clock": fp64_peak_tflops(sm_mhz)},
        "state_steps_per_s": jobs * B * 1e3 / r["ms"],
        "stage_ms": r["stages"],
        "kernels": kernel_rooflines(r["precision"], r["stages"], r["slots"], sm_mhz, r["solve_arith"], fp64_tf),
        "e2e": {"value": jobs * 1e3 / r["ms_e2e"], "unit": "steps/s", "h2d_bytes_per_step": r["bytes"],
                "d2h_bytes_per_step": r["bytes"], "copies": "pinned host, own streams, overlapping compute",
                "result_matches_device_step": r["e2e_same"]},
        "gpu_launches": launches * args.steps,
        "clocks": r["clocks"],
    }
    for name, _, _ in forms[1:]:
        f = results[name]
        line[name + "_form"] = {"value": world * 1e3 / f["ms"], "ms_per_step": f["ms"], "stage_ms": f["stages"],
                                "dtype": dtypes[name], "solve_layout": solve_layout(f),
                                "clocks": f["clocks"],
                                "kernels": kernel_rooflines(f["precision"], f["stages"], f["slots"], sm_mhz,
                                                            f["solve_arith"], fp64_tf)}
    if "ff_solve_form" in line:
        line["ff_solve_form"]["note"] = ("float-float solves and pole sum on the FP32 pipes: an extension outside "
                                         "the precision contract (binary64 solves), timed for comparison")
    if "fp64" in results and chosen != "fp64":
        f = results["fp64"]
        line["error_vs_fp64_form"] = float((results[chosen]["y"] - f["y"]).norm() / f["y"].norm())
    if "ff_solve" in results and "mixed" in results:
        f, y = results["mixed"]["y"], results["ff_solve"]["y"]
        line["ff_solve_form"]["vs_mixed_fp64_solves"] = {"rel_l2": float((y - f).norm() / f.norm()),
                                                         "bitwise_equal": bool(torch.equal(y, f))}
    if "fp64" in phi:
        line["phi_solver_form"] = {k: v for k, v in phi["fp64"].items() if k != "y0"}
    if "mixed" in phi:
        line["phi_solver_chosen_form"] = {k: v for k, v in phi["mixed"].items() if k != "y0"}
    for res in results.values():
        res.pop("y", None)
    torch.cuda.synchronize()

    if rank == 0 and not args.no_oracle:
        # the oracle's own grid step of state 0 (its own poles, transforms and banded solves):
        # every form's result for that state against it
        ref0, t_oracle = oracle_grid_step(x[0].cpu().numpy())
        errs = {name: relerr_fields(res["y0"], ref0) for name, res in results.items()}
        for name, pv in phi.items():
            errs["phi_solver_" + name] = relerr_fields(pv["y0"], ref0)
        line["error_vs_oracle"] = {
            "state": 0, "rel_l2": errs, "max_h_wind": {k: max(v["h"], v["wind"]) for k, v in errs.items()},
            "bound": {"fp64": 1e-10, "mixed": 1e-5, "ff_solve": 1e-5},
            "note": "the oracle's whole grid step of state 0 with its own poles (an independent refit: "
                    "responses agree to 6e-13); bounds on h' and the wind vector.  The Phi-only solver is a "
                    "different truncation (Sec. 5), so its difference from this delta-elimination oracle is "
                    "a discretisation difference, not a rounding error; its parity is tested against its "
                    "own oracle"}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = {
                "value": 1.0 / (B * t_oracle), "unit": "steps/s", "cores": host_threads(), "kind": "oracle",
                "sample": "state 0 of %d: the oracle's whole grid step (its transforms and all %d x %d x 2 banded "
                          "solves) timed once (%.1f s), times %d states; numpy/scipy as they stand, BLAS pools "
                          "of up to %d threads (the banded solves are single-threaded LAPACK calls)"
                          % (B, P, W["N"] + 1, t_oracle, B, host_threads()),
                "sample_seconds": t_oracle}
            try:
                line["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores(S[:1])
            except Exception as exc:  # a host without process support still gets the 1-core number
                line["cpu_baseline"]["all_cores"] = {"unavailable": repr(exc)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
