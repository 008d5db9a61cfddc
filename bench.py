#!/usr/bin/env python
"""REXI steps/s at T341, K=256 poles on one GB300 (or N replicas).

Workload: one T-REXI step (Algorithm 1) of the linear SWE for a batch of 16
seeded states (complex-normal n^-3 spectra, h' std 50 m, u,v std 5 m/s),
truncation T341 on a 1024 x 512 Gaussian grid, M = 256 Gaussian basis functions
per side (P = 535 poles), h = 0.2, tau = 1200 s, grid layout in and out (h', u, v
float64).  A step = longitude FFTs, Legendre analysis, the 535 x 342 x 2 banded
solves with the beta-weighted pole sum, Legendre synthesis, inverse FFTs.
Inputs (201 MB) and factors (4.5 GB) are larger than L2, so no flush is done.

`python bench.py [--gpus N --steps K --warmup W] [--impl reference]` prints
one JSON line.  For N > 1 (torchrun) every rank runs an independent replica
(the path has no exchange step) and value is the sum over ranks.
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
}
WORK = dict(WORKLOADS["t341_b16"])
METRIC = "REXI steps/s at T341, K=256 poles: chosen vs plain FP64 form at stated error"
# (name, transforms, solve arithmetic); the first is the chosen form.  mixed_fp32x2: 3xTF32
# Legendre and FP32 FFTs, float-float banded solves and pole sum; mixed: the same transforms
# with binary64 solves; fp64: every stage in binary64 (the plain form).
FORMS = [("mixed_fp32x2", "mixed", "fp32x2"), ("mixed", "mixed", "fp64"), ("fp64", "fp64", "fp64")]
FLOPS_PER_ROW = 72  # FP64 flops per (state, pole, row) of the fused solve: 36 FMAs
# FP32 operations per (state, pole, row) of the float-float solve: the same 36 real
# multiply-adds, each an error-free product and sum of 12 FP32 operations (1 mul, 3 FMA,
# 8 add); stored values stay unnormalised pairs, so there is no renormalisation
FF_OPS_PER_ROW = 36 * 12
# DRAM bytes (read + write) of one solve_kernel launch from ncu captures at T170, K=256,
# batch 16, by (pole slots, layout shape) (profiles/solve_kernel_t170_b16.md); traffic per
# row is constant, so a launch of the bench workload moves this times rows(T341) /
# rows(T170).  Re-captured after each change of the solve kernel.
SOLVE_TRAFFIC_T170 = {(32, 0): 12.64e9, (32, 1): 12.58e9}
SOLVE_FF_TRAFFIC_T170 = {(32, 0): 11.64e9}  # the float-float kernel (solve_kernel<true>)


def rows_of(N):
    return (N + 1) * (N + 2) // 2 - 1  # every (m, n) except (0, 0)


def fp64_peak_tflops(sm_mhz):
    # GB300: 152 SMs x 2 FP64 FMA/clk/SM (nominal 1.25 TFLOP/s at 2070 MHz)
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


def kernel_rooflines(form, stages, slots, sm_mhz, solve_arith="fp64"):
    """Every stage of the grid step against its own bound: algorithmic bytes (HBM-bound
    stages) or flops (ALU-bound stages) per launch / its live CUDA-event time."""
    W = WORK
    N, B, nlat, nlon = W["N"], W["batch"], W["nlat"], W["nlon"]
    P = 2 * (W["M"] + 11) + 1
    ns = (N + 1) * (N + 2) // 2
    hbm, bf16, src = measured_peaks()
    fp64 = fp64_peak_tflops(sm_mhz)
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
        put("fft_fwd", "alu", fl, "TFLOP/s", fp64, "derived FP64")
        put("fft_inv", "alu", fl, "TFLOP/s", fp64, "derived FP64")
        # FP64 Legendre: 10 FMAs per (n, lat pair, state) each way
        fl = 20.0 * ns * (nlat // 2) * B
        put("leg_ana", "alu", fl, "TFLOP/s", fp64, "derived FP64")
        put("leg_syn", "alu", fl, "TFLOP/s", fp64, "derived FP64")
    if solve_arith == "fp32x2":
        put("solve", "alu", FF_OPS_PER_ROW * B * P * rows_of(N), "Tops/s", fp32_peak_tops(sm_mhz),
            "derived FP32 (ops = adds, multiplies and FMAs)")
        # float-float reduction: reads every slot's partials once, writes the result
        put("reduce", "hbm", (slots + 2) * 3 * ns * B * 16, "GB/s", hbm, src + " HBM copy")
    else:
        put("solve", "alu", FLOPS_PER_ROW * B * P * rows_of(N), "TFLOP/s", fp64, "derived FP64")
        # reduction: one FP64 complex add per slot and output coefficient; the kernel is bound
        # by the FP64 issue rate (ncu: FP64 pipe 82 %, DRAM 47 %), where an add costs an FMA's slot
        put("reduce", "alu", 2.0 * slots * 3 * ns * B, "TFLOP/s", fp64 / 2, "derived FP64 add rate")
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
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


def cpu_baseline(sample_ms=None):
    """The CPU oracle as it stands on a bounded sample of the workload, extrapolated to one step."""
    from oracle import rexi_coeffs
    from oracle import step as ostep
    from paper_1812_03431_gb300 import inputs
    N, B = WORK["N"], WORK["batch"]
    al, be, _ = rexi_coeffs.rexi_coefficients(WORK["M"], WORK["h"])
    S = inputs.random_spectral(N, 1, WORK["seed"])
    ms = sample_ms if sample_ms is not None else list(range(0, N + 1, 3))  # ~10 s of CPU work
    t0 = time.perf_counter()
    ostep.rexi_step_spectral(S, N, al, be, WORK["tau"], ms=ms)
    t_solve = time.perf_counter() - t0
    rows_sample = sum(N - m + 1 for m in ms)
    rows_all = rows_of(N) + 1
    gs = ostep.GridStep(N, WORK["nlat"], WORK["nlon"], al[:1], be[:1], WORK["tau"])
    t0 = time.perf_counter()
    x = gs.synthesise(S)
    gs.analyse(x)
    t_tr = time.perf_counter() - t0
    t_step = B * (t_solve * rows_all / rows_sample + t_tr)
    cores = 1
    try:
        from threadpoolctl import threadpool_info
        cores = max([1] + [i.get("num_threads", 1) for i in threadpool_info()])
    except Exception:
        pass
    sample = ("1 of %d states; banded solves for m in %s (%d of %d coefficient rows, all %d poles) plus one "
              "analysis+synthesis, extrapolated linearly to the full step" % (B, ms, rows_sample, rows_all, len(al)))
    return {"value": 1.0 / t_step, "unit": "steps/s", "cores": cores, "kind": "oracle", "sample": sample,
            "sample_seconds": t_solve + t_tr}


def _oracle_solves(task):
    """Worker: the oracle's banded solves for a subset of zonal orders (one state)."""
    S, al, be, ms = task
    from oracle import step as ostep
    t0 = time.perf_counter()
    ostep.rexi_step_spectral(S, WORK["N"], al, be, WORK["tau"], ms=ms)
    return time.perf_counter() - t0


def cpu_baseline_all_cores(sample_ms=None):
    """The same oracle sample with its zonal orders spread over every host core (one
    process each, started by spawn); the oracle's code is unchanged."""
    import multiprocessing as mp
    from oracle import rexi_coeffs
    from paper_1812_03431_gb300 import inputs
    N, B = WORK["N"], WORK["batch"]
    al, be, _ = rexi_coeffs.rexi_coefficients(WORK["M"], WORK["h"])
    S = inputs.random_spectral(N, 1, WORK["seed"])
    ms = sample_ms if sample_ms is not None else list(range(0, N + 1, 3))
    n = max(1, min(os.cpu_count() or 1, len(ms)))
    # interleaved chunks balance the decreasing row counts of higher orders
    chunks = [ms[i::n] for i in range(n)]
    with mp.get_context("spawn").Pool(n) as pool:
        pool.map(_oracle_solves, [(S, al, be, [N]) for _ in range(n)], chunksize=1)  # start-up and imports
        t0 = time.perf_counter()
        pool.map(_oracle_solves, [(S, al, be, c) for c in chunks], chunksize=1)
        wall = time.perf_counter() - t0
    rows_sample = sum(N - m + 1 for m in ms)
    rows_all = rows_of(N) + 1
    return {"value": 1.0 / (B * wall * rows_all / rows_sample), "unit": "steps/s", "cores": n,
            "sample_seconds": wall, "sample": "the banded solves of the same sample on %d processes; "
            "transforms not included" % n}


def reference_arm(args, rank):
    if rank != 0:
        return
    per = []
    for i in range(args.warmup + args.steps):
        m0 = (37 * i) % (WORK["N"] + 1)
        r = cpu_baseline(sample_ms=[m0, (m0 + 171) % (WORK["N"] + 1)])
        if i >= args.warmup:
            per.append(1.0 / r["value"])
    ms_step = 1e3 * statistics.mean(per)
    v = 1e3 / ms_step
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(), "cpu_baseline": {**r, "value": v},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    return {"workload": "T-REXI step, linear SWE on the sphere: T%d, %dx%d Gaussian grid, K=M=%d (P=%d poles), "
                        "h=%g, tau=%g s, %d seeded n^-3 state%s, grid layout"
                        % (W["N"], W["nlon"], W["nlat"], W["M"], P, W["h"], W["tau"], W["batch"],
                           "s" if W["batch"] > 1 else ""),
            "global_batch": W["batch"], "truncation": W["N"], "grid": [W["nlat"], W["nlon"]],
            "poles": P, "parallelism": "replicas",
            "l2": "inputs (%.0f MB) and factors (%.1f GB) larger than L2, no flush" % (grid_mb, fac_gb)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="auto", choices=["auto"] + [f[0] for f in FORMS],
                    help="auto: time every form, the first (chosen) one gives value")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-phi-solver", action="store_true",
                    help="skip timing the paper's geopotential-only solver next to the default one")
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
    from paper_1812_03431_gb300 import inputs, rexi

    W = WORK
    B = W["batch"]
    forms = [f for f in FORMS if args.form in ("auto", f[0])]
    S = torch.from_numpy(inputs.random_spectral(W["N"], B, W["seed"])).cuda()
    results = {}
    stream = torch.cuda.current_stream()
    for name, prec, arith in forms:
        plan = rexi.Plan(W["N"], W["nlat"], W["nlon"], M=W["M"], h=W["h"], tau=W["tau"], max_batch=B,
                         precision=prec, solve_arith=arith)
        slots = plan.tune(B)  # the library's autotuner picks the pole-slot count for this batch
        x = plan.synthesize(S)
        y = torch.empty_like(x)
        for _ in range(args.warmup):
            plan.step(x, out=y)
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
            plan.step(x, out=y)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms = e0.elapsed_time(e1) / args.steps
        stages, ncalls = plan.profile_read()
        plan.profile_enable(0)
        ck = clocks.stop()
        ms = replica_max_ms(ms, dist)
        # e2e through the public API: every step copies its input from pinned host memory
        # and its result back inside the timed region.  The copies run on their own streams
        # with two device buffer pairs, so step i's result goes back and step i+1's input
        # comes in while step i+1 / i computes (what a user's pipelined rollout does).
        xh = x.cpu().pin_memory()
        yh = torch.empty(y.shape, dtype=y.dtype).pin_memory()
        xd = [torch.empty_like(x) for _ in range(2)]
        yd = [torch.empty_like(y) for _ in range(2)]
        # a compute stream of its own and two copy streams, none of them the legacy
        # default stream (which would serialise with the others)
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
                plan.step(xd[k], out=yd[k], stream=cs)
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
        ms_e2e = f0.elapsed_time(f1) / args.steps
        ms_e2e = replica_max_ms(ms_e2e, dist)
        e2e_same = bool(torch.equal(yh, y.cpu()))  # the copied-back result is the device step's, bit for bit
        results[name] = dict(ms=ms, ms_e2e=ms_e2e, stages={k: v / max(ncalls, 1) for k, v in stages.items()},
                             clocks=ck, y=y, bytes=x.numel() * 8, info=plan.info(), slots=slots,
                             shape=plan.layout_shape.get(B, 0), e2e_same=e2e_same, precision=prec,
                             solve_arith=arith)
        plan.close()

    # the paper's geopotential-only solver on the same workload, for comparison: in the
    # plain FP64 form, and in the chosen form's arithmetic (mixed transforms, float-float solves)
    phi = {}
    phi_forms = [("fp64", "fp64", "fp64"), ("mixed_fp32x2", "mixed", "fp32x2")]
    for name, prec, arith in phi_forms if not args.no_phi_solver else []:
        if name not in results:
            continue
        plan = rexi.Plan(W["N"], W["nlat"], W["nlon"], M=W["M"], h=W["h"], tau=W["tau"], max_batch=B,
                         precision=prec, solver="phi", solve_arith=arith)
        pslots = plan.tune(B)
        x = plan.synthesize(S)
        y = torch.empty_like(x)
        for _ in range(args.warmup):
            plan.step(x, out=y)
        plan.profile_enable(args.steps)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            plan.step(x, out=y)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = replica_max_ms(e0.elapsed_time(e1) / args.steps, dist)
        stages, ncalls = plan.profile_read()
        f = results[name]["y"]
        phi[name] = {"value": world * 1e3 / pms, "ms_per_step": pms, "pole_slots": pslots,
                     "stage_ms": {k: v / max(ncalls, 1) for k, v in stages.items()},
                     "difference_vs_delta_form": float((y - f).norm() / f.norm()),
                     "note": "REXI_SOLVER_PHI: the paper's Phi-only system (Sec. 4.3, 5), pentadiagonal per "
                             "(pole, m, parity); a different truncation, so it differs from the delta "
                             "elimination at the highest degrees; compared with the %s form" % name}
        plan.close()

    chosen = forms[0][0]
    r = results[chosen]
    P = 2 * (W["M"] + 11) + 1
    solve_ms = r["stages"]["solve"]
    sm_mhz = (r["clocks"] or {}).get("sm_max_mhz") or 2070.0
    if r["solve_arith"] == "fp32x2":
        amount, peak = FF_OPS_PER_ROW * B * P * rows_of(W["N"]), fp32_peak_tops(sm_mhz)
        traffic_t170, kname = SOLVE_FF_TRAFFIC_T170, "solve_kernel<true> (float-float banded solves + pole sum)"
        roof_unit, peak_source = "Tops/s", "derived: 152 SMs x 128 FP32 lanes x sm_max_mhz (ops = adds, mults, FMAs)"
    else:
        amount, peak = FLOPS_PER_ROW * B * P * rows_of(W["N"]), fp64_peak_tflops(sm_mhz)
        traffic_t170, kname = SOLVE_TRAFFIC_T170, "solve_kernel<false> (FP64 banded solves + pole sum)"
        roof_unit, peak_source = "TFLOP/s", "derived: 152 SMs x 2 FP64 FMA/clk x sm_max_mhz"
    achieved = amount / (solve_ms * 1e-3) / 1e12
    tkey = min(traffic_t170, key=lambda k: (k[1] != r["shape"], abs(k[0] - r["slots"])))
    traffic = traffic_t170[tkey] * rows_of(W["N"]) / rows_of(170)
    dtypes = {"mixed_fp32x2": "f64 i/o; float-float (2 x f32) solves + pole sum; 3xtf32 legendre; f32 fft",
              "mixed": "f64 solves + pole sum; 3xtf32 legendre; f32 fft", "fp64": "f64"}
    metric = METRIC if default_workload else "REXI steps/s at T%d, K=%d poles, %d state%s: chosen vs plain FP64 " \
        "form at stated error" % (W["N"], W["M"], B, "s" if B > 1 else "")
    if not default_workload:
        traffic = None  # the captured traffic is for 16 states; it does not scale by rows alone
    line = {
        "metric": metric, "value": world * 1e3 / r["ms"], "unit": "steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtypes[chosen],
        "data": "synthetic", "config": {**workload_config(), "form": chosen, "pole_slots": r["slots"], "layout_shape": r["shape"]},
        "roofline": {"bound": "alu", "kernel": kname,
                     "achieved": achieved, "peak": peak, "unit": roof_unit, "frac": achieved / peak,
                     "traffic": traffic,
                     "traffic_source": ("ncu dram bytes at T170/K256/B16 with %d pole slots, layout shape %d "
                                        "(the captured layout nearest the bench's %d, shape %d), scaled by rows "
                                        "to T341" % (tkey[0], tkey[1], r["slots"], r["shape"]))
                     if default_workload else "not captured for this workload",
                     "dram_gbs": traffic / (solve_ms * 1e-3) / 1e9 if traffic else None,
                     "peak_source": peak_source, "algorithmic_per_launch": amount, "launch_ms": solve_ms},
        "state_steps_per_s": world * B * 1e3 / r["ms"],
        "stage_ms": r["stages"],
        "kernels": kernel_rooflines(r["precision"], r["stages"], r["slots"], sm_mhz, r["solve_arith"]),
        "e2e": {"value": world * 1e3 / r["ms_e2e"], "unit": "steps/s", "h2d_bytes_per_step": r["bytes"],
                "d2h_bytes_per_step": r["bytes"], "copies": "pinned host, own streams, overlapping compute",
                "result_matches_device_step": r["e2e_same"]},
        "gpu_launches": (7 if r["solve_arith"] == "fp32x2" else 6) * args.steps,
        "clocks": r["clocks"],
    }
    for name, _, _ in forms[1:]:
        f = results[name]
        line[name + "_form"] = {"value": world * 1e3 / f["ms"], "ms_per_step": f["ms"], "stage_ms": f["stages"],
                                "pole_slots": f["slots"], "layout_shape": f["shape"],
                                "kernels": kernel_rooflines(f["precision"], f["stages"], f["slots"], sm_mhz,
                                                            f["solve_arith"])}
    if "fp64" in results and chosen != "fp64":
        f = results["fp64"]
        line["error_vs_fp64_form"] = float((results[chosen]["y"] - f["y"]).norm() / f["y"].norm())
    if "mixed" in results and chosen == "mixed_fp32x2":
        f = results["mixed"]["y"]
        y = results[chosen]["y"]
        line["vs_mixed_fp64_solves"] = {"rel_l2": float((y - f).norm() / f.norm()),
                                        "bitwise_equal": bool(torch.equal(y, f))}
    if "fp64" in phi:
        line["phi_solver_form"] = phi["fp64"]
    if "mixed_fp32x2" in phi:
        line["phi_solver_chosen_form"] = phi["mixed_fp32x2"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
        try:
            line["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores()
        except Exception as exc:  # a host without process support still gets the 1-core number
            line["cpu_baseline"]["all_cores"] = {"unavailable": repr(exc)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
