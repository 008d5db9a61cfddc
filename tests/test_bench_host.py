"""Host logic of bench.py that needs no GPU: the reference arm's line (the oracle timed
on a bounded sample, its extrapolation declared), the workload configurations, the
decoding of the tuned solve layout and the per-kernel roofline arithmetic."""
import json
import subprocess
import sys

from conftest import ROOT


def test_reference_arm_line_is_checkable():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "t63_c1", "--steps", "2",
                          "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    import bench
    bench.WORK.clear()
    bench.WORK.update(bench.WORKLOADS["t63_c1"])
    assert line["impl"] == "reference" and line["config"] == bench.workload_config()
    assert line["extrapolated"] is True and 0 < line["sample_fraction"] < 1
    # ms_per_step is what a timed (sampled) step took; value extrapolates by the fraction
    assert abs(line["value"] - line["sample_fraction"] * 1e3 / line["ms_per_step"]) < 1e-9 * line["value"]
    assert abs(line["ms_per_full_step_extrapolated"] - line["ms_per_step"] / line["sample_fraction"]) < 1e-6
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["steps"] == 2


def test_workload_configs_name_their_states():
    import bench
    for name, w in bench.WORKLOADS.items():
        bench.WORK.clear()
        bench.WORK.update(w)
        c = bench.workload_config()
        assert "T%d" % w["N"] in c["workload"] and c["global_batch"] == w["batch"]
        assert ("balanced" in c["workload"]) == (w.get("state") == "noisy_balanced")
        assert c["poles"] == 2 * (w["M"] + 11) + 1
        S = bench.make_states()
        assert S.shape == (w["batch"], 3, (w["N"] + 1) * (w["N"] + 2) // 2)


def test_solve_layout_and_kernel_rooflines():
    import bench
    # the fused solve's slot count packs tile + 256 x pole groups; shapes 2 to 4 are its forms
    assert bench.solve_layout({"slots": 2 + 256 * 2, "shape": 4}) == {
        "fused": "lean, two-warp CTAs", "tile": 2, "pole_groups": 2, "layout_shape": 4}
    assert bench.solve_layout({"slots": 8 + 256, "shape": 3})["fused"] == "lean"
    assert bench.solve_layout({"slots": 64, "shape": 0}) == {"pole_slots": 64, "layout_shape": 0}
    # the bench workload (T341, K = 256, 16 states): 36 FMAs per (state, pole, row)
    bench.WORK.clear()
    bench.WORK.update(bench.WORKLOADS["t341_b16"])
    flops = bench.FLOPS_PER_ROW * 16 * 535 * bench.rows_of(341)
    assert bench.rows_of(341) == 58652 and flops == 36148400640
    k = bench.kernel_rooflines("mixed", {"solve": 30.0, "fft_fwd": 0.128, "leg_syn": 0.184}, 0, 2070.0,
                               fp64_peak=1.25)
    assert k["solve"]["algorithmic"] == flops and k["solve"]["unit"] == "TFLOP/s"
    assert abs(k["solve"]["frac"] - flops / 30e-3 / 1e12 / 1.25) < 1e-12
    # the mixed FFT moves the FP64 grid and the FP32 Fourier array once each
    assert k["fft_fwd"]["algorithmic"] == 16 * 3 * 512 * 1024 * 8 + 512 * 342 * 48 * 8
    assert "reduce" not in k and "leg_ana" not in k  # stages without a time are left out
