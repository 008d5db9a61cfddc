"""Host logic of bench.py that needs no GPU: the reference arm's line (the oracle timed
on a bounded sample, its extrapolation declared) and the workload configurations."""
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
