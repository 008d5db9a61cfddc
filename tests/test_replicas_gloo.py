"""The bench's N > 1 path (independent replicas, max-over-ranks time) on CPU with gloo."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 40.0][rank]  # rank 1 is the slow replica
    out[rank] = bench.replica_max_ms(ms, dist)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_max_time():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == out[1] == 40.0
        # whole-job value: units of all ranks over the slowest rank's time
        assert 2 * 1e3 / out[0] == pytest.approx(50.0)


def test_kernel_rooflines_arithmetic():
    import bench
    st = {"fft_fwd": 0.2, "leg_ana": 0.15, "solve": 30.0, "reduce": 0.4, "leg_syn": 0.3, "fft_inv": 0.2}
    for form in ("mixed", "fp64"):
        k = bench.kernel_rooflines(form, st, 32, 2070.0)
        assert set(k) == set(st)
        for name, v in k.items():
            scale = 1e9 if v["unit"] == "GB/s" else 1e12
            assert abs(v["achieved"] - v["algorithmic"] / (v["ms"] * 1e-3) / scale) < 1e-9 * v["achieved"]
            assert abs(v["frac"] - v["achieved"] / v["peak"]) < 1e-12
        # the solve: 72 flops per (state, pole, row) at the derived FP64 rate
        W = bench.WORK
        P = 2 * (W["M"] + 11) + 1
        assert k["solve"]["algorithmic"] == 72 * W["batch"] * P * bench.rows_of(W["N"])
        assert abs(k["solve"]["peak"] - 152 * 4 * 2070e6 / 1e12) < 1e-12
    # the float-float solve: 36 multiply-adds of 12 FP32 operations at the derived FP32 rate;
    # its reduction is HBM-bound (every slot's partials read once, the result written)
    k = bench.kernel_rooflines("mixed", st, 32, 2070.0, "fp32x2")
    assert k["solve"]["algorithmic"] == 432 * W["batch"] * P * bench.rows_of(W["N"])
    assert abs(k["solve"]["peak"] - 152 * 128 * 2070e6 / 1e12) < 1e-12
    assert k["solve"]["unit"] == "Tops/s" and k["reduce"]["unit"] == "GB/s"
    ns = (W["N"] + 1) * (W["N"] + 2) // 2
    assert k["reduce"]["algorithmic"] == 34 * 3 * ns * W["batch"] * 16
    assert [f[0] for f in bench.FORMS] == ["mixed", "fp64", "ff_solve"]  # the chosen form first
    assert bench.rows_of(341) == 58652
