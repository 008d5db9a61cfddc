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
