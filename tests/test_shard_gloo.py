"""Pole sharding across ranks on the CPU (gloo, world size 2 and 3): each rank sums its
even share of the poles with the oracle (Sec. 6.4's split of the REXI terms), the bench's
reduction (bench.shard_allreduce) adds the partial steps, and every rank ends with the
full oracle step."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import bench
    from oracle import rexi_coeffs as rc
    from oracle import step as ostep
    from paper_1812_03431_gb300 import inputs
    from paper_1812_03431_gb300.rexi import pole_shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N, M, tau = 15, 16, 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    S = inputs.random_spectral(N, 2, 91)
    b, e = pole_shard(al.size, rank, world)
    y = torch.from_numpy(ostep.rexi_step_spectral(S, N, al[b:e], be[b:e], tau))
    bench.shard_allreduce(y, dist)
    full = ostep.rexi_step_spectral(S, N, al, be, tau)
    out[rank] = (float(np.linalg.norm(y.numpy() - full) / np.linalg.norm(full)), e - b)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_pole_shards_allreduce_to_the_full_step(world):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        errs = [out[r][0] for r in range(world)]
        sizes = [out[r][1] for r in range(world)]
    assert max(errs) < 1e-13
    assert sum(sizes) == 2 * (16 + 11) + 1 and max(sizes) - min(sizes) <= 1


def test_pole_shard_partitions_evenly():
    from paper_1812_03431_gb300.rexi import pole_shard
    for P in (25, 279, 535, 1047):
        for world in (1, 2, 3, 4, 8):
            parts = [pole_shard(P, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == P
            assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
            sizes = [e - b for b, e in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        pole_shard(3, 0, 4)
