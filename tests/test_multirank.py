"""The multi-rank path of the benchmark on CPU (gloo, world size 2): ranks
solve disjoint instance blocks, and the whole-job throughput takes the
slowest rank's time and every rank's solves."""
import os
import socket
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    insts = bench.instances("tree15_32", rank, 3)
    local_ms = 100.0 * (rank + 1)          # rank 1 is the slower one
    max_ms, total, value = bench.job_throughput(local_ms, len(insts) * 2, world, "cpu", dist)
    seeds = torch.tensor([float(w["instance"]) for w in insts])
    gathered = [torch.zeros_like(seeds) for _ in range(world)]
    dist.all_gather(gathered, seeds)
    out[rank] = (max_ms, total, value, sorted(float(v) for g in gathered for v in g.tolist()))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        max_ms, total, value, seeds = res[r]
        assert max_ms == 200.0
        assert total == 12                      # 2 ranks x 3 instances x 2 steps
        assert abs(value - 12 / 0.2) < 1e-9
        assert seeds == [0.0, 1.0, 2.0, 3.0, 4.0, 5.0]   # disjoint blocks covering 0..5
