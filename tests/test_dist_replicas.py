"""The multi-process (replicas) path of bench.py on CPU: two gloo ranks.  Each rank
reports its own timed-region length; the job's time is the maximum over ranks (the
replicas' regions end when the slowest one does), the job's rate counts every rank's
iterations, and only rank 0 runs and prints the reference arm."""
import argparse
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out_dir: str):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 * (rank + 1)                       # rank 1 is the slow replica
    dist.barrier()
    job_ms = bench.max_over_ranks(ms, dist)
    rate = bench.replica_rate(world, 10, job_ms / 1e3)
    ref = bench.run_reference(argparse.Namespace(steps=1, warmup=0, seed=1), rank, world) if rank != 0 else None
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(dict(job_ms=job_ms, rate=rate, ref_is_none=ref is None), f)
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_every_rank(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r in res:
        assert r["job_ms"] == 200.0                # the maximum over ranks, on every rank
        assert r["rate"] == pytest.approx(2 * 10 / 0.2)
    assert res[1]["ref_is_none"]                  # rank 1 does no reference work


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.replica_rate(1, 10, 2.0) == 5.0
