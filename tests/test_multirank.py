"""Several ranks on CPU (gloo, world size 2): the benchmark's replica sharding
(weak scaling, disjoint replica indices per rank), its barrier and the
max-over-ranks of the timed region, which are the only cross-rank steps --
replicas never exchange data."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, R, out_path):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench.dist_env()
    base, count = bench.shard(R, r, w)
    bench.barrier(w)
    mx = bench.reduce_max(float(10 * rank + 3), w)
    with open(f"{out_path}.{rank}", "w") as f:
        f.write(f"{w} {r} {base} {count} {mx}\n")
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_ranks_shard_and_reduce(tmp_path):
    import torch.multiprocessing as mp
    world, R = 2, 128
    out = str(tmp_path / "rank")
    mp.start_processes(_worker, args=(world, _free_port(), R, out), nprocs=world,
                       start_method="spawn", join=True)
    rows = [open(f"{out}.{k}").read().split() for k in range(world)]
    ranges = []
    for k, (w, r, base, count, mx) in enumerate(rows):
        assert int(w) == world and int(r) == k
        assert int(count) == R                 # weak scaling: fixed work per rank
        assert float(mx) == 13.0               # max over ranks
        ranges.append(range(int(base), int(base) + int(count)))
    got = sorted(i for rg in ranges for i in rg)
    assert got == list(range(world * R))       # disjoint, together all replica indices


def test_single_rank_defaults(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.shard(64, 0, 1) == (0, 64)
    assert bench.reduce_max(2.5, 1) == 2.5
    bench.barrier(1)
