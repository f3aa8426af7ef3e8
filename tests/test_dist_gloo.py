"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1).
Units shard round robin with no overlap and nothing left out, the job's
time is the max over ranks and its units the sum, as the benchmark reports
(value = units of all ranks / max time)."""
import json
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        mine = bench.shard(64, rank, ws)
        t = bench.max_over_ranks(1.5 + rank, dist, device="cpu")  # this rank's time: 1.5 s, 2.5 s
        n = bench.sum_over_ranks(len(mine), dist, device="cpu")
        everyone = [None] * ws
        dist.all_gather_object(everyone, mine)
        if rank == 0:
            with open(out, "w") as f:
                json.dump({"time": t, "units": n, "shards": everyone,
                           "value": n / t}, f)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_shard_and_reduce(tmp_path):
    out = str(tmp_path / "r.json")
    mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    r = json.load(open(out))
    a, b = r["shards"]
    assert not set(a) & set(b) and sorted(a + b) == list(range(64))
    assert abs(len(a) - len(b)) <= 1
    assert r["time"] == 2.5 and r["units"] == 64
    assert r["value"] == 64 / 2.5


def test_single_process_needs_no_group():
    import bench
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
    assert bench.max_over_ranks(3.0, None) == 3.0 and bench.sum_over_ranks(7, None) == 7.0
