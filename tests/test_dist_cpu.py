"""Multi-process host logic of bench.py on CPU: two ranks over gloo (127.0.0.1).

Each rank times its own replica of the workload; the bench takes the slowest rank's time
for every rank (all_reduce MAX after a barrier) and reports the units of all ranks over it
(weak scaling).  This test runs that path with world size 2 and CPU tensors: the ranks
report different times and must both end with the maximum and the same whole-job value.
"""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    rk = bench.Ranks(backend="gloo", device="cpu")
    rk.barrier()
    ms = 100.0 + 37.0 * rank          # this rank's own step time
    ms_max = rk.max(ms)
    value = rk.value(1_000_000, ms_max)
    rk.barrier()
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as fh:
        json.dump({"rank": rk.rank, "world": rk.world, "ms_max": ms_max, "value": value}, fh)
    rk.close()


def test_two_ranks_take_the_slowest_time(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, d in enumerate(res):
        assert d["rank"] == r and d["world"] == world
        assert d["ms_max"] == 137.0
        assert abs(d["value"] - world * 1_000_000 / 0.137) < 1e-6 * d["value"]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    rk = bench.Ranks(backend="gloo", device="cpu")
    assert rk.world == 1 and rk.max(3.5) == 3.5
    assert rk.value(10, 1000.0) == 10.0
    rk.barrier()
    rk.close()
