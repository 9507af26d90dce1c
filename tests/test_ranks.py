"""Multi-rank host logic (paper_1807_02431_gb300/ranks.py) on two gloo processes on the CPU: replica
sharding, the shard layout and the max-over-ranks time of the benchmark.  (The sharded run itself is
tested in test_sharded_run.py.)"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, samples, out_dir):
    import json

    import numpy as np
    import torch.distributed as dist

    from paper_1807_02431_gb300 import ranks

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    res = {}
    # sharding
    res["shards"] = [ranks.shard(n, world, rank) for n in (1, 7, 256, 1025)]
    res["tmax"] = ranks.max_over_ranks([0.5, 2.0][rank])
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump(res, f)


def test_two_rank_host_logic(tmp_path, oracle_mod):
    import json

    rng = np.random.default_rng(4)
    samples = rng.standard_normal((9, 40)) + np.linspace(0, 0.5, 9)[:, None]
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), samples, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    # shards are disjoint, contiguous and cover [0, n)
    for i, n in enumerate((1, 7, 256, 1025)):
        got = sorted(tuple(r["shards"][i]) for r in res)
        assert got[0][0] == 0 and got[0][0] + got[0][1] == got[1][0] and got[1][0] + got[1][1] == n
    for r in res:
        assert r["tmax"] == 2.0


def test_layout():
    """Shards of a run: contiguous, ordered, covering [0, N); shard_of finds the shard of every index."""
    from paper_1807_02431_gb300 import ranks

    L = ranks.Layout([10, 7, 15], [0, 1, 1])
    assert L.first == [0, 10, 17] and L.N == 32
    assert [L.shard_of(g) for g in (0, 9, 10, 16, 17, 31)] == [0, 0, 1, 1, 2, 2]
    assert L.of_rank(1) == [1, 2]
    L2 = ranks.Layout.by_rank(1025, 2, per_rank=2)
    assert L2.N == 1025 and L2.rank == [0, 0, 1, 1] and sum(L2.count) == 1025
    assert all(L2.shard_of(L2.first[s]) == s for s in range(4))
