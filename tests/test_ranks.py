"""Multi-rank host logic (paper_1807_02431_gb300/ranks.py) on two gloo processes on the CPU: replica
sharding, the global first exit of Eq. 5 (lowest check, then lowest global replica index), the
Gelman-Rubin ratio of Eq. 3 from per-rank sums (against the oracle's ratio on the whole sample set) and
the max-over-ranks time of the benchmark."""
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
    # first exit: rank 0 sees replica 5 at check 3, rank 1 replica 1 at check 3 (global 11): k = 6
    start, _ = ranks.shard(20, world, rank)
    local = [(3 << 32) | 5, (3 << 32) | 1][rank]
    res["exit_same_check"] = ranks.first_exit(local, start)
    # rank 1 exits one check earlier: its replica wins
    local = [(3 << 32) | 0, (2 << 32) | 4][rank]
    res["exit_earlier"] = ranks.first_exit(local, start)
    res["exit_none"] = ranks.first_exit(ranks.NO_EXIT, start)
    # Gelman-Rubin from per-rank sums
    s0, c0 = ranks.shard(samples.shape[0], world, rank)
    mine = samples[s0:s0 + c0]
    means = mine.mean(axis=1)
    variances = (mine * mine).mean(axis=1) - means * means
    res["rhat"] = float(ranks.gelman_rubin_global(means[:, None], variances[:, None])[0])
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
        assert tuple(r["exit_same_check"]) == (3, 6)
        assert tuple(r["exit_earlier"]) == (2, 10 + 4 + 1)
        assert r["exit_none"] is None
        assert r["tmax"] == 2.0
    ref = oracle_mod.gelman_rubin(samples)
    for r in res:
        assert abs(r["rhat"] - ref) < 1e-12 * ref
