"""One Gen. ParRep run sharded over two processes (paper_1807_02431_gb300/ranks.py, ShardedRun) on the
CPU with gloo: the event log of the loop of Fig. 1 equals the unsharded run's exactly.

Section 3.1 distributes a run's replicas over processes; the sharded loop exchanges exit flags, the
Fleming-Viot sources and rows, and the Gelman-Rubin sums of Eq. 3.  Here each process advances its shards
with the FP64 oracle (the CPU stand-in for a GPU; the GPU engine is tested in test_gpu_sharded.py), each
shard drawing the noise of its global replica indices, so the sharded run must reproduce
`run_genparrep` of the oracle on the whole replica set event for event: the transients, the F-V times,
the branch counts, M, k and tau of Eq. 5 and the clock of Eq. 6.  (The Gelman-Rubin sums are added in
another order than the unsharded oracle adds them; a convergence decision could only differ if a ratio
fell within rounding of 1 + TOL.)
"""
import json
import math
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_1807_02431_gb300 import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleShard:
    """Shard engine whose replicas the FP64 oracle advances (test infrastructure).  Observables are kept
    as sample histories and the Gelman-Rubin sums follow Eq. 3 literally, as the oracle's own loop does."""

    def __init__(self, o, s, first, n, seed):
        self.o, self.first, self.n, self.seed = o, first, n, seed
        self.no = len(s.observables)
        self.nd = s.n_atoms * s.dim
        self.q = np.repeat(np.asarray(s.q0, float).reshape(1, -1), n, 0)
        self.p = np.repeat(np.asarray(s.p0, float).reshape(1, -1), n, 0)
        f0 = o.forces(s.q0).reshape(-1)
        self.f = np.repeat(f0[None], n, 0)
        self.hist = np.zeros((n, self.no, 0))
        self.tg = self.tp = 0

    @property
    def row(self):
        return 3 * self.nd + self.no * self.hist.shape[2]

    def set_counters(self, t_global, t_phase):
        self.tg, self.tp = t_global, t_phase

    def advance(self, k, t_gr, n_active):
        q, p, f = self.q[:n_active], self.p[:n_active], self.f[:n_active]
        cap = k // t_gr + 1 if t_gr else 0
        smp = self.o.step_k_from(q, p, f, self.seed, self.first, self.tg, self.tp, k, t_gr, cap=cap)
        if t_gr and smp.shape[1]:
            assert n_active == self.n
            self.hist = np.concatenate([self.hist, np.transpose(smp, (0, 2, 1))], axis=2)
        self.tg += k
        self.tp += k

    def check(self, omega):
        lab = np.array([self.o.state_of(self.q[r]) for r in range(self.n)], np.int8)
        ex = np.array([self.o.exited(self.q[r], omega) for r in range(self.n)], np.uint8)
        return lab, ex

    def plan(self, exited_global):
        _, src = _oracle_mod().fv_branch(self.seed, self.tg, exited_global)
        return src[self.first: self.first + self.n]

    def pack(self, idx):
        return np.stack([np.concatenate([self.q[i], self.p[i], self.f[i], self.hist[i].ravel()]) for i in idx])

    def unpack(self, idx, rows):
        nd = self.nd
        for i, row in zip(idx, rows):
            self.q[i], self.p[i], self.f[i] = row[:nd], row[nd:2 * nd], row[2 * nd:3 * nd]
            self.hist[i] = row[3 * nd:].reshape(self.no, -1)

    def broadcast_local(self, src):
        for a in (self.q, self.p, self.f):
            a[:] = a[src]
        self.hist = np.zeros((self.n, self.no, 0))

    def _workers(self):
        return [i for i in range(self.n) if self.first + i >= 1]

    def gr1(self):
        out = np.zeros((self.no, 3))
        w = self._workers()
        if self.hist.shape[2] < 1:
            out[:, 2] = len(w)
        elif w:
            out[:, 0] = self.hist[w].mean(axis=2).sum(axis=0)
            out[:, 1] = len(w)
        return out

    def gr2(self, sums1):
        out = np.zeros((self.no, 2))
        w = self._workers()
        if self.hist.shape[2] < 1 or not w:
            return out
        h = self.hist[w]                                   # [workers, obs, samples]
        grand = (sums1[:, 0] / (sums1[:, 1] + sums1[:, 2]))[None, :, None]
        mk = h.mean(axis=2, keepdims=True)
        out[:, 0] = ((h - grand) ** 2).mean(axis=2).sum(axis=0)
        out[:, 1] = ((h - mk) ** 2).mean(axis=2).sum(axis=0)
        return out

    def gr_combine(self, sums1, sums2, tol):
        rhat = np.array([math.inf if (sums1[j, 2] > 0 or sums1[j, 1] < 1 or not sums2[j, 1] > 0)
                         else sums2[j, 0] / sums2[j, 1] for j in range(self.no)])
        return rhat, bool(np.all(rhat < 1.0 + tol))


def _oracle_mod():
    import oracle

    oracle.build()
    return oracle


RUN = dict(t_gr=10, t_check=100, tol=0.05, min_fv_steps=2000, max_steps=10 ** 8, max_exits=6)
SEED = 2431


def _worker(rank, world, port, counts, ranks_, out_dir):
    import torch.distributed as dist

    from paper_1807_02431_gb300 import ranks

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    s = W.double_well_2d()
    o = _oracle_mod().Oracle(s)
    layout = ranks.Layout(counts, ranks_)
    shards = {i: OracleShard(o, s, layout.first[i], layout.count[i], SEED) for i in layout.of_rank(rank)}
    run = ranks.ShardedRun(layout, shards, ranks.Comm())
    events, tsim = run.run(**RUN)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"events": events, "tsim": tsim, "t_global": run.t_global, "moved": run.rows_moved}, f)


def _reference():
    s = W.double_well_2d()
    o = _oracle_mod().Oracle(s)
    ev, tg = o.run_genparrep(s.n_replicas, SEED, RUN["t_gr"], RUN["t_check"], RUN["tol"], RUN["min_fv_steps"],
                             RUN["max_steps"], RUN["max_exits"], q0=s.q0, p0=s.p0)
    return ev, tg


def _run_sharded(tmp_path, counts, ranks_):
    world = max(ranks_) + 1
    mp.start_processes(_worker, args=(world, _free_port(), counts, ranks_, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    return [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]


def test_two_rank_run_equals_unsharded_oracle(tmp_path):
    """Two processes of 16 replicas each: the event log equals the oracle's whole run of 32 replicas."""
    ref, tg = _reference()
    kinds = {e["kind"] for e in ref}
    assert {0, 2, 3}.issubset(kinds) and len(ref) >= 10  # transients, converged F-V steps, parallel exits
    res = _run_sharded(tmp_path, [16, 16], [0, 1])
    assert sum(r["moved"]["between_processes"] for r in res) > 0  # branch copies crossed processes
    for r in res:
        assert r["events"] == ref
        assert r["tsim"] == ref[-1]["t_sim"]
        assert r["t_global"] == tg


def test_uneven_shards_two_per_process(tmp_path):
    """Three shards of 10, 7 and 15 replicas, the last two in the second process (a branch copy then
    crosses shards in one process as well as between processes): the same event log."""
    ref, _ = _reference()
    res = _run_sharded(tmp_path, [10, 7, 15], [0, 1, 1])
    for r in res:
        assert r["events"] == ref


def test_single_process_layout():
    """Without a process group the loop runs every shard in this process (four shards of 8)."""
    from paper_1807_02431_gb300 import ranks

    ref, tg = _reference()
    s = W.double_well_2d()
    o = _oracle_mod().Oracle(s)
    layout = ranks.Layout([8, 8, 8, 8], [0, 0, 0, 0])
    shards = {i: OracleShard(o, s, layout.first[i], 8, SEED) for i in range(4)}
    run = ranks.ShardedRun(layout, shards, ranks.Comm())
    events, tsim = run.run(**RUN)
    assert events == ref and run.t_global == tg
