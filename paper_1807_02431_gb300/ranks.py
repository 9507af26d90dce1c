"""Host logic for running the method on several GPUs, one process per GPU (torch.distributed).

Two modes:
  * independent replica sets per process (the benchmark's "replicas only" mode, weak scaling): each
    process runs its own set with its own noise key (`rank_seed`); only the benchmark's wall time is
    exchanged (`max_over_ranks`);
  * one run sharded over processes (`ShardedRun`): the run's replicas are cut into contiguous shards
    (`Layout`, `shard`), each process advances its shards on its GPU, and the small per-check data of
    the method are exchanged (see the comment above `Layout`).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def rank_seed(seed: int, rank: int) -> int:
    """Philox key of rank `rank` for independent replica sets (distinct noise streams per rank)."""
    return seed + 1000 * rank


def shard(n_total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous replica range (start, count) of `rank`; the first n_total % world ranks take one more."""
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def max_over_ranks(seconds: float, group=None, device=None) -> float:
    """Largest of the ranks' values (tensors on `device`: CUDA for NCCL, CPU for gloo)."""
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


# ----------------------------------------------------------------------------------------------------
# One Gen. ParRep run sharded over processes (Section 3.1: the replicas of a run are distributed over
# processes; Section 5: GPUs next).  The run's N replicas are cut into shards, contiguous ranges of global
# replica indices held by the processes (possibly several per process); the shard holding global replica
# 0 holds the reference walker.  Every shard draws the noise of its global indices, so the sharded run
# follows exactly the trajectory of one unsharded run of N replicas.  Per exit test the processes
# exchange, through torch.distributed:
#   * the exit flags and labels of every replica (an all-gather of N + N bytes);
#   * the Fleming-Viot sources of the exited workers (an all-gather of N int32), then the packed rows of
#     the copies whose survivor lives in another process (point-to-point), the rest copied locally;
#   * the Gelman-Rubin sums of Eq. 3, two all-reduces (SUM) of a few doubles per observable;
#   * in the parallel step, the first exit: the lowest (check, replica) among the gathered flags, and the
#     row of that replica sent to the reference walker's shard (Eq. 5).
# Each shard does its part through an engine with the methods of `LibraryShard` (its replica set on a
# GPU, the library's kernels); the arithmetic of the method stays in the engines.

class Layout:
    """Global layout of the shards: shard s holds global replicas [first[s], first[s] + count[s]) and
    lives in process rank[s].  Shards are contiguous and ordered by first index."""

    def __init__(self, counts, ranks_):
        assert len(counts) == len(ranks_) and all(c >= 1 for c in counts)
        self.count = [int(c) for c in counts]
        self.rank = [int(r) for r in ranks_]
        self.first = [0]
        for c in self.count[:-1]:
            self.first.append(self.first[-1] + c)
        self.N = self.first[-1] + self.count[-1]

    @staticmethod
    def by_rank(n_total: int, world: int, per_rank: int = 1) -> "Layout":
        """world * per_rank contiguous shards, process r holding shards r * per_rank ...  (shard sizes as
        `shard` gives them)."""
        parts = world * per_rank
        counts = [shard(n_total, parts, i)[1] for i in range(parts)]
        return Layout(counts, [i // per_rank for i in range(parts)])

    def shard_of(self, g: int) -> int:
        lo, hi = 0, len(self.first) - 1
        while lo < hi:
            mid = (lo + hi + 1) // 2
            if self.first[mid] <= g:
                lo = mid
            else:
                hi = mid - 1
        return lo

    def of_rank(self, rank: int):
        return [s for s in range(len(self.count)) if self.rank[s] == rank]


class Comm:
    """The exchanges of a sharded run over torch.distributed (gloo on host tensors, NCCL on `device`
    tensors), or within one process when no process group is initialised."""

    def __init__(self, group=None, device=None):
        self.group = group
        self.device = device
        self.dist = dist.is_available() and dist.is_initialized()
        self.rank = dist.get_rank(group) if self.dist else 0
        self.world = dist.get_world_size(group) if self.dist else 1

    def _t(self, a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(self.device if self.device is not None else "cpu")

    def allgather(self, local, size: int):
        """Every process's 1-D array (padded to `size` elements); returns the list over ranks."""
        if self.world == 1:
            return [local]
        buf = np.zeros(size, dtype=local.dtype)
        buf[: len(local)] = local
        t = self._t(buf)
        out = [torch.empty_like(t) for _ in range(self.world)]
        dist.all_gather(out, t, group=self.group)
        return [o.cpu().numpy() for o in out]

    def allreduce_sum(self, a):
        if self.world == 1:
            return a
        t = self._t(a)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t.cpu().numpy()

    def bcast(self, a, src: int):
        """`a` of process src to every process (the others pass an array of the same shape and type)."""
        if self.world == 1:
            return a
        t = self._t(a)
        dist.broadcast(t, src=src, group=self.group)
        return t.cpu().numpy()

    def exchange(self, sends: dict, recv_shapes: dict):
        """Point-to-point arrays: sends[rank] goes to that process; returns {rank: array} of the shapes
        recv_shapes[rank] (FP64).  Every receive is posted before the sends."""
        if not sends and not recv_shapes:
            return {}
        bufs = {r: torch.empty(shape, dtype=torch.float64, device=self.device or "cpu")
                for r, shape in recv_shapes.items()}
        reqs = [dist.irecv(bufs[r], src=r, group=self.group) for r in sorted(bufs)]
        keep = []
        for r in sorted(sends):
            t = self._t(sends[r])
            keep.append(t)
            reqs.append(dist.isend(t, dst=r, group=self.group))
        for q in reqs:
            q.wait()
        return {r: b.cpu().numpy() for r, b in bufs.items()}


class LibraryShard:
    """A shard on this process's GPU: a replica set of the library (grp_set_shard) and the library's
    shard calls.  Host arrays in and out; the kernels do the method's arithmetic."""

    def __init__(self, B, rep, first: int, n_global: int, stream=None):
        self.B, self.rep, self.first, self.n = B, rep, first, rep.R
        self.stream = stream
        B.grp_set_shard(rep, first, n_global)
        dev = "cuda"
        self.d_lab = torch.empty(self.n, dtype=torch.int8, device=dev)
        self.d_ex = torch.empty(self.n, dtype=torch.uint8, device=dev)
        self.d_src = torch.empty(self.n, dtype=torch.int32, device=dev)
        self.row = B.row_len(rep)

    def set_counters(self, t_global: int, t_phase: int):
        self.B.grp_set_state(self.rep, counters={"t_global": t_global, "t_phase": t_phase}, stream=self.stream)

    def advance(self, k: int, t_gr: int, n_active: int):
        self.B.grp_step_k(self.rep, k, t_gr, n_active, self.stream)

    def check(self, omega: int):
        self.B.grp_check_states(self.rep, omega, self.d_lab, self.d_ex, self.stream)
        torch.cuda.synchronize()
        return self.d_lab.cpu().numpy(), self.d_ex.cpu().numpy()

    def plan(self, exited_global):
        ex = torch.as_tensor(np.ascontiguousarray(exited_global, dtype=np.uint8), device="cuda")
        self.B.grp_fv_plan(self.rep, ex, self.d_src, self.stream)
        torch.cuda.synchronize()
        return self.d_src.cpu().numpy()

    def pack(self, idx):
        d_idx = torch.as_tensor(np.asarray(idx, dtype=np.int32), device="cuda")
        buf = torch.empty((len(idx), self.row), dtype=torch.float64, device="cuda")
        self.B.grp_pack_rows(self.rep, len(idx), d_idx, buf, self.stream)
        torch.cuda.synchronize()
        return buf.cpu().numpy()

    def unpack(self, idx, rows):
        d_idx = torch.as_tensor(np.asarray(idx, dtype=np.int32), device="cuda")
        buf = torch.as_tensor(np.ascontiguousarray(rows, dtype=np.float64), device="cuda")
        self.B.grp_unpack_rows(self.rep, len(idx), d_idx, buf, self.stream)
        torch.cuda.synchronize()

    def broadcast_local(self, src: int):
        self.B.grp_broadcast(self.rep, src, self.stream)

    def gr1(self):
        return self.B.grp_gr_partials(self.rep, 1, None, self.stream)

    def gr2(self, sums1):
        return self.B.grp_gr_partials(self.rep, 2, sums1, self.stream)

    def gr_combine(self, sums1, sums2, tol: float):
        return self.B.grp_gr_combine(sums1, sums2, tol)


EV_TRANSIENT, EV_REF_EXIT, EV_FV_CONVERGED, EV_PARALLEL_EXIT, EV_FV_ALL_EXITED = range(5)


class ShardedRun:
    """The loop of Fig. 1 (transient, convergence step with Fleming-Viot branching and the Gelman-Rubin
    test, parallel step with Eq. 5, the clock of Eq. 6) over the shards of `layout`; `shards` maps the
    index of each shard of this process to its engine.  Every process runs the same loop and logs the
    same events; the exchanges are those listed above."""

    def __init__(self, layout: Layout, shards: dict, comm: Comm):
        self.L, self.shards, self.comm = layout, shards, comm
        assert sorted(shards) == layout.of_rank(comm.rank)
        self.local = sorted(shards)
        self.n_local_max = max(sum(layout.count[s] for s in layout.of_rank(r)) for r in range(comm.world))
        self.t_global = 0
        self.rows_moved = {"within_process": 0, "between_processes": 0}

    # -- exchanges
    def _gather(self, per_shard, dtype):
        """Concatenation over all shards (global replica order) of per-shard 1-D arrays."""
        mine = np.concatenate([np.asarray(per_shard[s], dtype=dtype) for s in self.local])
        parts = self.comm.allgather(mine, self.n_local_max)
        out = np.empty(self.L.N, dtype=dtype)
        for r in range(self.comm.world):
            pos = 0
            for s in self.L.of_rank(r):
                out[self.L.first[s]: self.L.first[s] + self.L.count[s]] = parts[r][pos: pos + self.L.count[s]]
                pos += self.L.count[s]
        return out

    def _flags(self, omega):
        lab, ex = {}, {}
        for s in self.local:
            lab[s], ex[s] = self.shards[s].check(omega)
        return self._gather(lab, np.int8).astype(np.int64), self._gather(ex, np.uint8)

    def _advance(self, k, t_gr, t_phase, only_ref=False):
        for s in self.local:
            if only_ref and self.L.first[s] != 0:
                continue
            sh = self.shards[s]
            sh.set_counters(self.t_global, t_phase)
            sh.advance(k, t_gr, 1 if only_ref else sh.n)

    def _move_rows(self, pairs):
        """Copy rows src -> dst for the (dst, src) pairs of global indices (sources never destinations):
        local pairs within this process, the others packed per destination process in ascending
        destination order."""
        L, me = self.L, self.comm.rank
        sends, recv_shapes, incoming = {}, {}, {}
        by_src = {}
        for d, s in sorted(pairs):
            by_src.setdefault((L.shard_of(s), L.shard_of(d)), []).append((d, s))
        out_rows = {}
        for (ss, ds), lst in sorted(by_src.items()):
            if L.rank[ss] == me:
                rows = self.shards[ss].pack([s - L.first[ss] for _, s in lst])
                if L.rank[ds] == me:
                    self.shards[ds].unpack([d - L.first[ds] for d, _ in lst], rows)
                    self.rows_moved["within_process"] += len(lst)
                else:
                    self.rows_moved["between_processes"] += len(lst)
                    out_rows.setdefault(L.rank[ds], []).append(rows)
            elif L.rank[ds] == me:
                incoming.setdefault(L.rank[ss], []).append((ds, lst))
        row = next(iter(self.shards.values())).row
        for r, parts in out_rows.items():
            sends[r] = np.concatenate(parts)
        for r, groups in incoming.items():
            recv_shapes[r] = (sum(len(lst) for _, lst in groups), row)
        got = self.comm.exchange(sends, recv_shapes)
        for r, groups in incoming.items():
            pos = 0
            for ds, lst in groups:
                self.shards[ds].unpack([d - L.first[ds] for d, _ in lst], got[r][pos: pos + len(lst)])
                pos += len(lst)

    def _ref_owner(self):
        return self.L.shard_of(0)

    def _ref_label(self):
        s0 = self._ref_owner()
        lab = np.zeros(1, np.int64)
        if s0 in self.shards:
            lab[0] = int(self.shards[s0].check(0)[0][0])
        return int(self.comm.bcast(lab, self.L.rank[s0])[0])

    def _broadcast_ref(self):
        """Every replica of every shard takes the reference walker's state; accumulators cleared."""
        s0 = self._ref_owner()
        row = np.zeros((1, next(iter(self.shards.values())).row))
        if s0 in self.shards:
            row = self.shards[s0].pack([0])
        row = self.comm.bcast(row, self.L.rank[s0])
        for s in self.local:
            if s != s0:
                self.shards[s].unpack([0], row)
            self.shards[s].broadcast_local(0)

    def _gelman_rubin(self, tol):
        sh = [self.shards[s] for s in self.local]
        s1 = self.comm.allreduce_sum(np.sum([x.gr1() for x in sh], axis=0))
        s2 = self.comm.allreduce_sum(np.sum([x.gr2(s1) for x in sh], axis=0))
        return sh[0].gr_combine(s1, s2, tol)

    # -- the loop of Fig. 1
    def run(self, t_gr, t_check, tol, min_fv_steps, max_steps, max_exits, max_events=100000):
        N = self.L.N
        events, tsim, nexit = [], 0, 0

        def log(kind, omega, to, k, M, steps, nb):
            events.append({"kind": kind, "omega": int(omega), "label_to": int(to), "k": int(k), "M": int(M),
                           "steps": int(steps), "t_sim": int(tsim), "n_branch": int(nb)})

        while nexit < max_exits and self.t_global < max_steps and len(events) < max_events:
            # 1. transient propagation of the reference walker
            omega, treach = self._ref_label(), 0
            while omega < 0 and self.t_global < max_steps:
                self._advance(t_check, 0, treach, only_ref=True)
                self.t_global += t_check
                treach += t_check
                omega = self._ref_label()
            if omega < 0:
                break
            if treach > 0:
                tsim += treach
                log(EV_TRANSIENT, -1, omega, 0, 0, treach, 0)
            # 2. convergence step
            self._broadcast_ref()
            t_phase, nbranch, converged, ref_exit = 0, 0, False, False
            while self.t_global < max_steps:
                self._advance(t_check, t_gr, t_phase)
                self.t_global += t_check
                t_phase += t_check
                lab, ex = self._flags(omega)
                if ex[0]:  # (a) the reference walker left omega
                    tsim += t_phase
                    log(EV_REF_EXIT, omega, lab[0], 0, 0, t_phase, nbranch)
                    nexit += 1
                    ref_exit = True
                    break
                ex[0] = 0  # (b) Fleming-Viot branching of the exited workers
                nb = int(ex.sum())
                if nb > 0:
                    if nb == N - 1:
                        log(EV_FV_ALL_EXITED, omega, omega, 0, 0, t_phase, nb)
                    src = self._gather({s: self.shards[s].plan(ex) for s in self.local}, np.int32)
                    self._move_rows([(d, int(src[d])) for d in range(N) if src[d] >= 0])
                nbranch += nb
                if t_phase >= min_fv_steps and N > 1:  # (c) Gelman-Rubin test, Eq. 4
                    _, conv = self._gelman_rubin(tol)
                    if conv:
                        converged = True
                        break
            if ref_exit:
                continue
            if not converged:
                break
            tsim += t_phase
            log(EV_FV_CONVERGED, omega, omega, 0, 0, t_phase, nbranch)
            # 3. parallel dynamics step, Eqs. 5-6
            M, found = 0, False
            while self.t_global < max_steps:
                self._advance(t_check, 0, t_phase)
                self.t_global += t_check
                t_phase += t_check
                M += 1
                lab, ex = self._flags(omega)
                hit = np.nonzero(ex)[0]
                if len(hit):
                    k0 = int(hit[0])
                    tau = (N * (M - 1) + k0 + 1) * t_check
                    tsim += tau
                    log(EV_PARALLEL_EXIT, omega, lab[k0], k0 + 1, M, tau, 0)
                    if k0 != 0:
                        self._move_rows([(0, k0)])
                    found = True
                    break
            if not found:
                break
            nexit += 1
        return events, tsim
