"""Benchmark of the Gen. ParRep hot path on one GB300 (or N ranks, one GPU each, replicas only).

Workload: the 22-bead peptide-like chain (alanine-dipeptide stand-in, Section 4.1 shape), 256
replicas, mixed precision, t_check = 500 steps, t_GR = 10 steps.  One benchmark step is one pass of
the convergence-step loop body over the whole replica set: a 500-step BAOAB segment with force-field
evaluation, observable sampling every 10 steps and the fused exit test, the Fleming-Viot branching of
exited workers, the Gelman-Rubin reduction, and the host readback of the per-check status — i.e. one
exit test of the method (Section 2.4.1).  Metric: replica-atom-steps/s (whole job).

Also reported: the same step on the plain FP64 GPU path, accelerated simulation speed (ns/day of
simulated clock, Tables 2 and 4) from a bounded run of the whole loop, the oracle on the host cores,
the roofline of the dominant kernel and the SM clocks seen during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1807_02431_gb300 import workloads as W  # noqa: E402

WORKLOAD = "chain22_r256"
# DRAM bytes (read + write) of one launch of the chain's segment kernel in this workload, from an ncu
# capture of the current kernel (511,744 read, 0 written: the replicas' state is read once and stays on
# chip); to be re-measured whenever the kernel changes.
SEGMENT_DRAM_BYTES = 511744  # ncu dram__bytes_read + write of one chain launch (profiles/)
SEED = 2431


def algorithmic_flops_per_replica_step(s: W.System) -> float:
    """FP32 flops per replica-step of the force kernel: 40 per non-excluded pair (with a cutoff: per
    non-excluded pair within the cutoff in the initial configuration), 15 per bond, 40 per angle and
    100 per three-term dihedral (33 per term), FMA counted as 2."""
    n = s.n_atoms
    if s.cutoff > 0:
        d = np.linalg.norm(s.q0[:, None] - s.q0[None], axis=-1)
        within = np.triu(d < s.cutoff, 1)
        within[s.excl[:, 0], s.excl[:, 1]] = False
        within[s.excl[:, 1], s.excl[:, 0]] = False
        n_pairs = int(within.sum())
    else:
        excl = {tuple(sorted(x)) for x in s.excl.tolist()}
        n_pairs = n * (n - 1) // 2 - len(excl)
    return 40.0 * n_pairs + 15.0 * len(s.bonds) + 40.0 * len(s.angles) + 33.3 * len(s.dihedral_k)


def pme_flops_per_replica_step(s: W.System) -> float:
    """FP32 flops per replica-step of the periodic force kernel (particle mesh Ewald): 46 per
    non-excluded pair within the cutoff over minimum images in the initial configuration (the pair
    count of `algorithmic_flops_per_replica_step` plus 6 for the image; erfc and exp counted as one
    each), 20 per excluded pair, the bonded terms as there; on the mesh of G points, a real-data 3-D
    transform forward and back at 2.5 G log2 G each (half the complex transform's 5 G log2 G: the
    grid is real), 2 G for the influence function, 188 per atom for spreading (3 B-spline evaluations
    of 20 and 64 multiply-adds) and 512 per atom for the gather (64 points x 8)."""
    n, box = s.n_atoms, np.asarray(s.box)
    d = s.q0[:, None] - s.q0[None]
    d -= box * np.round(d / box)
    within = np.triu(np.linalg.norm(d, axis=-1) < s.cutoff, 1)
    within[s.excl[:, 0], s.excl[:, 1]] = False
    within[s.excl[:, 1], s.excl[:, 0]] = False
    G = int(np.prod(s.pme_grid))
    mesh = 5.0 * G * np.log2(G) + 2.0 * G + n * (188.0 + 512.0)
    bonded = 15.0 * len(s.bonds) + 40.0 * len(s.angles) + 33.3 * len(s.dihedral_k)
    return 46.0 * int(within.sum()) + 20.0 * len(s.excl) + bonded + mesh


def fp32_peak_tflops(sm_mhz: float) -> float:
    """152 SMs x 128 FP32 lanes x 2 flops (FMA) x SM clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


# ----------------------------------------------------------------------------- CPU oracle
def _oracle_worker(args):
    r0, r1, steps, seed = args
    import oracle

    s = W.chain()
    o = oracle.Oracle(s)
    q, p = W.replica_states(s, r1 - r0, seed=seed + r0, spread=0.002)
    f = np.stack([o.forces(q[i]) for i in range(r1 - r0)])
    t = time.time()
    o.step_k(q, p, f, SEED, 0, 0, steps, s.t_gr, cap=steps // s.t_gr)
    ex = np.array([o.exited(q[i], 1) for i in range(r1 - r0)], np.uint8)
    return time.time() - t, int(ex.sum())


def cpu_oracle(n_replicas: int, steps: int, cores: int, repeats: int = 1):
    """The FP64 oracle on the host cores: the replicas of the sample split over `cores` spawned
    processes (each single-threaded), `repeats` times with one pool.  Returns a list of
    (replica-atom-steps/s, wall time) per repeat."""
    s = W.chain()
    chunks = np.array_split(np.arange(n_replicas), cores)
    tasks = [(int(c[0]), int(c[-1]) + 1, steps, 7) for c in chunks if len(c)]
    ctx = mp.get_context("spawn")
    out = []
    with ctx.Pool(len(tasks)) as pool:
        pool.map(_oracle_worker, [(0, 1, 1, 7)] * len(tasks))  # start-up and build outside the clock
        for _ in range(repeats):
            t = time.time()
            pool.map(_oracle_worker, tasks)
            wall = time.time() - t
            out.append((n_replicas * steps * s.n_atoms / wall, wall))
    return out


# ----------------------------------------------------------------------------- GPU step
class Step:
    """One convergence-step check of the method over the whole replica set (see module doc)."""

    def __init__(self, B, s: W.System, precision: int, R: int, seed: int, device_index: int, omega: int = 1):
        import torch

        self.B, self.s, self.R, self.omega = B, s, R, omega
        self.sysh = B.grp_create_system(s, precision)
        q0, p0 = W.replica_states(s, R, seed=seed, spread=0.002)
        self.q0, self.p0 = q0, p0
        self.stream = torch.cuda.current_stream()
        self.rep = B.grp_init_replicas(self.sysh, R, seed, q0, p0, per_replica=True, stream=self.stream)
        self.launches_per_step = 4  # segment, branching, Gelman-Rubin, status
        self.status = B.FvStatus()

    def __call__(self):
        s = self.s
        # omega: the state the system starts in (the chain: 1, outside the paper's rectangle; the
        # ligand: 0, bound); min_fv_steps = 0 so that every check also evaluates the Gelman-Rubin ratios
        return self.B.grp_fv_check(self.rep, self.omega, s.t_check, s.t_gr, s.tol, 0, self.stream, self.status)

    def reset(self):
        self.B.grp_set_state(self.rep, self.q0, self.p0, np.zeros((self.R, len(self.s.observables), 4)),
                             {"t_global": 0, "t_phase": 0}, self.stream)


def time_steps(step, K, W_, flush, events_stream):
    import torch

    for _ in range(W_):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for i in range(K):
        flush.zero_()  # write 256 MB > L2 between timed iterations (outside the events)
        ev[i][0].record(events_stream)
        step()
        ev[i][1].record(events_stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def segment_kernel_ms(B, step, n):
    """Average duration of the segment kernel alone (CUDA events on the launching stream)."""
    import torch

    s = step.s
    st = step.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    B.grp_step_k(step.rep, s.t_check, s.t_gr, 0, st)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(n):
        B.grp_step_k(step.rep, s.t_check, s.t_gr, 0, st)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def e2e_steps(B, step, K):
    """The same step through the public API with host buffers: H2D of the replica state (positions and
    momenta) from pinned host memory, the step, D2H of the positions into pinned memory and of the
    Gelman-Rubin ratios (read by the step's status), every step."""
    import torch

    s, R = step.s, step.R
    nd = R * s.n_atoms * s.dim
    hq = torch.from_numpy(step.q0.copy()).pin_memory()
    hp = torch.from_numpy(step.p0.copy()).pin_memory()
    hout = torch.empty(nd, dtype=torch.float64).pin_memory()
    ctr = {"t_global": 0, "t_phase": 0}
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(K):
        B.grp_set_state(step.rep, hq.numpy(), hp.numpy(), None, ctr, step.stream)
        step()
        B.grp_get_state(step.rep, step.stream, q=hout.numpy().reshape(R, s.n_atoms, s.dim), copy=("q",))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t
    return wall, 2 * nd * 8, nd * 8 + 8 * len(s.observables)


def accelerated_speed(B, s, precision, R, seed, max_steps, max_exits=10 ** 6, unit_ns=True, original=False):
    """Simulated clock per wall time of the whole loop (Fig. 1): t_sim advances by t_reach, t_ref,
    t_FV and tau (Eq. 6); speed = t_sim / wall as in Tables 2 and 4.  original=True runs the original
    ParRep loop (Section 2.4.3) with t_corr = t_phase = the minimum F-V time instead."""
    import torch

    sysh = B.grp_create_system(s, precision)
    rep = B.grp_init_replicas(sysh, R, seed, s.q0, s.p0)
    torch.cuda.synchronize()
    t = time.perf_counter()
    if original:
        ev, tsim = B.grp_run_original(rep, s.t_check, s.min_fv_steps, s.min_fv_steps, max_steps, max_exits)
    else:
        ev, tsim = B.grp_run(rep, s.t_gr, s.t_check, s.tol, s.min_fv_steps, max_steps, max_exits)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t
    ctr = B.grp_get_state(rep)[3]
    sim = tsim * s.dt * (1e-3 if unit_ns else 1.0)
    kinds = ((("transient", 0), ("decorrelated", 5), ("dephased", 6), ("ref_exit", 1), ("parallel_exit", 3))
             if original else (("transient", 0), ("fv_converged", 2), ("ref_exit", 1), ("parallel_exit", 3)))
    out = {"t_sim": sim, "wall_s": wall, "global_steps": ctr["t_global"],
           "events": {k: sum(1 for e in ev if e["kind"] == v) for k, v in kinds}}
    if original:
        out["loop"] = "original ParRep, t_corr = t_phase = %d steps" % s.min_fv_steps
    out["ns_per_day" if unit_ns else "time_units_per_day"] = sim / (wall / 86400.0)
    return out


def same_error_bench(B, max_steps, n_runs=64):
    """The metric's comparison at the same error: the state-to-state loop on the alkane (81 rotamer
    states) run on both precision paths with the same seeds.  Mixed and FP64 trajectories decorrelate
    (chaos), so "same error" is judged on the output of the method, the distribution of residence times
    per visit: a two-sample Kolmogorov-Smirnov test of mixed against FP64, beside the accelerated time
    per wall time of each path."""
    from scipy import stats

    from paper_1807_02431_gb300 import analysis

    out = {}
    res = {}
    for prec, name in ((B.GRP_MIXED, "mixed"), (B.GRP_FP64, "fp64")):
        r = multistate_bench(B, max_steps, n_runs, precision=prec, keep_visits=True)
        res[name] = r.pop("_residences")
        out[name] = {"ns_per_day": r["ns_per_day"], "wall_s": r["wall_s"], "visits": r["visits"],
                     "mean_residence_ps": float(np.mean(res[name]))}
    out["ks_pvalue_mixed_vs_fp64"] = float(stats.ks_2samp(res["mixed"], res["fp64"]).pvalue)
    out["speedup_mixed_over_fp64_ns_per_day"] = out["mixed"]["ns_per_day"] / out["fp64"]["ns_per_day"]
    out["workload"] = f"alkane7, {n_runs} runs x 32 replicas, {max_steps} steps per run, both paths"
    return out


def multistate_bench(B, max_steps, n_runs=64, precision=None, keep_visits=False):
    """The state-to-state loop at scale: n_runs independent Gen. ParRep runs of the 7-bead alkane
    (81 rotamer states, transients between them), 32 replicas each, mixed precision, all advanced by
    grp_batch_run until each run's step counter reaches max_steps.  Reports the summed simulated time
    per wall time (Tables 2 and 4's speed, over all runs), the visits and the exit statistics of the
    most visited states (mean with its 95 % chi-square interval, Section 4)."""
    import torch

    from paper_1807_02431_gb300 import analysis

    s = W.alkane()
    reps = []
    for i in range(n_runs):
        sysh = B.grp_create_system(s, B.GRP_MIXED if precision is None else precision)
        reps.append((sysh, B.grp_init_replicas(sysh, s.n_replicas, 9000 + i, s.q0, s.p0)))
    b = B.grp_batch_create([r for _, r in reps])
    torch.cuda.synchronize()
    t = time.perf_counter()
    evs, tsims = B.grp_batch_run(b, s.t_gr, s.t_check, s.tol, s.min_fv_steps, max_steps, 10 ** 6)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t
    sim_ns = sum(tsims) * s.dt * 1e-3
    rep = analysis.state_report(evs, dt=s.dt)
    top = sorted(rep, key=lambda k: -rep[k]["n"])[:3]
    vis = [v for ev in evs for v in analysis.visits(ev)]
    out = {"system": f"alkane7 (81 rotamer states), {n_runs} runs x {s.n_replicas} replicas, "
                     f"{'FP64' if precision == B.GRP_FP64 else 'mixed'}, "
                     f"t_check {s.t_check}, TOL {s.tol}, {max_steps} steps per run",
            "wall_s": wall, "t_sim_ns": sim_ns, "ns_per_day": sim_ns / (wall / 86400.0),
            "visits": len(vis), "parallel_exits": sum(1 for v in vis if v[3]),
            "states_visited": len({v[0] for v in vis}),
            "top_states_ps": {str(k): {"n": rep[k]["n"], "mean": rep[k]["mean"], "ci95": list(rep[k]["ci"])}
                              for k in top}}
    if keep_visits:
        out["_residences"] = [v[1] * s.dt for v in vis]
    return out


def batched_bench(B, steps, warmup, flush, n_runs=64, R=128):
    """64 independent runs of chains with sizes drawn uniformly in 22..400 beads, 128 replicas each,
    mixed precision, one persistent kernel per exit test (autotuned block size)."""
    import torch

    systems = W.batched_chains(n_runs=n_runs, n_replicas=R)
    handles, reps = [], []
    for k, s in enumerate(systems):
        sysh = B.grp_create_system(s, B.GRP_MIXED)
        q0, p0 = W.replica_states(s, R, seed=3000 + k, spread=0.002)
        handles.append(sysh)
        reps.append(B.grp_init_replicas(sysh, R, SEED + k, q0, p0, per_replica=True))
    b = B.grp_batch_create(reps)
    threads = B.grp_batch_autotune(b, 10)
    st = torch.cuda.current_stream()
    t_check = systems[0].t_check
    omegas = [1] * n_runs

    def step():
        B.grp_batch_fv_check(b, omegas, t_check, 10, 0.01, 0, st)

    times = time_steps(step, steps, warmup, flush, st)
    t = float(np.sum(times)) / 1e3
    atoms = sum(s.n_atoms for s in systems)
    flops = sum(algorithmic_flops_per_replica_step(s) for s in systems) * R * t_check
    return {"workload": f"{n_runs} runs x {R} replicas, chains of 22..400 beads (mean {atoms / n_runs:.0f})",
            "value": R * atoms * t_check * steps / t, "unit": "replica-atom-steps/s", "ms_per_step": t * 1e3 / steps,
            "block_threads": threads, "fp32_tflops_achieved": flops * steps / t / 1e12,
            "fp32_frac_of_peak": flops * steps / t / 1e12 / fp32_peak_tflops(2070.0)}


def ligand_bench(B, steps, warmup, flush, fp64_steps):
    """Ligand bound in a surface pocket of a 2,000-bead globule (2,030 atoms, elastic network, LJ and
    Coulomb truncated at 1.2 nm), 1,024 replicas, one exit test of the convergence step per step
    (500 BAOAB steps sampling every 50, branching, Gelman-Rubin), mixed and FP64 paths."""
    s = W.ligand_receptor()
    R = s.n_replicas
    step = Step(B, s, B.GRP_MIXED, R, SEED, 0, omega=0)
    times = time_steps(step, steps, warmup, flush, step.stream)
    t = float(np.sum(times)) / 1e3
    units = R * s.n_atoms * s.t_check
    seg_ms = segment_kernel_ms(B, step, 2)
    flops = algorithmic_flops_per_replica_step(s) * R * s.t_check
    peak = fp32_peak_tflops(2070.0)
    out = {"workload": f"ligand_receptor{s.n_atoms}_r{R}", "value": units * steps / t, "unit": "replica-atom-steps/s",
           "ms_per_step": t * 1e3 / steps,
           "roofline": {"bound": "alu", "achieved": flops / (seg_ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                        "frac": flops / (seg_ms * 1e-3) / 1e12 / peak, "kernel_ms": seg_ms,
                        "flops_per_launch": flops}}
    # the same system with reaction-field electrostatics (eps_rf = 78.3) instead of eps = 4r
    import dataclasses

    srf = dataclasses.replace(s, coulomb_mode=W.COULOMB_REACTION_FIELD, rf_dielectric=78.3)
    srf.q0, srf.p0 = s.q0, s.p0
    step_rf = Step(B, srf, B.GRP_MIXED, R, SEED, 0, omega=0)
    t_rf = time_steps(step_rf, max(1, steps // 2), 1, flush, step_rf.stream)
    out["reaction_field"] = {"value": units * len(t_rf) / (float(np.sum(t_rf)) / 1e3),
                             "ms_per_step": float(np.mean(t_rf))}
    # the same system in OBC II implicit solvent with the 1.2 nm cutoff applied to the solvent sums too
    # (the paper's protein-ligand setup: OBC II, non-periodic cutoff)
    sgb = W.solvated(s)
    step_gb = Step(B, sgb, B.GRP_MIXED, R, SEED, 0, omega=0)
    t_gb = time_steps(step_gb, max(1, steps // 2), 1, flush, step_gb.stream)
    out["solvent_obc2"] = {"value": units * len(t_gb) / (float(np.sum(t_gb)) / 1e3),
                           "ms_per_step": float(np.mean(t_gb)),
                           "solvent_pairs": "Verlet-list pairs and excluded pairs within 1.2 nm, 5 passes per step"}
    # the paper's protein-ligand setup in full: OBC II solvent and constrained hydrogens on the ligand
    sh = W.solvated(W.ligand_receptor_h(n_replicas=R))
    step_h = Step(B, sh, B.GRP_MIXED, R, SEED, 0, omega=0)
    t_h = time_steps(step_h, max(1, steps // 2), 1, flush, step_h.stream)
    out["solvent_obc2_constrained_h"] = {
        "workload": f"{sh.name}_r{R} ({sh.n_atoms} atoms, {len(sh.constraints)} constrained hydrogen bonds, OBC II)",
        "value": R * sh.n_atoms * sh.t_check * len(t_h) / (float(np.sum(t_h)) / 1e3),
        "ms_per_step": float(np.mean(t_h))}
    if fp64_steps > 0:
        step64 = Step(B, s, B.GRP_FP64, R, SEED, 0, omega=0)
        t64 = time_steps(step64, fp64_steps, 1, flush, step64.stream)
        v64 = units * len(t64) / (float(np.sum(t64)) / 1e3)
        out["fp64_path"] = {"value": v64, "ms_per_step": float(np.mean(t64)), "speedup_of_mixed": out["value"] / v64}
    return out


def branch_bytes(s, n_branched):
    """Algorithmic HBM bytes of one branching: each branched worker reads and writes q, p, F (3 n dim
    doubles) and its observable accumulators (4 n_obs doubles)."""
    return n_branched * 2 * 8 * (3 * s.n_atoms * s.dim + 4 * len(s.observables))


def branch_bench(B, flush, reps=10):
    """Fleming-Viot branching bandwidth (Section 2.4.1, task 2) on the ligand system: 1,024 replicas of
    2,030 atoms (q, p, F of all replicas: 150 MB, more than the 129 MB L2); every odd worker exited, so
    511 workers each copy q, p, F and accumulators from a survivor.  Kernel time by CUDA events around
    the asynchronous calls: K launches each after an L2 flush, minus K flushes alone, so that the GPU
    never waits for the host between the events), against the measured HBM copy bandwidth."""
    import torch

    s = W.ligand_receptor()
    R = s.n_replicas
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, R, SEED, s.q0, s.p0)
    ex = torch.zeros(R, dtype=torch.uint8, device="cuda")
    ex[1::2] = 1
    src = torch.empty(R, dtype=torch.int32, device="cuda")
    nb = B.grp_fv_branch(rep, ex, src)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(with_branch):
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            flush.zero_()
            if with_branch:
                B.grp_fv_branch(rep, ex, src, count=False)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    timed(True)
    both = [timed(True) for _ in range(3)]
    alone = [timed(False) for _ in range(3)]
    ms = (float(np.median(both)) - float(np.median(alone))) / reps
    peak = measured_hbm_gbs()
    gbs = branch_bytes(s, nb) / (ms * 1e-3) / 1e9
    return {"workload": f"ligand_receptor{s.n_atoms}_r{R}, {nb} workers branched", "kernel_ms": ms,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "bytes_per_launch": branch_bytes(s, nb), "peak_basis": "measured HBM copy (MEASURED_PEAKS.json)"}}


def measured_hbm_gbs():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0  # the profiling recipe's fallback


def gradient_bench(B, reps, precision=None):
    """Differentiation through the dynamics (the gradient workload): 256 replicas of the 22-bead chain,
    one 1,000-step fixed-noise segment with the end-to-end distance sampled every 10 steps, forward
    pass + checkpoints every 100 steps + adjoint sweep (grp_adjoint_segment), FP64 or mixed (FP32
    forces and FP32 dual-number tangents in fixed point, FP64 adjoint vectors)."""
    import torch

    s = W.chain_gradient()
    R, k, t_gr, ck = s.n_replicas, 1000, 10, 100
    q0, p0 = W.replica_states(s, R, seed=24, spread=0.002)
    sysh = B.grp_create_system(s, B.GRP_FP64 if precision is None else precision)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    gth = torch.empty(B.grp_param_count(sysh), dtype=torch.float64, device="cuda")
    B.grp_adjoint_segment(rep, k, t_gr, ck, 4, d_grad_theta=gth)  # warm-up
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(reps):
        B.grp_adjoint_segment(rep, k, t_gr, ck, 4, d_grad_theta=gth)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t) / reps
    t = time.perf_counter()
    B.grp_step_k(rep, k, 0)
    torch.cuda.synchronize()
    fwd = time.perf_counter() - t
    return {"workload": f"chain{s.n_atoms}_gradient_r{R}_k{k}", "ms_per_segment": wall * 1e3,
            "forward_ms": fwd * 1e3, "adjoint_over_forward": wall / fwd,
            "value": R * s.n_atoms * k / wall, "unit": "replica-atom-steps/s (forward + adjoint)"}


def profile_case(B, case, replicas, steps, launches):
    """A small fixed case for ncu captures: `launches` launches of the case's main kernel."""
    import torch

    if case in ("chain", "pme", "pme_list", "constrained", "solvated"):
        s = {"chain": W.chain, "pme": W.chain_ions, "constrained": W.chain_h,
             "pme_list": lambda: W.chain_ions(n_chain=100, n_pairs=60, edge=4.0),
             "solvated": lambda: W.solvated(W.chain())}[case]()
        st = Step(B, s, B.GRP_MIXED, replicas, SEED, 0)
        for _ in range(launches):
            B.grp_step_k(st.rep, steps, s.t_gr, 0, st.stream)
    elif case == "batch":
        systems = W.batched_chains(n_runs=16, n_replicas=replicas)
        keep = []
        for k, s in enumerate(systems):
            sysh = B.grp_create_system(s, B.GRP_MIXED)
            q0, p0 = W.replica_states(s, replicas, seed=3000 + k, spread=0.002)
            keep.append((sysh, B.grp_init_replicas(sysh, replicas, SEED + k, q0, p0, per_replica=True)))
        b = B.grp_batch_create([r for _, r in keep])
        for _ in range(launches):
            B.grp_batch_step_k(b, steps, 10)
        torch.cuda.synchronize()
        del b
    elif case in ("ligand", "ligand_gb"):
        s = W.ligand_receptor() if case == "ligand" else W.solvated(W.ligand_receptor())
        st = Step(B, s, B.GRP_MIXED, replicas, SEED, 0, omega=0)
        for _ in range(launches):
            B.grp_step_k(st.rep, steps, s.t_gr, 0, st.stream)
    elif case == "branch":  # every odd worker exited; `replicas` ligand replicas
        s = W.ligand_receptor()
        sysh = B.grp_create_system(s, B.GRP_MIXED)
        rep = B.grp_init_replicas(sysh, replicas, SEED, s.q0, s.p0)
        ex = torch.zeros(replicas, dtype=torch.uint8, device="cuda")
        ex[1::2] = 1
        for _ in range(launches):
            B.grp_fv_branch(rep, ex)
    else:
        s = W.chain_gradient()
        q0, p0 = W.replica_states(s, replicas, seed=24, spread=0.002)
        sysh = B.grp_create_system(s, B.GRP_FP64)
        rep = B.grp_init_replicas(sysh, replicas, SEED, q0, p0, per_replica=True)
        for _ in range(launches):
            B.grp_adjoint_segment(rep, steps, 10, 100, 4)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": case, "replicas": replicas, "steps": steps, "launches": launches}))


def arm_config(s: W.System, R: int, world: int) -> dict:
    """The `config` of the benchmark line (both arms)."""
    return {"workload": WORKLOAD, "n_atoms": s.n_atoms, "n_replicas": R, "t_check": s.t_check, "t_gr": s.t_gr,
            "precision": "mixed (FP32 forces, int64 fixed point, double-single integration)",
            "parallelism": f"replicas-only x{world}",
            "l2": "flushed between timed steps (256 MB write outside the events)"}


def run_reference(args):
    """The oracle (FP64 C, as it stands) on the host cores, same workload and metric; each step is a
    bounded sample, the same as the GPU arm's cpu_baseline leg: the 256 replicas advanced ten t_check
    segments (5,000 steps) with sampling and the exit test."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    s = W.chain()
    R, steps = s.n_replicas, 10 * s.t_check
    vals = cpu_oracle(R, steps, cores, args.warmup + args.steps)[args.warmup:]
    value = float(np.mean([v for v, _ in vals]))
    ms = float(np.mean([w for _, w in vals])) * 1e3
    line = {"metric": "replica-atom-steps/s", "value": value, "unit": "replica-atom-steps/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": arm_config(s, R, args.gpus),
            "cpu_baseline": {"value": value, "unit": "replica-atom-steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{R} replicas x {steps} BAOAB steps (ten t_check segments, sampling every "
                                       f"{s.t_gr}) + exit test, split over {cores} spawned processes"},
            "e2e": {"value": value, "unit": "replica-atom-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="grp", choices=["grp", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--accel-steps", type=int, default=200000)
    ap.add_argument("--accel-ligand-steps", type=int, default=10000)
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--ligand-steps", type=int, default=3)
    ap.add_argument("--gradient-reps", type=int, default=2)
    ap.add_argument("--multistate-steps", type=int, default=40000)
    ap.add_argument("--branch-reps", type=int, default=20)
    ap.add_argument("--same-error-steps", type=int, default=40000)
    ap.add_argument("--profile-case", choices=["chain", "pme", "pme_list", "constrained", "solvated", "ligand", "ligand_gb", "adjoint", "batch",
                                                     "branch"],
                    default=None,
                    help="run a small case of one kernel for ncu captures and exit (no benchmark line)")
    ap.add_argument("--profile-replicas", type=int, default=152)
    ap.add_argument("--profile-steps", type=int, default=100)
    ap.add_argument("--profile-launches", type=int, default=3)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        import torch

        from paper_1807_02431_gb300 import binding as B
        from paper_1807_02431_gb300 import build as build_mod

        build_mod.build()
        B.load()
        return profile_case(B, args.profile_case, args.profile_replicas, args.profile_steps, args.profile_launches)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1807_02431_gb300 import binding as B
    from paper_1807_02431_gb300 import build as build_mod
    from paper_1807_02431_gb300 import ranks

    if rank == 0 or not os.path.exists(build_mod.LIB):
        build_mod.build()
    if world > 1:
        torch.distributed.barrier()
    B.load()
    s = W.chain()
    R = s.n_replicas
    seed = ranks.rank_seed(SEED, rank)
    step = Step(B, s, B.GRP_MIXED, R, seed, local)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        times = time_steps(step, args.steps, args.warmup, flush, step.stream)
    if world > 1:
        torch.distributed.barrier()
    t_total = float(np.sum(times)) / 1e3
    units_per_step = R * s.n_atoms * s.t_check
    if world > 1:
        t_total = ranks.max_over_ranks(t_total, device="cuda")
    value = world * units_per_step * args.steps / t_total
    clocks = clk.summary()
    out = None
    if rank == 0:
        # dominant kernel: the fused segment kernel, timed alone on its stream
        seg_ms = segment_kernel_ms(B, step, 10)
        flops = algorithmic_flops_per_replica_step(s) * R * s.t_check
        sm_mhz = clocks.get("sm_mhz") or 2070.0
        peak = fp32_peak_tflops(2070.0)
        achieved = flops / (seg_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": SEGMENT_DRAM_BYTES, "traffic_unit": "bytes per launch (ncu dram read + write)", "kernel": "ff_segment_kernel<PathMixed, 320, 2, kModeItems, 0>",
                "peak_basis": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz (max SM clock)",
                "kernel_ms": seg_ms, "flops_per_launch": flops, "median_sm_mhz": sm_mhz}
        # plain FP64 GPU path, same step
        fp64 = None
        if args.fp64_steps > 0:
            step64 = Step(B, s, B.GRP_FP64, R, seed, local)
            t64 = time_steps(step64, args.fp64_steps, 1, flush, step64.stream)
            fp64_value = units_per_step * len(t64) / (float(np.sum(t64)) / 1e3)
            fp64 = {"value": fp64_value, "unit": "replica-atom-steps/s", "ms_per_step": float(np.mean(t64)),
                    "speedup_of_mixed": value / world / fp64_value}
        # the same chain in Generalized Born implicit solvent (OBC II), mixed
        solvated = None
        if args.fp64_steps > 0:
            sg = W.solvated(s)
            step_gb = Step(B, sg, B.GRP_MIXED, R, seed, local)
            tg = time_steps(step_gb, args.fp64_steps, 1, flush, step_gb.stream)
            solvated = {"workload": f"{sg.name}_r{R} (OBC II, all {sg.n_atoms * (sg.n_atoms - 1) // 2} pairs)",
                        "value": units_per_step * len(tg) / (float(np.sum(tg)) / 1e3),
                        "unit": "replica-atom-steps/s", "ms_per_step": float(np.mean(tg))}
        # the chain with one constrained hydrogen per bead (SHAKE / RATTLE), mixed
        constrained = None
        if args.fp64_steps > 0:
            sh = W.chain_h(n_replicas=R)
            step_h = Step(B, sh, B.GRP_MIXED, R, seed, local)
            th = time_steps(step_h, args.fp64_steps, 1, flush, step_h.stream)
            constrained = {"workload": f"{sh.name}_r{R} ({sh.n_atoms} atoms, {len(sh.constraints)} constraints)",
                           "value": R * sh.n_atoms * sh.t_check * len(th) / (float(np.sum(th)) / 1e3),
                           "unit": "replica-atom-steps/s", "ms_per_step": float(np.mean(th))}
        # the chain with 20 ion pairs in a periodic box, particle mesh Ewald, mixed
        periodic = None
        if args.fp64_steps > 0:
            sp = W.chain_ions(n_replicas=R)
            step_p = Step(B, sp, B.GRP_MIXED, R, seed, local)
            tp = time_steps(step_p, args.fp64_steps, 1, flush, step_p.stream)
            pk_ms = segment_kernel_ms(B, step_p, 3)
            pflops = pme_flops_per_replica_step(sp) * R * sp.t_check
            pach = pflops / (pk_ms * 1e-3) / 1e12
            periodic = {"workload": f"{sp.name}_r{R} ({sp.n_atoms} atoms, box {sp.box[0]} nm, grid "
                                    f"{'x'.join(str(k) for k in sp.pme_grid)}, order {sp.pme_order}, cutoff {sp.cutoff} nm)",
                        "value": R * sp.n_atoms * sp.t_check * len(tp) / (float(np.sum(tp)) / 1e3),
                        "unit": "replica-atom-steps/s", "ms_per_step": float(np.mean(tp)),
                        "roofline": {"bound": "alu", "achieved": pach, "peak": peak, "unit": "TFLOP/s",
                                     "frac": pach / peak, "kernel": "ff_segment_kernel<PathMixed, 320, 2, kModeItems, 4>",
                                     "kernel_ms": pk_ms, "flops_per_launch": pflops}}
            # a larger periodic system on the Verlet-list path: the 100-bead chain with 60 ion pairs, 4.0 nm box
            sl = W.chain_ions(n_chain=100, n_pairs=60, edge=4.0, n_replicas=R)
            step_l = Step(B, sl, B.GRP_MIXED, R, seed, local)
            tl = time_steps(step_l, args.fp64_steps, 1, flush, step_l.stream)
            lk_ms = segment_kernel_ms(B, step_l, 2)
            lflops = pme_flops_per_replica_step(sl) * R * sl.t_check
            lach = lflops / (lk_ms * 1e-3) / 1e12
            periodic["verlet_list"] = {
                "workload": f"{sl.name}_r{R} ({sl.n_atoms} atoms, box {sl.box[0]} nm, grid "
                            f"{'x'.join(str(k) for k in sl.pme_grid)}, cutoff {sl.cutoff} nm, Verlet lists over nearest images)",
                "value": R * sl.n_atoms * sl.t_check * len(tl) / (float(np.sum(tl)) / 1e3),
                "unit": "replica-atom-steps/s", "ms_per_step": float(np.mean(tl)),
                "roofline": {"bound": "alu", "achieved": lach, "peak": peak, "unit": "TFLOP/s", "frac": lach / peak,
                             "kernel": "ff_segment_kernel<PathMixed, 512, 1, kModeList, 4>", "kernel_ms": lk_ms,
                             "flops_per_launch": lflops}}
        # end to end through the public API with host buffers
        step.reset()
        e2e_wall, bi, bo = e2e_steps(B, step, args.steps)
        e2e_value = units_per_step * args.steps / e2e_wall
        batched = batched_bench(B, args.batch_steps, 2, flush) if args.batch_steps > 0 else None
        ligand = (ligand_bench(B, args.ligand_steps, 1, flush, min(args.fp64_steps, 1))
                  if args.ligand_steps > 0 else None)
        gradient = gradient_bench(B, args.gradient_reps) if args.gradient_reps > 0 else None
        if gradient is not None:
            gm = gradient_bench(B, args.gradient_reps, precision=B.GRP_MIXED)
            gradient["mixed_path"] = {k: gm[k] for k in ("ms_per_segment", "forward_ms", "adjoint_over_forward", "value")}
            gradient["mixed_path"]["speedup_over_fp64"] = gradient["ms_per_segment"] / gm["ms_per_segment"]
        accel = None
        if args.accel_steps > 0:
            # the chain (bounded run) and the double-well validation system, where the loop cycles
            accel = {"chain22": accelerated_speed(B, s, B.GRP_MIXED, R, seed, args.accel_steps)}
            dw = W.double_well_2d()
            accel["double_well_2d"] = accelerated_speed(B, dw, B.GRP_FP64, dw.n_replicas, SEED, 10 ** 8,
                                                        max_exits=8, unit_ns=False)
            accel["double_well_2d_original"] = accelerated_speed(B, dw, B.GRP_FP64, dw.n_replicas, SEED, 10 ** 8,
                                                                 max_exits=8, unit_ns=False, original=True)
            if args.accel_ligand_steps > 0:
                # the ligand-receptor system (bounded run): its bound state is left within tens of ps, before
                # the Fleming-Viot step converges, so the loop cycles through reference exits
                lg = W.ligand_receptor()
                accel["ligand_receptor2030"] = accelerated_speed(B, lg, B.GRP_MIXED, lg.n_replicas, seed,
                                                                 args.accel_ligand_steps)
        multistate = multistate_bench(B, args.multistate_steps) if args.multistate_steps > 0 else None
        same_error = same_error_bench(B, args.same_error_steps) if args.same_error_steps > 0 else None
        branching = branch_bench(B, flush, args.branch_reps) if args.branch_reps > 0 else None
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cores = os.cpu_count() or 1
            cv, cwall = cpu_oracle(R, 10 * s.t_check, cores)[0]
            cpu = {"value": cv, "unit": "replica-atom-steps/s", "cores": cores, "kind": "oracle",
                   "sample": f"{R} replicas x {10 * s.t_check} BAOAB steps (ten t_check segments, sampling every "
                             f"{s.t_gr}) + exit test, split over {cores} spawned processes; wall {cwall:.2f} s "
                             f"({cwall * cores:.0f} core-seconds)"}
        out = {"metric": "replica-atom-steps/s", "value": value, "unit": "replica-atom-steps/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_total * 1e3 / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": arm_config(s, R, world),
               "gpu_launches": step.launches_per_step * args.steps,
               "roofline": roof, "clocks": clocks,
               "fp64_path": fp64,
               "solvated_chain": solvated,
               "constrained_chain": constrained,
               "periodic_pme": periodic,
               "batched": batched,
               "ligand_receptor": ligand,
               "gradient": gradient,
               "accelerated": accel,
               "multistate": multistate,
               "same_error": same_error,
               "branching": branching,
               "e2e": {"value": e2e_value, "unit": "replica-atom-steps/s", "h2d_bytes_per_step": bi,
                       "d2h_bytes_per_step": bo},
               "cpu_baseline": cpu}
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
