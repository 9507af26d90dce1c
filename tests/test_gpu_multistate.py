"""Many disjoint states, transients and batched whole runs (the loop of Fig. 1 for every run of a batch).

* Rotamer labels and exits of the GPU state check equal the oracle's on chains built from random
  torsions (both precisions keep the state in FP64 and test it in FP64).
* grp_batch_run gives every run exactly the event log and step counter of grp_run on that run alone,
  for runs in different phases at the same time (transients, convergence steps, parallel steps) and
  of different systems and sizes in one batch.
* On the FP64 path the first visit of each run equals the oracle's Gen. ParRep run of the alkane.
* The mixed-precision batched path's residence times in the all-trans state pass a two-sample KS
  test (p > 0.01) against brute-force dynamics of the FP64 oracle (the validation of Section 4.1).
"""
import multiprocessing as mp

import numpy as np
import pytest

from paper_1807_02431_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SEED = 2431


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_02431_gb300 import binding, build

    build.build()
    binding.load()
    return binding


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rotamer_labels_match_oracle(B, oracle_mod, prec):
    rng = np.random.default_rng(5)
    tors = rng.uniform(-180.0, 180.0, (96, 4))
    tors[:32] = rng.choice([60.0, 180.0, -60.0], (32, 4)) + rng.uniform(-40.0, 40.0, (32, 4))
    q = np.stack([W.alkane(torsions=t).q0 for t in tors])
    # random torsions can overlap beads: the nonbonded terms are switched off (the labels do not
    # depend on the forces, which grp_init_replicas evaluates and range-checks)
    import dataclasses

    s = dataclasses.replace(W.alkane(), epsilon=np.zeros(7))
    o = oracle_mod.Oracle(s)
    sysh = B.grp_create_system(s, B.GRP_FP64 if prec == "fp64" else B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, len(q), SEED, q, np.zeros_like(q), per_replica=True)
    import torch

    lo = [o.state_of(x) for x in q]
    for omega in (40, 13, 0, 80, -1):
        lab = torch.zeros(len(q), dtype=torch.int8, device="cuda")
        ex = torch.zeros(len(q), dtype=torch.uint8, device="cuda")
        B.grp_check_states(rep, omega, lab, ex)
        torch.cuda.synchronize()
        assert lab.cpu().tolist() == lo
        assert ex.cpu().tolist() == [o.exited(x, omega) for x in q]
    assert len(set(lo)) > 10 and -1 in lo


def _runs(B, prec, specs):
    reps = []
    for s, seed in specs:
        sysh = B.grp_create_system(s, prec)
        reps.append((sysh, B.grp_init_replicas(sysh, s.n_replicas, seed, s.q0, s.p0)))
    return reps


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_run_matches_single_runs(B, prec):
    P = B.GRP_FP64 if prec == "fp64" else B.GRP_MIXED
    specs = [(W.alkane(), SEED + i) for i in range(5)]
    specs.append((W.alkane(torsions=[100.0, 180.0, 180.0, 180.0]), SEED + 7))  # starts in the transient region
    specs.append((W.alkane(n_atoms=5, n_replicas=8), SEED + 8))               # 9 states, 8 replicas
    specs.append((W.chain(n_replicas=16), SEED + 9))                          # another system and size
    args = (10, 100, 0.05, 1000, 30000, 5)
    batch_reps = _runs(B, P, specs)
    b = B.grp_batch_create([r for _, r in batch_reps])
    evs, tsims = B.grp_batch_run(b, *args)
    ticks, graph_ticks = B.grp_batch_stats(b)
    assert ticks > 10 and graph_ticks == ticks - 1  # every tick after the first replayed as a CUDA graph
    kinds = set()
    for i, (s, seed) in enumerate(specs):
        sysh, rep = _runs(B, P, [(s, seed)])[0]
        ev, tsim = B.grp_run(rep, *args)
        assert evs[i] == ev, i
        assert tsims[i] == tsim
        assert B.grp_get_state(batch_reps[i][1])[3] == B.grp_get_state(rep)[3]
        kinds |= {e["kind"] for e in ev}
    assert {B.EV_TRANSIENT, B.EV_FV_CONVERGED, B.EV_PARALLEL_EXIT} <= kinds


def test_batch_run_fp64_matches_oracle(B, oracle_mod):
    """The first visit of each run (F-V convergence and parallel step, or a reference exit) exactly as
    in the oracle.  Later visits are compared by their statistics only: the FP64 path differs from the
    oracle by rounding (FMA contraction, the 2^-40 fixed-point force quantum), which the chain's
    dynamics amplifies until, some 10^4 steps on, a reference exit or a convergence test falls on the
    other side (measured: the third visit of one run)."""
    s = W.alkane()
    o = oracle_mod.Oracle(s)
    specs = [(s, seed) for seed in range(SEED + 20, SEED + 26)]
    reps = _runs(B, B.GRP_FP64, specs)
    b = B.grp_batch_create([r for _, r in reps])
    evs, _ = B.grp_batch_run(b, s.t_gr, s.t_check, s.tol, s.min_fv_steps, 30000, 1)
    kinds = set()
    for i, (_, seed) in enumerate(specs):
        evo, tgo = o.run_genparrep(s.n_replicas, seed, s.t_gr, s.t_check, s.tol, s.min_fv_steps, 30000, 1,
                                   q0=s.q0, p0=s.p0)
        assert evs[i] == evo
        assert B.grp_get_state(reps[i][1])[3]["t_global"] == tgo
        kinds |= {e["kind"] for e in evo}
    assert {B.EV_REF_EXIT, B.EV_FV_CONVERGED, B.EV_PARALLEL_EXIT} <= kinds


def _residences(ev, B, state=None):
    """Residence time per visit (t_FV + tau, or t_ref) after the first visit, optionally of one state."""
    out, fv = [], None
    for e in ev:
        if e["kind"] == B.EV_FV_CONVERGED:
            fv = e["steps"]
        elif e["kind"] == B.EV_PARALLEL_EXIT:
            out.append((e["omega"], fv + e["steps"]))
        elif e["kind"] == B.EV_REF_EXIT:
            out.append((e["omega"], e["steps"]))
    return [r for o, r in out[1:] if state is None or o == state]


def _brute(seed):
    import oracle

    s = W.alkane()
    res, frm = oracle.Oracle(s).run_bruteforce(seed, s.t_check, 4 * 10 ** 6, 100000)
    return list(zip(frm[1:].tolist(), res[1:].tolist()))


def test_mixed_batched_exit_times_match_brute_force(B):
    from scipy import stats

    s = W.alkane()
    reps = _runs(B, B.GRP_MIXED, [(s, 9000 + i) for i in range(64)])
    b = B.grp_batch_create([r for _, r in reps])
    evs, _ = B.grp_batch_run(b, s.t_gr, s.t_check, s.tol, s.min_fv_steps, 10 ** 9, 20)
    with mp.get_context("spawn").Pool(8) as pool:
        brute = [x for part in pool.map(_brute, [700 + w for w in range(8)]) for x in part]
    for state in (40, None):  # the all-trans state, and every state pooled
        gp = np.array([r for ev in evs for r in _residences(ev, B, state)], float)
        bf = np.array([r for o, r in brute if state is None or o == state], float)
        assert len(gp) >= 100 and len(bf) >= 500, (state, len(gp), len(bf))
        p = stats.ks_2samp(gp, bf).pvalue
        assert p > 0.01, (state, p, gp.mean(), bf.mean())
