"""Whole-method pin of the oracle: Gen. ParRep exit-time statistics against brute-force dynamics.

The paper validates gen.parRep by comparing its exit-time distribution with a long serial Langevin
run (Section 4.1, Table 1 and the ccdf figures).  Here the same comparison on the 2-D double well:
residence times per visit (t_FV + tau after a converged F-V step, Eq. 5; t_ref after a reference
exit) against residence times of plain trajectories, two-sample KS test at p > 0.01.
"""
import multiprocessing as mp

import numpy as np
import pytest

from paper_1807_02431_gb300 import workloads as W

N_WORKERS = 8


def _parrep_worker(seed, max_exits):
    import oracle

    s = W.double_well_2d()
    o = oracle.Oracle(s)
    ev, _ = o.run_genparrep(s.n_replicas, seed, s.t_gr, s.t_check, s.tol, s.min_fv_steps,
                            10 ** 10, max_exits)
    res, fv = [], None
    for e in ev:
        if e["kind"] == oracle.EV_FV_CONVERGED:
            fv = e["steps"]
        elif e["kind"] == oracle.EV_PARALLEL_EXIT:
            res.append(fv + e["steps"])
            fv = None
        elif e["kind"] == oracle.EV_REF_EXIT:
            res.append(e["steps"])
    taus = [e["steps"] for e in ev if e["kind"] == oracle.EV_PARALLEL_EXIT]
    return res[1:], taus, ev


def _brute_worker(seed, n):
    import oracle

    s = W.double_well_2d()
    o = oracle.Oracle(s)
    res, _ = o.run_bruteforce(seed, s.t_check, 10 ** 11, n + 1)
    return list(res[1:])


@pytest.fixture(scope="module")
def samples(oracle_mod):
    ctx = mp.get_context("spawn")
    with ctx.Pool(N_WORKERS) as pool:
        pr = pool.starmap(_parrep_worker, [(1000 + w, 13) for w in range(N_WORKERS)])
        bf = pool.starmap(_brute_worker, [(5000 + w, 40) for w in range(N_WORKERS)])
    parrep = np.concatenate([np.array(r[0], float) for r in pr])
    taus = np.concatenate([np.array(r[1], float) for r in pr])
    brute = np.concatenate([np.array(r, float) for r in bf])
    events = [r[2] for r in pr]
    return parrep, taus, brute, events


def test_parrep_exit_times_match_brute_force(samples):
    """Two-sample KS, Gen. ParRep residence times vs brute force (Section 4.1 validation style)."""
    from scipy import stats

    parrep, _, brute, _ = samples
    assert len(parrep) >= 80 and len(brute) >= 250
    p = stats.ks_2samp(parrep, brute).pvalue
    assert p > 0.01, (p, parrep.mean(), brute.mean())
    # the means agree within their 95% intervals' combined width
    se = np.sqrt(parrep.var() / len(parrep) + brute.var() / len(brute))
    assert abs(parrep.mean() - brute.mean()) < 3 * se


def test_parallel_phase_exit_time_is_exponential(samples):
    """Starting from the QSD the exit time is exponential (Section 2.3, property 3): the parallel
    phase's tau has coefficient of variation ~ 1 and passes a KS test against Exp(mean)."""
    from scipy import stats

    _, taus, _, _ = samples
    cv = taus.std() / taus.mean()
    assert 0.75 < cv < 1.25, cv
    assert stats.kstest(taus / taus.mean(), "expon").pvalue > 0.01


def test_clock_is_the_sum_of_event_times(samples):
    """Clock updates (Section 2.4.1 and Eq. 6): t_sim after each event is the running sum of t_reach,
    t_ref, t_FV and tau; a reference exit is never followed by a parallel exit of the same visit."""
    import oracle

    _, _, _, events = samples
    for ev in events:
        t = 0
        for a, e in enumerate(ev):
            if e["kind"] != oracle.EV_FV_ALL_EXITED:
                t += e["steps"]
            assert e["t_sim"] == t
            if e["kind"] == oracle.EV_PARALLEL_EXIT:
                prev = [x for x in ev[:a] if x["kind"] != oracle.EV_FV_ALL_EXITED][-1]
                assert prev["kind"] == oracle.EV_FV_CONVERGED
                assert 1 <= e["k"] <= W.double_well_2d().n_replicas
                assert e["steps"] == (32 * (e["M"] - 1) + e["k"]) * 100
