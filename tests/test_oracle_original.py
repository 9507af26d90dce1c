"""Pins of the oracle's original ParRep loop (Section 2.4.3: decorrelation, dephasing, parallel step).

(a) With one replica the method degenerates into plain dynamics as long as the dephasing restarts
nothing: the walker's trajectory is then the brute-force run's on the same random stream, and each
visit's counted time plus its uncounted dephasing time equals the brute-force residence time, step for
step; the global step counter is the clock plus the dephasing time.
(b) With 32 replicas the residence-time distribution matches brute force (two-sample KS, the
validation style of Section 4.1), and the event log follows the clock rules of Section 2.4.3.
"""
import multiprocessing as mp

import numpy as np
import pytest

from paper_1807_02431_gb300 import workloads as W

N_WORKERS = 8
T_CORR = 2000
T_PHASE = 2000


def _visits(ev, oracle, with_dephasing=False):
    """Residence time per visit: t_ref after a reference exit, t_corr + tau after a parallel exit (plus
    the dephasing steps when asked)."""
    res, frm, dec = [], [], None
    for e in ev:
        if e["kind"] == oracle.EV_DECORRELATED:
            dec = e["steps"]
        elif e["kind"] == oracle.EV_DEPHASED and with_dephasing:
            dec += e["steps"]
        elif e["kind"] == oracle.EV_PARALLEL_EXIT:
            res.append(dec + e["steps"])
            frm.append(e["omega"])
            dec = None
        elif e["kind"] == oracle.EV_REF_EXIT:
            res.append(e["steps"])
            frm.append(e["omega"])
    return res, frm


@pytest.mark.parametrize("seed", [11, 12])
def test_single_replica_reduces_to_brute_force(oracle_mod, seed):
    o = oracle_mod.Oracle(W.double_well_2d())
    s = o.system
    # one check of dephasing right after t_corr in the state: an exit there (a restart) is rare
    ev, tg = o.run_original(1, seed, s.t_check, T_CORR, 0, 10 ** 9, 6)
    deph = [e for e in ev if e["kind"] == oracle_mod.EV_DEPHASED]
    assert deph and all(e["n_branch"] == 0 and e["steps"] == s.t_check for e in deph)
    res, frm = _visits(ev, oracle_mod, with_dephasing=True)
    assert len(res) == 6
    bres, bfrm = o.run_bruteforce(seed, s.t_check, 10 ** 9, 6)
    assert list(bres) == res and list(bfrm) == frm
    assert tg == ev[-1]["t_sim"] + sum(e["steps"] for e in deph)
    # the parallel step of one replica: k = 1, tau = M t_check (Eq. 5 with N = 1)
    for e in ev:
        if e["kind"] == oracle_mod.EV_PARALLEL_EXIT:
            assert e["k"] == 1 and e["steps"] == e["M"] * s.t_check


def _original_worker(seed, max_exits):
    import oracle

    s = W.double_well_2d()
    o = oracle.Oracle(s)
    ev, tg = o.run_original(s.n_replicas, seed, s.t_check, T_CORR, T_PHASE, 10 ** 10, max_exits)
    res, _ = _visits(ev, oracle)
    return res[1:], ev, tg


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
        orig = pool.starmap(_original_worker, [(3000 + w, 13) for w in range(N_WORKERS)])
        bf = pool.starmap(_brute_worker, [(7000 + w, 40) for w in range(N_WORKERS)])
    original = np.concatenate([np.array(r[0], float) for r in orig])
    brute = np.concatenate([np.array(r, float) for r in bf])
    return original, brute, [(r[1], r[2]) for r in orig]


def test_original_exit_times_match_brute_force(samples):
    from scipy import stats

    original, brute, _ = samples
    assert len(original) >= 80 and len(brute) >= 250
    p = stats.ks_2samp(original, brute).pvalue
    assert p > 0.01, (p, original.mean(), brute.mean())
    se = np.sqrt(original.var() / len(original) + brute.var() / len(brute))
    assert abs(original.mean() - brute.mean()) < 3 * se


def test_original_event_log_follows_the_clock_rules(samples, oracle_mod):
    """t_sim advances by t_reach, t_ref, t_corr and tau, never by the dephasing time; each parallel exit
    follows a dephasing that follows a decorrelation of t_corr in the same state; the walltime spent
    (t_global) exceeds the simulated time only by the dephasing and the (N-1)-fold parallel work."""
    ev_kinds = oracle_mod
    n = W.double_well_2d().n_replicas
    t_check = W.double_well_2d().t_check
    for ev, tg in samples[2]:
        t, extra = 0, 0
        for a, e in enumerate(ev):
            if e["kind"] == ev_kinds.EV_DEPHASED:
                extra += e["steps"]
                assert e["steps"] >= T_PHASE
            else:
                t += e["steps"]
            assert e["t_sim"] == t
            if e["kind"] == ev_kinds.EV_DECORRELATED:
                assert e["steps"] == T_CORR and e["omega"] == e["label_to"]
            if e["kind"] == ev_kinds.EV_PARALLEL_EXIT:
                assert ev[a - 1]["kind"] == ev_kinds.EV_DEPHASED
                assert ev[a - 2]["kind"] == ev_kinds.EV_DECORRELATED
                assert ev[a - 2]["omega"] == e["omega"] != e["label_to"]
                assert 1 <= e["k"] <= n
                assert e["steps"] == (n * (e["M"] - 1) + e["k"]) * t_check
                extra += e["M"] * t_check - e["steps"]
            if e["kind"] == ev_kinds.EV_REF_EXIT:
                assert 0 < e["steps"] <= T_CORR
        # the global counter: the clock, plus dephasing, minus the parallel steps' N-fold credit
        assert tg == t + extra
