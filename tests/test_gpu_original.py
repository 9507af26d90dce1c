"""Original ParRep (Section 2.4.3) on the GPU against the FP64 oracle, through the C ABI.

On the double well the FP64 path and the oracle draw the same Philox numbers and round alike, so the
whole event log (transients, decorrelation, dephasing steps and restarts, M, k, tau, labels, clock)
and the global step counter must be identical.
"""
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


def _both(B, oracle_mod, n_rep, t_corr, t_phase, max_steps, max_exits, seed=SEED):
    s = W.double_well_2d()
    o = oracle_mod.Oracle(s)
    evo, tgo = o.run_original(n_rep, seed, s.t_check, t_corr, t_phase, max_steps, max_exits, q0=s.q0, p0=s.p0)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, n_rep, seed, s.q0, s.p0)
    ev, tsim = B.grp_run_original(rep, s.t_check, t_corr, t_phase, max_steps, max_exits)
    return ev, tsim, B.grp_get_state(rep)[3]["t_global"], evo, tgo


def test_original_loop_double_well_bit_exact(B, oracle_mod):
    ev, tsim, tg, evo, tgo = _both(B, oracle_mod, 32, 2000, 2000, 10 ** 8, 6)
    assert ev == evo
    assert tsim == evo[-1]["t_sim"] and tg == tgo
    kinds = {e["kind"] for e in ev}
    assert {B.EV_DECORRELATED, B.EV_DEPHASED, B.EV_PARALLEL_EXIT} <= kinds
    # the restart branch of the dephasing kernel ran
    assert sum(e["n_branch"] for e in ev if e["kind"] == B.EV_DEPHASED) > 0


@pytest.mark.parametrize("t_corr,t_phase,seed,kind", [(0, 0, SEED, None), (100, 5000, SEED + 5100, "restart"),
                                                       (10000, 100, SEED + 10000, "ref_exit")])
def test_original_degenerate_times_bit_exact(B, oracle_mod, t_corr, t_phase, seed, kind):
    """t_corr = 0 (no decorrelation) with t_phase = 0 (one check of dephasing); long dephasing with
    restarts; long decorrelation with reference exits."""
    ev, tsim, tg, evo, tgo = _both(B, oracle_mod, 16, t_corr, t_phase, 10 ** 8, 6 if kind else 4, seed=seed)
    assert ev == evo and tg == tgo
    if kind == "restart":
        assert sum(e["n_branch"] for e in ev if e["kind"] == B.EV_DEPHASED) > 0
    if kind == "ref_exit":
        assert any(e["kind"] == B.EV_REF_EXIT for e in ev)


def test_original_stops_at_max_steps(B, oracle_mod):
    """A step bound that falls inside a dephasing or a parallel step ends the run where the oracle's
    does, with the same events and step counter."""
    for max_steps in (2500, 4100, 9000):
        ev, tsim, tg, evo, tgo = _both(B, oracle_mod, 8, 2000, 2000, max_steps, 50)
        assert ev == evo and tg == tgo


def test_original_single_replica_is_brute_force(B, oracle_mod):
    """N = 1 with one check of dephasing and no restart: the walker follows the brute-force trajectory,
    so counted time plus dephasing time per visit equals the oracle's brute-force residence times."""
    s = W.double_well_2d()
    o = oracle_mod.Oracle(s)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, 1, SEED, s.q0, s.p0)
    ev, tsim = B.grp_run_original(rep, s.t_check, 2000, 0, 10 ** 9, 4)
    res, dec = [], None
    for e in ev:
        if e["kind"] == B.EV_DECORRELATED:
            dec = e["steps"]
        elif e["kind"] == B.EV_DEPHASED:
            assert e["n_branch"] == 0
            dec += e["steps"]
        elif e["kind"] == B.EV_PARALLEL_EXIT:
            res.append(dec + e["steps"])
        elif e["kind"] == B.EV_REF_EXIT:
            res.append(e["steps"])
    bres, _ = o.run_bruteforce(SEED, s.t_check, 10 ** 9, 4)
    assert res == list(bres)
    deph = sum(e["steps"] for e in ev if e["kind"] == B.EV_DEPHASED)
    assert tsim + deph == B.grp_get_state(rep)[3]["t_global"]


def test_original_mixed_chain_event_log_is_consistent(B):
    """Mixed precision, 22-bead chain, 64 replicas: the event log obeys the clock rules of Section
    2.4.3 (dephasing not counted; tau = (N (M - 1) + k) t_check) and the step counter adds up."""
    s = W.chain()
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    n = 64
    rep = B.grp_init_replicas(sysh, n, SEED, s.q0, s.p0)
    ev, tsim = B.grp_run_original(rep, s.t_check, 2 * s.t_check, 2 * s.t_check, 60 * s.t_check, 3)
    assert ev, "no event"
    t, extra = 0, 0
    for a, e in enumerate(ev):
        if e["kind"] == B.EV_DEPHASED:
            extra += e["steps"]
            assert e["steps"] >= 2 * s.t_check
        else:
            t += e["steps"]
        assert e["t_sim"] == t
        if e["kind"] == B.EV_PARALLEL_EXIT:
            assert ev[a - 1]["kind"] == B.EV_DEPHASED
            assert e["steps"] == (n * (e["M"] - 1) + e["k"]) * s.t_check
            extra += e["M"] * s.t_check - e["steps"]
    tg = B.grp_get_state(rep)[3]["t_global"]
    # the bound may stop a phase part-way: the counter covers at least the logged work
    assert tg >= t + extra and tsim == t


def test_original_invalid_arguments(B):
    s = W.double_well_2d()
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, 4, SEED, s.q0, s.p0)
    for bad in [(0, 100, 100), (100, -1, 100), (100, 100, -1)]:
        with pytest.raises(B.GrpError) as ei:
            B.grp_run_original(rep, bad[0], bad[1], bad[2], 1000, 1)
        assert ei.value.status == B.GRP_EINVAL
    # nothing ran
    assert B.grp_get_state(rep)[3]["t_global"] == 0
