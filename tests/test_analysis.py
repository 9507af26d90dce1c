"""Exit-time reports of Section 4: per-visit residence times from event logs, the empirical ccdf and
per-state chi-square intervals."""
import numpy as np

from paper_1807_02431_gb300 import analysis as A


def _ev(kind, steps, omega=0, to=0):
    return {"kind": kind, "omega": omega, "label_to": to, "k": 0, "M": 0, "steps": steps, "t_sim": 0, "n_branch": 0}


def test_visits_of_a_log():
    log = [_ev(A.EV_TRANSIENT, 300, -1, 4), _ev(A.EV_FV_ALL_EXITED, 100, 4, 4), _ev(A.EV_FV_CONVERGED, 2000, 4, 4),
           _ev(A.EV_PARALLEL_EXIT, 9000, 4, 5), _ev(A.EV_REF_EXIT, 700, 5, -1), _ev(A.EV_TRANSIENT, 200, -1, 4),
           _ev(A.EV_DECORRELATED, 1000, 4, 4), _ev(A.EV_DEPHASED, 2500, 4, 4), _ev(A.EV_PARALLEL_EXIT, 400, 4, 3)]
    assert A.visits(log) == [(4, 11000, 5, True), (5, 700, -1, False), (4, 1400, 3, True)]


def test_ccdf_definition():
    t, p = A.ccdf([3.0, 1.0, 2.0, 2.0])
    assert list(t) == [0.0, 1.0, 2.0, 3.0]
    assert list(p) == [1.0, 0.75, 0.25, 0.0]


def test_ccdf_of_exponential_samples():
    x = np.random.default_rng(1).exponential(5.0, 20000)
    t, p = A.ccdf(x)
    grid = np.array([1.0, 5.0, 10.0, 20.0])
    emp = p[np.searchsorted(t, grid, side="right") - 1]
    assert np.allclose(emp, np.exp(-grid / 5.0), atol=0.01)


def test_state_report():
    rng = np.random.default_rng(2)
    logs = []
    for run in range(40):
        log = []
        for v in range(6):
            om = v % 2
            log += [_ev(A.EV_FV_CONVERGED, 100, om, om), _ev(A.EV_PARALLEL_EXIT, int(rng.exponential(900 + 1000 * om)), om, 1 - om)]
        logs.append(log)
    rep = A.state_report(logs, dt=0.002)
    assert set(rep) == {0, 1}
    for om in (0, 1):
        r = rep[om]
        assert r["n"] == {0: 80, 1: 120}[om]  # the first visit (state 0) of each run is dropped
        lo, hi = r["ci"]
        assert lo < r["mean"] < hi
        assert r["to"] == {1 - om: r["n"]} and r["parallel_exits"] == r["n"]
        assert abs(r["mean"] - (1000 + 1000 * om) * 0.002) < 0.3 * (1000 + 1000 * om) * 0.002
        _, l2, h2 = A.exit_time_ci(r["mean"], n=r["n"])
        assert (l2, h2) == (lo, hi)
