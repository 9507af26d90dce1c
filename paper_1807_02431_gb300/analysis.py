"""Post-processing of Gen. ParRep exit-time samples and run speed (Section 4).

These follow the reporting conventions of the paper: the sample mean of exit times with a
chi-square confidence interval for (close to) exponential samples (start of Section 4), and the
speed / effective speedup / efficiency of Tables 2 and 4.
"""
from __future__ import annotations

import numpy as np


def exit_time_ci(samples_or_mean, n: int | None = None, alpha: float = 0.05):
    """Mean of exponential exit-time samples and its 1 - alpha confidence interval
    2 n tau_bar / chi2_{1-alpha/2, 2n} < E(tau) < 2 n tau_bar / chi2_{alpha/2, 2n}.

    Pass either the samples, or their mean together with n."""
    from scipy.stats import chi2

    if n is None:
        x = np.asarray(samples_or_mean, dtype=np.float64)
        n, tau_bar = x.size, float(x.mean())
    else:
        tau_bar = float(samples_or_mean)
    lo = 2 * n * tau_bar / chi2.ppf(1 - alpha / 2, 2 * n)
    hi = 2 * n * tau_bar / chi2.ppf(alpha / 2, 2 * n)
    return tau_bar, lo, hi


def speed_ns_per_day(t_sim_ns: float, wall_s: float) -> float:
    """Simulated clock divided by wall time, in ns/day (Table 2 caption)."""
    return t_sim_ns / (wall_s / 86400.0)


def effective_speedup(speed: float, serial_speed: float) -> float:
    """Speed divided by the speed of a plain serial Langevin run on the same hardware."""
    return speed / serial_speed


def efficiency(speedup: float, n_replicas: int) -> float:
    """Effective speedup over the maximum possible speedup N."""
    return speedup / n_replicas


# Event kinds of an event log (the values of grp_event.kind).
EV_TRANSIENT, EV_REF_EXIT, EV_FV_CONVERGED, EV_PARALLEL_EXIT, EV_FV_ALL_EXITED, EV_DECORRELATED, EV_DEPHASED = range(7)


def visits(events):
    """Per visit of a state, from one run's event log: (state, residence steps, destination, ended by a
    parallel step).  The residence time is the simulated time the visit added to the clock: t_FV + tau
    after a converged F-V step (Eq. 6), t_corr + tau in the original loop, t_ref after a reference exit.
    Transients and dephasing times are not part of any visit."""
    out, lead = [], 0
    for e in events:
        k = e["kind"]
        if k in (EV_FV_CONVERGED, EV_DECORRELATED):
            lead = e["steps"]
        elif k == EV_PARALLEL_EXIT:
            out.append((e["omega"], lead + e["steps"], e["label_to"], True))
            lead = 0
        elif k == EV_REF_EXIT:
            out.append((e["omega"], e["steps"], e["label_to"], False))
            lead = 0
    return out


def ccdf(samples):
    """Empirical complementary cumulative distribution P(tau > t) (the ccdf of Section 4.1): returns
    (t, P) with t = 0 and the distinct sample values in ascending order and P(tau > t) the fraction of
    samples strictly above t, so that P = 1 at t = 0 for positive samples."""
    x = np.sort(np.asarray(samples, dtype=np.float64))
    t = np.concatenate([[0.0], np.unique(x)])
    above = x.size - np.searchsorted(x, t, side="right")
    return t, above / max(x.size, 1)


def state_report(logs, dt: float = 1.0, alpha: float = 0.05, skip_first: bool = True):
    """Exit statistics per state over many runs' event logs: for each state, the number of visits n,
    the mean residence time with its chi-square 1 - alpha interval (exit_time_ci), the destinations of
    the exits, the number of visits ended by a parallel step, and the empirical ccdf.  Times are in
    steps times dt.  skip_first drops each run's first visit, which starts from the given initial
    configuration rather than from an entry into the state."""
    per = {}
    for ev in logs:
        vs = visits(ev)
        for omega, steps, to, par in (vs[1:] if skip_first else vs):
            d = per.setdefault(omega, {"t": [], "to": {}, "parallel": 0})
            d["t"].append(steps * dt)
            d["to"][to] = d["to"].get(to, 0) + 1
            d["parallel"] += int(par)
    report = {}
    for omega, d in sorted(per.items()):
        mean, lo, hi = exit_time_ci(d["t"], alpha=alpha)
        t, p = ccdf(d["t"])
        report[omega] = {"n": len(d["t"]), "mean": mean, "ci": (lo, hi), "to": d["to"],
                         "parallel_exits": d["parallel"], "ccdf": (t, p)}
    return report
