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
