"""Sensitivity of the 22-bead chain's dynamics, measured in the oracle alone (CPU).

Two oracle trajectories with the same noise whose initial positions differ by a relative 1e-10
separate by more than a factor 1e3 (median over replicas) within 1,000 steps: the dynamics is
chaotic.  Any path whose per-step rounding is ~1e-7 (FP32 forces) therefore cannot stay within 1e-4
of the FP64 oracle for 1,000 steps; this is why the mixed path is compared at 200 steps, by its
one-step local error and by labels, while the FP64 path is compared at 1,000 steps.
"""
import numpy as np

from paper_1807_02431_gb300 import workloads as W


def test_chain_dynamics_amplifies_perturbations(oracle_mod):
    s = W.chain()
    o = oracle_mod.Oracle(s)
    R, eps = 6, 1e-10
    q0, p0 = W.replica_states(s, R, seed=3, spread=0.003)
    qa, pa = q0.copy(), p0.copy()
    qb, pb = q0 * (1 + eps), p0.copy()
    fa = np.stack([o.forces(qa[r]) for r in range(R)])
    fb = np.stack([o.forces(qb[r]) for r in range(R)])
    o.step_k(qa, pa, fa, 2431, 0, 0, 1000, 0)
    o.step_k(qb, pb, fb, 2431, 0, 0, 1000, 0)
    growth = np.abs(qa - qb).max(axis=(1, 2)) / np.abs(qa).max() / eps
    assert np.median(growth) > 1e3, growth
