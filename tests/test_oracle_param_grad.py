"""Pins of the oracle's parameter derivatives dV/d theta (CPU only).

theta = (sigma_i, epsilon_i, dihedral k_t).  Each pin is a fact the derivative must satisfy that does
not come from re-typing its formula: central finite differences of the (separately pinned) potential,
the closed form of a Lennard-Jones pair at its minimum, and Euler relations of the homogeneous parts
of V.  A dropped factor 1/2 of the combination rules, a wrong power of s or a sign error fails one.
"""
import dataclasses

import numpy as np

from paper_1807_02431_gb300 import workloads as W


def _q(s, seed=5, spread=0.01):
    rng = np.random.default_rng(seed)
    return s.q0 + spread * rng.standard_normal(s.q0.shape)


def _theta(s):
    return np.concatenate([s.sigma, s.epsilon, s.dihedral_k])


def _with_theta(s, th):
    n = s.n_atoms
    return dataclasses.replace(s, sigma=th[:n].copy(), epsilon=th[n:2 * n].copy(), dihedral_k=th[2 * n:].copy())


def test_param_grad_matches_central_differences(oracle_mod):
    """Every component of dV/d theta against a central difference of V (h = 1e-6 relative)."""
    s = W.chain(22)
    q = _q(s)
    g = oracle_mod.Oracle(s).param_grad(q)
    th = _theta(s)
    assert g.shape == th.shape
    fd = np.zeros_like(th)
    for k in range(len(th)):
        h = 1e-6 * max(abs(th[k]), 1e-3)
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd[k] = (oracle_mod.Oracle(_with_theta(s, tp)).potential(q) -
                 oracle_mod.Oracle(_with_theta(s, tm)).potential(q)) / (2 * h)
    scale = np.abs(fd).max()
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-7 * scale)


def test_lj_pair_at_its_minimum(oracle_mod):
    """Two atoms at r = 2^(1/6) sigma_ij: V = -eps_ij for every sigma, so dV/d sigma_i = 0, and
    dV/d eps_ij = -1 gives dV/d eps_i = -eps_j / (2 eps_ij)."""
    sig = np.array([0.28, 0.34])
    eps = np.array([0.3, 0.7])
    sij = sig.mean()
    r = 2 ** (1 / 6) * sij
    s = W.System(name="pair", n_atoms=2, dim=3, potential=W.POT_FORCE_FIELD, mass=np.full(2, 12.0),
                 kT=1.0, gamma=1.0, dt=0.002, sigma=sig, epsilon=eps, charge=np.zeros(2),
                 excl=np.zeros((0, 2), np.int32), coulomb_k=W.COULOMB_K,
                 dihedrals=np.zeros((0, 4), np.int32), dihedral_n=np.zeros(0, np.int32),
                 dihedral_k=np.zeros(0), dihedral_delta=np.zeros(0),
                 q0=np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]]))
    o = oracle_mod.Oracle(s)
    g = o.param_grad(s.q0)
    eij = np.sqrt(eps[0] * eps[1])
    assert abs(o.potential(s.q0) + eij) < 1e-12
    np.testing.assert_allclose(g[:2], [0.0, 0.0], atol=1e-12)
    np.testing.assert_allclose(g[2:4], [-eps[1] / (2 * eij), -eps[0] / (2 * eij)], rtol=1e-12)


def _lj_only(s):
    z = lambda a: None if a is None else np.zeros_like(a)
    return dataclasses.replace(s, charge=np.zeros(s.n_atoms), bond_k=z(s.bond_k), angle_k=z(s.angle_k),
                               dihedral_k=z(s.dihedral_k))


def test_euler_relations(oracle_mod):
    """V_LJ is homogeneous of degree 1 in epsilon (eps_ij = sqrt(eps_i eps_j)): sum eps_i dV/d eps_i =
    V_LJ; the dihedral energy is linear in k: sum k_t dV/dk_t = V_dih; and V_LJ depends on sigma_ij / r
    only, so scaling sigma and q together leaves it unchanged: sum sigma_i dV/d sigma_i = q . F_LJ."""
    s = W.chain(22)
    q = _q(s, seed=9)
    n = s.n_atoms
    lj = _lj_only(s)
    olj = oracle_mod.Oracle(lj)
    g = olj.param_grad(q)
    v_lj = olj.potential(q)
    assert abs(np.dot(s.epsilon, g[n:2 * n]) - v_lj) < 1e-10 * max(1.0, abs(v_lj))
    f_lj = olj.forces(q)
    assert abs(np.dot(s.sigma, g[:n]) - np.sum(q * f_lj)) < 1e-9 * max(1.0, np.abs(g[:n]).sum())
    # dihedral part: V of a system with only dihedrals
    z = lambda a: None if a is None else np.zeros_like(a)
    dih = dataclasses.replace(s, charge=np.zeros(n), epsilon=np.zeros(n), bond_k=z(s.bond_k), angle_k=z(s.angle_k))
    od = oracle_mod.Oracle(dih)
    gk = oracle_mod.Oracle(s).param_grad(q)[2 * n:]
    assert abs(np.dot(s.dihedral_k, gk) - od.potential(q)) < 1e-10 * max(1.0, abs(od.potential(q)))
    # 0 <= 1 + cos(.) <= 2
    assert np.all(gk >= -1e-15) and np.all(gk <= 2 + 1e-15)
