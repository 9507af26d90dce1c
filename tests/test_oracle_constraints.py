"""Pins of the oracle's constrained BAOAB (SHAKE positions, RATTLE momenta), on facts that do not
restate its code: constrained lengths and zero relative velocity along every bond after long runs; a
free rigid rotor (no forces, no friction) keeps its kinetic energy and angular momentum; and the
kinetic energy follows equipartition over the 3N - N_c remaining degrees of freedom."""
import dataclasses

import numpy as np
import pytest

from paper_1807_02431_gb300 import workloads as W


def test_constraints_hold_along_trajectories(oracle_mod):
    s = W.chain_h()
    o = oracle_mod.Oracle(s)
    R = 3
    q = np.repeat(s.q0[None], R, 0).copy()
    p = np.stack([W.maxwell_boltzmann(s.mass, s.kT, 3, np.random.default_rng(r)) for r in range(R)])
    f = np.stack([o.forces(x) for x in q])
    o.step_k(q, p, f, 3, 0, 0, 600, 0)
    i, j = s.constraints[:, 0], s.constraints[:, 1]
    r = q[:, i] - q[:, j]
    assert np.abs(np.linalg.norm(r, axis=-1) - s.constraint_length).max() < 1e-9 * 0.109
    v = p[:, i] / s.mass[i][:, None] - p[:, j] / s.mass[j][:, None]
    assert np.abs((r * v).sum(-1)).max() < 1e-9 * 0.109 ** 2 / s.dt
    assert o.unconverged() == 0


def test_unconverged_projections_are_counted(oracle_mod):
    """One sweep cannot meet a 1e-14 tolerance from a thermal start, so projections that ran out of
    sweeps are counted; with the default tolerance and bound the same steps count none."""
    s = dataclasses.replace(W.chain_h(), constraint_max_iter=1, constraint_tol=1e-14)
    o = oracle_mod.Oracle(s)
    q = s.q0[None].copy()
    p = W.maxwell_boltzmann(s.mass, s.kT, 3, np.random.default_rng(0))[None]
    f = np.stack([o.forces(x) for x in q])
    o.step_k(q, p, f, 3, 0, 0, 5, 0)
    assert o.unconverged() > 0
    o2 = oracle_mod.Oracle(W.chain_h())
    q2, p2 = W.chain_h().q0[None].copy(), p.copy()
    o2.step_k(q2, p2, np.stack([o2.forces(x) for x in q2]), 3, 0, 0, 5, 0)
    assert o2.unconverged() == 0


def test_free_rigid_rotor(oracle_mod):
    """Two atoms joined by a constraint, no potential, gamma = 0: a free rotor whose kinetic energy
    and angular momentum stay constant."""
    base = W.chain(n_atoms=6)
    s = dataclasses.replace(base, n_atoms=2, mass=np.array([12.0, 1.008]), sigma=np.full(2, 0.3), epsilon=np.zeros(2),
                            charge=np.zeros(2), excl=np.zeros((0, 2), np.int32), gamma=0.0,
                            bonds=None, bond_k=None, bond_r0=None, angles=None, angle_k=None, angle_theta0=None,
                            dihedrals=None, dihedral_n=None, dihedral_k=None, dihedral_delta=None,
                            cv_kind=W.CV_COM_DISTANCE, cv_atoms=(), cv_params=(1.0,), groups=[[0], [1]],
                            observables=[(W.OBS_KINETIC, ())], constraints=np.array([[0, 1]], np.int32),
                            constraint_length=np.array([0.109]))
    o = oracle_mod.Oracle(s)
    q = np.array([[[0.0, 0.0, 0.0], [0.109, 0.0, 0.0]]])
    p = np.array([[[0.0, 0.0, 0.0], [0.0, 1.5, 0.3]]])  # tangent: perpendicular to the bond
    f = np.zeros_like(q)

    def invariants(q, p):
        ke = 0.5 * (p[0] ** 2 / s.mass[:, None]).sum()
        ang = np.cross(q[0], p[0]).sum(0)
        return ke, ang

    ke0, l0 = invariants(q, p)
    o.step_k(q, p, f, 1, 0, 0, 2000, 0)
    ke, ang = invariants(q, p)
    assert abs(ke - ke0) < 1e-8 * ke0
    assert np.abs(ang - l0).max() < 1e-8 * np.abs(l0).max()
    assert abs(np.linalg.norm(q[0, 0] - q[0, 1]) - 0.109) < 1e-10


def test_equipartition_over_unconstrained_degrees(oracle_mod):
    """<2K> / kT = 3N - N_c (110 for 44 atoms and 22 constraints; 132 without the constraints)."""
    s = dataclasses.replace(W.chain_h(), observables=[(W.OBS_KINETIC, ())])
    o = oracle_mod.Oracle(s)
    R = 4
    q = np.repeat(s.q0[None], R, 0).copy()
    p = np.stack([W.maxwell_boltzmann(s.mass, s.kT, 3, np.random.default_rng(10 + r)) for r in range(R)])
    f = np.stack([o.forces(x) for x in q])
    o.step_k(q, p, f, 5, 0, 0, 1500, 0)  # equilibration
    k = 8000
    samples = o.step_k(q, p, f, 5, 1500, 0, k, 20, cap=k // 20)
    dof = 2 * samples.mean() / s.kT
    assert dof == pytest.approx(3 * s.n_atoms - len(s.constraints), rel=0.04), dof
