"""Pins of the oracle's reaction-field electrostatics (the Coulomb model of a cutoff scheme).

Pinned against facts that do not restate the oracle's formula: the pair energy vanishes at the cutoff
(and so does the force for a conducting continuum); with eps_rf = 1 energy differences are those of
plain Coulomb; for a cutoff far beyond the pair the energy tends to plain Coulomb; forces are minus
the gradient of the energy (central differences) on a charged cluster.
"""
import dataclasses

import numpy as np
import pytest

from paper_1807_02431_gb300 import workloads as W


def _pair(rc, eps_rf, q=(0.7, -0.4)):
    """Two charged beads without Lennard-Jones."""
    s = W.chain(n_atoms=4)
    s = dataclasses.replace(s, n_atoms=2, mass=np.full(2, 12.0), sigma=np.full(2, 0.3), epsilon=np.zeros(2),
                            charge=np.array(q), excl=np.zeros((0, 2), np.int32), cutoff=rc,
                            coulomb_mode=W.COULOMB_REACTION_FIELD, rf_dielectric=eps_rf,
                            bonds=None, bond_k=None, bond_r0=None, angles=None, angle_k=None, angle_theta0=None,
                            dihedrals=None, dihedral_n=None, dihedral_k=None, dihedral_delta=None,
                            cv_kind=W.CV_COM_DISTANCE, cv_atoms=(), cv_params=(1.0,), groups=[[0], [1]],
                            observables=[(W.OBS_POTENTIAL, ())])
    s.q0 = np.zeros((2, 3))
    s.p0 = np.zeros((2, 3))
    return s


def _at(r):
    return np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])


@pytest.mark.parametrize("eps_rf", [0.0, 78.3, 4.0])
def test_energy_vanishes_at_the_cutoff(oracle_mod, eps_rf):
    rc = 1.2
    o = oracle_mod.Oracle(_pair(rc, eps_rf))
    e_in = o.potential(_at(rc * (1 - 1e-9)))
    e_mid = o.potential(_at(0.6))
    assert abs(e_in) < 1e-7 * abs(e_mid)
    assert o.potential(_at(rc * (1 + 1e-9))) == 0.0
    if eps_rf == 0.0:  # conductor: the force vanishes at the cutoff too
        f_in = o.forces(_at(rc * (1 - 1e-9)))
        assert np.abs(f_in).max() < 1e-7 * np.abs(o.forces(_at(0.6))).max()


def test_unit_continuum_is_shifted_coulomb(oracle_mod):
    s = _pair(1.5, 1.0)
    o = oracle_mod.Oracle(s)
    kqq = W.COULOMB_K * 0.7 * -0.4
    for r1, r2 in ((0.3, 0.9), (0.5, 1.4)):
        assert o.potential(_at(r1)) - o.potential(_at(r2)) == pytest.approx(kqq * (1 / r1 - 1 / r2), rel=1e-12)


def test_far_cutoff_tends_to_coulomb(oracle_mod):
    o = oracle_mod.Oracle(_pair(1.0e4, 78.3))
    kqq = W.COULOMB_K * 0.7 * -0.4
    assert o.potential(_at(0.5)) == pytest.approx(kqq / 0.5, rel=1e-3)
    f = o.forces(_at(0.5))
    assert f[1, 0] == pytest.approx(kqq / 0.25, rel=1e-6)  # force on the second bead along +x


def test_forces_are_minus_the_gradient(oracle_mod):
    s = dataclasses.replace(W.chain(), cutoff=1.0, coulomb_mode=W.COULOMB_REACTION_FIELD, rf_dielectric=78.3)
    s.q0 = W.chain().q0
    o = oracle_mod.Oracle(s)
    rng = np.random.default_rng(3)
    q = s.q0 + 0.01 * rng.standard_normal(s.q0.shape)
    f = o.forces(q)
    h = 1e-6
    for a, x in [(0, 0), (5, 1), (11, 2), (20, 0), (21, 1)]:
        qp, qm = q.copy(), q.copy()
        qp[a, x] += h
        qm[a, x] -= h
        fd = -(o.potential(qp) - o.potential(qm)) / (2 * h)
        assert fd == pytest.approx(f[a, x], rel=1e-6, abs=1e-5)
