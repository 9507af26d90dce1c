"""Pins of the oracle's Generalized Born implicit solvent (OBC model II, the solvent of the paper's
protein-ligand setup).

* The descreening sum of one neighbour equals a numerical quadrature of the integral it approximates:
  (1/4 pi) times the integral of |x|^-4 over the neighbour's scaled sphere outside atom i's sphere,
  shell by shell (the fraction of each shell inside a sphere is the spherical-cap formula).
* A lone ion has Born radius a = rho - 0.009 nm and the Born solvation energy -k_e tau q^2 / (2 a).
* Two ions far apart: the pair term is the screening of their Coulomb interaction, -k_e tau q1 q2 / r.
* Born radii never fall below a_i (descreening only adds), and grow when a neighbour comes closer.
* Forces are minus the gradient of the energy (central differences) on a charged chain in solvent.
"""
import dataclasses
import math

import numpy as np
import pytest

from paper_1807_02431_gb300 import workloads as W

OFFSET = 0.009


def _ions(q, rho, scale, pos):
    """Point charges without Lennard-Jones or bonded terms, in OBC II solvent."""
    n = len(q)
    s = W.chain(n_atoms=6)
    s = dataclasses.replace(s, n_atoms=n, mass=np.full(n, 12.0), sigma=np.full(n, 0.3), epsilon=np.zeros(n),
                            charge=np.array(q, float), excl=np.zeros((0, 2), np.int32), coulomb_k=W.COULOMB_K,
                            bonds=None, bond_k=None, bond_r0=None, angles=None, angle_k=None, angle_theta0=None,
                            dihedrals=None, dihedral_n=None, dihedral_k=None, dihedral_delta=None,
                            cv_kind=W.CV_COM_DISTANCE, cv_atoms=(), cv_params=(1.0,), groups=[[0], [n - 1]],
                            observables=[(W.OBS_POTENTIAL, ())], gb_radius=np.array(rho, float),
                            gb_scale=np.array(scale, float))
    s.q0 = np.array(pos, float)
    s.p0 = np.zeros_like(s.q0)
    return s


def _tau():
    return W.COULOMB_K * (1.0 / 1.0 - 1.0 / 78.5)


def _quadrature(r, ai, sj):
    """(1/4 pi) int |x|^-4 dV over {|x - c| < sj, |x| > ai}, |c| = r, by shells |x| = t."""
    from scipy.integrate import quad

    def frac(t):  # fraction of the shell of radius t inside the sphere
        if t <= abs(r - sj):
            return 1.0 if sj > r else 0.0
        if t >= r + sj:
            return 0.0
        return (sj * sj - (t - r) ** 2) / (4.0 * r * t)

    lo = ai
    pts = sorted({x for x in (abs(r - sj), r + sj) if x > lo})
    val, _ = quad(lambda t: frac(t) / (t * t), lo, r + sj, points=pts or None, limit=200, epsabs=1e-13, epsrel=1e-11)
    return val


@pytest.mark.parametrize("r,rho_i,rho_j,scale", [(0.35, 0.17, 0.15, 0.8), (0.20, 0.17, 0.19, 0.85),
                                                 (0.05, 0.12, 0.20, 1.0), (0.9, 0.15, 0.15, 0.72),
                                                 (0.02, 0.2, 0.12, 0.8)])
def test_descreening_sum_is_the_volume_integral(oracle_mod, r, rho_i, rho_j, scale):
    s = _ions([0.0, 0.0], [rho_i, rho_j], [scale, scale], [[0, 0, 0], [r, 0, 0]])
    o = oracle_mod.Oracle(s)
    _, integral = o.gb_born(s.q0)
    ref = _quadrature(r, rho_i - OFFSET, scale * (rho_j - OFFSET))
    assert integral[0] == pytest.approx(ref, rel=1e-8, abs=1e-12)


def test_lone_ion_is_a_born_sphere(oracle_mod):
    q, rho = -0.83, 0.16
    s = _ions([q], [rho], [0.8], [[0.1, 0.2, 0.3]])
    o = oracle_mod.Oracle(s)
    born, _ = o.gb_born(s.q0)
    assert born[0] == pytest.approx(rho - OFFSET, rel=1e-14)
    assert o.potential(s.q0) == pytest.approx(-_tau() * q * q / (2 * (rho - OFFSET)), rel=1e-13)


def test_distant_ions_screen_coulomb(oracle_mod):
    q1, q2, r = 0.7, -0.45, 80.0
    s = _ions([q1, q2], [0.16, 0.18], [0.8, 0.85], [[0, 0, 0], [r, 0, 0]])
    o = oracle_mod.Oracle(s)
    born, _ = o.gb_born(s.q0)
    self_e = -_tau() * (q1 * q1 / born[0] + q2 * q2 / born[1]) / 2
    vac = dataclasses.replace(s, gb_radius=None, gb_scale=None)
    vac.q0 = s.q0
    solvation = o.potential(s.q0) - oracle_mod.Oracle(vac).potential(s.q0)  # the vacuum terms cancel
    assert solvation - self_e == pytest.approx(-_tau() * q1 * q2 / r, rel=1e-6)


def test_born_radii_grow_with_burial(oracle_mod):
    rho = [0.16, 0.15, 0.17]
    prev = None
    for d in (0.8, 0.5, 0.35, 0.3):
        s = _ions([0.2, -0.1, 0.3], rho, [0.8, 0.8, 0.8], [[0, 0, 0], [d, 0, 0], [0, d, 0]])
        born, _ = oracle_mod.Oracle(s).gb_born(s.q0)
        assert np.all(born >= np.array(rho) - OFFSET - 1e-15)
        if prev is not None:
            assert born[0] > prev
        prev = born[0]


def test_forces_are_minus_the_gradient(oracle_mod):
    base = W.chain()
    rng = np.random.default_rng(2)
    s = dataclasses.replace(base, gb_radius=rng.uniform(0.14, 0.19, base.n_atoms),
                            gb_scale=rng.uniform(0.7, 0.9, base.n_atoms))
    s.q0, s.p0 = base.q0, base.p0
    o = oracle_mod.Oracle(s)
    q = s.q0 + 0.005 * rng.standard_normal(s.q0.shape)
    f = o.forces(q)
    e0 = oracle_mod.Oracle(base).potential(q)  # the same chain in vacuum
    assert abs(o.potential(q) - e0) > 1.0  # the solvent term is there
    h = 1e-6
    for a, x in [(0, 0), (3, 1), (10, 2), (17, 0), (21, 2)]:
        qp, qm = q.copy(), q.copy()
        qp[a, x] += h
        qm[a, x] -= h
        fd = -(o.potential(qp) - o.potential(qm)) / (2 * h)
        assert fd == pytest.approx(f[a, x], rel=1e-6, abs=1e-4)


# ----------------------------------------------------------------------------- with a cutoff
# A system with a cutoff truncates the solvent sums like its other nonbonded terms: a pair at r >= r_c
# enters neither the descreening sums nor the pair energy; the self terms always count.

def _with_cutoff(s, rc):
    t = dataclasses.replace(s, cutoff=rc)
    t.q0, t.p0 = s.q0, s.p0
    return t


def test_cutoff_beyond_every_pair_changes_nothing(oracle_mod):
    base = W.chain()
    rng = np.random.default_rng(3)
    s = dataclasses.replace(base, gb_radius=rng.uniform(0.14, 0.19, base.n_atoms),
                            gb_scale=rng.uniform(0.7, 0.9, base.n_atoms))
    s.q0, s.p0 = base.q0, base.p0
    q = s.q0 + 0.005 * rng.standard_normal(s.q0.shape)
    o, oc = oracle_mod.Oracle(s), oracle_mod.Oracle(_with_cutoff(s, 50.0))
    assert oc.potential(q) == o.potential(q)
    assert np.array_equal(oc.forces(q), o.forces(q))


def test_ions_beyond_the_cutoff_are_lone_born_spheres(oracle_mod):
    """Two ions 1.5 nm apart with a 1.2 nm cutoff: no descreening, no pair term, no Coulomb: the energy
    is the two Born energies exactly and there is no force; at 1.0 nm both couplings are back."""
    q1, q2, rho1, rho2 = 0.6, -0.8, 0.16, 0.18
    a1, a2 = rho1 - OFFSET, rho2 - OFFSET
    born_e = -_tau() * (q1 * q1 / a1 + q2 * q2 / a2) / 2
    far = _with_cutoff(_ions([q1, q2], [rho1, rho2], [0.8, 0.8], [[0, 0, 0], [1.5, 0, 0]]), 1.2)
    o = oracle_mod.Oracle(far)
    born, integral = o.gb_born(far.q0)
    assert np.array_equal(integral, [0.0, 0.0]) and born[0] == pytest.approx(a1, rel=1e-15)
    assert o.potential(far.q0) == pytest.approx(born_e, rel=1e-14)
    assert np.all(o.forces(far.q0) == 0.0)
    near = np.array([[0, 0, 0], [1.0, 0, 0]], float)
    assert abs(o.potential(near) - born_e) > 1.0
    assert np.all(o.gb_born(near)[1] > 0)


def test_cutoff_truncates_each_pair_separately(oracle_mod):
    """Three atoms on a line, 1.0 nm apart, cutoff 1.2 nm: atom 0 is descreened by atom 1 alone (its sum
    equals the two-atom value) while atom 1 is descreened by both; the pair (0, 2) at 2.0 nm is cut."""
    rho, sc = [0.16, 0.17, 0.15], [0.8, 0.75, 0.85]
    three = _with_cutoff(_ions([0.3, -0.2, 0.4], rho, sc, [[0, 0, 0], [1.0, 0, 0], [2.0, 0, 0]]), 1.2)
    _, i3 = oracle_mod.Oracle(three).gb_born(three.q0)
    pair01 = _ions([0.3, -0.2], rho[:2], sc[:2], [[0, 0, 0], [1.0, 0, 0]])
    pair12 = _ions([-0.2, 0.4], rho[1:], sc[1:], [[1.0, 0, 0], [2.0, 0, 0]])
    _, i01 = oracle_mod.Oracle(pair01).gb_born(pair01.q0)
    _, i12 = oracle_mod.Oracle(pair12).gb_born(pair12.q0)
    assert i3[0] == i01[0] and i3[2] == i12[1]
    assert i3[1] == pytest.approx(i01[1] + i12[0], rel=1e-15)


def test_forces_are_minus_the_gradient_with_a_cutoff(oracle_mod):
    """The chain in solvent with a 0.9 nm cutoff (some pairs beyond it): forces = -grad V where no pair
    lies within 1e-4 nm of the cutoff."""
    base = W.chain()
    rng = np.random.default_rng(4)
    s = dataclasses.replace(base, gb_radius=rng.uniform(0.14, 0.19, base.n_atoms),
                            gb_scale=rng.uniform(0.7, 0.9, base.n_atoms), cutoff=0.9)
    s.q0, s.p0 = base.q0, base.p0
    o = oracle_mod.Oracle(s)
    q = s.q0 + 0.005 * rng.standard_normal(s.q0.shape)
    d = np.linalg.norm(q[:, None] - q[None], axis=-1)[np.triu_indices(base.n_atoms, 1)]
    assert (d > 0.9).any() and (d < 0.9).any() and np.abs(d - 0.9).min() > 1e-4
    f = o.forces(q)
    h = 1e-6
    for a, x in [(0, 0), (4, 1), (11, 2), (16, 0), (21, 1)]:
        qp, qm = q.copy(), q.copy()
        qp[a, x] += h
        qm[a, x] -= h
        fd = -(o.potential(qp) - o.potential(qm)) / (2 * h)
        assert fd == pytest.approx(f[a, x], rel=1e-6, abs=1e-4)
