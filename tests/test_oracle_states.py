"""Pins of the oracle's centre-of-mass state rule and the ligand observables (CPU only).

The ligand-dissociation workload (Section 4.2, Gen. ParRep setup) labels a configuration bound
while the distance between two groups' centres of mass is below a threshold, and tracks the
convergence of the Fleming-Viot process with group distances and the ligand's root mean square
velocity.  The values below are worked out by hand on configurations small enough to check by eye,
and each test names the plausible misreading it rules out:

* an unweighted centre (the mean of the positions) instead of the mass-weighted one;
* the root mean square over Cartesian components instead of over atoms (speeds);
* ``<=`` instead of ``<`` at the threshold (the state is bound strictly below it).
"""
import math

import numpy as np
import pytest

from paper_1807_02431_gb300 import workloads as W


def _system(masses, groups, observables, threshold=1.0):
    n = len(masses)
    return W.System(
        name="pin", n_atoms=n, dim=3, potential=W.POT_FORCE_FIELD, mass=np.asarray(masses, float),
        kT=2.49434, gamma=1.0, dt=0.002,
        sigma=np.full(n, 0.3), epsilon=np.zeros(n), charge=np.zeros(n),
        cv_kind=W.CV_COM_DISTANCE, cv_params=(threshold,),
        groups=[list(g) for g in groups], observables=list(observables),
        q0=np.zeros((n, 3)), p0=np.zeros((n, 3)),
    )


def _oracle(oracle_mod, s):
    return oracle_mod.Oracle(s)


def test_com_distance_is_mass_weighted(oracle_mod):
    """Group 0: masses 1 and 3 at x = 0 and x = 4, centre (3, 0, 0) (the plain mean would be
    (2, 0, 0)).  Group 1: masses 2 and 6 at (3, 4, 0) and (3, 4, 4), centre (3, 4, 3) (plain mean
    (3, 4, 2)).  The distance is the 3-4-5 triangle's 5 exactly; unweighted centres give sqrt(21)."""
    s = _system([1.0, 3.0, 2.0, 6.0], [(0, 1), (2, 3)],
                [(W.OBS_GROUP_DISTANCE, (0, 1)), (W.OBS_GROUP_DISTANCE, (1, 0))], threshold=6.0)
    o = _oracle(oracle_mod, s)
    q = np.array([[0.0, 0, 0], [4.0, 0, 0], [3.0, 4, 0], [3.0, 4, 4]])
    p = np.zeros_like(q)
    assert o.cv(q)[0] == pytest.approx(5.0, abs=1e-15)
    assert o.observable(0, q, p) == pytest.approx(5.0, abs=1e-15)
    assert o.observable(1, q, p) == pytest.approx(5.0, abs=1e-15)  # symmetric in the two groups
    assert abs(o.cv(q)[0] - math.sqrt(21.0)) > 0.1


def test_com_distance_ignores_atoms_outside_the_groups(oracle_mod):
    """Atoms that belong to no group (here atom 2, far away and heavy) do not move either centre."""
    s = _system([1.0, 1.0, 100.0, 1.0], [(0,), (1, 3)], [(W.OBS_GROUP_DISTANCE, (0, 1))])
    o = _oracle(oracle_mod, s)
    q = np.array([[0.0, 0, 0], [0.0, 2, 0], [50.0, 50, 50], [0.0, 0, 2]])
    # centre of group 1 = (0, 1, 1): distance sqrt(2)
    assert o.observable(0, q, np.zeros_like(q)) == pytest.approx(math.sqrt(2.0), abs=1e-15)


def test_rms_velocity_is_over_atoms(oracle_mod):
    """Ligand root mean square velocity: sqrt(mean over the group's atoms of |p/m|^2).
    Atom 0: m = 2, p = (2, 4, 4), v = (1, 2, 2), |v|^2 = 9.  Atom 1: m = 1, p = (0, 0, 1), |v|^2 = 1.
    Atom 2 (not in the group) moves fast.  RMS = sqrt((9 + 1) / 2) = sqrt(5); over the six components
    it would be sqrt(10 / 6), and with momenta in place of velocities sqrt((36 + 1) / 2)."""
    s = _system([2.0, 1.0, 1.0], [(0, 1), (2,)], [(W.OBS_RMS_VELOCITY, (0,)), (W.OBS_RMS_VELOCITY, (1,))])
    o = _oracle(oracle_mod, s)
    q = np.zeros((3, 3))
    p = np.array([[2.0, 4, 4], [0.0, 0, 1], [30.0, 0, 40]])
    assert o.observable(0, q, p) == pytest.approx(math.sqrt(5.0), abs=1e-15)
    assert o.observable(1, q, p) == pytest.approx(50.0, abs=1e-13)
    assert abs(o.observable(0, q, p) - math.sqrt(10.0 / 6.0)) > 0.5


def test_rms_velocity_of_thermal_momenta(oracle_mod):
    """Momenta drawn from Maxwell-Boltzmann at kT: <|v|^2> = 3 kT / m per atom, so the squared RMS
    velocity of a large group of equal masses is 3 kT / m within its sampling error."""
    n, m, kT = 4000, 12.0, 2.49434
    s = _system([m] * n, [tuple(range(n))], [(W.OBS_RMS_VELOCITY, (0,))], threshold=1.0)
    s.kT = kT
    o = _oracle(oracle_mod, s)
    p = W.maxwell_boltzmann(np.full(n, m), kT, 3, np.random.default_rng(5))
    v2 = o.observable(0, np.zeros((n, 3)), p) ** 2
    # |v|^2 per atom is (kT/m) chi^2_3: variance 2 * 3 (kT/m)^2, mean over n atoms
    assert abs(v2 - 3 * kT / m) < 5 * math.sqrt(6.0 / n) * kT / m


@pytest.mark.parametrize("d,label", [(1.0 - 2.0 ** -52, 0), (1.0, 1), (1.0 + 2.0 ** -52, 1), (0.0, 0), (7.5, 1)])
def test_bound_state_is_strictly_below_threshold(oracle_mod, d, label):
    """Bound (state 0) while the centre-of-mass distance is strictly below the threshold, unbound
    (state 1) at and above it; a two-state partition, so exited(Omega) is the label changing."""
    s = _system([1.0, 1.0], [(0,), (1,)], [(W.OBS_GROUP_DISTANCE, (0, 1))], threshold=1.0)
    o = _oracle(oracle_mod, s)
    q = np.array([[0.0, 0, 0], [d, 0, 0]])
    assert o.cv(q)[0] == d
    assert o.state_of(q) == label
    assert o.exited(q, 0) == (label != 0)
    assert o.exited(q, 1) == (label != 1)


def test_threshold_is_read_from_the_state_definition(oracle_mod):
    """The threshold is the state definition's parameter, not a constant: at d = 1.1 the ligand
    is bound for a 1.2 nm threshold (the paper's FKBP value) and unbound for 1.0 nm."""
    q = np.array([[0.0, 0, 0], [0.0, 1.1, 0]])
    for thr, label in ((1.2, 0), (1.0, 1)):
        s = _system([1.0, 1.0], [(0,), (1,)], [], threshold=thr)
        assert _oracle(oracle_mod, s).state_of(q) == label


def test_ligand_workload_state_uses_mass_weighted_pocket(oracle_mod):
    """On the generated ligand-receptor system, the oracle's CV equals the distance between the
    mass-weighted centres of the ligand and the pocket-lining beads computed here with numpy, and
    the first configuration is bound."""
    s = W.ligand_receptor()
    o = _oracle(oracle_mod, s)
    q = s.q0
    m = s.mass

    def com(g):
        g = np.asarray(g)
        return (m[g, None] * q[g]).sum(0) / m[g].sum()

    d = np.linalg.norm(com(s.groups[0]) - com(s.groups[1]))
    assert o.cv(q)[0] == pytest.approx(d, rel=1e-13)
    assert d < s.cv_params[0] and o.state_of(q) == 0
