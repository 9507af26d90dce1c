"""Pins of the oracle's rotamer state definition (many disjoint states with a transient region between
them, the case of Section 2.4.1's transient propagation) on the united-atom alkane.

* Labels of chains built from chosen torsions (natural-extension geometry, so the torsions are known
  by construction): the base-3 well index when every torsion is in its core, -1 otherwise.
* The torsions equal an independent numpy dihedral (projection formula, not the oracle's atan2 of
  cross products), so a sign or atom-order error fails.
* Wells tile the circle: on any configuration exactly one state is not exited, and a configuration
  in a state has not exited it.
* Dynamics: butane's trans/gauche occupancy follows the Boltzmann weights of its torsion potential
  (the only phi-dependent term: no nonbonded pair is four bonds apart), within sampling error.
"""
import math

import numpy as np
import pytest

from paper_1807_02431_gb300 import workloads as W


def _label(tors, w=35.0):
    lab, scale = 0, 1
    for t in tors:
        t = (t + 180.0) % 360.0 - 180.0
        t = 180.0 if t == -180.0 else t
        well = 0 if 0 <= t < 120 else (2 if -120 <= t < 0 else 1)
        centre = (60.0, 180.0, -60.0)[well]
        dist = 180.0 - abs(t) if well == 1 else abs(t - centre)
        if not dist < w:
            return -1
        lab += well * scale
        scale *= 3
    return lab


def _dihedral_projection(a, b, c, d):
    """Dihedral in degrees by projecting the outer bonds on the plane normal to the central bond."""
    b0, b1, b2 = a - b, c - b, d - c
    b1 = b1 / np.linalg.norm(b1)
    v = b0 - np.dot(b0, b1) * b1
    w = b2 - np.dot(b2, b1) * b1
    x = np.dot(v, w)
    y = np.dot(np.cross(b1, v), w)
    return math.degrees(math.atan2(y, x))


@pytest.mark.parametrize("tors", [[180, 180, 180, 180], [60, 180, 180, 180], [-60, 180, -60, 180],
                                  [100, 180, 180, 180], [180, 180, 180, -150], [70, -50, 170, 60],
                                  [60, 60, 60, 60], [-60, -60, -60, -60], [0, 180, 180, 180],
                                  [-120, 180, 180, 180], [120, 180, 180, 180], [180, 146, 180, 180]])
def test_rotamer_labels_of_built_chains(oracle_mod, tors):
    s = W.alkane(torsions=tors)
    o = oracle_mod.Oracle(s)
    cv = o.cv(s.q0)
    for t in range(4):
        # the built torsion, and an independent formula on the built coordinates (angles mod 360)
        assert abs(((cv[t] - tors[t]) + 180.0) % 360.0 - 180.0) < 1e-9
        ref = _dihedral_projection(*s.q0[t:t + 4])
        assert abs(((cv[t] - ref) + 180.0) % 360.0 - 180.0) < 1e-9
    lab = o.state_of(s.q0)
    assert lab == _label(cv)


def test_labels_of_each_single_torsion_well(oracle_mod):
    """Moving one torsion through its three wells steps the label by 3^t."""
    for t in range(4):
        base = [180.0] * 4
        got = []
        for phi in (60.0, 180.0, -60.0):
            base[t] = phi
            got.append(oracle_mod.Oracle(W.alkane(torsions=base)).state_of(W.alkane(torsions=base).q0))
        assert got == [40 - 3 ** t, 40, 40 + 3 ** t]


def test_wells_tile_the_circle(oracle_mod):
    """On configurations along a trajectory exactly one of the 81 states is not exited, and it is the
    labelled state whenever the configuration is in a core."""
    s = W.alkane(temperature=300.0)
    o = oracle_mod.Oracle(s)
    R = 4
    q = np.repeat(s.q0[None], R, 0).copy()
    p = np.repeat(s.p0[None], R, 0).copy()
    f = np.stack([o.forces(q[r]) for r in range(R)])
    seen = set()
    for block in range(25):
        o.step_k(q, p, f, 11, block * 400, 0, 400, 0)
        for r in range(R):
            inside = [w for w in range(81) if not o.exited(q[r], w)]
            assert len(inside) == 1
            lab = o.state_of(q[r])
            seen.add(lab)
            if lab >= 0:
                assert inside == [lab]
    assert len(seen) >= 3  # the walkers visited several states (and the transient region)


def test_butane_trans_gauche_occupancy(oracle_mod):
    """Occupancy ratios of the three wells against the Boltzmann weights of the torsion potential."""
    import dataclasses

    s = dataclasses.replace(W.alkane(n_atoms=4, temperature=300.0), observables=[(W.OBS_DIHEDRAL, (0, 1, 2, 3))])
    o = oracle_mod.Oracle(s)
    R, k, t_gr = 48, 200_000, 50
    q = np.repeat(s.q0[None], R, 0).copy()
    p = np.stack([W.maxwell_boltzmann(s.mass, s.kT, 3, np.random.default_rng(100 + r)) for r in range(R)])
    f = np.stack([o.forces(q[r]) for r in range(R)])
    o.step_k(q, p, f, 5, 0, 0, 20_000, 0)  # equilibration
    samples = o.step_k(q, p, f, 5, 20_000, 0, k, t_gr, cap=k // t_gr)
    phi = np.degrees(samples[..., 0]).ravel()
    occ = np.array([np.mean((phi >= 0) & (phi < 120)), np.mean((phi >= 120) | (phi < -120)),
                    np.mean((phi >= -120) & (phi < 0))])
    # Boltzmann weights of V(phi) = sum_n k_n (1 + cos(n phi)) over each well
    grid = np.radians(np.linspace(-180, 180, 36001)[:-1] + 0.005)
    v = sum(kk * (1 + np.cos(nn * grid)) for nn, kk in zip(s.dihedral_n, s.dihedral_k))
    wgt = np.exp(-(v - v.min()) / s.kT)
    deg = np.degrees(grid)
    ref = np.array([wgt[(deg >= 0) & (deg < 120)].sum(), wgt[(deg >= 120) | (deg < -120)].sum(),
                    wgt[(deg >= -120) & (deg < 0)].sum()])
    ref /= ref.sum()
    # ~ 3 standard errors: ~1,000 well changes give sd(log odds of trans) ~ 0.1, sd(g+ - g-) ~ 0.03
    assert abs(math.log(occ[1] / (occ[0] + occ[2])) - math.log(ref[1] / (ref[0] + ref[2]))) < 0.3, (occ, ref)
    assert abs(occ[0] - occ[2]) < 0.1, occ  # mirror symmetry of gauche+ and gauche-
