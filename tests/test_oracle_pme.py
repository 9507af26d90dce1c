"""Pins of the oracle's periodic electrostatics: the plain Ewald sum and smooth particle mesh Ewald.

Pinned against facts that do not restate the oracle's formulas:
  * the Madelung constants of the rock-salt and caesium-chloride lattices (lattice energy per ion pair
    -M k_e q^2 / r_0, r_0 the nearest-neighbour distance; M = 1.747564595 and 1.762674773, tabulated
    e.g. by Kittel, Introduction to Solid State Physics, Ch. 3, and Glasser & Zucker, Theoretical
    Chemistry 5 (1980) 67, to more digits);
  * the total Ewald energy does not depend on the splitting parameter beta (the real-space,
    excluded-pair, self, reciprocal and background parts all change with it), also with a net charge;
  * excluding a pair removes exactly its nearest image's plain Coulomb energy k_e q_i q_j / r;
  * particle mesh Ewald tends to the Ewald sum as the grid and the B-spline order grow (Essmann et al.
    1995: the error falls with the grid spacing to the power of the order);
  * forces are minus the gradient of the energy (central differences);
  * invariances: the Ewald energy under any translation and a box-vector move of one atom; the mesh
    energy under a translation by whole grid spacings; Lennard-Jones through a face of the box equals
    the isolated pair's.
"""
import dataclasses
import itertools
import math

import numpy as np
import pytest

from paper_1807_02431_gb300 import workloads as W

NACL_M = 1.747564595
CSCL_M = 1.762674773
ORTHO = dict(edge=(2.6, 2.9, 2.45), grid=(16, 8, 32))  # an orthorhombic box with unequal grids
LIST_SHAPE = dict(n_chain=100, n_pairs=60, edge=4.0)  # the Verlet-list variant, 220 atoms


def _ions(pos, charges, box, mode, beta, cutoff, kmax=0, grid=(16, 16, 16), order=4, sigma=0.0, eps=0.0,
          excl=None):
    n = len(pos)
    s = W.System(name="ions", n_atoms=n, dim=3, potential=W.POT_FORCE_FIELD, mass=np.full(n, 20.0), kT=2.5,
                 gamma=1.0, dt=0.002, sigma=np.full(n, sigma), epsilon=np.full(n, eps),
                 charge=np.asarray(charges, float),
                 excl=np.zeros((0, 2), np.int32) if excl is None else np.asarray(excl, np.int32),
                 cutoff=cutoff, coulomb_k=W.COULOMB_K, coulomb_mode=mode, box=tuple(box), ewald_beta=beta,
                 pme_grid=tuple(grid), pme_order=order, ewald_kmax=kmax, cv_kind=W.CV_COM_DISTANCE,
                 cv_params=(1.0,), groups=[[0], [n - 1]], observables=[(W.OBS_POTENTIAL, ())])
    s.q0 = np.asarray(pos, float)
    s.p0 = np.zeros((n, 3))
    return s


def _kmax(beta, edge, digits=25.0):
    """Reciprocal vectors up to exp(-pi^2 k^2 / (beta L)^2) < e^-digits."""
    return int(math.ceil(math.sqrt(digits) * beta * edge / math.pi))


def _crystal(basis, charges, reps):
    pos = [np.add(c, b) for c in itertools.product(range(reps), repeat=3) for b in basis]
    return np.array(pos, float), np.tile(charges, reps ** 3)


@pytest.mark.parametrize("lattice", ["NaCl", "CsCl"])
def test_madelung_constants(oracle_mod, lattice):
    """2 x 2 x 2 conventional cells of edge 1 nm, unit charges, beta r_c = 5."""
    if lattice == "NaCl":
        basis = [(0, 0, 0), (.5, .5, 0), (.5, 0, .5), (0, .5, .5), (.5, 0, 0), (0, .5, 0), (0, 0, .5), (.5, .5, .5)]
        zs, r0, M = [1, 1, 1, 1, -1, -1, -1, -1], 0.5, NACL_M
    else:
        basis, zs, r0, M = [(0, 0, 0), (.5, .5, .5)], [1, -1], math.sqrt(3) / 2, CSCL_M
    pos, q = _crystal(basis, zs, 2)
    rc = 0.999
    beta = 5.0 / rc
    o = oracle_mod.Oracle(_ions(pos, q, (2, 2, 2), W.COULOMB_EWALD, beta, rc, kmax=_kmax(beta, 2.0)))
    e = o.potential(pos)
    assert -e / (len(pos) / 2 * W.COULOMB_K / r0) == pytest.approx(M, rel=1e-8)


@pytest.mark.parametrize("net", [0.0, 0.6])
def test_ewald_total_does_not_depend_on_beta(oracle_mod, net):
    s = W.chain_ions()
    q = s.q0
    charge = s.charge + net / s.n_atoms
    totals, selfs = [], []
    for brc in (4.5, 5.0, 5.5):
        beta = brc / s.cutoff
        e = dataclasses.replace(s, coulomb_mode=W.COULOMB_EWALD, ewald_beta=beta, ewald_kmax=_kmax(beta, s.box[0]),
                                charge=charge)
        parts = oracle_mod.Oracle(e).ewald_parts(q)
        totals.append(parts.sum())
        selfs.append(parts[2])
        if net:
            assert parts[4] < 0.0
    assert abs(selfs[2] / selfs[0] - 5.5 / 4.5) < 1e-12
    assert np.ptp(totals) < 1e-9 * abs(totals[0])


def test_excluding_a_pair_removes_its_coulomb(oracle_mod):
    s = W.chain_ions()
    q = s.q0
    beta = 4.5 / s.cutoff
    base = dataclasses.replace(s, coulomb_mode=W.COULOMB_EWALD, ewald_beta=beta, ewald_kmax=_kmax(beta, s.box[0]),
                               epsilon=np.zeros(s.n_atoms))
    i, j = 30, 41  # two ions; their nearest image
    d = q[i] - q[j]
    d -= np.asarray(s.box) * np.round(d / np.asarray(s.box))
    r = np.linalg.norm(d)
    assert r < s.cutoff
    ex = dataclasses.replace(base, excl=np.concatenate([base.excl, [[i, j]]]).astype(np.int32))
    e0 = oracle_mod.Oracle(base).potential(q)
    e1 = oracle_mod.Oracle(ex).potential(q)
    assert e1 - e0 == pytest.approx(-W.COULOMB_K * s.charge[i] * s.charge[j] / r, rel=1e-9)


@pytest.mark.parametrize("shape", [{}, ORTHO, LIST_SHAPE])
def test_mesh_tends_to_the_ewald_sum(oracle_mod, shape):
    s = W.chain_ions(**shape)
    q = s.q0
    beta = s.ewald_beta
    ew = oracle_mod.Oracle(dataclasses.replace(s, coulomb_mode=W.COULOMB_EWALD, ewald_kmax=_kmax(beta, max(s.box))))
    e_ref, f_ref = ew.ewald_parts(q)[3], ew.forces(q)
    errs = []
    for grid, order in ((16, 4), (32, 4), (32, 6), (48, 6)):
        g = tuple(int(round(grid * b / s.box[0])) for b in s.box)
        o = oracle_mod.Oracle(dataclasses.replace(s, pme_grid=g, pme_order=order))
        errs.append((abs(o.ewald_parts(q)[3] - e_ref) / abs(e_ref), np.abs(o.forces(q) - f_ref).max() / np.abs(f_ref).max()))
    for a, b in zip(errs, errs[1:]):
        assert b[0] < a[0] and b[1] < a[1]
    # the 4.0 nm box has a coarser mesh at the same point counts (0.25 nm spacing at 16 points against
    # 0.16 nm; measured 1.0e-2 / 1.3e-2 at 16^3, order 4, and 6e-7 / 2.8e-6 at 48^3, order 6)
    coarse, fine = (2e-2, 5e-6) if shape is LIST_SHAPE else (1e-2, 1e-6)
    assert errs[0][0] < coarse and errs[0][1] < coarse
    assert errs[-1][0] < fine and errs[-1][1] < fine


@pytest.mark.parametrize("mode", [W.COULOMB_PME, W.COULOMB_EWALD])
@pytest.mark.parametrize("shape", [{}, ORTHO])
def test_forces_are_minus_the_gradient(oracle_mod, mode, shape):
    s = W.chain_ions(**shape)
    s = dataclasses.replace(s, coulomb_mode=mode, ewald_kmax=_kmax(s.ewald_beta, s.box[0], 16.0))
    o = oracle_mod.Oracle(s)
    rng = np.random.default_rng(5)
    q = s.q0 + 0.01 * rng.standard_normal(s.q0.shape)
    f = o.forces(q)
    h = 1e-5
    for a in (0, 11, 21, 22, 45, 61):
        for x in range(3):
            qp, qm = q.copy(), q.copy()
            qp[a, x] += h
            qm[a, x] -= h
            fd = -(o.potential(qp) - o.potential(qm)) / (2 * h)
            assert fd == pytest.approx(f[a, x], abs=2e-6 * np.abs(f).max())


def test_invariances(oracle_mod):
    s = W.chain_ions()
    q = s.q0
    L = np.asarray(s.box)
    ew = oracle_mod.Oracle(dataclasses.replace(s, coulomb_mode=W.COULOMB_EWALD, ewald_kmax=_kmax(s.ewald_beta, L[0])))
    pm = oracle_mod.Oracle(s)
    e_ew, e_pm = ew.potential(q), pm.potential(q)
    shift = np.array([0.3137, -0.771, 1.9])
    assert ew.potential(q + shift) == pytest.approx(e_ew, rel=1e-11)
    moved = q.copy()
    moved[40] += L * np.array([1, -2, 1])
    assert ew.potential(moved) == pytest.approx(e_ew, rel=1e-11)
    assert pm.potential(moved) == pytest.approx(e_pm, rel=1e-11)
    h = L / np.asarray(s.pme_grid)
    assert pm.potential(q + h * np.array([1, 3, -2])) == pytest.approx(e_pm, rel=1e-11)
    # a translation by a fraction of a grid spacing changes the mesh energy within its error only
    assert pm.potential(q + 0.37 * h) == pytest.approx(e_pm, rel=1e-3)


def test_lennard_jones_through_a_face(oracle_mod):
    """Two uncharged atoms 0.1 nm inside opposite faces are 0.2 nm apart through the face."""
    edge, sig, eps = 2.0, 0.25, 0.7
    pos = np.array([[-0.9, 0.1, 0.0], [0.9, 0.1, 0.0]])
    s = _ions(pos, [0.0, 0.0], (edge, edge, edge), W.COULOMB_PME, 3.0, 0.9, sigma=sig, eps=eps)
    o = oracle_mod.Oracle(s)
    sr6 = (sig / 0.2) ** 6
    assert o.potential(pos) == pytest.approx(4 * eps * (sr6 * sr6 - sr6), rel=1e-12)
    f = o.forces(pos)
    g = 24 * eps * (2 * sr6 * sr6 - sr6) / 0.2  # repulsive: atom 0 moves away from atom 1's image at x = -1.1
    assert f[0, 0] == pytest.approx(g, rel=1e-10) and f[1, 0] == pytest.approx(-g, rel=1e-10)


@pytest.mark.parametrize("shape", [{}, ORTHO, LIST_SHAPE])
def test_chain_ions_recipe(shape):
    """The periodic workload as documented: neutral, every ion at least 0.3 nm (minimum image) from
    every other atom, erfc(beta r_c) = 1e-5, the cutoff within half the shortest edge; the Verlet-list
    variant (64 atoms or more) also keeps cutoff + skin (7/6 of the cutoff) within half the shortest
    edge, and no chain bead comes within 0.25 nm of another bead's periodic image."""
    s = W.chain_ions(**shape)
    box = np.asarray(s.box)
    assert abs(s.charge.sum()) < 1e-12
    assert math.erfc(s.ewald_beta * s.cutoff) == pytest.approx(1e-5, rel=1e-9)
    assert s.cutoff <= 0.5 * box.min()
    n_chain = shape.get("n_chain", 22)
    assert s.n_atoms == n_chain + 2 * shape.get("n_pairs", 20)
    if s.n_atoms >= 64:
        assert 7.0 / 6.0 * s.cutoff <= 0.5 * box.min()
        dc = s.q0[:n_chain, None] - s.q0[None, :n_chain]
        dc -= box * np.round(dc / box)
        iu = np.triu_indices(n_chain, 3)
        assert np.linalg.norm(dc, axis=-1)[iu].min() >= 0.25
    d = s.q0[n_chain:, None] - s.q0[None]
    d -= box * np.round(d / box)
    r = np.linalg.norm(d, axis=-1)
    r[np.arange(s.n_atoms - n_chain), n_chain + np.arange(s.n_atoms - n_chain)] = np.inf  # self
    assert r.min() >= 0.3 - 1e-12
