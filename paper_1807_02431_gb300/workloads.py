"""Seeded synthetic workloads shaped like the paper's systems.

This module is shared by the CUDA binding, the oracle, the tests and the benchmark.  It holds none
of the method's arithmetic: it only builds geometries (a chain from internal coordinates) and draws
force-field parameters, initial momenta and system sizes from seeded numpy generators.

Systems (stand-ins for the paper's workloads, whose force fields and structures are not available):
  * ``double_well_2d``  - one particle in V(x, y) = 5 (x^2 - 1)^2 + 2.5 y^2 (dimensionless, kT = 1),
    two states = the cores |x| > 0.3 of the two basins; used for the brute-force exit-time check.
  * ``chain``           - a 22-bead (or n-bead) peptide-like chain shaped like alanine dipeptide
    (Section 4.1): harmonic bonds and angles, periodic dihedrals, LJ + Coulomb with eps = 4r; the
    two states are the paper's (phi, psi) rectangle and its complement.
  * ``batched_chains``  - independent chains of uneven sizes for the batched path.
  * ``alkane``          - a united-atom n-alkane whose backbone torsions have three rotamer wells:
    3^(n-3) disjoint states (all torsions in their well cores) separated by a transient region, the
    many-state, non-partition case of Section 2.4.1's transient propagation.
  * ``chain_ions``      - the chain with ion pairs in a periodic box, electrostatics by particle
    mesh Ewald.
  * ``ligand_receptor`` - a packed-globule receptor with an elastic network and a short ligand chain
    in a surface pocket, shaped like the FKBP-DMSO dissociation problem (Section 4.2).

Units for the particle systems: nm, ps, amu, kJ/mol, elementary charge.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

KB_KJ_PER_MOL_K = 0.0083144626
COULOMB_K = 138.935458  # kJ mol^-1 nm e^-2

POT_DOUBLE_WELL_2D = 0
POT_FORCE_FIELD = 1

CV_DOUBLE_WELL = 0
CV_DIHEDRAL_RECT = 1
CV_COM_DISTANCE = 2
CV_ROTAMERS = 3

COULOMB_EPS4R = 0
COULOMB_REACTION_FIELD = 1
COULOMB_PME = 2     # periodic box, smooth particle mesh Ewald
COULOMB_EWALD = 3   # periodic box, plain Ewald sum over reciprocal vectors (oracle only)

OBS_COORD = 0
OBS_POTENTIAL = 1
OBS_KINETIC = 2
OBS_DIHEDRAL = 3
OBS_GROUP_DISTANCE = 4
OBS_RMS_VELOCITY = 5


@dataclasses.dataclass
class System:
    name: str
    n_atoms: int
    dim: int
    potential: int
    mass: np.ndarray
    kT: float
    gamma: float
    dt: float
    dw_a: float = 0.0
    dw_b: float = 0.0
    sigma: np.ndarray | None = None
    epsilon: np.ndarray | None = None
    charge: np.ndarray | None = None
    excl: np.ndarray | None = None          # [m, 2] int32
    cutoff: float = 0.0
    coulomb_k: float = 0.0
    coulomb_mode: int = COULOMB_EPS4R       # or COULOMB_REACTION_FIELD (needs a cutoff)
    rf_dielectric: float = 78.3             # eps_rf of the reaction field; 0 = conductor
    gb_radius: np.ndarray | None = None     # Generalized Born (OBC II) intrinsic radii, nm; None = off
    gb_scale: np.ndarray | None = None      # descreening scale factors S_i
    gb_solute_dielectric: float = 1.0
    gb_solvent_dielectric: float = 78.5
    constraints: np.ndarray | None = None   # [m, 2] atom pairs of fixed bond length
    constraint_length: np.ndarray | None = None
    constraint_tol: float = 1e-10           # relative tolerance of SHAKE / RATTLE
    constraint_max_iter: int = 1000
    box: tuple | None = None                # periodic box edges (nm) of the Ewald modes
    ewald_beta: float = 0.0                 # splitting parameter, nm^-1
    pme_grid: tuple = (16, 16, 16)          # PME grid points per axis
    pme_order: int = 4                      # B-spline order
    ewald_kmax: int = 8                     # plain Ewald: |k_d| <= kmax
    bonds: np.ndarray | None = None         # [nb, 2]
    bond_k: np.ndarray | None = None
    bond_r0: np.ndarray | None = None
    angles: np.ndarray | None = None        # [na, 3]
    angle_k: np.ndarray | None = None
    angle_theta0: np.ndarray | None = None
    dihedrals: np.ndarray | None = None     # [nd, 4]
    dihedral_n: np.ndarray | None = None
    dihedral_k: np.ndarray | None = None
    dihedral_delta: np.ndarray | None = None
    cv_kind: int = CV_DOUBLE_WELL
    cv_atoms: tuple = ()
    cv_params: tuple = ()
    groups: list = dataclasses.field(default_factory=list)
    observables: list = dataclasses.field(default_factory=list)  # (kind, (args...))
    q0: np.ndarray | None = None            # [n, dim]
    p0: np.ndarray | None = None            # [n, dim]
    # Gen. ParRep parameters (Sections 2.4.1 and 3.4)
    n_replicas: int = 32
    t_gr: int = 10
    t_check: int = 100
    tol: float = 0.01
    min_fv_steps: int = 0

    def empty_arrays(self):
        """Return zero-length arrays for the force-field fields a system does not use."""
        z_i2 = np.zeros((0, 2), np.int32)
        out = {}
        out["sigma"] = self.sigma if self.sigma is not None else np.zeros(self.n_atoms)
        out["epsilon"] = self.epsilon if self.epsilon is not None else np.zeros(self.n_atoms)
        out["charge"] = self.charge if self.charge is not None else np.zeros(self.n_atoms)
        out["excl"] = self.excl if self.excl is not None else z_i2
        out["bonds"] = self.bonds if self.bonds is not None else z_i2
        out["bond_k"] = self.bond_k if self.bond_k is not None else np.zeros(0)
        out["bond_r0"] = self.bond_r0 if self.bond_r0 is not None else np.zeros(0)
        out["angles"] = self.angles if self.angles is not None else np.zeros((0, 3), np.int32)
        out["angle_k"] = self.angle_k if self.angle_k is not None else np.zeros(0)
        out["angle_theta0"] = self.angle_theta0 if self.angle_theta0 is not None else np.zeros(0)
        out["dihedrals"] = self.dihedrals if self.dihedrals is not None else np.zeros((0, 4), np.int32)
        out["dihedral_n"] = self.dihedral_n if self.dihedral_n is not None else np.zeros(0, np.int32)
        out["dihedral_k"] = self.dihedral_k if self.dihedral_k is not None else np.zeros(0)
        out["dihedral_delta"] = self.dihedral_delta if self.dihedral_delta is not None else np.zeros(0)
        return out


def maxwell_boltzmann(mass: np.ndarray, kT: float, dim: int, rng: np.random.Generator) -> np.ndarray:
    """Momenta p_i ~ N(0, m_i kT) per component."""
    return rng.standard_normal((mass.shape[0], dim)) * np.sqrt(mass * kT)[:, None]


def double_well_2d(seed: int = 2431, n_replicas: int = 32) -> System:
    """One particle, V = 5 (x^2-1)^2 + 2.5 y^2, kT = 1, m = 1, gamma = 1, dt = 1e-3, q0 = (-1, 0)."""
    rng = np.random.default_rng(seed)
    mass = np.ones(1)
    s = System(
        name="double_well_2d", n_atoms=1, dim=2, potential=POT_DOUBLE_WELL_2D, mass=mass,
        kT=1.0, gamma=1.0, dt=1e-3, dw_a=5.0, dw_b=2.5,
        cv_kind=CV_DOUBLE_WELL, cv_params=(0.3,),
        observables=[(OBS_COORD, (0, 0)), (OBS_POTENTIAL, ())],
        n_replicas=n_replicas, t_gr=10, t_check=100, tol=0.01, min_fv_steps=2000,
    )
    s.q0 = np.array([[-1.0, 0.0]])
    s.p0 = maxwell_boltzmann(mass, s.kT, 2, rng)
    return s


def _place(a, b, c, bond, angle, torsion):
    """Natural-extension reference frame: the point d with |cd| = bond, angle(b, c, d) = angle and
    dihedral(a, b, c, d) = torsion (radians)."""
    bc = c - b
    bc /= np.linalg.norm(bc)
    n = np.cross(b - a, bc)
    n /= np.linalg.norm(n)
    m = np.cross(n, bc)
    d2 = np.array([-bond * math.cos(angle),
                   bond * math.sin(angle) * math.cos(torsion),
                   bond * math.sin(angle) * math.sin(torsion)])
    return c + d2[0] * bc + d2[1] * m + d2[2] * n


def _grow_chain(n, bond, angle, sigma, rng, fixed):
    """Place beads one by one from internal coordinates: torsions drawn 70 % trans (180 +- 20 deg),
    30 % gauche (+-65 +- 10 deg), except the `fixed` ones; a bead closer than 0.8 sigma_ij to any
    earlier bead (|i - j| >= 3) has its torsion redrawn, and the chain restarts after 100 failures."""
    while True:
        x = np.zeros((n, 3))
        x[1] = [bond, 0.0, 0.0]
        if n > 2:
            x[2] = x[1] + bond * np.array([-math.cos(angle), math.sin(angle), 0.0])
        ok = True
        for i in range(3, n):
            t = i - 3
            for _attempt in range(100):
                if t in fixed:
                    tor = fixed[t]
                elif rng.random() < 0.7:
                    tor = math.radians(180.0 + rng.uniform(-20.0, 20.0))
                else:
                    tor = math.radians(rng.choice([-65.0, 65.0]) + rng.uniform(-10.0, 10.0))
                xi = _place(x[i - 3], x[i - 2], x[i - 1], bond, angle, tor)
                d = np.linalg.norm(x[: i - 2] - xi, axis=1)
                if np.all(d >= 0.8 * 0.5 * (sigma[: i - 2] + sigma[i])):
                    x[i] = xi
                    break
            else:
                ok = False
                break
        if ok:
            return x


def _chain_geometry(n, bond, angle, torsions):
    x = np.zeros((n, 3))
    x[1] = [bond, 0.0, 0.0]
    x[2] = x[1] + bond * np.array([-math.cos(angle), math.sin(angle), 0.0])
    for i in range(3, n):
        x[i] = _place(x[i - 3], x[i - 2], x[i - 1], bond, angle, torsions[i - 3])
    return x


def chain(n_atoms: int = 22, seed: int = 1807, dyn_seed: int = 2431, n_replicas: int = 256,
          temperature: float = 300.0, dihedral_terms: str = "triple") -> System:
    """Peptide-like bead chain shaped like alanine dipeptide (Section 4.1 stand-in).

    Bonds k = 3e5 kJ/mol/nm^2, r0 = 0.15 nm; angles k = 400 kJ/mol/rad^2, theta0 = 110 deg; each
    dihedral (i, i+1, i+2, i+3) has terms n = 1, 2, 3 with k ~ U[0, 8] kJ/mol, delta in {0, pi};
    LJ sigma ~ U[0.25, 0.35] nm, eps ~ U[0.2, 0.8] kJ/mol (Lorentz-Berthelot); charges ~ N(0, 0.3)
    shifted to zero net; Coulomb with eps = 4r; 1-2 and 1-3 pairs excluded; no cutoff; mass 12 amu;
    gamma = 1/ps, dt = 2 fs.  States: phi = dihedral(c-2, c-1, c, c+1), psi = dihedral(c-1, c, c+1,
    c+2) around the central bead c = n//2 - 1 (beads 9..13 for n = 22); state 0 is the paper's
    rectangle phi in [0, 120], psi in [-170, 0] (degrees), state 1 its complement.  The initial
    central angles are the paper's starting point (phi, psi) = (-81, 70) degrees, in state 1.
    """
    rng = np.random.default_rng(seed)
    n = n_atoms
    mass = np.full(n, 12.0)
    sigma = rng.uniform(0.25, 0.35, n)
    epsilon = rng.uniform(0.2, 0.8, n)
    charge = rng.normal(0.0, 0.3, n)
    charge -= charge.mean()
    bonds = np.array([[i, i + 1] for i in range(n - 1)], np.int32)
    angles = np.array([[i, i + 1, i + 2] for i in range(n - 2)], np.int32)
    dih, dn, dk, dd = [], [], [], []
    for i in range(n - 3):
        if dihedral_terms == "triple":  # terms n = 1, 2, 3, each with its own k
            mults = (1, 2, 3)
        else:  # "single": one term whose multiplicity is drawn from 1..3
            mults = (int(rng.integers(1, 4)),)
        for mult in mults:
            dih.append([i, i + 1, i + 2, i + 3])
            dn.append(mult)
            dk.append(rng.uniform(0.0, 8.0))
            dd.append(math.pi * rng.integers(0, 2))
    excl = np.array([[i, j] for i in range(n) for j in range(i + 1, min(n, i + 3))], np.int32)
    c = n // 2 - 1
    phi_idx, psi_idx = c - 2, c - 1  # torsion index t describes dihedral (t, t+1, t+2, t+3)
    bond, angle = 0.15, math.radians(110.0)
    x = _grow_chain(n, bond, angle, sigma, rng, {phi_idx: math.radians(-81.0), psi_idx: math.radians(70.0)})
    x -= x.mean(axis=0)
    kT = KB_KJ_PER_MOL_K * temperature
    s = System(
        name=f"chain{n}", n_atoms=n, dim=3, potential=POT_FORCE_FIELD, mass=mass,
        kT=kT, gamma=1.0, dt=0.002, sigma=sigma, epsilon=epsilon, charge=charge, excl=excl,
        cutoff=0.0, coulomb_k=COULOMB_K,
        bonds=bonds, bond_k=np.full(n - 1, 3.0e5), bond_r0=np.full(n - 1, bond),
        angles=angles, angle_k=np.full(n - 2, 400.0), angle_theta0=np.full(n - 2, angle),
        dihedrals=np.array(dih, np.int32).reshape(-1, 4), dihedral_n=np.array(dn, np.int32),
        dihedral_k=np.array(dk), dihedral_delta=np.array(dd),
        cv_kind=CV_DIHEDRAL_RECT, cv_atoms=(c - 2, c - 1, c, c + 1, c + 2),
        cv_params=(0.0, 120.0, -170.0, 0.0),
        observables=[(OBS_POTENTIAL, ()), (OBS_KINETIC, ()),
                     (OBS_DIHEDRAL, (c - 2, c - 1, c, c + 1)),
                     (OBS_DIHEDRAL, (c - 1, c, c + 1, c + 2))],
        n_replicas=n_replicas, t_gr=10, t_check=500, tol=0.01, min_fv_steps=0,
    )
    s.q0 = x
    s.p0 = maxwell_boltzmann(mass, kT, 3, np.random.default_rng(dyn_seed))
    return s


def alkane(n_atoms: int = 7, dyn_seed: int = 2431, n_replicas: int = 32, temperature: float = 250.0,
           core_half_width: float = 35.0, torsions=None) -> System:
    """United-atom n-alkane with rotamer states (a many-state stand-in; no dataset of the paper).

    Beads of 14 amu along a chain; bonds k = 3e5 kJ/mol/nm^2, r0 = 0.154 nm; angles k = 520
    kJ/mol/rad^2, theta0 = 114 deg; each backbone torsion V(phi) = 1/2 V1 (1 + cos phi) + 1/2 V2
    (1 - cos 2 phi) + 1/2 V3 (1 + cos 3 phi) with (V1, V2, V3) = (5.9046, -1.1339, 13.1606) kJ/mol
    (trans at 180 deg, gauche wells at +-60 deg, 3.6 kJ/mol above trans, barriers 10-14 kJ/mol),
    written as terms k (1 + cos(n phi - delta)) up to a constant: (n, k, delta) = (1, V1/2, 0),
    (2, |V2|/2, 0), (3, V3/2, 0); LJ sigma = 0.395 nm, eps = 0.382 kJ/mol between beads four or more
    bonds apart (1-2, 1-3 and 1-4 pairs excluded); no charges, no cutoff; gamma = 1/ps, dt = 2 fs.
    States: the rotamer wells of the n-3 torsions (gauche+ [0, 120), trans, gauche- [-120, 0)
    degrees); a configuration is in state sum_t well_t 3^t when every torsion is within
    `core_half_width` degrees of its well's centre, and leaves it when a torsion changes well.  The
    initial chain is all-trans (or has the given torsions, degrees).  Observables for the
    Gelman-Rubin test: the potential energy and the end-to-end distance, TOL = 0.05, at least 1,000
    F-V steps.  At 250 K a state lasts ~10^4 steps and the convergence step needs ~8 x 10^3, so
    about 40 % of the visits end in a parallel step (at 300 K with TOL = 0.01 the reference walker
    leaves before convergence in most visits)."""
    n = n_atoms
    if not 4 <= n <= 7:
        raise ValueError("the rotamer state index covers 1 to 4 torsions (4 to 7 beads)")
    m = n - 3
    mass = np.full(n, 14.0)
    sigma = np.full(n, 0.395)
    epsilon = np.full(n, 0.382)
    bonds = np.array([[i, i + 1] for i in range(n - 1)], np.int32)
    angles = np.array([[i, i + 1, i + 2] for i in range(n - 2)], np.int32)
    v1, v2, v3 = 5.9046, -1.1339, 13.1606
    dih, dn, dk, dd = [], [], [], []
    for i in range(m):
        for mult, k in ((1, v1 / 2), (2, abs(v2) / 2), (3, v3 / 2)):
            dih.append([i, i + 1, i + 2, i + 3])
            dn.append(mult)
            dk.append(k)
            dd.append(0.0)
    excl = np.array([[i, j] for i in range(n) for j in range(i + 1, min(n, i + 4))], np.int32)
    bond, angle = 0.154, math.radians(114.0)
    tors = [180.0] * m if torsions is None else list(torsions)
    x = _chain_geometry(n, bond, angle, [math.radians(t) for t in tors])
    x -= x.mean(axis=0)
    kT = KB_KJ_PER_MOL_K * temperature
    s = System(
        name=f"alkane{n}", n_atoms=n, dim=3, potential=POT_FORCE_FIELD, mass=mass,
        kT=kT, gamma=1.0, dt=0.002, sigma=sigma, epsilon=epsilon, charge=np.zeros(n), excl=excl,
        cutoff=0.0, coulomb_k=COULOMB_K,
        bonds=bonds, bond_k=np.full(n - 1, 3.0e5), bond_r0=np.full(n - 1, bond),
        angles=angles, angle_k=np.full(n - 2, 520.0), angle_theta0=np.full(n - 2, angle),
        dihedrals=np.array(dih, np.int32).reshape(-1, 4), dihedral_n=np.array(dn, np.int32),
        dihedral_k=np.array(dk), dihedral_delta=np.array(dd),
        cv_kind=CV_ROTAMERS, cv_atoms=tuple(range(n)), cv_params=(float(m), float(core_half_width)),
        groups=[[0], [n - 1]],
        observables=[(OBS_POTENTIAL, ()), (OBS_GROUP_DISTANCE, (0, 1))],
        n_replicas=n_replicas, t_gr=10, t_check=100, tol=0.05, min_fv_steps=1000,
    )
    s.q0 = x
    s.p0 = maxwell_boltzmann(mass, kT, 3, np.random.default_rng(dyn_seed))
    return s


def solvated(s: System, seed: int = 77) -> System:
    """A copy of a force-field system in Generalized Born implicit solvent (OBC II, as the paper's
    protein-ligand setup, Section 4.2): intrinsic radii 0.55 sigma_i (0.14-0.19 nm for the chain's
    beads), descreening scales ~ U[0.72, 0.85] (the range of the usual carbon to oxygen values),
    solute and solvent dielectric constants 1 and 78.5."""
    rng = np.random.default_rng(seed)
    out = dataclasses.replace(s, name=s.name + "_gb", gb_radius=0.55 * np.asarray(s.sigma, float),
                              gb_scale=rng.uniform(0.72, 0.85, s.n_atoms), gb_solute_dielectric=1.0,
                              gb_solvent_dielectric=78.5)
    out.q0, out.p0 = s.q0, s.p0
    return out


def chain_h(n_heavy: int = 22, seed: int = 1807, dyn_seed: int = 2431, n_replicas: int = 256) -> System:
    """The peptide-like chain with one hydrogen (1.008 amu) on every bead, its bond of 0.109 nm held
    fixed by a constraint (as the paper's setups constrain the bonds of hydrogens, Section 4): 2 x 22
    atoms.  Each hydrogen carries 0.1 e taken from its bead's charge, LJ sigma 0.25 nm and eps 0.1
    kJ/mol, angles H-C-C of k = 300 kJ/mol/rad^2 and 109.5 deg with each neighbour of its bead; 1-2 and
    1-3 pairs through the hydrogens excluded.  Hydrogens are placed opposite the bisector of their
    bead's neighbours.  States, observables and the Gen. ParRep parameters are the chain's."""
    base = chain(n_atoms=n_heavy, seed=seed, dyn_seed=dyn_seed, n_replicas=n_replicas)
    nh = n_heavy
    x = base.q0
    hpos = np.zeros((nh, 3))
    for i in range(nh):
        nb = [k for k in (i - 1, i + 1) if 0 <= k < nh]
        if len(nb) == 2:  # opposite the bisector of the two bonds
            u = sum((x[i] - x[k]) / np.linalg.norm(x[i] - x[k]) for k in nb)
        else:  # an end bead: 109.5 deg from its one bond, in the plane of the next bond
            b = (x[nb[0]] - x[i]) / np.linalg.norm(x[nb[0]] - x[i])
            other = x[nb[0] + (1 if nb[0] > i else -1)] - x[nb[0]]
            perp = other - np.dot(other, b) * b
            perp /= np.linalg.norm(perp)
            u = math.cos(math.radians(109.5)) * b - math.sin(math.radians(109.5)) * perp
        hpos[i] = x[i] + 0.109 * u / np.linalg.norm(u)
    n = 2 * nh
    mass = np.concatenate([base.mass, np.full(nh, 1.008)])
    charge = np.concatenate([base.charge - 0.1, np.full(nh, 0.1)])
    sigma = np.concatenate([base.sigma, np.full(nh, 0.25)])
    epsilon = np.concatenate([base.epsilon, np.full(nh, 0.1)])
    angles = [list(a) for a in base.angles]
    angle_k = list(base.angle_k)
    angle_t0 = list(base.angle_theta0)
    excl = {tuple(e) for e in base.excl.tolist()}
    for i in range(nh):
        h = nh + i
        excl.add((i, h))
        for k in (i - 1, i + 1):
            if 0 <= k < nh:
                angles.append([h, i, k])
                angle_k.append(300.0)
                angle_t0.append(math.radians(109.5))
                excl.add((min(k, h), max(k, h)))
    excl = np.array(sorted(excl), np.int32)
    s = dataclasses.replace(
        base, name=f"chain{nh}h", n_atoms=n, mass=mass, charge=charge, sigma=sigma, epsilon=epsilon,
        excl=excl, angles=np.array(angles, np.int32), angle_k=np.array(angle_k), angle_theta0=np.array(angle_t0),
        constraints=np.array([[i, nh + i] for i in range(nh)], np.int32), constraint_length=np.full(nh, 0.109))
    s.q0 = np.concatenate([x, hpos])
    s.p0 = maxwell_boltzmann(mass, s.kT, 3, np.random.default_rng(dyn_seed))
    return s


def chain_ions(n_pairs: int = 20, edge=2.6, seed: int = 1807, dyn_seed: int = 2431,
               n_replicas: int = 256, grid=16, order: int = 4, ewald_rtol: float = 1e-5,
               n_chain: int = 22) -> System:
    """The `n_chain`-bead chain (22 by default) with `n_pairs` ion pairs in a periodic box of edge `edge`
    nm (or edges), its electrostatics summed over all periodic images by particle mesh Ewald (an
    optimisation the paper expects of an MD engine, Section 3.2): 62 atoms for 20 pairs; 220 atoms for
    the 100-bead chain with 60 pairs in a 4.0 nm box (a system of 64 atoms or more keeps Verlet lists
    over nearest images).  Ions of 20 amu, LJ sigma 0.3 nm and
    eps 0.5 kJ/mol, charges +-0.3 e, placed uniformly at least 0.3 nm from every atom placed before;
    plain Coulomb (eps = 1) with real-space cutoff 1.2 nm, beta such that erfc(beta r_c) = ewald_rtol
    (2.6 nm^-1 for 1e-5, the usual MD setting), a grid x grid x grid mesh (0.16 nm spacing for 16) and
    B-splines of order `order`; Lennard-Jones cut at the same distance over minimum images.  States,
    observables and the Gen. ParRep parameters are the chain's."""
    base = chain(n_atoms=n_chain, seed=seed, dyn_seed=dyn_seed, n_replicas=n_replicas)
    rng = np.random.default_rng(seed + 7)
    box = np.broadcast_to(np.asarray(edge, float), 3)
    grid = tuple(int(g) for g in np.broadcast_to(grid, 3))
    x = [v for v in base.q0]
    ions = []
    while len(ions) < 2 * n_pairs:
        cand = rng.uniform(-0.5 * box, 0.5 * box)
        d = np.asarray(x) - cand
        d -= box * np.round(d / box)
        if np.min(np.linalg.norm(d, axis=1)) >= 0.3:
            x.append(cand)
            ions.append(cand)
    n = base.n_atoms + 2 * n_pairs
    ni = 2 * n_pairs
    cutoff = 1.2
    beta = _erfc_inverse(ewald_rtol) / cutoff
    mass = np.concatenate([base.mass, np.full(ni, 20.0)])
    s = dataclasses.replace(
        base, name=f"chain{base.n_atoms}_ions{ni}", n_atoms=n, mass=mass,
        charge=np.concatenate([base.charge, np.tile([0.3, -0.3], n_pairs)]),
        sigma=np.concatenate([base.sigma, np.full(ni, 0.3)]),
        epsilon=np.concatenate([base.epsilon, np.full(ni, 0.5)]),
        cutoff=cutoff, coulomb_mode=COULOMB_PME, box=tuple(float(b) for b in box), ewald_beta=beta,
        pme_grid=grid, pme_order=order, ewald_kmax=int(math.ceil(3.5 * beta * box.max() / math.pi)))
    s.q0 = np.asarray(x)
    s.p0 = maxwell_boltzmann(mass, s.kT, 3, np.random.default_rng(dyn_seed))
    return s


def _erfc_inverse(y: float) -> float:
    """x with erfc(x) = y (bisection; 0 < y < 1)."""
    lo, hi = 0.0, 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if math.erfc(mid) > y else (lo, mid)
    return 0.5 * (lo + hi)


def _kd_order(x, leaf=32):
    """Order of points by recursive bisection along the longest extent, each cut at a multiple of
    `leaf` points, so that every consecutive block of `leaf` points is spatially compact."""
    idx = np.arange(len(x))

    def rec(ids):
        if len(ids) <= leaf:
            return [ids]
        ext = x[ids].max(axis=0) - x[ids].min(axis=0)
        ax = int(np.argmax(ext))
        srt = ids[np.argsort(x[ids, ax], kind="stable")]
        cut = max(leaf, (len(ids) // (2 * leaf)) * leaf)
        return rec(srt[:cut]) + rec(srt[cut:])

    return np.concatenate(rec(idx))


def ligand_receptor(n_receptor: int = 2000, n_ligand: int = 30, seed: int = 1807, dyn_seed: int = 2431,
                    n_replicas: int = 1024, temperature: float = 300.0) -> System:
    """Ligand bound in a surface pocket of a packed globule (Section 4.2 stand-in, FKBP-DMSO shaped).

    Receptor: n_receptor beads at density 7.7 nm^-3 (a jittered cubic lattice of spacing 0.506 nm,
    jitter U[-0.05, 0.05] nm per axis) filling a sphere (radius 3.96 nm for 2,000 beads) from which a
    pocket of radius 0.9 nm centred 0.5 nm below the surface is carved; beads are held by an elastic
    network: a harmonic spring k = 500 kJ/mol/nm^2 with r0 = the generated distance between every pair
    closer than 0.9 nm (those pairs are excluded from the nonbonded terms).  Beads are numbered by
    recursive bisection, so every block of 32 consecutive beads is spatially compact.
    Ligand: an n_ligand-bead chain grown inside the pocket (bond 0.15 nm, k = 3e5; angle 110 deg,
    k = 400; one dihedral term per torsion with n ~ U{1,2,3}, k ~ U[0, 8] kJ/mol, delta in {0, pi};
    1-2 and 1-3 pairs excluded), numbered after the receptor.
    Both: LJ sigma ~ U[0.25, 0.35] nm, eps ~ U[0.2, 0.8] kJ/mol (Lorentz-Berthelot); charges
    N(0, 0.2) (receptor) and N(0, 0.3) (ligand) shifted to zero net; Coulomb with eps = 4r; plain
    truncation of LJ and Coulomb at 1.2 nm; mass 12 amu; gamma = 1/ps; dt = 2 fs.
    Groups: 0 = ligand, 1 = pocket (receptor beads within 1.5 nm of the pocket centre), 2 = first and
    3 = last ligand bead.  States: d = |COM(ligand) - COM(pocket)|; state 0 = bound (d < 1.0 nm),
    state 1 = its complement.  Observables (sampled every 50 steps): d, the ligand's RMS velocity and
    the distances of the two ligand ends to the pocket.
    """
    rng = np.random.default_rng(seed)
    rho, a = 7.7, 0.506
    rg = (3.0 * n_receptor / (4.0 * math.pi * rho)) ** (1.0 / 3.0)
    cp = np.array([0.0, 0.0, rg - 0.5])
    rp = 0.9
    m = int(math.ceil((rg + 1.5) / a))
    g = np.arange(-m, m + 1)
    ijk = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    x = ijk * a + rng.uniform(-0.05, 0.05, ijk.shape)
    keep = np.linalg.norm(x - cp, axis=1) >= rp
    ijk, x = ijk[keep], x[keep]
    order = np.argsort(np.linalg.norm(x, axis=1), kind="stable")[:n_receptor]
    ijk, x = ijk[order], x[order]
    xr = x[_kd_order(x)]
    nl = n_ligand
    n = n_receptor + nl
    sigma = rng.uniform(0.25, 0.35, n)
    epsilon = rng.uniform(0.2, 0.8, n)
    charge = np.concatenate([rng.normal(0.0, 0.2, n_receptor), rng.normal(0.0, 0.3, nl)])
    charge -= charge.mean()
    # elastic network
    d = np.linalg.norm(xr[:, None] - xr[None], axis=-1)
    iu, ju = np.nonzero(np.triu(d < 0.9, 1))
    enm = np.stack([iu, ju], 1).astype(np.int32)
    enm_r0 = d[iu, ju]
    # ligand chain grown inside the pocket
    bond, angle = 0.15, math.radians(110.0)
    sl = sigma[n_receptor:]

    def clash_free(p, i, xl):
        dr = np.linalg.norm(xr - p, axis=1)
        if np.any(dr < 0.8 * 0.5 * (sigma[:n_receptor] + sl[i])):
            return False
        if i >= 3 and np.any(np.linalg.norm(xl[: i - 2] - p, axis=1) < 0.8 * 0.5 * (sl[: i - 2] + sl[i])):
            return False
        return np.linalg.norm(p - cp) <= rp - 0.15

    for _restart in range(1000):
        xl = np.zeros((nl, 3))
        xl[0] = cp
        u = rng.standard_normal(3)
        xl[1] = cp + bond * u / np.linalg.norm(u)
        v = np.cross(u, rng.standard_normal(3))
        v /= np.linalg.norm(v)
        b01 = (xl[1] - xl[0]) / bond
        xl[2] = xl[1] + bond * (-math.cos(angle) * b01 + math.sin(angle) * v)
        ok = clash_free(xl[1], 1, xl) and clash_free(xl[2], 2, xl)
        for i in range(3, nl):
            if not ok:
                break
            for _attempt in range(200):
                p = _place(xl[i - 3], xl[i - 2], xl[i - 1], bond, angle, rng.uniform(-math.pi, math.pi))
                if clash_free(p, i, xl):
                    xl[i] = p
                    break
            else:
                ok = False
        if ok:
            break
    else:
        raise RuntimeError("ligand growth failed")
    q0 = np.concatenate([xr, xl])
    L = n_receptor + np.arange(nl)
    lbonds = np.stack([L[:-1], L[1:]], 1).astype(np.int32)
    langles = np.stack([L[:-2], L[1:-1], L[2:]], 1).astype(np.int32)
    ldih = np.stack([L[:-3], L[1:-2], L[2:-1], L[3:]], 1).astype(np.int32)
    nt = len(ldih)
    dn = rng.integers(1, 4, nt).astype(np.int32)
    dk = rng.uniform(0.0, 8.0, nt)
    dd = math.pi * rng.integers(0, 2, nt)
    lexcl = np.array([[L[i], L[j]] for i in range(nl) for j in range(i + 1, min(nl, i + 3))], np.int32)
    pocket = np.nonzero(np.linalg.norm(xr - cp, axis=1) < rp + 0.6)[0].astype(np.int32)
    kT = KB_KJ_PER_MOL_K * temperature
    mass = np.full(n, 12.0)
    s = System(
        name=f"ligand_receptor{n}", n_atoms=n, dim=3, potential=POT_FORCE_FIELD, mass=mass,
        kT=kT, gamma=1.0, dt=0.002, sigma=sigma, epsilon=epsilon, charge=charge,
        excl=np.concatenate([enm, lexcl]), cutoff=1.2, coulomb_k=COULOMB_K,
        bonds=np.concatenate([enm, lbonds]),
        bond_k=np.concatenate([np.full(len(enm), 500.0), np.full(nl - 1, 3.0e5)]),
        bond_r0=np.concatenate([enm_r0, np.full(nl - 1, bond)]),
        angles=langles, angle_k=np.full(nl - 2, 400.0), angle_theta0=np.full(nl - 2, angle),
        dihedrals=ldih, dihedral_n=dn, dihedral_k=dk, dihedral_delta=dd,
        cv_kind=CV_COM_DISTANCE, cv_params=(1.0,),
        groups=[L.astype(np.int32), pocket, L[:1].astype(np.int32), L[-1:].astype(np.int32)],
        observables=[(OBS_GROUP_DISTANCE, (0, 1)), (OBS_RMS_VELOCITY, (0,)),
                     (OBS_GROUP_DISTANCE, (2, 1)), (OBS_GROUP_DISTANCE, (3, 1))],
        n_replicas=n_replicas, t_gr=50, t_check=500, tol=0.01, min_fv_steps=0,
    )
    s.q0 = q0
    s.p0 = maxwell_boltzmann(mass, kT, 3, np.random.default_rng(dyn_seed))
    return s


def ligand_receptor_h(n_replicas: int = 1024, seed: int = 1807, dyn_seed: int = 2431) -> System:
    """The ligand-receptor system with one hydrogen (1.008 amu) on every ligand bead, its bond of
    0.109 nm held by a constraint (the paper's protein-ligand setup constrains the bonds of hydrogens,
    Section 4.2): 2,030 + 30 atoms.  As in ``chain_h``: each hydrogen carries 0.1 e taken from its bead,
    LJ sigma 0.25 nm and eps 0.1 kJ/mol, angles H-C-C of k = 300 kJ/mol/rad^2 at 109.5 deg with the bead's
    neighbours, 1-2 and 1-3 pairs through the hydrogen excluded.  A hydrogen sits opposite the bisector
    of its bead's bonds, turned about the bead's neighbour axis to the 10-deg step that keeps it furthest
    (in units of sigma_ij, at least 0.8) from every atom it interacts with.  Groups, states and observables are the ligand's
    (the centres of mass are those of the heavy beads)."""
    base = ligand_receptor(n_replicas=n_replicas, seed=seed, dyn_seed=dyn_seed)
    nb = base.n_atoms
    L = np.asarray(base.groups[0])
    nl = len(L)
    x = base.q0
    sig_h = 0.25
    excl = {tuple(sorted(e)) for e in base.excl.tolist()}
    hpos = np.zeros((nl, 3))
    for k, i in enumerate(L):
        nbrs = [L[m] for m in (k - 1, k + 1) if 0 <= m < nl]
        if len(nbrs) == 2:
            u = sum((x[i] - x[j]) / np.linalg.norm(x[i] - x[j]) for j in nbrs)
            axis = x[nbrs[1]] - x[nbrs[0]]
        else:  # an end bead: 109.5 deg from its one bond
            b = (x[nbrs[0]] - x[i]) / np.linalg.norm(x[nbrs[0]] - x[i])
            perp = np.cross(b, [0.3, 0.5, 0.8])
            perp /= np.linalg.norm(perp)
            u = math.cos(math.radians(109.5)) * b - math.sin(math.radians(109.5)) * perp
            axis = b
        u /= np.linalg.norm(u)
        axis /= np.linalg.norm(axis)
        skip = {i} | set(nbrs)  # the bead and its neighbours are excluded partners of the hydrogen
        others = [j for j in range(nb) if j not in skip]
        best, best_ratio = None, -1.0
        for turn in range(36):  # the turn about the axis that keeps the hydrogen furthest from clashes
            a = math.radians(10.0 * turn)
            v = u * math.cos(a) + np.cross(axis, u) * math.sin(a) + axis * np.dot(axis, u) * (1 - math.cos(a))
            ph = x[i] + 0.109 * v
            ratio = (np.linalg.norm(x[others] - ph, axis=1) / (0.5 * (base.sigma[others] + sig_h))).min()
            if k:
                ratio = min(ratio, (np.linalg.norm(hpos[:k] - ph, axis=1) / sig_h).min())
            if ratio > best_ratio:
                best, best_ratio = ph, ratio
        if best_ratio < 0.8:
            raise RuntimeError("no clash-free hydrogen position")
        hpos[k] = best
    n = nb + nl
    H = nb + np.arange(nl)
    mass = np.concatenate([base.mass, np.full(nl, 1.008)])
    charge = np.concatenate([base.charge, np.full(nl, 0.1)])
    charge[L] -= 0.1
    sigma = np.concatenate([base.sigma, np.full(nl, sig_h)])
    epsilon = np.concatenate([base.epsilon, np.full(nl, 0.1)])
    angles = [list(a) for a in base.angles]
    angle_k = list(base.angle_k)
    angle_t0 = list(base.angle_theta0)
    for k, i in enumerate(L):
        h = int(H[k])
        excl.add((min(i, h), max(i, h)))
        for m in (k - 1, k + 1):
            if 0 <= m < nl:
                angles.append([h, int(i), int(L[m])])
                angle_k.append(300.0)
                angle_t0.append(math.radians(109.5))
                excl.add((min(int(L[m]), h), max(int(L[m]), h)))
    s = dataclasses.replace(
        base, name=f"ligand_receptor{n}h", n_atoms=n, mass=mass, charge=charge, sigma=sigma, epsilon=epsilon,
        excl=np.array(sorted(excl), np.int32), angles=np.array(angles, np.int32), angle_k=np.array(angle_k),
        angle_theta0=np.array(angle_t0),
        constraints=np.stack([L, H], 1).astype(np.int32), constraint_length=np.full(nl, 0.109))
    s.q0 = np.concatenate([x, hpos])
    s.p0 = maxwell_boltzmann(mass, s.kT, 3, np.random.default_rng(dyn_seed))
    return s


def chain_gradient(n_atoms: int = 22, seed: int = 1807, dyn_seed: int = 2431, n_replicas: int = 256) -> System:
    """The chain of ``chain`` for differentiation through the dynamics: groups 0 = first bead and
    1 = last bead, and one more observable, their distance (the end-to-end distance, observable 4)."""
    s = chain(n_atoms, seed=seed, dyn_seed=dyn_seed, n_replicas=n_replicas)
    s.name = f"chain{n_atoms}_gradient"
    s.groups = [np.array([0], np.int32), np.array([n_atoms - 1], np.int32)]
    s.observables = s.observables + [(OBS_GROUP_DISTANCE, (0, 1))]
    return s


def batched_sizes(n_runs: int = 64, seed: int = 1807, lo: int = 22, hi: int = 400) -> np.ndarray:
    """Chain sizes drawn uniformly in [lo, hi] for the batched workload."""
    return np.random.default_rng(seed).integers(lo, hi + 1, n_runs)


def batched_chains(n_runs: int = 64, seed: int = 1807, n_replicas: int = 128, lo: int = 22,
                   hi: int = 400) -> list[System]:
    """Independent chains of uneven sizes, one Gen. ParRep run each (seeds 1807 + run)."""
    sizes = batched_sizes(n_runs, seed, lo, hi)
    return [chain(int(nb), seed=seed + r, dyn_seed=2431 + r, n_replicas=n_replicas)
            for r, nb in enumerate(sizes)]


def replica_states(s: System, n_replicas: int, seed: int, spread: float = 0.0):
    """Per-replica (q, p) [R, n, dim]: the system's q0 plus optional Gaussian displacement of scale
    `spread`, and Maxwell-Boltzmann momenta; used by parity tests that need distinct replicas."""
    rng = np.random.default_rng(seed)
    q = np.repeat(s.q0[None], n_replicas, axis=0).astype(np.float64)
    if spread > 0:
        q = q + spread * rng.standard_normal(q.shape)
    p = np.stack([maxwell_boltzmann(s.mass, s.kT, s.dim, rng) for _ in range(n_replicas)])
    return np.ascontiguousarray(q), np.ascontiguousarray(p)
