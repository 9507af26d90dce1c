"""Reaction-field electrostatics on the GPU against the oracle, on the three nonbonded paths: the
explicit pair items (22-bead chain with a 1.0 nm cutoff), the Verlet list (ligand-receptor, 1.2 nm),
and the dual-number Hessian-vector products of the adjoint (chain).

Tolerances as for the dielectric eps = 4r model: FP64 forces 1e-11 and mixed 2e-6 of the largest
component; the atoms of pairs within rounding of the cutoff are left out of the mixed comparison (a
pair there may be counted on one side and not on the other; the reaction-field energy is continuous at
the cutoff but its force is not).
"""
import dataclasses

import numpy as np
import pytest

from paper_1807_02431_gb300 import workloads as W

pytestmark = pytest.mark.gpu
SEED = 2431


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_02431_gb300 import binding, build

    build.build()
    binding.load()
    return binding


def _rf(s, cutoff):
    out = dataclasses.replace(s, cutoff=cutoff, coulomb_mode=W.COULOMB_REACTION_FIELD, rf_dielectric=78.3)
    out.q0, out.p0 = s.q0, s.p0
    return out


def _near_cutoff_atoms(s, q, rel):
    n = s.n_atoms
    d = np.linalg.norm(q[:, None] - q[None], axis=-1)
    ex = np.zeros((n, n), bool)
    ex[s.excl[:, 0], s.excl[:, 1]] = True
    ex |= ex.T
    np.fill_diagonal(ex, True)
    i, j = np.nonzero((np.abs(d - s.cutoff) < rel * s.cutoff) & ~ex)
    return np.unique(np.concatenate([i, j]))


def _check(B, oracle_mod, s, qs, prec):
    import torch

    o = oracle_mod.Oracle(s)
    sysh = B.grp_create_system(s, prec)
    dq = torch.tensor(qs, device="cuda", dtype=torch.float64)
    de = torch.zeros(len(qs), device="cuda", dtype=torch.float64)
    df = torch.zeros_like(dq)
    B.grp_energy_forces(sysh, len(qs), dq, de, df)
    fg, eg = df.cpu().numpy(), de.cpu().numpy()
    for b, q in enumerate(qs):
        fo, eo = o.forces(q), o.potential(q)
        scale = np.abs(fo).max()
        if prec == B.GRP_FP64:
            assert len(_near_cutoff_atoms(s, q, 1e-9)) == 0
            assert np.abs(fg[b] - fo).max() < 1e-11 * scale
            assert abs(eg[b] - eo) < 1e-11 * max(abs(eo), scale)
        else:
            keep = np.setdiff1d(np.arange(s.n_atoms), _near_cutoff_atoms(s, q, 1e-5))
            assert np.abs(fg[b][keep] - fo[keep]).max() < 2e-6 * scale
            assert abs(eg[b] - eo) < 2e-6 * max(abs(eo), scale) + 1e-3 * s.n_atoms


@pytest.mark.parametrize("prec", [0, 1])
def test_chain_items_reaction_field(B, oracle_mod, prec):
    s = _rf(W.chain(), 1.0)
    rng = np.random.default_rng(4)
    qs = np.stack([s.q0 + 0.01 * rng.standard_normal(s.q0.shape) for _ in range(8)])
    _check(B, oracle_mod, s, qs, prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_ligand_list_reaction_field(B, oracle_mod, prec):
    s = _rf(W.ligand_receptor(), 1.2)
    rng = np.random.default_rng(5)
    qs = np.stack([s.q0 + 0.01 * rng.standard_normal(s.q0.shape) for _ in range(2)])
    _check(B, oracle_mod, s, qs, prec)


def test_reaction_field_trajectory_fp64(B, oracle_mod):
    """200 FP64 steps of the cutoff chain: positions within 1e-9 of the oracle's."""
    s = _rf(W.chain(), 1.0)
    R = 4
    q0, p0 = W.replica_states(s, R, seed=8, spread=0.002)
    o = oracle_mod.Oracle(s)
    q, p = q0.copy(), p0.copy()
    f = np.stack([o.forces(x) for x in q])
    o.step_k(q, p, f, SEED, 0, 0, 200, 0)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 200, 0)
    qg, pg, _, _ = B.grp_get_state(rep)
    assert np.abs(qg - q).max() < 1e-9 * np.abs(q).max()
    assert np.abs(pg - p).max() < 1e-8 * np.abs(p).max()


def test_reaction_field_adjoint(B, oracle_mod):
    """The adjoint's Hessian-vector products (dual numbers) through the reaction field.  The cutoff is
    1.6 nm (the paper's), beyond every distance in the chain (1.3 nm at most): the oracle takes its
    Hessian-vector products by central differences of the forces, which a pair crossing a truncated
    force's cutoff within the difference step would spoil, while the reaction-field terms k_rf and
    c_rf still act on every pair."""
    import torch

    s = _rf(W.chain_gradient(), 1.6)
    R, k, t_gr = 2, 100, 10
    q0, p0 = W.replica_states(s, R, seed=21, spread=0.002)
    o = oracle_mod.Oracle(s)
    f0 = np.stack([o.forces(x) for x in q0])
    Lo, gtho, gqo, gpo = o.adjoint_segment(q0.copy(), p0.copy(), f0.copy(), SEED, 0, 0, k, t_gr, 4, 0, 0.0, 1.0)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    gth = torch.empty(B.grp_param_count(sysh), dtype=torch.float64, device="cuda")
    gq = torch.empty((R, s.n_atoms, 3), dtype=torch.float64, device="cuda")
    gp = torch.empty_like(gq)
    L = B.grp_adjoint_segment(rep, k, t_gr, 50, d_grad_theta=gth, d_grad_q0=gq, d_grad_p0=gp, obs=4, transform=0,
                              center=0.0, width=1.0)
    assert abs(L - Lo) < 1e-12 * max(1.0, abs(Lo))
    for g, go in ((gth, gtho), (gq, gqo), (gp, gpo)):
        g = g.cpu().numpy()
        assert np.abs(g - go).max() < 1e-8 * np.abs(go).max()


def test_reaction_field_needs_a_cutoff(B):
    s = dataclasses.replace(W.chain(), coulomb_mode=W.COULOMB_REACTION_FIELD)
    with pytest.raises(B.GrpError) as e:
        B.grp_create_system(s, B.GRP_FP64)
    assert e.value.status == B.GRP_EINVAL
