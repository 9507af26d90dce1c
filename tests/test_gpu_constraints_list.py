"""Bond constraints on the Verlet-list path: the ligand-receptor system with constrained hydrogens on the
ligand (2,060 atoms), alone and in OBC II solvent (the paper's protein-ligand setup constrains the bonds of
hydrogens and runs in OBC II with a cutoff, Section 4.2), against the oracle.

In the list kernel the atoms of a constraint group are integrated by the group's thread (SHAKE/RATTLE,
FP64 on the FP64 path, double-single for single-bond groups on the mixed path) with the noise drawn from
the same counter-based stream as the free atoms, and their displacements take part in the list's rebuild
test.  Tolerances as for the constrained chain: FP64 trajectories within 1e-9 (positions) and 1e-8
(momenta) with no projection out of sweeps in the oracle; the mixed one-step local error 1e-9 and 1e-6;
constraint lengths within 1e-9 relative after a full segment."""
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


@pytest.fixture(scope="module")
def lh():
    return W.ligand_receptor_h()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _lengths(s, q):
    c = s.constraints
    return np.linalg.norm(q[..., c[:, 0], :] - q[..., c[:, 1], :], axis=-1)


@pytest.mark.parametrize("solvent", [False, True])
def test_constrained_ligand_fp64_trajectory(B, oracle_mod, lh, solvent):
    s = W.solvated(lh) if solvent else lh
    o = oracle_mod.Oracle(s)
    R, k = 2, 100 if not solvent else 50
    q0, p0 = W.replica_states(s, R, seed=5, spread=0.003)
    # a replica's constrained bonds start at their lengths: project the spread hydrogens back onto them
    c = s.constraints
    for r in range(R):
        v = q0[r, c[:, 1]] - q0[r, c[:, 0]]
        q0[r, c[:, 1]] = q0[r, c[:, 0]] + 0.109 * v / np.linalg.norm(v, axis=1)[:, None]
    q, p = q0.copy(), p0.copy()
    f = np.stack([o.forces(q[r]) for r in range(R)])
    o.step_k(q, p, f, SEED, 0, 0, k, 0)
    assert o.unconverged() == 0
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, k, 0)
    qg, pg, _, _ = B.grp_get_state(rep)
    print(solvent, _rel(qg, q), _rel(pg, p))
    assert _rel(qg, q) < 1e-9 and _rel(pg, p) < 1e-8
    assert np.abs(_lengths(s, qg) / 0.109 - 1).max() < 1e-9


def test_constrained_ligand_mixed_one_step(B, oracle_mod, lh):
    s = lh
    o = oracle_mod.Oracle(s)
    R = 2
    q0, p0 = W.replica_states(s, R, seed=6, spread=0.0)
    q, p = q0.copy(), p0.copy()
    f = np.stack([o.forces(q[r]) for r in range(R)])
    o.step_k(q, p, f, SEED, 0, 0, 1, 0)
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 1, 0)
    qg, pg, _, _ = B.grp_get_state(rep)
    for r in range(R):
        assert np.abs(qg[r] - q[r]).max() < 1e-9 * np.abs(q[r]).max()
        assert np.abs(pg[r] - p[r]).max() < 1e-6 * np.abs(p[r]).max()


def test_constrained_solvated_ligand_full_launch(B, lh):
    """The benchmark's launch configuration in the paper's setup (solvent and constrained hydrogens,
    1,024 replicas, one 500-step exit test of the convergence step, mixed): the state stays finite, the
    constrained bonds keep their lengths, every replica keeps its samples."""
    s = W.solvated(lh)
    R = s.n_replicas
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, R, SEED, s.q0, s.p0)
    st = B.grp_fv_check(rep, 0, s.t_check, s.t_gr, s.tol, 0)
    assert st.t_phase == s.t_check
    qg, pg, acc, _ = B.grp_get_state(rep)
    assert np.all(np.isfinite(qg)) and np.all(np.isfinite(pg))
    assert np.abs(_lengths(s, qg) / 0.109 - 1).max() < 1e-9
    assert np.all(acc[..., 3] == s.t_check // s.t_gr)


def test_constraints_with_reaction_field_on_lists_declined(B, lh):
    bad = dataclasses.replace(lh, coulomb_mode=W.COULOMB_REACTION_FIELD)
    bad.q0, bad.p0 = lh.q0, lh.p0
    with pytest.raises(B.GrpError) as e:
        B.grp_create_system(bad, B.GRP_MIXED)
    assert e.value.status == B.GRP_ENOTIMPL
