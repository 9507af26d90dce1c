"""Generalized Born implicit solvent (OBC II) on the GPU against the oracle: the 22-bead chain in
solvent, forces and energies on both paths, an FP64 trajectory, the Gen. ParRep loop running, and the
combinations the library declines (GRP_ENOTIMPL)."""
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


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-6)])
def test_solvated_chain_forces(B, oracle_mod, prec, tol):
    import torch

    s = W.solvated(W.chain())
    o = oracle_mod.Oracle(s)
    vac = oracle_mod.Oracle(W.chain())
    rng = np.random.default_rng(6)
    qs = np.stack([s.q0 + 0.01 * rng.standard_normal(s.q0.shape) for _ in range(8)])
    sysh = B.grp_create_system(s, prec)
    dq = torch.tensor(qs, device="cuda", dtype=torch.float64)
    de = torch.zeros(len(qs), device="cuda", dtype=torch.float64)
    df = torch.zeros_like(dq)
    B.grp_energy_forces(sysh, len(qs), dq, de, df)
    fg, eg = df.cpu().numpy(), de.cpu().numpy()
    for b, q in enumerate(qs):
        fo, eo = o.forces(q), o.potential(q)
        assert abs(eo - vac.potential(q)) > 10.0  # the solvent term is present and sizeable
        scale = np.abs(fo).max()
        assert np.abs(fg[b] - fo).max() < tol * scale
        assert abs(eg[b] - eo) < tol * max(abs(eo), scale)


def test_solvated_chain_trajectory_fp64(B, oracle_mod):
    s = W.solvated(W.chain())
    R = 4
    q0, p0 = W.replica_states(s, R, seed=12, spread=0.002)
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


def test_solvated_mixed_one_step(B, oracle_mod):
    """Mixed path, one step from the same state: positions 1e-9 and momenta 1e-6 relative (as in
    vacuum)."""
    s = W.solvated(W.chain())
    R = 8
    q0, p0 = W.replica_states(s, R, seed=13, spread=0.002)
    o = oracle_mod.Oracle(s)
    q, p = q0.copy(), p0.copy()
    f = np.stack([o.forces(x) for x in q])
    o.step_k(q, p, f, SEED, 0, 0, 1, 0)
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 1, 0)
    qg, pg, _, _ = B.grp_get_state(rep)
    assert np.abs(qg - q).max() < 1e-9 * np.abs(q).max()
    assert np.abs(pg - p).max() < 1e-6 * np.abs(p).max()


def test_solvated_loop_runs(B):
    """The whole loop of Fig. 1 on the solvated chain (mixed), with observables sampled in solvent."""
    s = W.solvated(W.chain())
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, 64, SEED, s.q0, s.p0)
    ev, tsim = B.grp_run(rep, s.t_gr, s.t_check, s.tol, 0, 20 * s.t_check, 3)
    assert B.grp_get_state(rep)[3]["t_global"] >= 20 * s.t_check or len(ev) > 0


def test_declined_combinations(B):
    s = W.solvated(W.chain())
    for bad in (dataclasses.replace(s, cutoff=1.2), W.solvated(W.chain(n_atoms=64))):
        with pytest.raises(B.GrpError) as e:
            B.grp_create_system(bad, B.GRP_MIXED)
        assert e.value.status == B.GRP_ENOTIMPL
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, 2, SEED, s.q0, s.p0)
    with pytest.raises(B.GrpError) as e:
        B.grp_batch_create([rep])
    assert e.value.status == B.GRP_ENOTIMPL
    with pytest.raises(B.GrpError) as e:
        B.grp_adjoint_segment(rep, 10, 10, 5, obs=0)
    assert e.value.status == B.GRP_ENOTIMPL
