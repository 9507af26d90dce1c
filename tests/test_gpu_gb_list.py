"""Generalized Born implicit solvent (OBC II) with a cutoff on the Verlet-list path, against the oracle:
the 2,030-atom ligand-receptor system in solvent (the paper's protein-ligand setup runs OBC II with a
non-periodic cutoff, Section 4.2).  The solvent sums take the pairs within the cutoff, excluded
(elastic-network and bonded) pairs included; plain truncation as the oracle reads it.

A pair within rounding of the cutoff may enter the sums or not, and through the Born radii its
decision reaches every neighbour, so these tests use configurations in which no pair (excluded ones
included) lies within 1e-6 relative of the cutoff: FP32 distances then take every decision as FP64
does.  Tolerances as for the solvated chain: forces 1e-11 (FP64) and 2e-6 (mixed) of the largest
component; an FP64 trajectory within 1e-9 (positions) and 1e-8 (momenta); the mixed one-step local
error 1e-9 and 1e-6."""
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
def sl():
    return W.solvated(W.ligand_receptor())


def _min_rel_to_cutoff(s, q):
    iu = np.triu_indices(s.n_atoms, 1)
    d = np.linalg.norm(q[:, None] - q[None], axis=-1)[iu]
    return np.abs(d - s.cutoff).min() / s.cutoff


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-6)])
def test_solvated_ligand_forces(B, oracle_mod, sl, prec, tol):
    import torch

    s = sl
    o = oracle_mod.Oracle(s)
    vac = oracle_mod.Oracle(W.ligand_receptor())
    rng = np.random.default_rng(11)
    qs = np.stack([s.q0 + 0.01 * rng.standard_normal(s.q0.shape) for _ in range(2)])
    sysh = B.grp_create_system(s, prec)
    dq = torch.tensor(qs, device="cuda")
    de = torch.zeros(len(qs), device="cuda", dtype=torch.float64)
    df = torch.zeros_like(dq)
    B.grp_energy_forces(sysh, len(qs), dq, de, df)
    fg, eg = df.cpu().numpy(), de.cpu().numpy()
    for b, q in enumerate(qs):
        assert _min_rel_to_cutoff(s, q) > 1e-6
        fo, eo = o.forces(q), o.potential(q)
        assert np.abs(fo - vac.forces(q)).max() > 10.0  # the solvent forces are there
        assert _rel(fg[b], fo) < tol
        assert abs(eg[b] - eo) < tol * max(abs(eo), np.abs(fo).max())


def test_solvated_ligand_fp64_trajectory(B, oracle_mod, sl):
    """FP64 path: 100 steps sampling every 50 (segment kernel, solvent passes over the Verlet list and
    the excluded pairs), positions, momenta and the observable means against the oracle."""
    s = sl
    o = oracle_mod.Oracle(s)
    R, k = 2, 100
    q0, p0 = W.replica_states(s, R, seed=5, spread=0.005)
    q, p = q0.copy(), p0.copy()
    f = np.stack([o.forces(q[r]) for r in range(R)])
    samples = o.step_k(q, p, f, SEED, 0, 0, k, s.t_gr, cap=k // s.t_gr)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, k, s.t_gr)
    qg, pg, acc, _ = B.grp_get_state(rep)
    mean = acc[..., 0] + acc[..., 1] / acc[..., 3]
    assert _rel(qg, q) < 1e-9 and _rel(pg, p) < 1e-8
    assert np.abs(mean - samples.mean(axis=1)).max() < 1e-9 * np.abs(samples).max()


def test_solvated_ligand_mixed_one_step(B, oracle_mod, sl):
    s = sl
    o = oracle_mod.Oracle(s)
    R = 2
    q0, p0 = W.replica_states(s, R, seed=6, spread=0.005)
    q, p = q0.copy(), p0.copy()
    f = np.stack([o.forces(q[r]) for r in range(R)])
    o.step_k(q, p, f, SEED, 0, 0, 1, 0)
    for r in range(R):
        assert _min_rel_to_cutoff(s, q0[r]) > 1e-6 and _min_rel_to_cutoff(s, q[r]) > 1e-6
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 1, 0)
    qg, pg, _, _ = B.grp_get_state(rep)
    for r in range(R):
        assert np.abs(qg[r] - q[r]).max() < 1e-9 * np.abs(q[r]).max()
        assert np.abs(pg[r] - p[r]).max() < 1e-6 * np.abs(p[r]).max()


def test_solvated_ligand_segment_full_launch(B, oracle_mod, sl):
    """The benchmark's launch configuration in solvent (1,024 replicas, one 500-step exit test of the
    convergence step, mixed): the state stays finite, every replica keeps its samples, sampled replicas'
    labels match the oracle's state of their final configuration, and the solvent energy of sampled
    final states on the FP64 force kernel matches the oracle's."""
    import torch

    s = sl
    o = oracle_mod.Oracle(s)
    R = s.n_replicas
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, R, SEED, s.q0, s.p0)
    st = B.grp_fv_check(rep, 0, s.t_check, s.t_gr, s.tol, 0)
    assert st.t_phase == s.t_check
    view = B.device_tensors(rep)
    lab = view["labels"].cpu().numpy()
    qg, pg, acc, _ = B.grp_get_state(rep)
    assert np.all(np.isfinite(qg)) and np.all(np.isfinite(pg))
    sample = [0, 1, 512, 1023]
    sys64 = B.grp_create_system(s, B.GRP_FP64)
    de = torch.zeros(len(sample), dtype=torch.float64, device="cuda")
    B.grp_energy_forces(sys64, len(sample), torch.tensor(qg[sample], device="cuda"), de)
    for b, r in enumerate(sample):
        if lab[r] >= 0 and st.n_branched == 0:
            assert lab[r] == o.state_of(qg[r])
        if _min_rel_to_cutoff(s, qg[r]) > 1e-9:
            assert abs(de[b].item() - o.potential(qg[r])) < 1e-9 * abs(o.potential(qg[r])) + 1e-8
