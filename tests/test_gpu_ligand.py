"""Parity of the ligand-receptor workload (2,030 atoms: elastic network, LJ + Coulomb truncated at
1.2 nm, COM-distance states, group observables) against the FP64 oracle.  The system is large enough
that the segment kernel reads atom parameters from the global table and draws its noise inline.

Cutoff: a pair whose distance lies within rounding of 1.2 nm may be counted or not, so its force (up to
~2 kJ/mol/nm from Coulomb at 1.2 nm) is not unique.  FP64 comparisons first assert that no pair lies
within 1e-9 relative of the cutoff (every decision is then unique); mixed comparisons leave out the
atoms of pairs within 1e-5 relative of the cutoff and compare the rest.  Other tolerances as for the
chain: FP64 forces 1e-11 of the largest component, FP64 trajectories 1e-9 on positions, mixed forces
2e-6, mixed one-step local error 1e-9 on positions and 1e-6 on momenta.  Labels, exit flags and branch
sources are compared exactly.
"""
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
def lr():
    return W.ligand_receptor()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _near_cutoff_atoms(s, q, rel):
    """Atoms of non-excluded pairs whose distance is within `rel` (relative) of the cutoff."""
    n = s.n_atoms
    d = np.linalg.norm(q[:, None] - q[None], axis=-1)
    ex = np.zeros((n, n), bool)
    ex[s.excl[:, 0], s.excl[:, 1]] = True
    ex |= ex.T
    np.fill_diagonal(ex, True)
    i, j = np.nonzero((np.abs(d - s.cutoff) < rel * s.cutoff) & ~ex)
    return np.unique(np.concatenate([i, j]))


def _configs(s, n, seed, spread=0.01):
    rng = np.random.default_rng(seed)
    return np.stack([s.q0 + spread * rng.standard_normal(s.q0.shape) for _ in range(n)])


@pytest.mark.parametrize("prec", [0, 1])
def test_ligand_energy_forces(B, oracle_mod, lr, prec):
    import torch

    s = lr
    o = oracle_mod.Oracle(s)
    qs = _configs(s, 3, seed=11)
    sysh = B.grp_create_system(s, prec)
    dq = torch.tensor(qs, device="cuda")
    de = torch.zeros(len(qs), device="cuda", dtype=torch.float64)
    df = torch.zeros_like(dq)
    B.grp_energy_forces(sysh, len(qs), dq, de, df)
    fg, eg = df.cpu().numpy(), de.cpu().numpy()
    for b, q in enumerate(qs):
        fo, eo = o.forces(q), o.potential(q)
        if prec == 0:
            assert len(_near_cutoff_atoms(s, q, 1e-9)) == 0
            assert _rel(fg[b], fo) < 1e-11
            assert abs(eg[b] - eo) < 1e-11 * max(abs(eo), np.abs(fo).max())
        else:
            amb = _near_cutoff_atoms(s, q, 1e-5)
            keep = np.setdiff1d(np.arange(s.n_atoms), amb)
            assert _rel(fg[b][keep], fo[keep]) < 2e-6
            # each ambiguous pair moves the energy by at most ~1 kJ/mol (Coulomb at 1.2 nm)
            assert abs(eg[b] - eo) < 2e-6 * np.abs(fo).max() + 2.0 * len(amb)


def test_ligand_fp64_trajectory(B, oracle_mod, lr):
    """FP64 path, 100 steps sampling every 50, then the exit test: positions, momenta, the observable
    means (COM distance, RMS velocity, end distances) and the labels against the oracle."""
    import torch

    s = lr
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
    assert np.all(acc[..., 3] == k // s.t_gr)
    assert _rel(qg, q) < 1e-9 and _rel(pg, p) < 1e-8
    assert np.abs(mean - samples.mean(axis=1)).max() < 1e-9 * np.abs(samples).max()
    lab = torch.zeros(R, dtype=torch.int8, device="cuda")
    ex = torch.zeros(R, dtype=torch.uint8, device="cuda")
    B.grp_check_states(rep, 0, lab, ex)
    assert lab.cpu().tolist() == [o.state_of(q[r]) for r in range(R)]
    assert ex.cpu().tolist() == [o.exited(q[r], 0) for r in range(R)]


def test_ligand_mixed_local_error(B, oracle_mod, lr):
    s = lr
    o = oracle_mod.Oracle(s)
    R = 2
    q0, p0 = W.replica_states(s, R, seed=6, spread=0.005)
    q, p = q0.copy(), p0.copy()
    f = np.stack([o.forces(q[r]) for r in range(R)])
    o.step_k(q, p, f, SEED, 0, 0, 1, 0)
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 1, 0)
    qg, pg, _, _ = B.grp_get_state(rep)
    for r in range(R):
        amb = set(_near_cutoff_atoms(s, q0[r], 1e-5)) | set(_near_cutoff_atoms(s, q[r], 1e-5))
        keep = np.setdiff1d(np.arange(s.n_atoms), sorted(amb))
        assert np.abs(qg[r][keep] - q[r][keep]).max() < 1e-9 * np.abs(q[r]).max()
        assert np.abs(pg[r][keep] - p[r][keep]).max() < 1e-6 * np.abs(p[r]).max()


def test_ligand_states(B, oracle_mod, lr):
    """The ligand pulled out of the pocket step by step: COM-distance labels and exit flags exactly as
    the oracle's, for both precisions (the exit test runs in FP64 on both paths)."""
    import torch

    s = lr
    o = oracle_mod.Oracle(s)
    lig = s.groups[0]
    shifts = [0.0, 0.3, 0.45, 0.5, 0.55, 0.8, 1.5, 3.0]
    qs = []
    for z in shifts:
        q = s.q0.copy()
        q[lig, 2] += z
        qs.append(q)
    qs = np.stack(qs)
    R = len(qs)
    lo = [o.state_of(x) for x in qs]
    assert 0 in lo and 1 in lo
    for prec in (0, 1):
        sysh = B.grp_create_system(s, prec)
        rep = B.grp_init_replicas(sysh, R, SEED, qs, np.zeros_like(qs), per_replica=True)
        for omega in (0, 1):
            lab = torch.zeros(R, dtype=torch.int8, device="cuda")
            ex = torch.zeros(R, dtype=torch.uint8, device="cuda")
            B.grp_check_states(rep, omega, lab, ex)
            assert lab.cpu().tolist() == lo
            assert ex.cpu().tolist() == [o.exited(x, omega) for x in qs]


def test_ligand_full_size_segment(B, oracle_mod, lr):
    """The benchmark's launch: 1,024 replicas, one 500-step exit test of the convergence step on the
    mixed path.  Sampled replicas are checked one by one against the oracle: their labels against the
    oracle's state of their final configuration, their energies against the oracle's potential (via
    the FP64 force kernel); the branching of the same exited mask against the oracle's draw."""
    import torch

    s = lr
    o = oracle_mod.Oracle(s)
    R = s.n_replicas
    sysm = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysm, R, SEED, s.q0, s.p0)
    # exit test without branching first, to read the labels of the final states
    B.grp_step_k(rep, s.t_check, s.t_gr)
    lab = torch.zeros(R, dtype=torch.int8, device="cuda")
    ex = torch.zeros(R, dtype=torch.uint8, device="cuda")
    B.grp_check_states(rep, 0, lab, ex)
    qg, pg, acc, ctr = B.grp_get_state(rep)
    assert np.all(np.isfinite(qg)) and np.all(np.isfinite(pg))
    assert np.all(acc[..., 3] == s.t_check // s.t_gr)
    sample = [0, 1, 511, 1023]
    lab_h = lab.cpu().numpy()
    for r in sample:
        assert lab_h[r] == o.state_of(qg[r])
    sys64 = B.grp_create_system(s, B.GRP_FP64)
    dq = torch.tensor(qg[sample], device="cuda")
    de = torch.zeros(len(sample), dtype=torch.float64, device="cuda")
    B.grp_energy_forces(sys64, len(sample), dq, de)
    for b, r in enumerate(sample):
        assert len(_near_cutoff_atoms(s, qg[r], 1e-9)) == 0
        assert abs(de[b].item() - o.potential(qg[r])) < 1e-9 * abs(o.potential(qg[r])) + 1e-8
    # replicas differ after 500 steps (distinct noise streams)
    assert not np.array_equal(qg[0], qg[1])
    # branching at this size against the oracle's draw, on a synthetic exited mask
    rng = np.random.default_rng(3)
    exm = (rng.random(R) < 0.4).astype(np.uint8)
    dsrc = torch.zeros(R, dtype=torch.int32, device="cuda")
    nb = B.grp_fv_branch(rep, torch.tensor(exm, device="cuda"), dsrc)
    nbo, srco = oracle_mod.fv_branch(SEED, ctr["t_global"], exm)
    assert nb == nbo and np.array_equal(dsrc.cpu().numpy(), srco)


def test_ligand_fp64_full_size_sampled(B, oracle_mod, lr):
    """FP64 path in the full launch (1,024 replicas, 20 steps): sampled replicas against the oracle."""
    s = lr
    o = oracle_mod.Oracle(s)
    R, k = s.n_replicas, 20
    q0, p0 = W.replica_states(s, R, seed=12, spread=0.002)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, k, 0)
    qg, pg, _, _ = B.grp_get_state(rep)
    for r in (0, 700, 1023):
        q, p = q0[r:r + 1].copy(), p0[r:r + 1].copy()
        f = o.forces(q[0])[None].copy()
        for t in range(k):
            o.baoab_step(q[0], p[0], f[0], SEED, r, t)
        assert _rel(qg[r], q[0]) < 1e-10 and _rel(pg[r], p[0]) < 1e-9
