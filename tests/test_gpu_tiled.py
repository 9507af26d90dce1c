"""Parity of the tiled nonbonded path (systems of 64 atoms and more: 32x32 atom tiles per warp) with
the FP64 oracle, with and without a cutoff.  Tolerances as in test_gpu_parity.py: FP64 forces
1e-11 relative to the largest component, mixed 2e-6; FP64 trajectories 1e-9 relative positions over
a horizon shorter than the chain's chaotic amplification; mixed one-step local error."""
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


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


SYSTEMS = {
    "chain100": lambda: W.chain(n_atoms=100),
    "chain400": lambda: W.chain(n_atoms=400),
    "chain200_cut1.0": lambda: dataclasses.replace(W.chain(n_atoms=200), cutoff=1.0),
}


@pytest.mark.parametrize("name", list(SYSTEMS))
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-6)])
def test_tiled_energy_forces(B, oracle_mod, name, prec, tol):
    import torch

    s = SYSTEMS[name]()
    o = oracle_mod.Oracle(s)
    rng = np.random.default_rng(2)
    n = 4
    qs = np.stack([s.q0 + 0.005 * rng.standard_normal(s.q0.shape) for _ in range(n)])
    sysh = B.grp_create_system(s, prec)
    dq = torch.tensor(qs, device="cuda", dtype=torch.float64)
    de = torch.zeros(n, device="cuda", dtype=torch.float64)
    df = torch.zeros_like(dq)
    B.grp_energy_forces(sysh, n, dq, de, df)
    torch.cuda.synchronize()
    fo = np.stack([o.forces(q) for q in qs])
    eo = np.array([o.potential(q) for q in qs])
    ferr = _rel(df.cpu().numpy(), fo)
    eerr = np.abs(de.cpu().numpy() - eo).max() / np.abs(eo).max()
    print(f"{name} prec={prec} force {ferr:.2e} energy {eerr:.2e}")
    assert ferr < tol and eerr < tol


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_tiled_fp64_trajectory(B, oracle_mod, name):
    """FP64 path, 300 steps with sampling, against the oracle (1e-9 on positions)."""
    s = SYSTEMS[name]()
    o = oracle_mod.Oracle(s)
    R, k = 3, 300
    q0, p0 = W.replica_states(s, R, seed=5, spread=0.002)
    q, p = q0.copy(), p0.copy()
    f = np.stack([o.forces(q[r]) for r in range(R)])
    samples = o.step_k(q, p, f, SEED, 0, 0, k, s.t_gr, cap=k // s.t_gr)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, k, s.t_gr)
    qg, pg, acc, _ = B.grp_get_state(rep)
    mean = acc[..., 0] + acc[..., 1] / acc[..., 3]
    em = np.abs(mean - samples.mean(axis=1)).max() / np.abs(samples).max()
    print(f"{name} fp64 q {_rel(qg, q):.2e} p {_rel(pg, p):.2e} obs {em:.2e}")
    assert _rel(qg, q) < 1e-9 and _rel(pg, p) < 1e-8 and em < 1e-9


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_tiled_mixed_local_error(B, oracle_mod, name):
    s = SYSTEMS[name]()
    o = oracle_mod.Oracle(s)
    R = 3
    q0, p0 = W.replica_states(s, R, seed=6, spread=0.002)
    q, p = q0.copy(), p0.copy()
    f = np.stack([o.forces(q[r]) for r in range(R)])
    o.step_k(q, p, f, SEED, 0, 0, 1, 0)
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 1, 0)
    qg, pg, _, _ = B.grp_get_state(rep)
    print(f"{name} mixed one step q {_rel(qg, q):.2e} p {_rel(pg, p):.2e}")
    assert _rel(qg, q) < 1e-9 and _rel(pg, p) < 1e-6


def test_tiled_mixed_deterministic(B):
    s = W.chain(n_atoms=400)
    R = 4
    q0, p0 = W.replica_states(s, R, seed=7, spread=0.002)
    out = []
    for _ in range(2):
        sysh = B.grp_create_system(s, B.GRP_MIXED)
        rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
        B.grp_step_k(rep, 100, s.t_gr)
        out.append(B.grp_get_state(rep)[:3])
    for a, b in zip(*out):
        assert np.array_equal(a, b)
