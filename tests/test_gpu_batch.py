"""Batched runs (one persistent kernel over many replica sets of uneven sizes) against the same runs
advanced one by one: the fixed-point force sums make every result independent of the block size and
of the order in which units are taken, so the comparison is exact (bit for bit)."""
import numpy as np
import pytest

from paper_1807_02431_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_02431_gb300 import binding, build

    build.build()
    binding.load()
    return binding


SIZES = [22, 100, 37, 200]


def _runs(B, prec, R=6):
    runs = []
    for k, n in enumerate(SIZES):
        s = W.chain(n_atoms=n, seed=1807 + k, dyn_seed=2431 + k)
        sysh = B.grp_create_system(s, prec)
        q0, p0 = W.replica_states(s, R, seed=100 + k, spread=0.002)
        runs.append((s, sysh, B.grp_init_replicas(sysh, R, 2431 + k, q0, p0, per_replica=True)))
    return runs


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_step_matches_single_runs(B, prec):
    single = _runs(B, prec)
    batched = _runs(B, prec)
    for s, _, rep in single:
        B.grp_step_k(rep, 300, s.t_gr)
    b = B.grp_batch_create([rep for _, _, rep in batched])
    B.grp_batch_step_k(b, 300, 10)
    for (_, _, r1), (_, _, r2) in zip(single, batched):
        a1, a2 = B.grp_get_state(r1), B.grp_get_state(r2)
        for x, y in zip(a1[:3], a2[:3]):
            assert np.array_equal(x, y)
        assert a1[3] == a2[3]


def test_batch_fv_check_matches_single_runs(B):
    single = _runs(B, 1, R=8)
    batched = _runs(B, 1, R=8)
    omegas = [1] * len(SIZES)
    b = B.grp_batch_create([rep for _, _, rep in batched])
    for check in range(3):
        ref = [B.grp_fv_check(rep, 1, 100, 10, 0.01, 0) for _, _, rep in single]
        got = B.grp_batch_fv_check(b, omegas, 100, 10, 0.01, 0)
        for st1, st2 in zip(ref, got):
            assert (st1.ref_exited, st1.label0, st1.n_branched, st1.converged, st1.t_phase) == \
                   (st2.ref_exited, st2.label0, st2.n_branched, st2.converged, st2.t_phase)
            assert list(st1.rhat) == list(st2.rhat)
    for (_, _, r1), (_, _, r2) in zip(single, batched):
        a1, a2 = B.grp_get_state(r1), B.grp_get_state(r2)
        for x, y in zip(a1[:3], a2[:3]):
            assert np.array_equal(x, y)


def test_batch_autotune_restores_state(B):
    runs = _runs(B, 1)
    b = B.grp_batch_create([rep for _, _, rep in runs])
    before = [B.grp_get_state(rep) for _, _, rep in runs]
    t = B.grp_batch_autotune(b, 10)
    assert t in (128, 256, 384, 512)
    after = [B.grp_get_state(rep) for _, _, rep in runs]
    for a1, a2 in zip(before, after):
        for x, y in zip(a1[:3], a2[:3]):
            assert np.array_equal(x, y)
        assert a1[3] == a2[3]


@pytest.mark.parametrize("prec,tol", [(1, 1e-6), (0, 1e-12)])
def test_batch_full_size_sampled(B, oracle_mod, prec, tol):
    """The benchmark's batch at full size and in its launch configuration (64 runs x 128 replicas,
    chains of 22..400 beads, the autotuned block size): 50 steps of every replica with sampling every
    10, then sampled replicas -- six runs across the size range, two replicas each -- against the oracle
    advancing them alone with their own noise indices.  Positions relative to their largest component:
    FP64 1e-12 (measured ~1e-15: the oracle's arithmetic in another order); mixed 1e-6 (measured 1-3e-8
    from the FP32 forces; a missing or doubled pair term gives ~1e-3)."""
    n_runs, R, k = 64, 128, 50
    systems = W.batched_chains(n_runs=n_runs, n_replicas=R)
    inits, reps = [], []
    for i, s in enumerate(systems):
        sysh = B.grp_create_system(s, prec)
        q0, p0 = W.replica_states(s, R, seed=3000 + i, spread=0.002)
        inits.append((q0, p0))
        reps.append(B.grp_init_replicas(sysh, R, 2431 + i, q0, p0, per_replica=True))
    b = B.grp_batch_create(reps)
    B.grp_batch_autotune(b, 10)  # restores every replica's state and counters
    B.grp_batch_step_k(b, k, 10)
    order = np.argsort([s.n_atoms for s in systems], kind="stable")
    for i in order[np.linspace(0, n_runs - 1, 6).astype(int)]:
        s = systems[i]
        o = oracle_mod.Oracle(s)
        q, p, _, ctr = B.grp_get_state(reps[i])
        assert ctr["t_global"] == k
        for r in (0, 77):
            qo, po = inits[i][0][r:r + 1].copy(), inits[i][1][r:r + 1].copy()
            fo = o.forces(qo[0])[None]
            o.step_k_from(qo, po, fo, 2431 + i, r, 0, 0, k, 10, cap=k // 10)
            err = np.abs(q[r] - qo[0]).max() / np.abs(qo[0]).max()
            print(f"run {i} ({s.n_atoms} beads) replica {r} prec {prec}: q {err:.2e}")
            assert err < tol
