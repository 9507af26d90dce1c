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
