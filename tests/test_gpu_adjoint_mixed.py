"""The adjoint on the mixed path (grp_adjoint_segment on a GRP_MIXED system): the recomputation runs the
mixed path's own arithmetic (FP32 forces into fixed point, double-single integration), the reverse
sweep's Hessian-vector products and mixed parameter derivatives come from FP32 dual numbers summed in
fixed point, the adjoint vectors and dL/d theta stay FP64.

Checks in FP64: the FP64 adjoint (pinned to the oracle's finite-difference adjoint in
test_gpu_adjoint.py) of the same segment.  The two paths follow trajectories that differ by the mixed
path's rounding, which the chain's chaos amplifies (x1e5 in 1,000 steps, test_oracle_sensitivity.py), so the
gradients agree over short segments only: measured on GB300, 1e-6 of their largest component after 100
steps and 6e-6 after 200 (the tests allow 2e-5 and 1e-4); the losses agree to 4e-8.  Over 1,000 steps
each path differentiates its own trajectory (the gradients then differ at O(1), the losses by 3e-4)."""
import numpy as np
import pytest

from paper_1807_02431_gb300 import workloads as W

pytestmark = pytest.mark.gpu
SEED = 2431

LOSSES = {
    "end_to_end": dict(obs=4, transform=0, center=0.0, width=1.0),
    "phi_occupancy": dict(obs=2, transform=1, center=np.radians(-81.0), width=np.radians(10.0)),
}


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_02431_gb300 import binding, build

    build.build()
    binding.load()
    return binding


def _adjoint(B, prec, s, q0, p0, k, ck, loss):
    import torch

    R = q0.shape[0]
    sysh = B.grp_create_system(s, prec)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    gth = torch.empty(B.grp_param_count(sysh), dtype=torch.float64, device="cuda")
    gq = torch.empty((R, s.n_atoms, 3), dtype=torch.float64, device="cuda")
    gp = torch.empty_like(gq)
    L = B.grp_adjoint_segment(rep, k, 10, ck, d_grad_theta=gth, d_grad_q0=gq, d_grad_p0=gp, **loss)
    return L, gth.cpu().numpy(), gq.cpu().numpy(), gp.cpu().numpy(), B.grp_get_state(rep)


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("k,tol", [(100, 2e-5), (200, 1e-4)])
@pytest.mark.parametrize("name", sorted(LOSSES))
def test_mixed_adjoint_against_fp64_adjoint(B, name, k, tol):
    s = W.chain_gradient()
    q0, p0 = W.replica_states(s, 4, seed=21, spread=0.002)
    lo = LOSSES[name]
    L64, g64, q64, p64, _ = _adjoint(B, B.GRP_FP64, s, q0, p0, k, 100, lo)
    L32, g32, q32, p32, _ = _adjoint(B, B.GRP_MIXED, s, q0, p0, k, 100, lo)
    print(name, k, abs(L32 - L64) / abs(L64), _rel(g32, g64), _rel(q32, q64), _rel(p32, p64))
    assert abs(L32 - L64) < 1e-6 * abs(L64)
    assert _rel(g32, g64) < tol and _rel(q32, q64) < tol and _rel(p32, p64) < tol


def test_mixed_adjoint_recomputes_the_forward_exactly(B):
    """The recomputed trajectory is the forward one bit for bit: the gradients do not depend on the
    checkpoint interval, and the replica set ends where grp_step_k on the mixed path leaves it."""
    s = W.chain_gradient()
    R, k = 3, 120
    q0, p0 = W.replica_states(s, R, seed=22, spread=0.002)
    lo = LOSSES["end_to_end"]
    L1, g1, q1, p1, st1 = _adjoint(B, B.GRP_MIXED, s, q0, p0, k, 120, lo)
    L2, g2, q2, p2, _ = _adjoint(B, B.GRP_MIXED, s, q0, p0, k, 7, lo)
    assert L1 == L2 and np.array_equal(g1, g2) and np.array_equal(q1, q2) and np.array_equal(p1, p2)
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, k, 0)
    ref = B.grp_get_state(rep)
    assert np.array_equal(st1[0], ref[0]) and np.array_equal(st1[1], ref[1])


def test_mixed_adjoint_full_launch(B):
    """The gradient workload's launch on the mixed path (256 replicas, 1,000 steps, checkpoints every
    100): finite gradients, and the replica-averaged loss within 1e-3 of the FP64 path's."""
    s = W.chain_gradient()
    R = s.n_replicas
    q0, p0 = W.replica_states(s, R, seed=24, spread=0.002)
    lo = LOSSES["end_to_end"]
    L32, g32, q32, p32, _ = _adjoint(B, B.GRP_MIXED, s, q0, p0, 1000, 100, lo)
    L64, _, _, _, _ = _adjoint(B, B.GRP_FP64, s, q0, p0, 1000, 100, lo)
    assert np.all(np.isfinite(g32)) and np.all(np.isfinite(q32)) and np.all(np.isfinite(p32))
    assert abs(L32 - L64) < 1e-3 * abs(L64)
