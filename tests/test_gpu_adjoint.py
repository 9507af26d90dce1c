"""Adjoint differentiation through the dynamics (grp_adjoint_segment) against the oracle's adjoint.

The library's reverse sweep takes its Hessian-vector products from dual numbers (exact up to
rounding); the oracle's from Richardson-extrapolated central differences (error ~1e-10 relative).  Both
differentiate the same discrete map with the same noise; the trajectories differ only by rounding
(~1e-16), which the chain's chaos amplifies over the segment.  Measured on GB300: gradients agree to
1.3e-10 of their largest component after 200 steps and to 1.6e-9 after 1,000 steps (sampled replicas
of the full launch); the tests allow 1e-8 and 1e-6.  Losses agree to 1e-12.
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


LOSSES = {
    "end_to_end": dict(obs=4, transform=0, center=0.0, width=1.0),
    "phi_occupancy": dict(obs=2, transform=1, center=np.radians(-81.0), width=np.radians(10.0)),
}


def _gpu(B, s, q0, p0, k, t_gr, ck, loss):
    import torch

    R = q0.shape[0]
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    gth = torch.empty(B.grp_param_count(sysh), dtype=torch.float64, device="cuda")
    gq = torch.empty((R, s.n_atoms, 3), dtype=torch.float64, device="cuda")
    gp = torch.empty_like(gq)
    L = B.grp_adjoint_segment(rep, k, t_gr, ck, d_grad_theta=gth, d_grad_q0=gq, d_grad_p0=gp, **loss)
    return L, gth.cpu().numpy(), gq.cpu().numpy(), gp.cpu().numpy(), B.grp_get_state(rep)


@pytest.mark.parametrize("name", sorted(LOSSES))
def test_adjoint_matches_oracle(B, oracle_mod, name):
    s = W.chain_gradient()
    R, k, t_gr = 4, 200, 10
    q0, p0 = W.replica_states(s, R, seed=21, spread=0.002)
    o = oracle_mod.Oracle(s)
    f0 = np.stack([o.forces(x) for x in q0])
    lo = LOSSES[name]
    Lo, gtho, gqo, gpo = o.adjoint_segment(q0.copy(), p0.copy(), f0.copy(), SEED, 0, 0, k, t_gr, lo["obs"],
                                           lo["transform"], lo["center"], lo["width"])
    L, gth, gq, gp, _ = _gpu(B, s, q0, p0, k, t_gr, 50, lo)
    print(name, L, Lo, np.abs(gth - gtho).max() / np.abs(gtho).max(), np.abs(gq - gqo).max() / np.abs(gqo).max(),
          np.abs(gp - gpo).max() / np.abs(gpo).max())
    assert abs(L - Lo) < 1e-12 * max(1.0, abs(Lo))
    assert np.abs(gth - gtho).max() < 1e-8 * np.abs(gtho).max()
    assert np.abs(gq - gqo).max() < 1e-8 * np.abs(gqo).max()
    assert np.abs(gp - gpo).max() < 1e-8 * np.abs(gpo).max()


def test_adjoint_advances_like_step_k_and_ignores_checkpoint_interval(B):
    """The replica set ends exactly where grp_step_k leaves it, and the gradients do not depend on the
    checkpoint interval (recomputed states are bit-identical)."""
    s = W.chain_gradient()
    R, k = 3, 120
    q0, p0 = W.replica_states(s, R, seed=22, spread=0.002)
    lo = LOSSES["end_to_end"]
    L1, g1, q1, p1, st1 = _gpu(B, s, q0, p0, k, 10, 120, lo)
    L2, g2, q2, p2, st2 = _gpu(B, s, q0, p0, k, 10, 7, lo)
    assert L1 == L2 and np.array_equal(g1, g2) and np.array_equal(q1, q2) and np.array_equal(p1, p2)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, k, 0)
    ref = B.grp_get_state(rep)
    assert np.array_equal(st1[0], ref[0]) and np.array_equal(st1[1], ref[1])
    assert st1[3] == ref[3]


def test_adjoint_against_gpu_finite_differences(B):
    """dL/dtheta for a few parameters against central differences of the library's own loss (set
    through grp_set_params), 100 steps."""
    import torch

    s = W.chain_gradient()
    R, k, t_gr = 8, 100, 10
    q0, p0 = W.replica_states(s, R, seed=23, spread=0.002)
    lo = LOSSES["phi_occupancy"]
    L, gth, _, _, _ = _gpu(B, s, q0, p0, k, t_gr, 100, lo)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    th0 = torch.empty(B.grp_param_count(sysh), dtype=torch.float64, device="cuda")
    B.grp_get_params(sysh, th0)
    th0 = th0.cpu().numpy()
    for j in (0, 7, s.n_atoms + 3, 2 * s.n_atoms + 10, len(th0) - 1):
        vals = []
        for sgn in (1, -1):
            th = th0.copy()
            h = 1e-6 * abs(th[j])
            th[j] += sgn * h
            B.grp_set_params(sysh, torch.tensor(th, device="cuda"))
            rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
            vals.append(B.grp_adjoint_segment(rep, k, t_gr, 100, **lo))
        fd = (vals[0] - vals[1]) / (2 * 1e-6 * abs(th0[j]))
        assert abs(fd - gth[j]) < 1e-5 * np.abs(gth).max(), (j, fd, gth[j])


def test_adjoint_full_launch_sampled(B, oracle_mod):
    """The gradient workload's launch: 256 replicas, 1,000 steps, checkpoints every 100.  The gradient
    with respect to the initial state of sampled replicas against the oracle's adjoint of the same
    replica alone (scaled by R for the replica average)."""
    s = W.chain_gradient()
    R, k, t_gr = s.n_replicas, 1000, 10
    q0, p0 = W.replica_states(s, R, seed=24, spread=0.002)
    lo = LOSSES["end_to_end"]
    L, gth, gq, gp, _ = _gpu(B, s, q0, p0, k, t_gr, 100, lo)
    assert np.all(np.isfinite(gth)) and np.all(np.isfinite(gq))
    o = oracle_mod.Oracle(s)
    errs = []
    for r in (0, 101, 255):
        f0 = o.forces(q0[r])[None]
        _, _, gqo, gpo = o.adjoint_segment(q0[r:r + 1].copy(), p0[r:r + 1].copy(), f0.copy(), SEED, 0, 0, k, t_gr,
                                           lo["obs"], lo["transform"], lo["center"], lo["width"], replica0=r)
        eq = np.abs(gq[r] * R - gqo[0]).max() / np.abs(gqo).max()
        ep = np.abs(gp[r] * R - gpo[0]).max() / np.abs(gpo).max()
        errs.append((eq, ep))
    print("full launch sampled errors", errs)
    assert max(max(e) for e in errs) < 1e-6


def test_segment_loss_autograd(B):
    import torch

    from paper_1807_02431_gb300 import autograd as AG

    s = W.chain_gradient()
    R = 4
    q0, p0 = W.replica_states(s, R, seed=25, spread=0.002)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    theta = AG.current_params(sysh).requires_grad_(True)
    lo = LOSSES["end_to_end"]
    L = AG.segment_loss(rep, theta, 60, 10, lo["obs"])
    (3.0 * L).backward()
    L2, g2, _, _, _ = _gpu(B, s, q0, p0, 60, 10, 100, lo)
    assert abs(L.item() - L2) < 1e-14
    assert np.array_equal(theta.grad.cpu().numpy(), 3.0 * g2)
