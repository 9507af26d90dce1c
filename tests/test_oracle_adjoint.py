"""Pins of the oracle's adjoint of a dynamics segment (CPU only).

The adjoint returns dL/dtheta, dL/dq0 and dL/dp0 of L = mean over replicas and sampling steps of
g(O(q_t)) with the noise fixed.  Each is compared with central finite differences of L computed by
the forward dynamics alone (orc_step_k and its observable samples, pinned elsewhere), so the reverse
sweep (transposed drifts, friction factor c1, the half-kick weights, the loss-sample gradient, the
Hessian-vector products and mixed parameter derivatives) is checked against something other than
itself: a transposed factor or a dropped half kick moves the result far outside the tolerance.
"""
import dataclasses

import numpy as np
import pytest

from paper_1807_02431_gb300 import workloads as W

SEED = 2431


def _theta(s):
    return np.concatenate([s.sigma, s.epsilon, s.dihedral_k])


def _with_theta(s, th):
    n = s.n_atoms
    return dataclasses.replace(s, sigma=th[:n].copy(), epsilon=th[n:2 * n].copy(), dihedral_k=th[2 * n:].copy())


def _g(x, transform, center, width):
    return x if transform == 0 else 1.0 / (1.0 + np.exp(-(x - center) / width))


def _loss_forward(oracle_mod, s, q0, p0, k, t_gr, obs, transform, center, width):
    o = oracle_mod.Oracle(s)
    q, p = q0.copy(), p0.copy()
    f = np.stack([o.forces(x) for x in q])
    cap = k // t_gr
    samples = o.step_k(q, p, f, SEED, 0, 0, k, t_gr, cap=cap)  # [R, cap, n_obs]
    return float(np.mean(_g(samples[:, :, obs], transform, center, width)))


LOSSES = [
    ("end_to_end", 4, 0, 0.0, 1.0),
    ("phi_occupancy", 2, 1, np.radians(-81.0), np.radians(10.0)),
]


@pytest.mark.parametrize("name,obs,transform,center,width", LOSSES)
def test_adjoint_theta_gradient_matches_finite_differences(oracle_mod, name, obs, transform, center, width):
    s = W.chain_gradient()
    R, k, t_gr = 2, 40, 10
    q0, p0 = W.replica_states(s, R, seed=4, spread=0.002)
    o = oracle_mod.Oracle(s)
    f0 = np.stack([o.forces(x) for x in q0])
    L, gth, _, _ = o.adjoint_segment(q0.copy(), p0.copy(), f0.copy(), SEED, 0, 0, k, t_gr, obs, transform, center,
                                     width)
    assert abs(L - _loss_forward(oracle_mod, s, q0, p0, k, t_gr, obs, transform, center, width)) < 1e-13
    th = _theta(s)
    fd = np.zeros_like(th)
    for j in range(len(th)):
        h = 1e-6 * abs(th[j])
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        fd[j] = (_loss_forward(oracle_mod, _with_theta(s, tp), q0, p0, k, t_gr, obs, transform, center, width) -
                 _loss_forward(oracle_mod, _with_theta(s, tm), q0, p0, k, t_gr, obs, transform, center, width)) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0
    np.testing.assert_allclose(gth, fd, rtol=0, atol=2e-5 * scale)


@pytest.mark.parametrize("name,obs,transform,center,width", LOSSES)
def test_adjoint_state_gradient_matches_finite_differences(oracle_mod, name, obs, transform, center, width):
    s = W.chain_gradient()
    R, k, t_gr = 2, 40, 10
    q0, p0 = W.replica_states(s, R, seed=5, spread=0.002)
    o = oracle_mod.Oracle(s)
    f0 = np.stack([o.forces(x) for x in q0])
    _, _, gq, gp = o.adjoint_segment(q0.copy(), p0.copy(), f0.copy(), SEED, 0, 0, k, t_gr, obs, transform, center,
                                     width)
    rng = np.random.default_rng(1)
    idx = [tuple(int(v) for v in (rng.integers(R), rng.integers(s.n_atoms), rng.integers(3))) for _ in range(10)]
    for which, grad, base in (("q", gq, q0), ("p", gp, p0)):
        for (r, a, x) in idx:
            h = 1e-6 if which == "q" else 1e-4
            plus, minus = base.copy(), base.copy()
            plus[r, a, x] += h
            minus[r, a, x] -= h
            args = (plus, p0) if which == "q" else (q0, plus)
            argm = (minus, p0) if which == "q" else (q0, minus)
            fd = (_loss_forward(oracle_mod, s, *args, k, t_gr, obs, transform, center, width) -
                  _loss_forward(oracle_mod, s, *argm, k, t_gr, obs, transform, center, width)) / (2 * h)
            scale = np.abs(grad).max()
            assert abs(grad[r, a, x] - fd) < 1e-5 * scale + 1e-9, (which, r, a, x, grad[r, a, x], fd)
