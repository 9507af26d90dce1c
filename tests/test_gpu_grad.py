"""Differentiation of V(q; theta) through the C ABI against the FP64 oracle (dV/dq = -F and the
parameter derivatives of orc_param_grad), and the torch.autograd wrapper.

Tolerances: the FP64 path sums every term in 2^-40 fixed point (quantum 9e-13 per term), so energies,
position gradients and parameter gradients agree with the oracle to ~1e-10 of their largest
component; the mixed path evaluates terms in FP32 (relative rounding ~1e-7 per term, amplified by
cancellation between repulsive and attractive terms) and is held to 2e-4 of the largest component.
"""
import dataclasses

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


def _configs(s, n_conf, seed, spread=0.02):
    rng = np.random.default_rng(seed)
    return s.q0[None] + spread * rng.standard_normal((n_conf,) + s.q0.shape)


def _theta(s):
    return np.concatenate([s.sigma, s.epsilon, s.dihedral_k])


def _reference(oracle_mod, s, q, w):
    o = oracle_mod.Oracle(s)
    e = np.array([o.potential(x) for x in q])
    gq = np.stack([-wb * o.forces(x) for wb, x in zip(w, q)])
    gth = sum(wb * o.param_grad(x) for wb, x in zip(w, q))
    return e, gq, gth


def _run(B, s, precision, q, w):
    import torch

    sysh = B.grp_create_system(s, precision)
    dq = torch.tensor(q, device="cuda")
    dw = torch.tensor(w, device="cuda")
    n_theta = B.grp_param_count(sysh)
    e = torch.empty(len(q), dtype=torch.float64, device="cuda")
    gq = torch.empty_like(dq)
    gth = torch.empty(n_theta, dtype=torch.float64, device="cuda")
    B.grp_energy_grad(sysh, len(q), dq, dw, e, gq, gth)
    return e.cpu().numpy(), gq.cpu().numpy(), gth.cpu().numpy()


def _close(a, b, rel):
    scale = max(np.abs(b).max(), 1e-30)
    assert np.abs(a - b).max() <= rel * scale, (np.abs(a - b).max() / scale, rel)


CASES = {
    "chain22": lambda: W.chain(22),
    "chain100_tiled": lambda: W.chain(100, seed=1811),
    "chain100_cutoff": lambda: dataclasses.replace(W.chain(100, seed=1811), cutoff=1.0),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_energy_grad_matches_oracle(B, oracle_mod, case, precision):
    s = CASES[case]()
    q = _configs(s, 6, seed=17)
    if s.cutoff > 0:  # no pair within rounding of the cutoff (the inclusion decision is then unique)
        for x in q:
            d = np.linalg.norm(x[:, None] - x[None], axis=-1)
            assert np.abs(d - s.cutoff).min() > 1e-9
    w = np.linspace(-1.5, 2.0, len(q))
    e_ref, gq_ref, gth_ref = _reference(oracle_mod, s, q, w)
    prec = B.GRP_FP64 if precision == "fp64" else B.GRP_MIXED
    e, gq, gth = _run(B, s, prec, q, w)
    assert gth.shape == _theta(s).shape
    rel = 1e-10 if precision == "fp64" else 2e-4
    _close(e, e_ref, rel)
    _close(gq, gq_ref, rel)
    n = s.n_atoms
    _close(gth[:n], gth_ref[:n], rel)
    _close(gth[n:2 * n], gth_ref[n:2 * n], rel)
    _close(gth[2 * n:], gth_ref[2 * n:], rel)


def test_set_params_changes_the_potential(B, oracle_mod):
    import torch

    s = W.chain(22)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    th0 = torch.empty(B.grp_param_count(sysh), dtype=torch.float64, device="cuda")
    B.grp_get_params(sysh, th0)
    np.testing.assert_array_equal(th0.cpu().numpy(), _theta(s))
    rng = np.random.default_rng(3)
    th = _theta(s) * (1 + 0.1 * rng.standard_normal(len(th0)))
    th[:s.n_atoms] = np.abs(th[:s.n_atoms])
    th[s.n_atoms:2 * s.n_atoms] = np.abs(th[s.n_atoms:2 * s.n_atoms])
    B.grp_set_params(sysh, torch.tensor(th, device="cuda"))
    n = s.n_atoms
    s2 = dataclasses.replace(s, sigma=th[:n], epsilon=th[n:2 * n], dihedral_k=th[2 * n:])
    q = _configs(s, 3, seed=4)
    e = torch.empty(3, dtype=torch.float64, device="cuda")
    B.grp_energy_grad(sysh, 3, torch.tensor(q, device="cuda"), None, e)
    o2 = oracle_mod.Oracle(s2)
    np.testing.assert_allclose(e.cpu().numpy(), [o2.potential(x) for x in q], rtol=1e-11, atol=1e-9)
    # invalid parameters are rejected and leave the system unchanged
    bad = th.copy()
    bad[0] = -0.1
    with pytest.raises(B.GrpError):
        B.grp_set_params(sysh, torch.tensor(bad, device="cuda"))
    th1 = torch.empty_like(th0)
    B.grp_get_params(sysh, th1)
    np.testing.assert_array_equal(th1.cpu().numpy(), th)


def test_autograd_function(B, oracle_mod):
    import torch

    from paper_1807_02431_gb300 import autograd as AG

    s = W.chain(22)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    q_np = _configs(s, 4, seed=8)
    q = torch.tensor(q_np, device="cuda", requires_grad=True)
    theta = torch.tensor(_theta(s), device="cuda", requires_grad=True)
    e = AG.potential_energy(sysh, q, theta)
    loss = (e * torch.arange(1, 5, dtype=torch.float64, device="cuda")).sum()
    loss.backward()
    w = np.arange(1, 5, dtype=np.float64)
    e_ref, gq_ref, gth_ref = _reference(oracle_mod, s, q_np, w)
    _close(e.detach().cpu().numpy(), e_ref, 1e-10)
    _close(q.grad.cpu().numpy(), gq_ref, 1e-10)
    _close(theta.grad.cpu().numpy(), gth_ref, 1e-10)
    # finite-difference check of the whole Function in a few random directions
    qd = torch.tensor(q_np[:1], device="cuda", requires_grad=True)
    td = theta.detach().clone().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda a, b: AG.potential_energy(sysh, a, b), (qd, td), eps=1e-6,
                                    atol=1e-4, rtol=1e-4, fast_mode=True)
