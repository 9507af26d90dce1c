"""Periodic electrostatics by particle mesh Ewald on the GPU against the oracle, on the chain with 20 ion
pairs in a 2.6 nm box (62 atoms; real-space cutoff 1.2 nm, beta = 2.6 / nm, 16^3 grid, cubic
B-splines).

Tolerances: the FP64 path does the oracle's arithmetic in another order (the grid sums in fixed point,
radix-2 transforms instead of the oracle's direct sums): 1e-12 of the largest force (measured 7e-14).
The mixed path transforms and interpolates in FP32: a 16-point transform loses a few ulp per axis and
each grid point sums ~60 overlapping charges, so the reciprocal forces carry relative errors of a few
1e-7 of the largest force (measured 3e-7 for forces, 5e-8 of the Coulomb energy's scale, the sum of
the magnitudes of its parts); 3e-6 bounds both.
"""
import dataclasses

import numpy as np
import pytest

from paper_1807_02431_gb300 import workloads as W

pytestmark = pytest.mark.gpu
SEED = 2431
TOL = {0: 1e-12, 1: 3e-6}


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_02431_gb300 import binding, build

    build.build()
    binding.load()
    return binding


def _forces(B, s, qs, prec):
    import torch

    sysh = B.grp_create_system(s, prec)
    dq = torch.tensor(qs, device="cuda", dtype=torch.float64)
    de = torch.zeros(len(qs), device="cuda", dtype=torch.float64)
    df = torch.zeros_like(dq)
    B.grp_energy_forces(sysh, len(qs), dq, de, df)
    return df.cpu().numpy(), de.cpu().numpy()


def _configs(s, k, seed, spread=0.01):
    rng = np.random.default_rng(seed)
    return np.stack([s.q0 + spread * rng.standard_normal(s.q0.shape) for _ in range(k)])


# grids of 8 points on the first and third axes take the 8-point real-to-complex and fused passes
SHAPES = {"cube": {}, "ortho": dict(edge=(2.6, 2.9, 2.45), grid=(16, 8, 16)), "coarse": dict(grid=(8, 16, 8))}


@pytest.mark.parametrize("shape", list(SHAPES))
@pytest.mark.parametrize("prec", [0, 1])
def test_energy_forces(B, oracle_mod, shape, prec):
    s = W.chain_ions(**SHAPES[shape])
    o = oracle_mod.Oracle(s)
    qs = _configs(s, 3, 11)
    fg, eg = _forces(B, s, qs, prec)
    for b, q in enumerate(qs):
        fo, eo = o.forces(q), o.potential(q)
        escale = np.abs(o.ewald_parts(q)).sum()
        ferr = np.abs(fg[b] - fo).max() / np.abs(fo).max()
        eerr = abs(eg[b] - eo) / escale
        assert ferr < TOL[prec], f"force error {ferr:.3e}"
        assert eerr < TOL[prec], f"energy error {eerr:.3e}"


@pytest.mark.parametrize("prec", [0, 1])
def test_positions_outside_the_box(B, oracle_mod, prec):
    """Unwrapped positions several boxes away give the forces of the wrapped ones."""
    s = W.chain_ions()
    o = oracle_mod.Oracle(s)
    q = _configs(s, 1, 12)[0]
    far = q + np.asarray(s.box) * np.array([3, -2, 5])
    moved = q.copy()
    moved[30:] += np.asarray(s.box) * np.array([1, 1, -1])  # the ions one box over
    fg, _ = _forces(B, s, np.stack([q, far, moved]), prec)
    fo = o.forces(q)
    for b in range(3):
        assert np.abs(fg[b] - fo).max() < TOL[prec] * np.abs(fo).max()


def test_fp64_trajectory(B, oracle_mod):
    s = W.chain_ions()
    o = oracle_mod.Oracle(s)
    q0, p0 = W.replica_states(s, 4, seed=3, spread=0.005)
    q, p = q0.copy(), p0.copy()
    f = np.stack([o.forces(x) for x in q])
    o.step_k(q, p, f, SEED, 0, 0, 200, 0)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, 4, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 200, 0)
    qg, pg, _, _ = B.grp_get_state(rep)
    assert np.abs(qg - q).max() < 1e-9 * np.abs(q).max()
    assert np.abs(pg - p).max() < 1e-8 * np.abs(p).max()


def test_mixed_one_step(B, oracle_mod):
    s = W.chain_ions()
    o = oracle_mod.Oracle(s)
    q0, p0 = W.replica_states(s, 8, seed=4, spread=0.005)
    q, p = q0.copy(), p0.copy()
    f = np.stack([o.forces(x) for x in q])
    o.step_k(q, p, f, SEED, 0, 0, 1, 0)
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, 8, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 1, 0)
    qg, pg, _, _ = B.grp_get_state(rep)
    assert np.abs(qg - q).max() < 1e-9 * np.abs(q).max()
    assert np.abs(pg - p).max() < 2e-5 * np.abs(p).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_potential_observable_and_equipartition(B, oracle_mod, prec):
    """3,000 steps of equilibration and 3,000 of sampling: the kinetic energy gives 2<K>/kT = 3N within
    3 %, and the final configurations' energies match the oracle's to the path's tolerance."""
    s = W.chain_ions()
    R = 256 if prec else 64
    sysh = B.grp_create_system(s, prec)
    rep = B.grp_init_replicas(sysh, R, SEED, s.q0, s.p0)
    B.grp_step_k(rep, 3000, 0)
    B.grp_set_state(rep, acc=np.zeros((R, len(s.observables), 4)))
    B.grp_step_k(rep, 3000, 10)
    q, p, acc, _ = B.grp_get_state(rep)
    assert np.all(np.isfinite(q)) and np.all(np.isfinite(p))
    kin = [k for k, (kind, _) in enumerate(s.observables) if kind == W.OBS_KINETIC][0]
    a = acc.reshape(R, len(s.observables), 4)[:, kin]
    mean_k = (a[:, 0] + a[:, 1] / a[:, 3]).mean()
    assert 2 * mean_k / s.kT == pytest.approx(3 * s.n_atoms, rel=0.03)
    o = oracle_mod.Oracle(s)
    f, e = _forces(B, s, q[:4], prec)
    for r in range(4):
        assert abs(e[r] - o.potential(q[r])) < TOL[prec] * np.abs(o.ewald_parts(q[r])).sum()


def test_loop_runs(B):
    s = W.chain_ions()
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, 64, SEED, s.q0, s.p0)
    ev, _ = B.grp_run(rep, s.t_gr, s.t_check, s.tol, 0, 10 * s.t_check, 3)
    assert B.grp_get_state(rep)[3]["t_global"] >= 10 * s.t_check or ev


def test_declined_and_invalid(B):
    s = W.chain_ions()
    for bad, code in ((dataclasses.replace(s, pme_grid=(32, 16, 16)), B.GRP_ENOTIMPL),
                      (dataclasses.replace(s, pme_order=6), B.GRP_ENOTIMPL),
                      (dataclasses.replace(s, cutoff=1.31), B.GRP_EINVAL),
                      (dataclasses.replace(s, ewald_beta=0.0), B.GRP_EINVAL),
                      (dataclasses.replace(s, box=(2.6, 0.0, 2.6)), B.GRP_EINVAL),
                      # 64 atoms take the Verlet list, whose cutoff + skin (1.4 nm) exceeds half the box
                      (W.chain_ions(n_pairs=21), B.GRP_EINVAL)):
        with pytest.raises(B.GrpError) as e:
            B.grp_create_system(bad, B.GRP_MIXED)
        assert e.value.status == code
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, 2, SEED, s.q0, s.p0)
    with pytest.raises(B.GrpError) as e:
        B.grp_batch_create([rep])
    assert e.value.status == B.GRP_ENOTIMPL
    with pytest.raises(B.GrpError) as e:
        B.grp_adjoint_segment(rep, 10, 10, 5, obs=0)
    assert e.value.status == B.GRP_ENOTIMPL
