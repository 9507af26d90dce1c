"""Particle mesh Ewald on the Verlet-list path (systems of 64 atoms and more) against the oracle: the
100-bead chain with 60 ion pairs in a periodic 4.0 nm box (220 atoms; real-space cutoff 1.2 nm over
nearest images, beta = 2.6 / nm, 16^3 grid, cubic B-splines).  The list is built over nearest images
(tile gaps from the box centres' nearest image, pair distances likewise), so a pair within cutoff +
skin has one image, which cutoff + skin <= half the box guarantees.

Tolerances as for the small periodic system: FP64 1e-12 of the largest force (the oracle's
arithmetic in another order), mixed 3e-6 (FP32 transforms and interpolation); trajectories 1e-9 on
FP64 positions over 200 steps, one mixed step within the local error of its FP32 forces.
"""
import dataclasses

import numpy as np
import pytest

from paper_1807_02431_gb300 import workloads as W

pytestmark = pytest.mark.gpu
SEED = 2431
TOL = {0: 1e-12, 1: 3e-6}


def _system(**kw):
    return W.chain_ions(n_chain=100, n_pairs=60, edge=4.0, **kw)


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


def test_system_takes_the_list_path(B):
    s = _system()
    assert s.n_atoms == 220 and s.n_atoms >= 64
    assert 7.0 / 6.0 * s.cutoff <= 0.5 * min(s.box)


@pytest.mark.parametrize("prec", [0, 1])
def test_energy_forces(B, oracle_mod, prec):
    s = _system()
    o = oracle_mod.Oracle(s)
    qs = _configs(s, 2, 21)
    fg, eg = _forces(B, s, qs, prec)
    for b, q in enumerate(qs):
        fo, eo = o.forces(q), o.potential(q)
        escale = np.abs(o.ewald_parts(q)).sum()
        ferr = np.abs(fg[b] - fo).max() / np.abs(fo).max()
        eerr = abs(eg[b] - eo) / escale
        print(f"prec={prec} force {ferr:.2e} energy {eerr:.2e}")
        assert ferr < TOL[prec], f"force error {ferr:.3e}"
        assert eerr < TOL[prec], f"energy error {eerr:.3e}"


@pytest.mark.parametrize("prec", [0, 1])
def test_positions_outside_the_box(B, oracle_mod, prec):
    """Unwrapped positions several boxes away, and the ions moved one box over, give the forces of the
    original configuration."""
    s = _system()
    o = oracle_mod.Oracle(s)
    q = _configs(s, 1, 22)[0]
    far = q + np.asarray(s.box) * np.array([2, -3, 4])
    moved = q.copy()
    moved[100:] += np.asarray(s.box) * np.array([-1, 1, 1])
    fg, _ = _forces(B, s, np.stack([q, far, moved]), prec)
    fo = o.forces(q)
    for b in range(3):
        assert np.abs(fg[b] - fo).max() < TOL[prec] * np.abs(fo).max()


def test_fp64_trajectory(B, oracle_mod):
    """200 FP64 steps (Verlet-list rebuilds included) against the oracle's all-pairs dynamics."""
    s = _system()
    o = oracle_mod.Oracle(s)
    R = 3
    q0, p0 = W.replica_states(s, R, seed=23, spread=0.005)
    q, p = q0.copy(), p0.copy()
    f = np.stack([o.forces(x) for x in q])
    o.step_k(q, p, f, SEED, 0, 0, 200, 0)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 200, 0)
    qg, pg, _, _ = B.grp_get_state(rep)
    print(f"fp64 200 steps q {np.abs(qg - q).max() / np.abs(q).max():.2e} p {np.abs(pg - p).max() / np.abs(p).max():.2e}")
    assert np.abs(qg - q).max() < 1e-9 * np.abs(q).max()
    assert np.abs(pg - p).max() < 1e-8 * np.abs(p).max()


def test_mixed_one_step(B, oracle_mod):
    s = _system()
    o = oracle_mod.Oracle(s)
    R = 4
    q0, p0 = W.replica_states(s, R, seed=24, spread=0.005)
    q, p = q0.copy(), p0.copy()
    f = np.stack([o.forces(x) for x in q])
    o.step_k(q, p, f, SEED, 0, 0, 1, 0)
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 1, 0)
    qg, pg, _, _ = B.grp_get_state(rep)
    assert np.abs(qg - q).max() < 1e-9 * np.abs(q).max()
    assert np.abs(pg - p).max() < 2e-5 * np.abs(p).max()


def test_equipartition_and_final_energies(B, oracle_mod):
    """Mixed path, 256 replicas: 6,000 steps of equilibration and 4,000 of sampling (many list
    rebuilds, while the ions condense and the pair count grows); 2<K>/kT = 3N within 3 %, and the final
    configurations' energies match the oracle's.  (The ions' condensation releases heat: 2<K>/(3N kT)
    is 1.71 over the first 2,000 steps and 1.003 over steps 6,000-8,000, on both precision paths.)"""
    s = _system()
    R = 256
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, R, SEED, s.q0, s.p0)
    B.grp_step_k(rep, 6000, 0)
    B.grp_set_state(rep, acc=np.zeros((R, len(s.observables), 4)))
    B.grp_step_k(rep, 4000, 10)
    q, p, acc, _ = B.grp_get_state(rep)
    assert np.all(np.isfinite(q)) and np.all(np.isfinite(p))
    kin = [k for k, (kind, _) in enumerate(s.observables) if kind == W.OBS_KINETIC][0]
    a = acc.reshape(R, len(s.observables), 4)[:, kin]
    mean_k = (a[:, 0] + a[:, 1] / a[:, 3]).mean()
    assert 2 * mean_k / s.kT == pytest.approx(3 * s.n_atoms, rel=0.03)
    o = oracle_mod.Oracle(s)
    _, e = _forces(B, s, q[:3], B.GRP_MIXED)
    for r in range(3):
        assert abs(e[r] - o.potential(q[r])) < TOL[1] * np.abs(o.ewald_parts(q[r])).sum()


def test_box_too_small_for_the_list(B):
    """A 64-atom-or-larger periodic system keeps a Verlet list, which needs cutoff + skin (7/6 of the
    cutoff) within half the shortest edge: 1.4 nm in a 2.6 nm box is declined."""
    for bad in (W.chain_ions(n_chain=100, n_pairs=60, edge=2.6),
                dataclasses.replace(_system(), cutoff=1.75)):
        with pytest.raises(B.GrpError) as e:
            B.grp_create_system(bad, B.GRP_MIXED)
        assert e.value.status == B.GRP_EINVAL


def test_loop_runs(B):
    """The loop of Fig. 1 on the periodic list system (mixed): ten exit tests without an error."""
    s = _system()
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, 64, SEED, s.q0, s.p0)
    ev, _ = B.grp_run(rep, s.t_gr, s.t_check, s.tol, 0, 10 * s.t_check, 3)
    assert B.grp_get_state(rep)[3]["t_global"] >= 10 * s.t_check or ev
