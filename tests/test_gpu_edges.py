"""Edge cases of the CUDA path against the oracle: system sizes at and around the boundaries of the
force-field paths (the explicit item table below 64 atoms, 32-atom tiles from 64 on, ragged last
tiles), degenerate systems (one atom, one pair), segments longer than one launch, many replicas, and
a system without observables.
"""
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


def _forces(B, s, qs, prec):
    import torch

    sysh = B.grp_create_system(s, prec)
    dq = torch.tensor(qs, device="cuda", dtype=torch.float64)
    de = torch.zeros(len(qs), device="cuda", dtype=torch.float64)
    df = torch.zeros_like(dq)
    B.grp_energy_forces(sysh, len(qs), dq, de, df)
    return df.cpu().numpy(), de.cpu().numpy()


def _tiny(n):
    """n beads (1 or 2) with Lennard-Jones and charges, no bonded terms, COM-distance states."""
    s = W.chain(n_atoms=6)
    s = dataclasses.replace(s, n_atoms=n, mass=s.mass[:n], sigma=s.sigma[:n], epsilon=s.epsilon[:n],
                            charge=np.array([0.5, -0.5][:n]), excl=np.zeros((0, 2), np.int32),
                            bonds=None, bond_k=None, bond_r0=None, angles=None, angle_k=None, angle_theta0=None,
                            dihedrals=None, dihedral_n=None, dihedral_k=None, dihedral_delta=None,
                            cv_kind=W.CV_COM_DISTANCE, cv_atoms=(), cv_params=(1.0,),
                            groups=[[0], [n - 1]], observables=[(W.OBS_POTENTIAL, ())])
    s.q0 = np.array([[0.0, 0.0, 0.0], [0.37, 0.05, -0.02]])[:n]
    s.p0 = np.zeros((n, 3))
    return s


@pytest.mark.parametrize("n", [1, 2, 6, 7, 23, 63, 64, 65, 97])
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-6)])
def test_forces_across_path_boundaries(B, oracle_mod, n, prec, tol):
    s = _tiny(n) if n <= 2 else W.chain(n_atoms=n)
    o = oracle_mod.Oracle(s)
    rng = np.random.default_rng(n)
    qs = np.stack([s.q0 + 0.003 * rng.standard_normal(s.q0.shape) for _ in range(3)])
    fg, eg = _forces(B, s, qs, prec)
    for b, q in enumerate(qs):
        fo, eo = o.forces(q), o.potential(q)
        scale = max(np.abs(fo).max(), 1e-300)
        if n == 1:
            assert np.all(fg[b] == 0.0) and eg[b] == 0.0 and eo == 0.0
            continue
        assert np.abs(fg[b] - fo).max() < tol * scale
        assert abs(eg[b] - eo) < tol * max(abs(eo), scale)


def test_segment_longer_than_one_launch(B, oracle_mod):
    """45,000 steps are three launches (20,000 at most each): positions, momenta and the observable
    means match the oracle's single 45,000-step run (double well, FP64; the kernel's FMA contractions
    leave ~1e-16 per step, the same tolerance as a single launch), and the sample count and step
    counter carry over the launch boundaries exactly."""
    s = W.double_well_2d()
    R = 4
    q0, p0 = W.replica_states(s, R, seed=3, spread=0.05)
    o = oracle_mod.Oracle(s)
    q, p = q0.copy(), p0.copy()
    f = np.stack([o.forces(x) for x in q])
    samples = o.step_k(q, p, f, SEED, 0, 0, 45000, 10, cap=4500)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 45000, 10)
    qg, pg, acc, ctr = B.grp_get_state(rep)
    assert np.abs(qg - q).max() < 1e-9 * np.abs(q).max() and np.abs(pg - p).max() < 1e-9 * np.abs(p).max()
    assert ctr["t_global"] == 45000
    # accumulators (shift c, sum (O - c), sum (O - c)^2, n): the sample mean of each observable
    mean_o = samples.mean(axis=1)
    acc = acc.reshape(R, len(s.observables), 4)
    mean_g = acc[..., 0] + acc[..., 1] / acc[..., 3]
    assert np.all(acc[..., 3] == 4500)
    assert np.abs(mean_g - mean_o).max() < 1e-9 * max(1.0, np.abs(mean_o).max())


def test_many_replicas_sampled(B, oracle_mod):
    """4,096 replicas of the chain (FP64, 100 steps, 16 blocks per SM's worth of work): sampled
    replicas against the oracle, each drawing its own replica's noise."""
    s = W.chain(n_replicas=4096)
    R = 4096
    q0, p0 = W.replica_states(s, R, seed=9, spread=0.002)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 100, 0)
    qg, pg, _, _ = B.grp_get_state(rep)
    o = oracle_mod.Oracle(s)
    for r in (0, 1, 2047, 4095):
        q, p = q0[r].copy(), p0[r].copy()
        f = o.forces(q)
        for t in range(100):
            o.baoab_step(q, p, f, SEED, r, t)
        assert np.abs(qg[r] - q).max() < 1e-9 * np.abs(q).max()
        assert np.abs(pg[r] - p).max() < 1e-8 * np.abs(p).max()


def test_system_without_observables(B):
    """No observables: the convergence step never evaluates Eq. 4 and never converges; the whole
    loop stops at its step bound with reference exits only."""
    s = dataclasses.replace(W.alkane(), observables=[])
    s.q0, s.p0 = W.alkane().q0, W.alkane().p0
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, 8, SEED, s.q0, s.p0)
    st = B.grp_fv_check(rep, 40, 100, 10, 0.05, 0)
    assert st.gr_evaluated == 0 and st.converged == 0
    ev, _ = B.grp_run(rep, 10, 100, 0.05, 0, 5000, 100)
    assert all(e["kind"] in (B.EV_TRANSIENT, B.EV_REF_EXIT, B.EV_FV_ALL_EXITED) for e in ev)
    assert B.grp_get_state(rep)[3]["t_global"] >= 5000
