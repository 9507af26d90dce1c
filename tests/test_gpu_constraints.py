"""Bond constraints (SHAKE / RATTLE in BAOAB) on the GPU against the oracle, on the chain with one
constrained hydrogen per bead (44 atoms, 22 constraints)."""
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


@pytest.fixture(scope="module")
def ch():
    return W.chain_h()


def _states(s, R, seed):
    """The built configuration (bonds at their lengths) with Maxwell-Boltzmann momenta, which the
    first B step's RATTLE projects onto the constraints."""
    rng = np.random.default_rng(seed)
    q = np.repeat(s.q0[None], R, 0) + 0.0
    p = np.stack([W.maxwell_boltzmann(s.mass, s.kT, 3, rng) for _ in range(R)])
    return q, p


def _oracle_run(o, q0, p0, k, seed=SEED):
    q, p = q0.copy(), p0.copy()
    f = np.stack([o.forces(x) for x in q])
    o.step_k(q, p, f, seed, 0, 0, k, 0)
    return q, p


def test_fp64_trajectory(B, oracle_mod, ch):
    o = oracle_mod.Oracle(ch)
    q0, p0 = _states(ch, 4, 1)
    q, p = _oracle_run(o, q0, p0, 200)
    sysh = B.grp_create_system(ch, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, 4, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 200, 0)
    qg, pg, _, _ = B.grp_get_state(rep)
    assert np.abs(qg - q).max() < 1e-9 * np.abs(q).max()
    assert np.abs(pg - p).max() < 1e-8 * np.abs(p).max()


def test_mixed_one_step(B, oracle_mod, ch):
    o = oracle_mod.Oracle(ch)
    q0, p0 = _states(ch, 8, 2)
    q, p = _oracle_run(o, q0, p0, 1)
    sysh = B.grp_create_system(ch, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, 8, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 1, 0)
    qg, pg, _, _ = B.grp_get_state(rep)
    assert np.abs(qg - q).max() < 1e-9 * np.abs(q).max()
    assert np.abs(pg - p).max() < 1e-6 * np.abs(p).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_constraints_hold_and_equipartition(B, ch, prec):
    """After 15,000 steps of 256 replicas every bond holds to 1e-9 of its length with no relative
    velocity along it, and the kinetic energy sampled over the last 5,000 steps gives
    2<K>/kT = 3N - N_c = 110 within 3 % (the built chain is strained: its first ~5 ps are warmer, as
    in the oracle)."""
    R = 256
    q0, p0 = _states(ch, R, 3)
    sysh = B.grp_create_system(ch, prec)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 10000, 0)  # equilibration
    B.grp_set_state(rep, acc=np.zeros((R, len(ch.observables), 4)))
    B.grp_step_k(rep, 5000, 20)
    q, p, acc, _ = B.grp_get_state(rep)
    i, j = ch.constraints[:, 0], ch.constraints[:, 1]
    r = q[:, i] - q[:, j]
    assert np.abs(np.linalg.norm(r, axis=-1) - ch.constraint_length).max() < 1e-9 * 0.109
    v = p[:, i] / ch.mass[i][:, None] - p[:, j] / ch.mass[j][:, None]
    assert np.abs((r * v).sum(-1)).max() < 1e-8 * 0.109 ** 2 / ch.dt
    kin = [k for k, (kind, _) in enumerate(ch.observables) if kind == W.OBS_KINETIC][0]
    a = acc.reshape(R, len(ch.observables), 4)[:, kin]
    mean_k = (a[:, 0] + a[:, 1] / a[:, 3]).mean()
    assert 2 * mean_k / ch.kT == pytest.approx(3 * ch.n_atoms - len(ch.constraints), rel=0.03)


def test_loop_runs_with_constraints(B, ch):
    sysh = B.grp_create_system(ch, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, 64, SEED, ch.q0, ch.p0)
    ev, _ = B.grp_run(rep, ch.t_gr, ch.t_check, ch.tol, 0, 10 * ch.t_check, 3)
    assert B.grp_get_state(rep)[3]["t_global"] >= 10 * ch.t_check or ev


def test_unconverged_sweeps_are_reported(B, ch):
    """A sweep bound too small for the tolerance is reported as GRP_ETIMEOUT (the kernel flags it and
    finishes the segment; nothing waits)."""
    s = dataclasses.replace(ch, constraint_max_iter=1, constraint_tol=1e-14)
    q0, p0 = _states(s, 4, 4)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, 4, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 10, 0)
    with pytest.raises(B.GrpError) as e:
        B.grp_fv_check(rep, 0, 10, 10, 0.01, 0)
    assert e.value.status == B.GRP_ETIMEOUT


def test_declined_combinations(B, ch):
    for bad in (dataclasses.replace(ch, cutoff=1.2, coulomb_mode=W.COULOMB_REACTION_FIELD),
                W.solvated(ch)):
        with pytest.raises(B.GrpError) as e:
            B.grp_create_system(bad, B.GRP_MIXED)
        assert e.value.status == B.GRP_ENOTIMPL
    sysh = B.grp_create_system(ch, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, 2, SEED, ch.q0, ch.p0)
    with pytest.raises(B.GrpError) as e:
        B.grp_batch_create([rep])
    assert e.value.status == B.GRP_ENOTIMPL
    with pytest.raises(B.GrpError) as e:
        B.grp_adjoint_segment(rep, 10, 10, 5, obs=0)
    assert e.value.status == B.GRP_ENOTIMPL
