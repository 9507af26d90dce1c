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
    assert o.unconverged() == 0  # the reference itself met the tolerance at every projection
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


def _with_second_hydrogens(s, beads=(3, 7, 11, 15)):
    """The hydrogenated chain with a second constrained hydrogen on some beads: their two C-H bonds
    form one group of two coupled constraints (the FP64 group code on both paths), next to the
    single-bond groups (double-single on the mixed path).  The new hydrogen sits 0.109 nm from its bead
    along the normal of the plane of the bead and its two neighbours (90 degrees from the first
    hydrogen and from both C-C bonds); it is excluded from its bead, the bead's neighbours and the first
    hydrogen, and carries no angle term."""
    nh = len(s.constraints)
    q0 = [v for v in s.q0]
    extra, excl, cons = [], [tuple(e) for e in s.excl.tolist()], [tuple(c) for c in s.constraints.tolist()]
    for b in beads:
        h1 = nh + b
        nrm = np.cross(s.q0[b + 1] - s.q0[b], s.q0[b - 1] - s.q0[b])
        k = len(q0)
        q0.append(s.q0[b] + 0.109 * nrm / np.linalg.norm(nrm))
        extra.append(k)
        cons.append((b, k))
        for j in (b - 1, b, b + 1, h1):
            excl.append((min(j, k), max(j, k)))
    n = len(q0)
    ne = len(extra)
    s2 = dataclasses.replace(
        s, name=s.name + "h2", n_atoms=n, mass=np.concatenate([s.mass, np.full(ne, 1.008)]),
        charge=np.concatenate([s.charge, np.zeros(ne)]), sigma=np.concatenate([s.sigma, np.full(ne, 0.25)]),
        epsilon=np.concatenate([s.epsilon, np.full(ne, 0.1)]), excl=np.array(sorted(set(excl)), np.int32),
        constraints=np.array(cons, np.int32), constraint_length=np.full(len(cons), 0.109))
    s2.q0 = np.asarray(q0)
    s2.p0 = W.maxwell_boltzmann(s2.mass, s2.kT, 3, np.random.default_rng(5))
    return s2


@pytest.mark.parametrize("prec,steps,tq,tp", [(0, 200, 1e-9, 1e-8), (1, 1, 1e-8, 1e-6)])
def test_coupled_and_single_groups(B, oracle_mod, ch, prec, steps, tq, tp):
    """Groups of two coupled bonds (FP64 sweeps) beside single bonds (double-single on the mixed path)
    in one system: the FP64 path over 200 steps and the mixed path over one step against the oracle,
    with every bond at its length after 200 mixed steps.  The mixed bound on positions is that of its
    FP32 forces moving a hydrogen: 2e-6 of the largest force (1,880 kJ/mol/nm here) over one step of
    two half-kicks and two half-drifts, 2 h^2 dF / m_H ~ 7e-9 nm (measured 1.4e-9 nm)."""
    s = _with_second_hydrogens(ch)
    o = oracle_mod.Oracle(s)
    q0, p0 = _states(s, 4, 6)
    q, p = _oracle_run(o, q0, p0, steps)
    sysh = B.grp_create_system(s, prec)
    rep = B.grp_init_replicas(sysh, 4, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, steps, 0)
    qg, pg, _, _ = B.grp_get_state(rep)
    assert np.abs(qg - q).max() < tq * np.abs(q).max()
    assert np.abs(pg - p).max() < tp * np.abs(p).max()
    if prec == 1:
        B.grp_step_k(rep, 199, 0)
        qg = B.grp_get_state(rep)[0]
        i, j = s.constraints[:, 0], s.constraints[:, 1]
        assert np.abs(np.linalg.norm(qg[:, i] - qg[:, j], axis=-1) - 0.109).max() < 1e-9 * 0.109
