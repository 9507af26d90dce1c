"""Parity of the CUDA path (through the C ABI) against the FP64 oracle on identical seeded inputs.

Tolerances (stated for the two precisions of the library):
  FP64 path: positions and momenta within 1e-9 relative to the largest |q| (|p|) after 1,000 steps;
             labels, exit indices and branch sources bit-exact.
  mixed path: positions within 1e-4 relative after 1,000 steps (FP32 forces into fixed point,
             double-single integration, FP32 noise); labels/exits/branches bit-exact against the GPU
             FP64 path when both restart from the same FP64 state (one segment).
Integer and index outputs (labels, exited flags, branch sources, M, k, tau) are compared exactly.
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


@pytest.fixture(scope="module")
def chain():
    return W.chain()


def _oracle(oracle_mod, s):
    return oracle_mod.Oracle(s)


def _oracle_step(o, q0, p0, t0, tp0, k, t_gr):
    q, p = q0.copy(), p0.copy()
    f = np.stack([o.forces(q[r]) for r in range(q.shape[0])])
    cap = k // t_gr if t_gr else 0
    samples = o.step_k(q, p, f, SEED, t0, tp0, k, t_gr, cap=cap)
    return q, p, f, samples


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# ----------------------------------------------------------------------------- forces
@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 2e-4)])
def test_energy_forces_match_oracle(B, oracle_mod, chain, prec, tol):
    import torch

    o = _oracle(oracle_mod, chain)
    rng = np.random.default_rng(1)
    n = 16
    qs = np.stack([chain.q0 + 0.01 * rng.standard_normal(chain.q0.shape) for _ in range(n)])
    sysh = B.grp_create_system(chain, prec)
    dq = torch.tensor(qs, device="cuda", dtype=torch.float64)
    de = torch.zeros(n, device="cuda", dtype=torch.float64)
    df = torch.zeros_like(dq)
    B.grp_energy_forces(sysh, n, dq, de, df)
    torch.cuda.synchronize()
    fo = np.stack([o.forces(q) for q in qs])
    eo = np.array([o.potential(q) for q in qs])
    ferr = _rel(df.cpu().numpy(), fo)
    eerr = np.abs(de.cpu().numpy() - eo).max() / np.abs(eo).max()
    print(f"prec={prec} force rel err {ferr:.3e} energy rel err {eerr:.3e}")
    assert ferr < tol and eerr < tol


# ----------------------------------------------------------------------------- step_k
@pytest.mark.parametrize("prec", [0, 1])
def test_step_k_chain_matches_oracle(B, oracle_mod, chain, prec):
    """1,000 BAOAB steps of 8 distinct replicas with sampling every t_GR = 10 steps."""
    s = chain
    o = _oracle(oracle_mod, s)
    R, k = 8, 1000
    q0, p0 = W.replica_states(s, R, seed=3, spread=0.003)
    qo, po, _, samples = _oracle_step(o, q0, p0, 0, 0, k, s.t_gr)
    sysh = B.grp_create_system(s, prec)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, k, s.t_gr)
    q, p, acc, ctr = B.grp_get_state(rep)
    eq, ep = _rel(q, qo), _rel(p, po)
    # accumulators -> per-replica means and variances of every observable
    n = acc[..., 3]
    mean = acc[..., 0] + acc[..., 1] / n
    var = acc[..., 2] / n - (acc[..., 1] / n) ** 2
    mo, vo = samples.mean(axis=1), samples.var(axis=1)
    em = np.abs(mean - mo).max(axis=0) / np.abs(mo).max(axis=0)
    ev = np.abs(var - vo).max(axis=0) / np.abs(vo).max(axis=0)
    print(f"prec={prec} q {eq:.3e} p {ep:.3e} obs-mean {em} obs-var {ev}")
    assert ctr["t_global"] == k and ctr["t_phase"] == k
    assert np.all(n == k // s.t_gr)
    tol = 1e-9 if prec == 0 else 1e-4
    assert eq < tol
    assert ep < (1e-9 if prec == 0 else 1e-3)
    assert np.all(em < (1e-9 if prec == 0 else 1e-3))


def test_step_k_double_well_matches_oracle(B, oracle_mod):
    s = W.double_well_2d()
    o = _oracle(oracle_mod, s)
    R, k = 32, 5000
    q0, p0 = W.replica_states(s, R, seed=4, spread=0.3)
    qo, po, _, samples = _oracle_step(o, q0, p0, 123, 7, k, s.t_gr)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_set_state(rep, counters={"t_global": 123, "t_phase": 7})
    B.grp_step_k(rep, k, s.t_gr)
    q, p, acc, _ = B.grp_get_state(rep)
    n = acc[..., 3]
    mean = acc[..., 0] + acc[..., 1] / n
    print("dw", _rel(q, qo), _rel(p, po), np.abs(mean - samples.mean(axis=1)).max())
    assert _rel(q, qo) < 1e-9 and _rel(p, po) < 1e-9
    assert np.all(n == samples.shape[1])
    assert np.abs(mean - samples.mean(axis=1)).max() < 1e-9


# ----------------------------------------------------------------------------- checks and branching
@pytest.mark.parametrize("prec", [0, 1])
def test_check_states_bit_exact(B, oracle_mod, chain, prec):
    import torch

    s = chain
    o = _oracle(oracle_mod, s)
    R = 64
    q0, p0 = W.replica_states(s, R, seed=5)
    rng = np.random.default_rng(5)
    # rotate the central dihedrals by random amounts so that both states are populated
    c = s.cv_atoms
    for r in range(R):
        ang = rng.uniform(-np.pi, np.pi)
        axis = q0[r, c[2]] - q0[r, c[1]]
        axis /= np.linalg.norm(axis)
        K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
        Rm = np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K
        tail = np.arange(c[2] + 1, s.n_atoms)
        q0[r, tail] = (q0[r, tail] - q0[r, c[2]]) @ Rm.T + q0[r, c[2]]
    sysh = B.grp_create_system(s, prec)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    for omega in (0, 1):
        lab = torch.zeros(R, dtype=torch.int8, device="cuda")
        ex = torch.zeros(R, dtype=torch.uint8, device="cuda")
        B.grp_check_states(rep, omega, lab, ex)
        torch.cuda.synchronize()
        lo = np.array([o.state_of(q0[r]) for r in range(R)])
        eo = np.array([o.exited(q0[r], omega) for r in range(R)])
        assert np.array_equal(lab.cpu().numpy(), lo)
        assert np.array_equal(ex.cpu().numpy(), eo)
    assert 0 < (lo == 0).sum() < R


def test_fv_branch_bit_exact(B, oracle_mod, chain):
    import torch

    s = chain
    R = 96
    q0, p0 = W.replica_states(s, R, seed=6, spread=0.01)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_set_state(rep, counters={"t_global": 777, "t_phase": 0})
    rng = np.random.default_rng(7)
    for trial in range(4):
        exm = (rng.random(R) < [0.3, 0.9, 1.0, 0.0][trial]).astype(np.uint8)
        dex = torch.tensor(exm, device="cuda")
        dsrc = torch.zeros(R, dtype=torch.int32, device="cuda")
        qb, pb, _, _ = B.grp_get_state(rep)
        nb = B.grp_fv_branch(rep, dex, dsrc)
        nbo, srco = oracle_mod.fv_branch(SEED, 777, exm)
        assert nb == nbo
        assert np.array_equal(dsrc.cpu().numpy(), srco)
        qa, pa, _, _ = B.grp_get_state(rep)
        for r in range(R):
            src = srco[r] if srco[r] >= 0 else r
            assert np.array_equal(qa[r], qb[src]) and np.array_equal(pa[r], pb[src])


def test_gelman_rubin_matches_oracle(B, oracle_mod, chain):
    s = chain
    o = _oracle(oracle_mod, s)
    R, k = 12, 2000
    q0, p0 = W.replica_states(s, R, seed=8, spread=0.002)
    _, _, _, samples = _oracle_step(o, q0, p0, 0, 0, k, s.t_gr)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, k, s.t_gr)
    rhat, conv = B.grp_gelman_rubin(rep, 0.01)
    ro = np.array([oracle_mod.gelman_rubin(samples[1:, :, j]) for j in range(len(s.observables))])
    print("rhat", rhat, ro)
    assert np.all(np.abs(rhat - ro) <= 1e-9 * ro)
    assert conv == bool(np.all(ro < 1.01))


# ----------------------------------------------------------------------------- Eq. 5 and the loop
def test_parallel_phase_double_well_bit_exact(B, oracle_mod):
    s = W.double_well_2d()
    o = _oracle(oracle_mod, s)
    R = 32
    q0, p0 = W.replica_states(s, R, seed=9, spread=0.05)
    q0[:, 0, 0] = -0.6
    qo, po = q0.copy(), p0.copy()
    fo = np.stack([o.forces(qo[r]) for r in range(R)])
    found, exo = o.parallel_phase(qo, po, fo, SEED, 0, 0, s.t_check, 10 ** 5)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    ex = B.grp_run_parallel_phase(rep, 0, s.t_check, 10 ** 5)
    print(ex, exo)
    assert found and ex is not None
    assert (ex["M"], ex["k"], ex["tau_steps"], ex["label_to"]) == (exo["M"], exo["k"], exo["tau_steps"], exo["label_to"])


def test_genparrep_loop_double_well_bit_exact(B, oracle_mod):
    """The whole loop of Fig. 1 on the double well: the event log (phases, t_FV, t_ref, M, k, tau,
    labels, branch counts, clock) equals the oracle's exactly."""
    s = W.double_well_2d()
    o = _oracle(oracle_mod, s)
    evo, tgo = o.run_genparrep(s.n_replicas, SEED, s.t_gr, s.t_check, 0.05, s.min_fv_steps, 10 ** 8, 6,
                               q0=s.q0, p0=s.p0)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, s.n_replicas, SEED, s.q0, s.p0)
    ev, tsim = B.grp_run(rep, s.t_gr, s.t_check, 0.05, s.min_fv_steps, 10 ** 8, 6)
    for a, b in zip(ev, evo):
        print(a, b)
    assert ev == evo
    assert tsim == evo[-1]["t_sim"]


# ----------------------------------------------------------------------------- mixed vs FP64 GPU
def test_mixed_vs_fp64_segment_labels(B, chain):
    """Segment protocol: both paths restart from the same FP64 state, run one 1,000-step segment with
    the same Philox stream; labels and exited flags agree exactly, positions within 1e-4."""
    import torch

    s = chain
    R = 64
    q0, p0 = W.replica_states(s, R, seed=10, spread=0.003)
    out = {}
    for prec in (0, 1):
        sysh = B.grp_create_system(s, prec)
        rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
        B.grp_step_k(rep, 1000, s.t_gr)
        lab = torch.zeros(R, dtype=torch.int8, device="cuda")
        ex = torch.zeros(R, dtype=torch.uint8, device="cuda")
        B.grp_check_states(rep, 1, lab, ex)
        q, _, _, _ = B.grp_get_state(rep)
        out[prec] = (lab.cpu().numpy(), ex.cpu().numpy(), q)
    print("mixed vs fp64", _rel(out[1][2], out[0][2]))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert _rel(out[1][2], out[0][2]) < 1e-4


def test_deterministic(B, chain):
    s = chain
    R = 16
    q0, p0 = W.replica_states(s, R, seed=12, spread=0.003)
    res = []
    for _ in range(2):
        sysh = B.grp_create_system(s, B.GRP_MIXED)
        rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
        B.grp_step_k(rep, 500, s.t_gr)
        q, p, acc, _ = B.grp_get_state(rep)
        res.append((q, p, acc))
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)


# ----------------------------------------------------------------------------- full size
def test_full_size_chain_sampled_replicas(B, oracle_mod, chain):
    """256 replicas of the 22-bead chain, the benchmark's launch configuration: one 500-step F-V
    segment of the mixed path; sampled replicas against the oracle (1e-4)."""
    s = chain
    o = _oracle(oracle_mod, s)
    R = s.n_replicas
    q0, p0 = W.replica_states(s, R, seed=13, spread=0.002)
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, s.t_check, s.t_gr)
    q, _, _, _ = B.grp_get_state(rep)
    for r in (0, 1, 127, 255):
        qo, po = q0[r:r + 1].copy(), p0[r:r + 1].copy()
        fo = o.forces(qo[0])[None].copy()
        # the oracle's batch index is the replica index of the noise stream: run replica r alone by
        # stepping a batch of r + 1 replicas would be wasteful, so step one replica with index r
        for t in range(s.t_check):
            o.baoab_step(qo[0], po[0], fo[0], SEED, r, t)
        assert _rel(q[r], qo[0]) < 1e-4


# ----------------------------------------------------------------------------- edge cases
def test_invalid_arguments(B, chain):
    import copy

    bad = copy.deepcopy(chain)
    bad.bonds = bad.bonds.copy()
    bad.bonds[0, 1] = 999
    with pytest.raises(B.GrpError) as e:
        B.grp_create_system(bad, B.GRP_FP64)
    assert e.value.status == B.GRP_EINVAL
    sysh = B.grp_create_system(chain, B.GRP_FP64)
    with pytest.raises(B.GrpError):
        B.grp_init_replicas(sysh, 0, SEED, chain.q0, chain.p0)
    rep = B.grp_init_replicas(sysh, 1, SEED, chain.q0, chain.p0)
    B.grp_step_k(rep, 0, 10)  # empty segment is a no-op
    with pytest.raises(B.GrpError):
        B.grp_step_k(rep, 10, 10, n_active=5)
    with pytest.raises(B.GrpError):
        B.grp_gelman_rubin(rep, 0.01)  # one replica: no F-V worker


def test_transient_steps_reference_only(B, chain):
    s = chain
    R = 4
    q0, p0 = W.replica_states(s, R, seed=14, spread=0.003)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 50, 0, n_active=1)
    q, _, _, _ = B.grp_get_state(rep)
    assert not np.array_equal(q[0], q0[0])
    assert np.array_equal(q[1:], q0[1:])
