"""Parity of the CUDA path (through the C ABI) against the FP64 oracle on identical seeded inputs.

Tolerances, derived for the 22-bead chain whose dynamics is chaotic: in the oracle itself a relative
position perturbation of 1e-13 grows by x1e5 (median) to x2e6 (worst of 8 replicas) in 1,000 steps
(tests/test_oracle_sensitivity.py pins this).  Hence:
  FP64 path: positions within 1e-9 and momenta within 1e-8 relative (to the largest |q|, |p|) after
             1,000 steps
             (the library's per-step differences from the oracle are ~1e-16: FMA contraction, the
             2^-40 fixed-point quantum of the force sum, and the transcendental functions of the
             Box-Muller normals, CUDA's log and sincospi against glibc's log, cos and sin, a few ulps
             apart on identical Philox words); labels, exit indices, branch sources exact.
  mixed path: FP32 forces and FP32 normals carry ~1e-7 relative rounding every step, which the chain
             amplifies beyond any fixed tolerance after ~500 steps; so the mixed path is held to (i) the one-step local
             error (positions 1e-9, momenta 1e-6 relative), (ii) positions within 1e-4 relative after
             200 steps, (iii) labels identical to the GPU FP64 path after one 500-step exit-test
             segment from the same FP64 state for every replica whose CV is further than 2 degrees from
             a boundary.
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


def _oracle_step(o, q0, p0, t0, tp0, k, t_gr, replicas=None):
    """Advance copies of (q0, p0) k steps in the oracle; `replicas` gives each row's noise index."""
    q, p = q0.copy(), p0.copy()
    f = np.stack([o.forces(q[r]) for r in range(q.shape[0])])
    if replicas is None:
        cap = k // t_gr if t_gr else 0
        samples = o.step_k(q, p, f, SEED, t0, tp0, k, t_gr, cap=cap)
        return q, p, f, samples
    for row, rid in enumerate(replicas):
        for t in range(k):
            o.baoab_step(q[row], p[row], f[row], SEED, rid, t0 + t)
    return q, p, f, None


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _rotate_tail(q, axis_from, axis_to, first, ang):
    axis = q[axis_to] - q[axis_from]
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    Rm = np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K
    q[first:] = (q[first:] - q[axis_to]) @ Rm.T + q[axis_to]


def _spread_states(s, R, seed):
    """Replicas whose central (phi, psi) cover both states: the chain is turned about the two
    central bonds by random angles, redrawn while any non-excluded pair is closer than 0.8 sigma."""
    q0, p0 = W.replica_states(s, R, seed=seed)
    rng = np.random.default_rng(seed)
    c = s.cv_atoms
    excl = {tuple(x) for x in s.excl.tolist()}
    sig = 0.5 * (s.sigma[:, None] + s.sigma[None, :])
    for r in range(R):
        while True:
            q = q0[r].copy()
            _rotate_tail(q, c[1], c[2], c[3], rng.uniform(-np.pi, np.pi))
            _rotate_tail(q, c[2], c[3], c[4], rng.uniform(-np.pi, np.pi))
            d = np.linalg.norm(q[:, None] - q[None], axis=-1)
            ok = all(d[i, j] >= 0.8 * sig[i, j] for i in range(s.n_atoms) for j in range(i + 1, s.n_atoms)
                     if (i, j) not in excl)
            if ok:
                q0[r] = q
                break
    return q0, p0


# ----------------------------------------------------------------------------- forces
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-6)])
def test_energy_forces_match_oracle(B, oracle_mod, chain, prec, tol):
    """Forces and energies of 16 perturbed configurations (relative to the largest component)."""
    import torch

    o = oracle_mod.Oracle(chain)
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
def test_step_k_chain_fp64_matches_oracle(B, oracle_mod, chain):
    """FP64 path: 1,000 BAOAB steps of 8 distinct replicas with sampling every t_GR = 10 steps."""
    s = chain
    o = oracle_mod.Oracle(s)
    R, k = 8, 1000
    q0, p0 = W.replica_states(s, R, seed=3, spread=0.003)
    qo, po, _, samples = _oracle_step(o, q0, p0, 0, 0, k, s.t_gr)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, k, s.t_gr)
    q, p, acc, ctr = B.grp_get_state(rep)
    n = acc[..., 3]
    mean = acc[..., 0] + acc[..., 1] / n
    var = acc[..., 2] / n - (acc[..., 1] / n) ** 2
    mo, vo = samples.mean(axis=1), samples.var(axis=1)
    em = np.abs(mean - mo).max() / np.abs(mo).max()
    ev = (np.abs(var - vo) / np.abs(vo).max(axis=0)).max()
    print(f"fp64 q {_rel(q, qo):.3e} p {_rel(p, po):.3e} obs-mean {em:.3e} obs-var {ev:.3e}")
    assert ctr["t_global"] == k and ctr["t_phase"] == k
    assert np.all(n == k // s.t_gr)
    assert _rel(q, qo) < 1e-9 and _rel(p, po) < 1e-8
    assert em < 1e-9 and ev < 1e-6


def test_mixed_one_step_local_error(B, oracle_mod, chain):
    """Mixed path, one step from identical FP64 states: positions 1e-9, momenta 1e-6 relative."""
    s = chain
    o = oracle_mod.Oracle(s)
    R = 16
    q0, p0 = W.replica_states(s, R, seed=21, spread=0.003)
    qo, po, _, _ = _oracle_step(o, q0, p0, 0, 0, 1, 0)
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 1, 0)
    q, p, _, _ = B.grp_get_state(rep)
    print(f"mixed one step: q {_rel(q, qo):.3e} p {_rel(p, po):.3e}")
    assert _rel(q, qo) < 1e-9 and _rel(p, po) < 1e-6


def test_mixed_200_steps_matches_oracle(B, oracle_mod, chain):
    """Mixed path: 200 steps (before the chain's chaos amplifies FP32 rounding) within 1e-4; the
    observable accumulators of the same run within 1e-3 of the oracle's sample means."""
    s = chain
    o = oracle_mod.Oracle(s)
    R, k = 8, 200
    q0, p0 = W.replica_states(s, R, seed=3, spread=0.003)
    qo, po, _, samples = _oracle_step(o, q0, p0, 0, 0, k, s.t_gr)
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, k, s.t_gr)
    q, p, acc, _ = B.grp_get_state(rep)
    mean = acc[..., 0] + acc[..., 1] / acc[..., 3]
    em = np.abs(mean - samples.mean(axis=1)).max(axis=0) / np.abs(samples).max(axis=(0, 1))
    print(f"mixed 200 steps: q {_rel(q, qo):.3e} p {_rel(p, po):.3e} obs-mean {em}")
    assert _rel(q, qo) < 1e-4
    assert np.all(em < 1e-3)


def test_step_k_double_well_matches_oracle(B, oracle_mod):
    s = W.double_well_2d()
    o = oracle_mod.Oracle(s)
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
    assert _rel(q, qo) < 1e-9 and _rel(p, po) < 1e-9
    assert np.all(n == samples.shape[1])
    assert np.abs(mean - samples.mean(axis=1)).max() < 1e-9


# ----------------------------------------------------------------------------- checks and branching
@pytest.mark.parametrize("prec", [0, 1])
def test_check_states_bit_exact(B, oracle_mod, chain, prec):
    import torch

    s = chain
    o = oracle_mod.Oracle(s)
    R = 96
    q0, p0 = _spread_states(s, R, seed=5)
    sysh = B.grp_create_system(s, prec)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    lo = np.array([o.state_of(q0[r]) for r in range(R)])
    assert 0 < (lo == 0).sum() < R
    for omega in (0, 1):
        lab = torch.zeros(R, dtype=torch.int8, device="cuda")
        ex = torch.zeros(R, dtype=torch.uint8, device="cuda")
        B.grp_check_states(rep, omega, lab, ex)
        torch.cuda.synchronize()
        eo = np.array([o.exited(q0[r], omega) for r in range(R)])
        assert np.array_equal(lab.cpu().numpy(), lo)
        assert np.array_equal(ex.cpu().numpy(), eo)


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
        qb, pb, ab, _ = B.grp_get_state(rep)
        nb = B.grp_fv_branch(rep, dex, dsrc)
        nbo, srco = oracle_mod.fv_branch(SEED, 777, exm)
        assert nb == nbo
        assert np.array_equal(dsrc.cpu().numpy(), srco)
        qa, pa, aa, _ = B.grp_get_state(rep)
        for r in range(R):
            src = srco[r] if srco[r] >= 0 else r
            assert np.array_equal(qa[r], qb[src]) and np.array_equal(pa[r], pb[src])
            assert np.array_equal(aa[r], ab[src])


def test_gelman_rubin_kernel_from_oracle_samples(B, oracle_mod, chain):
    """Eq. 3 on the device from accumulators built from the oracle's own samples (shift = first
    sample), against the oracle's literal two-pass ratio: 1e-12 relative on R - 1."""
    s = chain
    o = oracle_mod.Oracle(s)
    R, k = 12, 2000
    q0, p0 = W.replica_states(s, R, seed=8, spread=0.002)
    _, _, _, samples = _oracle_step(o, q0, p0, 0, 0, k, s.t_gr)  # [R, n, obs]
    c = samples[:, 0, :]
    d = samples - c[:, None, :]
    acc = np.stack([c, d.sum(axis=1), (d * d).sum(axis=1), np.full(c.shape, samples.shape[1])], axis=-1)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_set_state(rep, acc=acc)
    rhat, conv = B.grp_gelman_rubin(rep, 0.01)
    ro = np.array([oracle_mod.gelman_rubin(samples[1:, :, j]) for j in range(len(s.observables))])
    print("rhat", rhat, ro)
    assert np.all(np.abs(rhat - ro) <= 1e-12 * (ro - 1) + 1e-15)
    assert conv == bool(np.all(ro < 1.01))


def test_gelman_rubin_end_to_end_fp64(B, oracle_mod, chain):
    """Sampling in the segment kernel plus the reduction, FP64 path, 400 steps: R within 1e-9."""
    s = chain
    o = oracle_mod.Oracle(s)
    R, k = 12, 400
    q0, p0 = W.replica_states(s, R, seed=8, spread=0.002)
    _, _, _, samples = _oracle_step(o, q0, p0, 0, 0, k, s.t_gr)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, k, s.t_gr)
    rhat, _ = B.grp_gelman_rubin(rep, 0.01)
    ro = np.array([oracle_mod.gelman_rubin(samples[1:, :, j]) for j in range(len(s.observables))])
    assert np.all(np.abs(rhat - ro) <= 1e-9 * ro)


# ----------------------------------------------------------------------------- Eq. 5 and the loop
def test_parallel_phase_double_well_bit_exact(B, oracle_mod):
    s = W.double_well_2d()
    o = oracle_mod.Oracle(s)
    R = 32
    q0, p0 = W.replica_states(s, R, seed=9, spread=0.05)
    q0[:, 0, 0] = -0.6
    qo, po = q0.copy(), p0.copy()
    fo = np.stack([o.forces(qo[r]) for r in range(R)])
    found, exo = o.parallel_phase(qo, po, fo, SEED, 0, 0, s.t_check, 10 ** 5)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    ex = B.grp_run_parallel_phase(rep, 0, s.t_check, 10 ** 5)
    assert found and ex is not None
    assert (ex["M"], ex["k"], ex["tau_steps"], ex["label_to"]) == (exo["M"], exo["k"], exo["tau_steps"], exo["label_to"])
    q, _, _, ctr = B.grp_get_state(rep)
    assert ctr["t_global"] == ex["M"] * s.t_check
    assert _rel(q, qo) < 1e-9


@pytest.mark.parametrize("order", [(0, 1, 2, 3, 4, 5, 6, 7), (5, 6, 7, 0, 1, 2, 3, 4)])
def test_parallel_phase_chain_fp64_bit_exact(B, oracle_mod, chain, order):
    """Eq. 5 on the chain (FP64 path): eight replicas in state 1 (outside the rectangle), several of
    them a few degrees from its edge, so that an exit comes within 40 checks of 50 steps (the oracle
    finds one at the third check; in the second ordering the first exit is replica k = 7, so the
    tie-break over indices is exercised).  An exit must be found; M, k, tau, the label entered and
    the positions at the exit check are those of the oracle."""
    s = chain
    o = oracle_mod.Oracle(s)
    R, tc = 16, 50
    q0, p0 = _spread_states(s, R, seed=31)
    keep = [r for r in range(R) if o.state_of(q0[r]) == 1]
    assert len(keep) >= 8
    q0, p0 = q0[keep][:8], p0[keep][:8]
    q0, p0 = q0[list(order)].copy(), p0[list(order)].copy()
    R = len(q0)
    qo, po = q0.copy(), p0.copy()
    fo = np.stack([o.forces(qo[r]) for r in range(R)])
    found, exo = o.parallel_phase(qo, po, fo, SEED, 0, 1, tc, 40)
    assert found, "the starts were chosen so that the oracle sees an exit within 40 checks"
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    ex = B.grp_run_parallel_phase(rep, 1, tc, 40)
    print(ex, exo)
    assert ex is not None
    assert (ex["M"], ex["k"], ex["tau_steps"], ex["label_to"]) == (exo["M"], exo["k"], exo["tau_steps"], exo["label_to"])
    assert exo["tau_steps"] == (R * (exo["M"] - 1) + exo["k"]) * tc
    q, _, _, ctr = B.grp_get_state(rep)
    assert ctr["t_global"] == ex["M"] * tc
    assert _rel(q, qo) < 1e-9


def test_genparrep_loop_double_well_bit_exact(B, oracle_mod):
    """The whole loop of Fig. 1 on the double well: the event log (phases, t_FV, t_ref, M, k, tau,
    labels, branch counts, clock) equals the oracle's exactly."""
    s = W.double_well_2d()
    o = oracle_mod.Oracle(s)
    evo, tgo = o.run_genparrep(s.n_replicas, SEED, s.t_gr, s.t_check, 0.05, s.min_fv_steps, 10 ** 8, 6,
                               q0=s.q0, p0=s.p0)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, s.n_replicas, SEED, s.q0, s.p0)
    ev, tsim = B.grp_run(rep, s.t_gr, s.t_check, 0.05, s.min_fv_steps, 10 ** 8, 6)
    assert ev == evo
    assert tsim == evo[-1]["t_sim"]
    assert B.grp_get_state(rep)[3]["t_global"] == tgo


# ----------------------------------------------------------------------------- mixed vs FP64 GPU
def test_mixed_vs_fp64_segment_labels(B, oracle_mod, chain):
    """Segment protocol: both paths restart from the same FP64 state and run one exit-test segment
    (t_check = 500 steps) with the same Philox stream; every replica whose FP64 CV is more than 2 degrees
    from a boundary of the rectangle has the same label and exit flag in both paths.  (Over 1,000 steps
    the chain's chaos, which amplifies differences up to x2e6, once moved a replica across a boundary
    from 2 degrees away: agreement is a per-segment property.)"""
    import torch

    s = chain
    o = oracle_mod.Oracle(s)
    R = 128
    q0, p0 = _spread_states(s, R, seed=10)
    out = {}
    for prec in (0, 1):
        sysh = B.grp_create_system(s, prec)
        rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
        B.grp_step_k(rep, s.t_check, s.t_gr)
        lab = torch.zeros(R, dtype=torch.int8, device="cuda")
        ex = torch.zeros(R, dtype=torch.uint8, device="cuda")
        B.grp_check_states(rep, 1, lab, ex)
        q, _, _, _ = B.grp_get_state(rep)
        out[prec] = (lab.cpu().numpy(), ex.cpu().numpy(), q)
    lo, hi = np.array(s.cv_params[0:2]), np.array(s.cv_params[2:4])
    far = []
    for r in range(R):
        phi, psi = o.cv(out[0][2][r])
        dist = min(abs(phi - lo[0]), abs(phi - lo[1]), abs(psi - hi[0]), abs(psi - hi[1]))
        far.append(dist > 2.0)
    far = np.array(far)
    agree = (out[0][0] == out[1][0]) & (out[0][1] == out[1][1])
    print(f"labels agree {agree.sum()}/{R}; far from boundary {far.sum()}; both states: "
          f"{np.bincount(out[0][0], minlength=2)}")
    assert np.all(agree[far])
    assert far.sum() >= R // 2


def test_deterministic(B, chain):
    """Fixed-point accumulation: two runs give identical bits."""
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
    """256 replicas of the 22-bead chain in the benchmark's launch configuration (mixed path, one
    exit test of the convergence step = 500-step segment with sampling, exit test, branching and
    Gelman-Rubin).  (i) Sampled replicas advanced alone by the oracle agree after 200 steps (1e-4
    relative).  (ii) After the full 500-step segment, 32 sampled replicas spread over both states
    are advanced alone by the oracle: every one whose oracle CV ends more than 2 degrees from a
    boundary of the rectangle has the oracle's label and exit flag (the margin of the mixed-path
    segment protocol).  (iii) The number of branched workers is the oracle's Fleming-Viot count for
    the device's exit mask."""
    s = chain
    o = oracle_mod.Oracle(s)
    R = s.n_replicas
    q0, p0 = W.replica_states(s, R, seed=13, spread=0.002)
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(rep, 200, s.t_gr)
    q, _, _, _ = B.grp_get_state(rep)
    sample = [0, 1, 127, 255]
    qo, _, _, _ = _oracle_step(o, q0[sample], p0[sample], 0, 0, 200, 0, replicas=sample)
    for row, r in enumerate(sample):
        assert _rel(q[r], qo[row]) < 1e-4

    q0, p0 = _spread_states(s, R, seed=13)
    omega = 1
    B.grp_set_state(rep, q0, p0, np.zeros((R, len(s.observables), 4)), {"t_global": 0, "t_phase": 0})
    st = B.grp_fv_check(rep, omega, s.t_check, s.t_gr, s.tol, 0)
    view = B.device_tensors(rep)
    lab = view["labels"].cpu().numpy().astype(np.int64)
    exm = view["exited"].cpu().numpy()
    assert st.t_phase == s.t_check and st.gr_evaluated == 1
    assert all(np.isfinite(st.rhat[j]) and st.rhat[j] >= 1.0 for j in range(len(s.observables)))
    assert st.ref_exited == exm[0] and st.label0 == lab[0]
    nbo, _ = oracle_mod.fv_branch(SEED, s.t_check, np.concatenate([[0], exm[1:]]).astype(np.uint8))
    assert st.n_branched == nbo and 0 <= st.n_branched < R

    sample = list(range(0, R, 8))
    qo, _, _, _ = _oracle_step(o, q0[sample], p0[sample], 0, 0, s.t_check, 0, replicas=sample)
    lo, hi = np.array(s.cv_params[0:2]), np.array(s.cv_params[2:4])
    far, labo = [], []
    for row in range(len(sample)):
        phi, psi = o.cv(qo[row])
        far.append(min(abs(phi - lo[0]), abs(phi - lo[1]), abs(psi - hi[0]), abs(psi - hi[1])) > 2.0)
        labo.append(o.state_of(qo[row]))
    far, labo = np.array(far), np.array(labo)
    got = lab[sample]
    print(f"sampled {len(sample)}, far {far.sum()}, oracle labels {np.bincount(labo, minlength=2)}")
    assert far.sum() >= len(sample) // 2
    assert len(set(labo[far].tolist())) == 2, "the sample covers both states"
    assert np.array_equal(got[far], labo[far])
    assert np.array_equal(exm[sample][far], (labo[far] != omega).astype(np.uint8))


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
    B.grp_step_k(rep, 0, 10)  # an empty segment is a no-op
    with pytest.raises(B.GrpError):
        B.grp_step_k(rep, 10, 10, n_active=5)
    with pytest.raises(B.GrpError):
        B.grp_gelman_rubin(rep, 0.01)  # one replica: no F-V worker
    with pytest.raises(B.GrpError):
        B.grp_broadcast(rep, 3)


def test_non_finite_state_is_reported(B, chain):
    """A NaN position (made on the host) is caught by the kernel's check and returned as GRP_ENAN."""
    R = 2
    q0, p0 = W.replica_states(chain, R, seed=15)
    sysh = B.grp_create_system(chain, B.GRP_MIXED)
    rep = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    q0[1, 3, 0] = np.nan
    with pytest.raises(B.GrpError) as e:
        B.grp_set_state(rep, q=q0)
        B.grp_step_k(rep, 5, 0)
        B.grp_get_state(rep)
    assert e.value.status in (B.GRP_ENAN, B.GRP_EOVERFLOW)


def test_checkpoint_resume_is_bit_exact(B, chain):
    """Checkpoint and resume (FP64 path): 1,000 steps in one go, or 500 steps, a copy of the state
    (positions, momenta, observable accumulators, step counters) to the host, a fresh replica set
    restored from it and 500 more steps, give identical bits: the noise is keyed by (seed, replica,
    step) and the forces are recomputed exactly (fixed-point sums) on restore."""
    s = chain
    R = 8
    q0, p0 = W.replica_states(s, R, seed=16, spread=0.003)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    one = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(one, 1000, s.t_gr)
    ref = B.grp_get_state(one)
    first = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(first, 500, s.t_gr)
    q, p, acc, ctr = B.grp_get_state(first)
    del first
    second = B.grp_init_replicas(sysh, R, SEED, q, p, per_replica=True)
    B.grp_set_state(second, acc=acc, counters=ctr)
    B.grp_step_k(second, 500, s.t_gr)
    got = B.grp_get_state(second)
    for a, b in zip(got[:3], ref[:3]):
        assert np.array_equal(a, b)
    assert got[3] == ref[3]


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


def test_single_replica_parallel_phase_is_plain_dynamics(B, oracle_mod):
    """N = 1 edge case of Eq. 5 on the GPU: tau = M t_check equals the oracle's brute-force
    first-check exit time."""
    s = W.double_well_2d()
    o = oracle_mod.Oracle(s)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    rep = B.grp_init_replicas(sysh, 1, SEED, s.q0, s.p0)
    ex = B.grp_run_parallel_phase(rep, 0, s.t_check, 10 ** 6)
    res, _ = o.run_bruteforce(SEED, s.t_check, 10 ** 9, 1)
    assert ex["k"] == 1 and ex["tau_steps"] == ex["M"] * s.t_check == res[0]
