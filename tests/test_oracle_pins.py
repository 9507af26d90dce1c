"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics (CPU only).

Each test names what it pins and why a plausible mistake in the oracle would fail it.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

from paper_1807_02431_gb300 import analysis
from paper_1807_02431_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- RNG
def test_philox_matches_triton_interpreter(oracle_mod):
    """Philox4x32-10 against an independent library implementation (Triton's tl.philox, run by its
    CPU interpreter).  A wrong multiplier, Weyl constant, word order or round count fails."""
    pytest.importorskip("triton")
    import subprocess
    import sys

    code = r"""
import os, sys, numpy as np, torch, triton, triton.language as tl
sys.path.insert(0, sys.argv[1])
import oracle as O
@triton.jit
def k(seed, c0p, c1p, c2p, c3p, o0, o1, o2, o3, N: tl.constexpr):
    i = tl.arange(0, N)
    a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i), tl.load(c3p + i))
    tl.store(o0 + i, a); tl.store(o1 + i, b); tl.store(o2 + i, c); tl.store(o3 + i, d)
N = 64
rng = np.random.default_rng(7)
cs = [torch.tensor(rng.integers(0, 2**32, N, dtype=np.uint64).astype(np.uint32).view(np.int32)) for _ in range(4)]
outs = [torch.zeros(N, dtype=torch.int32) for _ in range(4)]
for seed in (0, 2431, 0xFEDCBA9876543210 & 0x7FFFFFFFFFFFFFFF):
    k[(1,)](seed, *cs, *outs, N=N)
    for t in range(N):
        ctr = [int(c[t].item()) & 0xffffffff for c in cs]
        ref = O.philox4x32_10(ctr, [seed & 0xffffffff, seed >> 32])
        got = [int(o[t].item()) & 0xffffffff for o in outs]
        assert ref == got, (seed, t, ref, got)
print("OK")
"""
    env = dict(os.environ, TRITON_INTERPRET="1")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code, root], env=env, capture_output=True, text=True,
                       timeout=600)
    if r.returncode != 0 and "No module named" in r.stderr:
        pytest.skip(r.stderr.strip().splitlines()[-1])
    assert r.returncode == 0 and "OK" in r.stdout, r.stderr[-2000:]


def test_normals_are_standard_normal(oracle_mod):
    """Box-Muller output: mean 0, variance 1, KS against N(0,1), and the two members of a pair
    uncorrelated.  A wrong scale (ln vs log2, missing factor 2) or a cos/sin mix-up fails."""
    from scipy import stats

    xs = np.array([oracle_mod.normals(2431, step, r, a)
                   for step in range(250) for r in range(4) for a in range(10)])
    flat = xs.ravel()
    assert abs(flat.mean()) < 5 / math.sqrt(flat.size)
    assert abs(flat.var() - 1.0) < 5 * math.sqrt(2.0 / flat.size)
    assert stats.kstest(flat, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(xs[:, 0], xs[:, 1])[0, 1]) < 5 / math.sqrt(xs.shape[0])
    assert abs(np.corrcoef(xs[:, 0], xs[:, 2])[0, 1]) < 5 / math.sqrt(xs.shape[0])


def test_branch_draw_is_uniform(oracle_mod):
    """The Fleming-Viot source is drawn uniformly among survivors (Section 2.4.1, task 2):
    chi-square test of the chosen source over many draws with 5 survivors."""
    from scipy import stats

    ex = np.array([0, 1, 0, 1, 0, 0, 1, 0, 1, 0], np.uint8)  # survivors 2, 4, 5, 7, 9
    counts = {r: 0 for r in (2, 4, 5, 7, 9)}
    for step in range(4000):
        nb, src = oracle_mod.fv_branch(11, step, ex)
        assert nb == 4
        for r in (1, 3, 6, 8):
            counts[int(src[r])] += 1
    obs = np.array(list(counts.values()))
    assert stats.chisquare(obs).pvalue > 1e-3


# ----------------------------------------------------------------------------- potential and forces
def _fd_forces(o, q, h=1e-6):
    fd = np.zeros_like(q)
    for a in range(q.shape[0]):
        for x in range(q.shape[1]):
            qp, qm = q.copy(), q.copy()
            qp[a, x] += h
            qm[a, x] -= h
            fd[a, x] = -(o.potential(qp) - o.potential(qm)) / (2 * h)
    return fd


@pytest.mark.parametrize("which", ["chain", "double_well"])
def test_forces_match_central_differences(oracle_mod, which):
    """F = -grad V (Eq. 1) against central finite differences of V (FP64, h = 1e-6): a wrong sign or
    a dropped term in any bonded or nonbonded gradient fails."""
    s = W.chain() if which == "chain" else W.double_well_2d()
    o = oracle_mod.Oracle(s)
    rng = np.random.default_rng(3)
    for _ in range(3):
        q = s.q0 + (0.01 if which == "chain" else 0.5) * rng.standard_normal(s.q0.shape)
        f = o.forces(q)
        fd = _fd_forces(o, q)
        assert np.abs(f - fd).max() <= 1e-8 * np.abs(f).max() + 1e-6


def _two_atom_system(**kw):
    base = dict(name="t", n_atoms=4, dim=3, potential=W.POT_FORCE_FIELD, mass=np.ones(4), kT=1.0,
                gamma=1.0, dt=0.001, sigma=np.full(4, 0.3), epsilon=np.zeros(4), charge=np.zeros(4),
                excl=np.zeros((0, 2), np.int32), coulomb_k=0.0)
    base.update(kw)
    return W.System(**base)


def test_potential_closed_forms(oracle_mod):
    """Closed-form energies: LJ minimum -eps at r = 2^(1/6) sigma; Coulomb k q q / (4 r^2); a bond
    stretched by d gives k d^2 / 2; a right angle with theta0 = 110 deg; a trans dihedral."""
    far = np.array([[0, 0, 0], [0.3 * 2 ** (1 / 6), 0, 0], [50, 0, 0], [-50, 0, 0]], float)
    excl = np.array([[0, 2], [0, 3], [1, 2], [1, 3], [2, 3]], np.int32)
    s = _two_atom_system(epsilon=np.array([0.5, 0.5, 0, 0]), excl=excl)
    assert oracle_mod.Oracle(s).potential(far) == pytest.approx(-0.5, rel=1e-12)
    s = _two_atom_system(charge=np.array([0.4, -0.3, 0, 0]), coulomb_k=W.COULOMB_K, excl=excl)
    q = far.copy()
    q[1, 0] = 0.7
    assert oracle_mod.Oracle(s).potential(q) == pytest.approx(W.COULOMB_K * 0.4 * -0.3 / (4 * 0.49), rel=1e-12)
    allx = np.array([[i, j] for i in range(4) for j in range(i + 1, 4)], np.int32)
    s = _two_atom_system(excl=allx, bonds=np.array([[0, 1]], np.int32), bond_k=np.array([1000.0]),
                         bond_r0=np.array([0.15]))
    q = far.copy()
    q[1, 0] = 0.17
    assert oracle_mod.Oracle(s).potential(q) == pytest.approx(0.5 * 1000 * 0.02 ** 2, rel=1e-9)
    s = _two_atom_system(excl=allx, angles=np.array([[0, 1, 2]], np.int32), angle_k=np.array([400.0]),
                         angle_theta0=np.array([math.radians(110)]))
    q = np.array([[1, 0, 0], [0, 0, 0], [0, 1, 0], [9, 9, 9]], float)
    assert oracle_mod.Oracle(s).potential(q) == pytest.approx(0.5 * 400 * math.radians(20) ** 2, rel=1e-12)
    s = _two_atom_system(excl=allx, dihedrals=np.array([[0, 1, 2, 3]], np.int32),
                         dihedral_n=np.array([2], np.int32), dihedral_k=np.array([3.0]),
                         dihedral_delta=np.array([0.0]))
    q = np.array([[1, 0, 0], [0, 0, 0], [0, 0, 1], [-1, 0, 1]], float)  # trans: phi = 180 deg
    assert oracle_mod.Oracle(s).potential(q) == pytest.approx(3.0 * (1 + math.cos(2 * math.pi)), rel=1e-12)


def test_dihedral_sign_convention(oracle_mod):
    """IUPAC convention: looking along j->k, a clockwise turn of the front bond onto the back bond
    is positive.  Geometry with the back bond turned +60 deg about +z gives +60; its mirror -60."""
    s = W.chain()
    o = oracle_mod.Oracle(s)
    c0 = s.cv_atoms[0]
    q = s.q0.copy()
    q[c0] = [1, 0, 0]
    q[c0 + 1] = [0, 0, 0]
    q[c0 + 2] = [0, 0, 1]
    q[c0 + 3] = [math.cos(math.radians(60)), math.sin(math.radians(60)), 1]
    q[c0 + 4] = q[c0 + 3] + [0, 0, 1]
    assert o.cv(q)[0] == pytest.approx(60.0, abs=1e-9)
    q[c0 + 3, 1] *= -1
    assert o.cv(q)[0] == pytest.approx(-60.0, abs=1e-9)


def test_chain_generator_initial_state(oracle_mod):
    """The generated chain starts at the paper's (phi, psi) = (-81, 70) deg (Section 4.1), outside
    the rectangle, i.e. in state 1."""
    s = W.chain()
    o = oracle_mod.Oracle(s)
    phi, psi = o.cv(s.q0)
    assert phi == pytest.approx(-81.0, abs=1e-9) and psi == pytest.approx(70.0, abs=1e-9)
    assert o.state_of(s.q0) == 1


# ----------------------------------------------------------------------------- BAOAB
def test_baoab_harmonic_configurational_variance_is_exact(oracle_mod):
    """BAOAB samples the configurational marginal of a harmonic oscillator exactly at any stable dt
    (Leimkuhler & Matthews 2013): Var(y) = kT / k with k = 2 * 2.5 = 5 for the y-direction of the
    double well.  A large step (omega dt = 0.67) makes O(dt^2) errors of other splittings (ABOBA,
    OBABO, Euler-Maruyama) several standard errors large."""
    s = dataclasses.replace(W.double_well_2d(), dt=0.3, gamma=1.0)
    o = oracle_mod.Oracle(s)
    R = 64
    q, p = W.replica_states(s, R, seed=5)
    f = np.stack([o.forces(q[r]) for r in range(R)])
    o.step_k(q, p, f, 99, 0, 0, 200, 0)  # burn-in
    ys = []
    for blk in range(100):
        o.step_k(q, p, f, 99, 200 + 40 * blk, 0, 40, 0)
        ys.append(q[:, 0, 1].copy())
    ys = np.array(ys)  # [100 blocks, 64 replicas], blocks separated by 40 steps = 12 time units
    var = ys.var()
    se = math.sqrt(2.0 / ys.size) * 0.2
    assert abs(var - 0.2) < 3.5 * se, (var, se)
    # ABOBA-like position bias at this dt is (1 - (omega dt / 2)^2)^-1 ~ 12%: far outside 3.5 se
    assert 3.5 * se < 0.2 * 0.1


# ----------------------------------------------------------------------------- Gelman-Rubin
def test_gelman_rubin_hand_computed(oracle_mod):
    """Eq. 3 on N = 2 replicas with samples {0, 2} and {4, 6}: Obar^1 = 1, Obar^2 = 5, Obar = 3;
    numerator = 1/2 [ (9 + 1)/2 + (1 + 9)/2 ] = 5; denominator = 1/2 [ (1 + 1)/2 + (1 + 1)/2 ] = 1."""
    assert oracle_mod.gelman_rubin(np.array([[0.0, 2.0], [4.0, 6.0]])) == pytest.approx(5.0, rel=1e-15)
    # identical replicas: numerator equals denominator
    assert oracle_mod.gelman_rubin(np.array([[1.0, 3.0], [1.0, 3.0]])) == pytest.approx(1.0, rel=1e-15)
    # no within-replica spread: not converged
    assert math.isinf(oracle_mod.gelman_rubin(np.array([[1.0, 1.0], [2.0, 2.0]])))


def test_gelman_rubin_variance_decomposition(oracle_mod):
    """R = 1 + B / W with B = mean_k (Obar^k - Obar)^2 and W = mean_k var_k (the numerator of Eq. 3
    splits into within and between parts), so R >= 1; R is invariant under affine maps of O."""
    rng = np.random.default_rng(4)
    for N, n in [(2, 3), (7, 50), (31, 400)]:
        x = rng.standard_normal((N, n)) + rng.standard_normal((N, 1)) * 0.3
        R = oracle_mod.gelman_rubin(x)
        mk = x.mean(axis=1)
        B = ((mk - mk.mean()) ** 2).mean()
        Wv = x.var(axis=1).mean()
        assert R == pytest.approx(1 + B / Wv, rel=1e-12)
        assert R >= 1.0
        assert oracle_mod.gelman_rubin(3.5 * x - 2.0) == pytest.approx(R, rel=1e-10)


# ----------------------------------------------------------------------------- Fleming-Viot
def test_fv_branch_keeps_population(oracle_mod):
    """Fleming-Viot keeps N particles: every exited worker gets a source, every source is a
    surviving worker, the reference (replica 0) is never branched, survivors keep their state.
    With no surviving worker every exited worker branches from the reference."""
    rng = np.random.default_rng(6)
    for trial in range(200):
        N = int(rng.integers(2, 40))
        ex = (rng.random(N) < rng.random()).astype(np.uint8)
        ex[0] = rng.integers(0, 2)  # the reference's flag is ignored by branching
        nb, src = oracle_mod.fv_branch(2431, trial, ex)
        workers_exited = [r for r in range(1, N) if ex[r]]
        survivors = [r for r in range(1, N) if not ex[r]]
        assert nb == len(workers_exited)
        assert src[0] == -1
        for r in range(1, N):
            if ex[r]:
                assert (src[r] in survivors) if survivors else (src[r] == 0)
            else:
                assert src[r] == -1


# ----------------------------------------------------------------------------- Eq. 5
def test_parallel_phase_single_replica_is_brute_force(oracle_mod):
    """With N = 1, Eq. 5 gives tau = M t_check: the first-check exit time of a plain trajectory.
    Same seed and same stream, so the oracle's parallel phase and its brute-force driver agree
    exactly (the brute-force residence of the first visit, started inside the state)."""
    s = W.double_well_2d()
    o = oracle_mod.Oracle(s)
    for seed in (1, 2, 3):
        q = s.q0.copy()[None]
        p = s.p0.copy()[None]
        f = o.forces(q[0])[None].copy()
        found, ex = o.parallel_phase(q, p, f, seed, 0, 0, s.t_check, 10 ** 6)
        res, frm = o.run_bruteforce(seed, s.t_check, 10 ** 9, 1)
        assert found and ex["k"] == 1
        assert ex["tau_steps"] == ex["M"] * s.t_check == res[0]
        assert frm[0] == 0


def test_parallel_phase_index_rule(oracle_mod):
    """Eq. 5 with N > 1: record each replica's first-exit check while the whole batch runs on
    (so that every replica keeps its own noise stream), then M = the earliest first exit, k = the
    lowest 1-based index exited at check M, and tau = [N (M - 1) + k] t_check."""
    s = W.double_well_2d()
    o = oracle_mod.Oracle(s)
    N, tc = 6, s.t_check
    q0, p0 = W.replica_states(s, N, seed=9, spread=0.0)
    q0[:, 0, 0] = -0.35  # near the barrier so that exits happen quickly
    qa, pa = q0.copy(), p0.copy()
    fa = np.stack([o.forces(qa[r]) for r in range(N)])
    firsts = [None] * N
    t = 0
    M = 0
    while any(x is None for x in firsts):
        o.step_k(qa, pa, fa, 17, t, 0, tc, 0)
        t += tc
        M += 1
        for r in range(N):
            if firsts[r] is None and o.exited(qa[r], 0):
                firsts[r] = M
        if M > 10 ** 5:
            break
    Mmin = min(firsts)
    k = min(r for r in range(N) if firsts[r] == Mmin) + 1
    qb, pb = q0.copy(), p0.copy()
    fb = np.stack([o.forces(qb[r]) for r in range(N)])
    found, ex = o.parallel_phase(qb, pb, fb, 17, 0, 0, tc, 10 ** 5)
    assert found and ex["M"] == Mmin and ex["k"] == k
    assert ex["tau_steps"] == (N * (Mmin - 1) + k) * tc


# ----------------------------------------------------------------------------- paper's tables
def _golden_rows(kind):
    rows = []
    with open(os.path.join(GOLDEN, "paper_tables.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if parts[0] == kind:
                rows.append(parts)
    return rows


def test_confidence_interval_matches_paper_tables():
    """Chi-square interval (start of Section 4) reproduces the intervals printed in Tables 1 and 3."""
    rows = _golden_rows("ci")
    assert len(rows) >= 9
    for _, src, n, tau, lo, hi, dec in rows:
        _, l, h = analysis.exit_time_ci(float(tau), n=int(n))
        tol = 0.5 * 10 ** -int(dec) + 1e-9 + 0.006 * float(tau) * (int(dec) == 2 and float(tau) < 2)
        assert abs(l - float(lo)) <= max(tol, 0.011), (src, n, l, lo)
        assert abs(h - float(hi)) <= max(tol, 0.011), (src, n, h, hi)


def test_speed_metrics_match_paper_tables():
    """Speed = t_sim / WT in ns/day, effective speedup = speed / serial speed, efficiency = speedup / N
    (Tables 2 and 4)."""
    for _, src, wt, tsim, speed, serial, N, sp, eff in _golden_rows("speed"):
        v = analysis.speed_ns_per_day(float(tsim), float(wt))
        # t_sim and WT are printed rounded (to 1 ns / 0.1 ns and 1 s): up to ~2e-4 relative
        assert abs(v - float(speed)) <= 3e-4 * float(speed), (src, v, speed)
        s = analysis.effective_speedup(float(speed), float(serial))
        assert abs(s - float(sp)) < 0.6, (src, s, sp)
        # Table 2 prints whole percentages (181 / 224 = 80.8 % appears as 80 %)
        assert abs(100 * analysis.efficiency(float(sp), int(N)) - float(eff)) < 1.0
