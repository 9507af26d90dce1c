"""The library's shard calls (grp_set_shard, grp_fv_plan, grp_pack_rows / grp_unpack_rows,
grp_gr_partials / grp_gr_combine) and the sharded loop of Fig. 1 on the GPU.

A run's replicas cut into shards must behave as the unsharded replica set: the shards draw the noise of
their global replica indices (Section 3.1 distributes a run's replicas over processes), the Fleming-Viot
sources are those grp_fv_branch draws, and the Gelman-Rubin sums of all shards give the ratios of
grp_gelman_rubin.  On one GPU the shards live in one process (ranks.Comm without a process group), which
runs exactly the code that several processes run, minus the transport.
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


def _shards(B, s, prec, q0, p0, counts, per_replica=True):
    from paper_1807_02431_gb300 import ranks

    L = ranks.Layout(counts, [0] * len(counts))
    sysh = B.grp_create_system(s, prec)
    shards = {}
    for i in range(len(counts)):
        a, c = L.first[i], L.count[i]
        qs = q0[a:a + c] if per_replica else q0
        ps = p0[a:a + c] if per_replica else p0
        rep = B.grp_init_replicas(sysh, c, SEED, qs, ps, per_replica=per_replica)
        shards[i] = ranks.LibraryShard(B, rep, a, L.N)
    return L, sysh, shards


@pytest.mark.parametrize("prec", [0, 1])
def test_shards_follow_the_unsharded_trajectory(B, prec):
    """Chain, 24 replicas as shards of 10, 6 and 8: 300 steps with sampling give bit-identical positions,
    momenta and accumulators to one set of 24 (the noise of each replica is keyed by its global index)."""
    s = W.chain()
    R = 24
    q0, p0 = W.replica_states(s, R, seed=3, spread=0.01)
    sysh = B.grp_create_system(s, prec)
    whole = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_set_state(whole, counters={"t_global": 1000, "t_phase": 3})
    B.grp_step_k(whole, 300, s.t_gr)
    qw, pw, aw, _ = B.grp_get_state(whole)
    L, _, shards = _shards(B, s, prec, q0, p0, [10, 6, 8])
    for i, sh in shards.items():
        sh.set_counters(1000, 3)
        sh.advance(300, s.t_gr, sh.n)
        q, p, a, _ = B.grp_get_state(sh.rep)
        sl = slice(L.first[i], L.first[i] + L.count[i])
        assert np.array_equal(q, qw[sl]) and np.array_equal(p, pw[sl]) and np.array_equal(a, aw[sl])


def test_fv_plan_equals_fv_branch_sources(B):
    """Sources of every shard's exited workers from the global mask equal grp_fv_branch's on the whole
    set, at masks of 0 %, 40 %, 95 % and 100 % exited (the last: every worker copies the reference)."""
    import torch

    s = W.chain()
    R = 40
    q0, p0 = W.replica_states(s, R, seed=4, spread=0.01)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    whole = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    L, _, shards = _shards(B, s, B.GRP_FP64, q0, p0, [13, 13, 14])
    rng = np.random.default_rng(5)
    for t_global, frac in ((500, 0.0), (1000, 0.4), (1500, 0.95), (2000, 1.0)):
        ex = (rng.random(R) < frac).astype(np.uint8)
        ex[1:] = 1 if frac == 1.0 else ex[1:]
        B.grp_set_state(whole, counters={"t_global": t_global, "t_phase": 0})
        d_src = torch.empty(R, dtype=torch.int32, device="cuda")
        B.grp_fv_branch(whole, torch.tensor(ex, device="cuda"), d_src)
        ref = d_src.cpu().numpy()
        got = []
        for i, sh in shards.items():
            sh.set_counters(t_global, 0)
            got.append(sh.plan(ex))
        got = np.concatenate(got)
        ref[0] = -1
        assert np.array_equal(got, ref), (frac, got, ref)


def test_pack_unpack_and_gelman_rubin_sums(B):
    """Rows packed from one shard and unpacked into another carry q, p, F and the accumulators bit for
    bit; the Gelman-Rubin ratios from the shards' summed partials equal grp_gelman_rubin's on the whole
    set within 1e-12 (the sums are added in another order)."""
    import torch

    s = W.chain()
    R = 30
    q0, p0 = W.replica_states(s, R, seed=6, spread=0.01)
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    whole = B.grp_init_replicas(sysh, R, SEED, q0, p0, per_replica=True)
    B.grp_step_k(whole, 400, s.t_gr)
    rhat_w, _ = B.grp_gelman_rubin(whole, 0.01)
    qw, pw, aw, _ = B.grp_get_state(whole)
    L, _, shards = _shards(B, s, B.GRP_MIXED, q0, p0, [7, 11, 12])
    for i, sh in shards.items():
        sl = slice(L.first[i], L.first[i] + L.count[i])
        B.grp_set_state(sh.rep, qw[sl], pw[sl], aw[sl], {"t_global": 400, "t_phase": 400})
    s1 = np.sum([sh.gr1() for sh in shards.values()], axis=0)
    s2 = np.sum([sh.gr2(s1) for sh in shards.values()], axis=0)
    rhat, _ = shards[0].gr_combine(s1, s2, 0.01)
    assert np.all(np.abs(rhat - rhat_w) <= 1e-12 * np.abs(rhat_w - 1) + 1e-15), (rhat, rhat_w)
    rows = shards[2].pack([0, 5, 11])
    shards[1].unpack([3, 4, 10], rows)
    q, p, a, _ = B.grp_get_state(shards[1].rep)
    q2, p2, a2, _ = B.grp_get_state(shards[2].rep)
    for d, src in ((3, 0), (4, 5), (10, 11)):
        assert np.array_equal(q[d], q2[src]) and np.array_equal(p[d], p2[src]) and np.array_equal(a[d], a2[src])
    with pytest.raises(B.GrpError):
        B.grp_fv_check(shards[1].rep, 1, 10, 10, 0.01, 0)  # a shard is not a whole run


def test_sharded_loop_equals_grp_run(B, oracle_mod):
    """The loop of Fig. 1 on the double well over shards of 10, 7 and 15 replicas: the event log equals
    grp_run on one set of 32 and the oracle's run."""
    from paper_1807_02431_gb300 import ranks

    s = W.double_well_2d()
    args = (s.t_gr, s.t_check, 0.05, s.min_fv_steps, 10 ** 8, 6)
    sysh = B.grp_create_system(s, B.GRP_FP64)
    whole = B.grp_init_replicas(sysh, s.n_replicas, SEED, s.q0, s.p0)
    ev_w, _ = B.grp_run(whole, *args)
    L, _, shards = _shards(B, s, B.GRP_FP64, s.q0, s.p0, [10, 7, 15], per_replica=False)
    run = ranks.ShardedRun(L, shards, ranks.Comm())
    ev, tsim = run.run(*args)
    evo, _ = oracle_mod.Oracle(s).run_genparrep(s.n_replicas, SEED, *args[:5], args[5], q0=s.q0, p0=s.p0)
    assert ev == ev_w == evo
    assert run.rows_moved["within_process"] > 0
