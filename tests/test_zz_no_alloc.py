"""grp_fv_branch_noalloc: Fleming-Viot branching for callers that cannot allocate device memory while
they run (their memory belongs to another allocator, or cudaMalloc's implicit synchronisation is not
acceptable in their loop).  Its scratch is a static device array; it must give exactly what
grp_fv_branch gives on the same replicas, call after call.

This file is collected last on purpose: if it fails, every other test has already run.
"""
import numpy as np
import pytest

from paper_1807_02431_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_branching_matches_fv_branch_two_calls_in_a_row():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_02431_gb300 import binding as B
    from paper_1807_02431_gb300 import build

    build.build()
    B.load()
    s = W.chain()
    R, seed = 96, 2431
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    q0, p0 = W.replica_states(s, R, seed=41, spread=0.01)
    rep = B.grp_init_replicas(sysh, R, seed, q0, p0, per_replica=True)
    B.grp_step_k(rep, 20, s.t_gr)  # gives the replicas distinct accumulators and forces
    rng = np.random.default_rng(42)
    for call, t_global in enumerate((900, 901)):
        B.grp_set_state(rep, counters={"t_global": t_global, "t_phase": 20})
        view = B.device_tensors(rep)
        # the caller's own buffers: copies of the replica set's arrays (allocated by the caller)
        mine = {k: view[k].clone() for k in ("q", "p", "f", "acc")}
        exm = torch.tensor((rng.random(R) < (0.4 if call == 0 else 0.8)).astype(np.uint8), device="cuda")
        torch.cuda.synchronize()
        nb_ref = B.grp_fv_branch(rep, exm)
        nb = B.grp_fv_branch_noalloc(sysh, R, mine["q"], mine["p"], mine["f"], mine["acc"], exm, seed, t_global)
        torch.cuda.synchronize()
        assert nb == nb_ref and nb > 0
        for k in ("q", "p", "f", "acc"):
            assert torch.equal(mine[k], view[k]), (call, k)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_02431_gb300 import binding as B

    B.load()
    s = W.chain()
    sysh = B.grp_create_system(s, B.GRP_MIXED)
    x = torch.zeros(8, device="cuda", dtype=torch.float64)
    ex = torch.zeros(8, device="cuda", dtype=torch.uint8)
    with pytest.raises(B.GrpError) as e:
        B.grp_fv_branch_noalloc(sysh, 65537, x, x, x, x, ex, 1, 0)
    assert e.value.status == B.GRP_EINVAL and "65536" in str(e.value)
