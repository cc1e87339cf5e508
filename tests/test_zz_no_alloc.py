"""The batched entry point that allocates no device memory.

Some callers cannot call cudaMalloc: code running inside a component that
owns the whole device memory budget (a server's fixed arena, a framework
allocator that must account for every byte), or code on a path where an
allocation's implicit synchronisation or possible failure is not
acceptable.  ot_assign_solve_batched_noalloc keeps its launch metadata in a
static device array instead.  This file runs last (pytest collects files in
name order) so that a failure here leaves every other test already run; it
passes alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest
import torch

from paper_2005_01182_gb300 import otassign as ot
from paper_2005_01182_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _instances():
    sizes = W.batch_sizes(300, 16, 300, seed=4242)
    Cs = [W.embedding_costs(int(n), seed=4242 + i) for i, n in enumerate(sizes)]
    Cs += [W.pixel_sqdist(n, n + 7, seed=n) for n in (700, 1500)]
    return [torch.from_numpy(C).cuda() for C in Cs]


@pytest.mark.parametrize("algo", [ot.OT_KM, ot.OT_BKM])
def test_noalloc_matches_batched_twice(lib_path, algo):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dC = _instances()
    ctx = ot.Context()
    try:
        ref = ot.ot_assign_solve_batched(ctx, dC, algo)
        torch.cuda.synchronize()
        ref_cost = ref.cost.cpu().numpy().copy()
        ref_out = [[x.cpu().numpy() for x in o] for o in ref.outs]
    finally:
        ctx.close()
    free_before = None
    for call in range(2):
        a = ot.BatchArgs(dC)
        # poison the outputs so that stale results cannot pass
        a.cost.fill_(-12345)
        for o in a.outs:
            o[0].fill_(-1)
        torch.cuda.synchronize()
        if call == 1:
            free_before = torch.cuda.mem_get_info()[0]
        rc = ot.ot_assign_solve_batched_noalloc(a, algo)
        assert rc == ot.OT_OK
        torch.cuda.synchronize()
        if call == 1:
            # the second call allocates nothing on the device
            assert torch.cuda.mem_get_info()[0] == free_before
        assert (a.status.cpu().numpy() == 0).all()
        np.testing.assert_array_equal(a.cost.cpu().numpy(), ref_cost)
        for o, r in zip(a.outs, ref_out):
            for x, y in zip(o, r):
                np.testing.assert_array_equal(x.cpu().numpy(), y)


def test_noalloc_rejects_what_it_cannot_hold(lib_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    small = [torch.zeros((4, 4), dtype=torch.int32, device="cuda")] * (ot.OT_NOALLOC_MAX_INSTANCES + 1)
    assert ot.ot_assign_solve_batched_noalloc(ot.BatchArgs(small)) == ot.OT_ERR_UNSUPPORTED
    wide = [torch.zeros((8, 5000), dtype=torch.int32, device="cuda")]
    assert ot.ot_assign_solve_batched_noalloc(ot.BatchArgs(wide)) == ot.OT_ERR_UNSUPPORTED
    host = [torch.zeros((4, 4), dtype=torch.int32)]
    a = ot.BatchArgs(host, device="cpu")
    assert ot.ot_assign_solve_batched_noalloc(a) == ot.OT_ERR_ARG
    # device costs, but one output array on the host: refused before any
    # launch (the kernel would write through a host address)
    dev = [torch.zeros((4, 4), dtype=torch.int32, device="cuda")]
    for which in ("rp", "up", "vp"):
        a = ot.BatchArgs(dev)
        hosted = torch.empty(4, dtype=torch.int32 if which == "rp" else torch.int64)
        getattr(a, which)[0] = hosted.data_ptr()
        assert ot.ot_assign_solve_batched_noalloc(a) == ot.OT_ERR_ARG, which
    torch.cuda.synchronize()


def test_noalloc_empty_instance_in_a_mix(lib_path):
    """n == 0 gives cost 0 and status 0, as the context path returns it."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Cs = [torch.from_numpy(W.pixel_sqdist(n, n + 3, seed=n)).cuda() for n in (5, 40)]
    Cs.insert(1, torch.zeros((0, 6), dtype=torch.int32, device="cuda"))
    a = ot.BatchArgs(Cs)
    a.cost.fill_(-7)
    a.status.fill_(-7)
    a.outs[1][2].fill_(-7)
    assert ot.ot_assign_solve_batched_noalloc(a, ot.OT_KM) == ot.OT_OK
    torch.cuda.synchronize()
    ctx = ot.Context()
    try:
        ref = ot.ot_assign_solve_batched(ctx, Cs, ot.OT_KM)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(a.cost.cpu().numpy(), ref.cost.cpu().numpy())
    finally:
        ctx.close()
    assert a.cost[1].item() == 0
    assert (a.status.cpu().numpy() == 0).all()
    assert (a.outs[1][2].cpu().numpy() == 0).all()
