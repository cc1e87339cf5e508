"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle.

Bar (integer problem, exact arithmetic): the optimal cost is bit-exact
(tolerance 0) everywhere; KM's assignment, duals and counters are
bit-identical to the oracle's KM (same tie-breaks); batched KM may return a
different optimal assignment/duals, so its result is checked through the LP
certificate plus cost equality.
"""
import math

import numpy as np
import pytest
import torch

from paper_2005_01182_gb300 import otassign as ot
from paper_2005_01182_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [(32, 1), (32, 2), (32, 4), (32, 8), (64, 4), (128, 2), (128, 4), (256, 2), (256, 4),
          (512, 2), (512, 4), (1024, 2), (1024, 4)]


def gpu_solve(ctx, C_np, algo):
    C = torch.from_numpy(np.ascontiguousarray(C_np)).cuda()
    r, c, u, v = ot.ot_assign_solve(ctx, C, algo)
    torch.cuda.synchronize()
    return r.cpu().numpy(), int(c.item()), u.cpu().numpy(), v.cpu().numpy()


def check_km(oracle, ctx, C):
    a0, c0, u0, v0 = oracle.km(C)
    a, c, u, v = gpu_solve(ctx, C, ot.OT_KM)
    assert c == c0
    np.testing.assert_array_equal(a, a0)
    np.testing.assert_array_equal(u, u0)
    np.testing.assert_array_equal(v, v0)
    return c0


def check_bkm(oracle, ctx, C, cost):
    a, c, u, v = gpu_solve(ctx, C, ot.OT_BKM)
    assert c == cost
    assert oracle.check_certificate(C, a, u, v, c) == 0
    assert (v <= 0).all()


@pytest.fixture(autouse=True)
def _reset_table(ctx):
    yield
    # restore the built-in table after tests that force shapes
    for algo in (0, 1):
        for m, (t, k) in zip([32, 64, 128, 256, 512, 1024, 2048, 4096],
                             [(32, 1), (32, 2), (32, 4), (32, 8), (128, 4), (256, 4), (512, 4), (1024, 4)]):
            ot.ot_tune_set(ctx, algo, m, t, k)


def test_single_256(oracle_mod, ctx):
    C = W.single_256()
    cost = check_km(oracle_mod, ctx, C)
    check_bkm(oracle_mod, ctx, C, cost)
    assert oracle_mod.bkm(C)[1] == cost


def test_km_counters_match_oracle(oracle_mod, ctx):
    C = W.single_256()
    *_, st0 = oracle_mod.km(C, stats=True)
    *_, st = ot.ot_assign_solve_stats(ctx, torch.from_numpy(C).cuda(), ot.OT_KM)
    assert st["steps"] == st0["steps"]
    assert st["cost_bytes"] == st0["bytes"]
    assert st["augmentations"] == st0["augmentations"] == 256


@pytest.mark.parametrize("tpi,k", SHAPES)
def test_every_shape_ragged(oracle_mod, ctx, tpi, k):
    M = tpi * k
    rng = np.random.default_rng(M + tpi)
    sizes = sorted({max(1, M // 2 + 1), max(1, M - 1), M, max(1, M // 4 + 3)})
    for m in sizes:
        if m > 1024 and k > 1:
            sizes_n = [m - 5]
        else:
            sizes_n = [m, max(1, m - 3)]
        for n in sizes_n:
            for algo in (ot.OT_KM, ot.OT_BKM):
                ot.ot_tune_set(ctx, algo, m, tpi, k)
            seed = int(rng.integers(1 << 30))
            C = W.pixel_sqdist(n, m, seed=seed) if (n + m) % 2 else W.uniform_costs(n, m, hi=1000, seed=seed)
            cost = check_km(oracle_mod, ctx, C)
            check_bkm(oracle_mod, ctx, C, cost)


def test_rectangular_and_negative(oracle_mod, ctx):
    r = np.random.default_rng(9)
    for n, m in [(1, 1), (1, 300), (7, 100), (100, 101), (250, 256), (600, 1000), (1500, 2048)]:
        C = r.integers(-(1 << 20), 1 << 20, size=(n, m)).astype(np.int32)
        cost = check_km(oracle_mod, ctx, C)
        check_bkm(oracle_mod, ctx, C, cost)


def test_extreme_values(oracle_mod, ctx):
    r = np.random.default_rng(10)
    for n in (5, 64, 200):
        C = r.integers(-(1 << 31), (1 << 31) - 1, size=(n, n), dtype=np.int64).astype(np.int32)
        cost = check_km(oracle_mod, ctx, C)
        check_bkm(oracle_mod, ctx, C, cost)


def test_packed_32bit_path_limits(oracle_mod, ctx):
    """Rows packed to 16 bits run on 32-bit distances and duals.  At the
    bound of that path -- every row spans exactly 65535 above an offset near
    the int32 extremes, n = m = 4096 -- KM must still equal the oracle bit
    for bit, and a batch mixing packable rows with one row of range 65536
    (64-bit path) must agree instance by instance."""
    r = np.random.default_rng(23)
    n = 4096
    base = r.integers(-(1 << 31) + 70000, (1 << 31) - 70000, size=(n, 1))
    C = (base + r.integers(0, 65536, size=(n, n))).astype(np.int64)
    C[:, 0] = base[:, 0]
    C[:, 1] = base[:, 0] + 65535
    C = C.astype(np.int32)
    cost = check_km(oracle_mod, ctx, C)
    check_bkm(oracle_mod, ctx, C, cost)
    mats = []
    for t in range(6):
        M = r.integers(0, 65536, size=(200 + t, 220)).astype(np.int32)
        if t == 3:
            M[7, 5] = 65536  # this instance cannot be packed
            M[7, 6] = 0
        mats.append(M)
    b = ot.ot_assign_solve_batched(ctx, [torch.from_numpy(M).cuda() for M in mats], ot.OT_KM)
    torch.cuda.synchronize()
    for t, M in enumerate(mats):
        a0, c0, u0, v0 = oracle_mod.km(M)
        r_, u_, v_ = (x.cpu().numpy() for x in b.outs[t])
        assert int(b.cost[t]) == c0
        np.testing.assert_array_equal(r_, a0)
        np.testing.assert_array_equal(u_, u0)
        np.testing.assert_array_equal(v_, v0)


def test_degenerate(oracle_mod, ctx):
    for n, m in [(0, 0), (0, 7)]:
        C = torch.zeros((n, m), dtype=torch.int32, device="cuda")
        for algo in (ot.OT_KM, ot.OT_BKM):
            r, c, u, v = ot.ot_assign_solve(ctx, C, algo)
            torch.cuda.synchronize()
            assert int(c.item()) == 0
    C = np.zeros((50, 60), np.int32)
    a, c, u, v = gpu_solve(ctx, C, ot.OT_KM)
    assert c == 0 and a.tolist() == list(range(50))
    C = np.full((77, 77), 3, np.int32)
    cost = check_km(oracle_mod, ctx, C)
    check_bkm(oracle_mod, ctx, C, cost)
    C = np.array([[-5]], np.int32)
    assert check_km(oracle_mod, ctx, C) == -5


def test_closed_forms_on_gpu(ctx, oracle_mod):
    r = np.random.default_rng(11)
    n = 700
    a = r.integers(-1000, 1000, n)
    b = r.integers(-1000, 1000, n)
    C = (a[:, None] + b[None, :]).astype(np.int32)
    for algo in (ot.OT_KM, ot.OT_BKM):
        _, c, u, v = gpu_solve(ctx, C, algo)
        assert c == int(a.sum() + b.sum())
    p = r.permutation(n)
    C = r.integers(1, 500, size=(n, n)).astype(np.int32)
    C[np.arange(n), p] = 0
    for algo in (ot.OT_KM, ot.OT_BKM):
        asg, c, u, v = gpu_solve(ctx, C, algo)
        assert c == 0 and asg.tolist() == p.tolist()


def test_bad_arguments(ctx):
    C = torch.zeros((5, 3), dtype=torch.int32, device="cuda")
    with pytest.raises(ot.OtError) as e:
        ot.ot_assign_solve(ctx, C, ot.OT_KM)
    assert e.value.code == ot.OT_ERR_ARG
    C = torch.zeros((3, 5), dtype=torch.int32, device="cuda")
    with pytest.raises(ot.OtError) as e:
        ot.ot_assign_solve(ctx, C, 7)
    assert e.value.code == ot.OT_ERR_ARG


def test_empty_batch(ctx):
    """k = 0 is a valid batch: nothing is launched and the call succeeds."""
    for algo in (ot.OT_KM, ot.OT_BKM, ot.OT_AUTO):
        a = ot.ot_assign_solve_batched(ctx, [], algo)
        assert a.k == 0


def _batch(k, lo, hi, seed):
    sizes = W.batch_sizes(k, lo, hi, seed)
    return [W.embedding_costs(int(n), seed=seed + 1 + i) for i, n in enumerate(sizes)]


@pytest.mark.parametrize("algo", [ot.OT_KM, ot.OT_BKM])
def test_batched_equals_solo_and_oracle(oracle_mod, ctx, algo):
    Cs = _batch(300, 8, 300, 123) + [W.pixel_sqdist(int(n), seed=7 + int(n)) for n in (16, 33, 517, 1030)]
    dev = [torch.from_numpy(C).cuda() for C in Cs]
    a = ot.ot_assign_solve_batched(ctx, dev, algo)
    torch.cuda.synchronize()
    cost = a.cost.cpu().numpy()
    assert (a.status.cpu().numpy() == 0).all()
    for t, C in enumerate(Cs):
        r, u, v = (x.cpu().numpy() for x in a.outs[t])
        if algo == ot.OT_KM:
            a0, c0, u0, v0 = oracle_mod.km(C)
            assert cost[t] == c0
            np.testing.assert_array_equal(r, a0)
            np.testing.assert_array_equal(u, u0)
            np.testing.assert_array_equal(v, v0)
        else:
            assert oracle_mod.check_certificate(C, r, u, v, int(cost[t])) == 0
        if t % 37 == 0 or algo == ot.OT_BKM and t % 5 == 0:
            rs, cs, us, vs = gpu_solve(ctx, C, algo)
            assert cs == cost[t]
            np.testing.assert_array_equal(rs, r)
            np.testing.assert_array_equal(us, u)
            np.testing.assert_array_equal(vs, v)


def test_batched_full_size_embeddings(oracle_mod, ctx):
    """4096 instances, n ~ U{32..256}, 300-d embedding costs: certificate for
    every instance, oracle KM identity on a sample, KM cost == bKM cost."""
    Cs = W.batch_embeddings(4096)
    dev = [torch.from_numpy(C).cuda() for C in Cs]
    res = {}
    for algo in (ot.OT_KM, ot.OT_BKM):
        a = ot.ot_assign_solve_batched(ctx, dev, algo)
        torch.cuda.synchronize()
        assert (a.status.cpu().numpy() == 0).all()
        res[algo] = a.cost.cpu().numpy().copy()
        for t in range(0, 4096, 7):
            r, u, v = (x.cpu().numpy() for x in a.outs[t])
            assert oracle_mod.check_certificate(Cs[t], r, u, v, int(res[algo][t])) == 0
        if algo == ot.OT_KM:
            for t in range(0, 4096, 128):
                a0, c0, u0, v0 = oracle_mod.km(Cs[t])
                assert res[algo][t] == c0
                np.testing.assert_array_equal(a.outs[t][0].cpu().numpy(), a0)
    np.testing.assert_array_equal(res[ot.OT_KM], res[ot.OT_BKM])


def test_single_4096(oracle_mod, ctx):
    """n = m = 4096: uniform costs (oracle KM identity) and circle/square
    shapes (certificate, KM cost == bKM cost)."""
    C = W.single_4096("uniform")
    cost = check_km(oracle_mod, ctx, C)
    check_bkm(oracle_mod, ctx, C, cost)
    C = W.single_4096("circle-square")
    a, c, u, v = gpu_solve(ctx, C, ot.OT_KM)
    assert oracle_mod.check_certificate(C, a, u, v, c) == 0
    check_bkm(oracle_mod, ctx, C, c)


def test_default_stream_ordering(oracle_mod, ctx):
    """NULL stream = the caller's default stream: a solve issued right after
    torch writes the matrix on that stream sees the written values, and
    torch's reads of the results after the call see the solve's output,
    with no explicit synchronisation in between."""
    C = W.uniform_costs(700, hi=50000, seed=31)
    a0, c0, _, _ = oracle_mod.km(C)
    src = torch.from_numpy(C).cuda()
    for _ in range(3):
        dst = torch.zeros_like(src)
        big = torch.randn(4096, 4096, device="cuda")
        for _ in range(4):
            big = big @ big  # keeps the default stream busy before the copy
        dst.copy_(src)
        r, c, u, v = ot.ot_assign_solve(ctx, dst, ot.OT_KM, stream=0)
        got_c = int(c.cpu().item())
        assert got_c == c0
        np.testing.assert_array_equal(r.cpu().numpy(), a0)
        del big


def test_host_pointers(oracle_mod, ctx):
    """The C-ABI with host buffers (pinned and pageable) stages through the
    device and returns the same result as the device path."""
    C = W.pixel_sqdist(300, 310, seed=5)
    a0, c0, u0, v0 = oracle_mod.km(C)
    for pin in (False, True):
        Ct = torch.from_numpy(C)
        if pin:
            Ct = Ct.pin_memory()
        r, c, u, v = ot.ot_assign_solve(ctx, Ct, ot.OT_KM)
        assert int(c.item()) == c0
        np.testing.assert_array_equal(r.numpy(), a0)
        np.testing.assert_array_equal(v.numpy(), v0)
    Cs = [torch.from_numpy(W.embedding_costs(n, seed=n)) for n in (40, 90, 250)]
    a = ot.ot_assign_solve_batched(ctx, Cs, ot.OT_BKM)
    for t, Ct in enumerate(Cs):
        C = Ct.numpy()
        r, u, v = (x.numpy() for x in a.outs[t])
        assert oracle_mod.check_certificate(C, r, u, v, int(a.cost[t])) == 0


@pytest.mark.parametrize("mode", ["pinned", "pageable"])
def test_host_slab_batch_pipelined(oracle_mod, ctx, mode):
    """A large batch in one host slab (>= 256 instances, >= 64 MB) is copied
    and solved chunk by chunk; results equal the device path bit for bit
    (KM), including a skipped empty instance, an instance whose rows span
    more than 16 bits and a ragged tail."""
    rng = np.random.default_rng(17)
    sizes = [int(x) for x in rng.integers(240, 301, size=300)] + [0, 37]
    # instance 5 spans more than 16 bits (not packed: solved from the staged copy)
    mats = [W.uniform_costs(n, hi=(1 << 20) if i == 5 else 60000, seed=i) if n else np.zeros((0, 5), np.int32)
            for i, n in enumerate(sizes)]
    total = sum(C.size for C in mats)
    assert 4 * total >= 64 << 20
    slab = torch.empty(total, dtype=torch.int32)
    if mode != "pageable":
        slab = slab.pin_memory()
    hC, o = [], 0
    for C in mats:
        v = slab[o:o + C.size].view(C.shape)
        v.copy_(torch.from_numpy(C))
        hC.append(v)
        o += C.size
    ah = ot.ot_assign_solve_batched(ctx, hC, ot.OT_KM)
    ad = ot.ot_assign_solve_batched(ctx, [torch.from_numpy(C).cuda() for C in mats], ot.OT_KM)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ah.cost.numpy(), ad.cost.cpu().numpy())
    assert (ah.status.numpy() == 0).all()
    for t, C in enumerate(mats):
        if C.shape[0] == 0:
            continue
        np.testing.assert_array_equal(ah.outs[t][0].numpy(), ad.outs[t][0].cpu().numpy())
        np.testing.assert_array_equal(ah.outs[t][2].numpy(), ad.outs[t][2].cpu().numpy())
    for t in (0, 5, 150, 301):
        assert int(ah.cost[t]) == oracle_mod.km(mats[t])[1]
    st = ot.ot_last_call_stats(ctx)
    assert st["launches"] >= 1


def test_last_call_counters_and_launches(oracle_mod, ctx):
    """ot_last_call_stats sums the oracle's KM counters over the instances of
    the last batched call; ot_last_call_launches lists one entry per bucket
    kernel whose instance counts add up to the batch, with device times."""
    mats = [W.embedding_costs(n, seed=n) for n in (20, 33, 70, 130, 250, 250)]
    b = ot.ot_assign_solve_batched(ctx, [torch.from_numpy(C).cuda() for C in mats], ot.OT_KM)
    st = ot.ot_last_call_stats(ctx)
    launches = ot.ot_last_call_launches(ctx)
    want_steps = want_bytes = 0
    for C in mats:
        *_, s0 = oracle_mod.km(C, stats=True)
        want_steps += s0["steps"]
        want_bytes += s0["bytes"]
    assert st["steps"] == want_steps
    assert st["cost_bytes"] == want_bytes
    assert 0 < st["read_bytes"] <= st["cost_bytes"]
    assert sum(L["instances"] for L in launches) == len(mats)
    assert all(L["algo"] == ot.OT_KM and L["ms"] > 0 for L in launches)
    assert sum(L["read_bytes"] for L in launches) == st["read_bytes"]
    assert st["launches"] == len(launches) + 1  # the bucket kernels and the packing pass
    for t, C in enumerate(mats):
        assert int(b.cost[t]) == oracle_mod.km(C)[1]


def test_serving_results_equal_solo(oracle_mod, ctx):
    """Requests submitted while others run are admitted and solved in
    overlapping waves; every result equals the solo solve bit for bit."""
    reqs = W.served_requests(160, rate_per_s=1e9, lo=16, hi=700, seed=99)
    served = ot.Context(hbm_budget_bytes=64 << 20, wave_streams=3)
    try:
        tickets = []
        for i, (_, C) in enumerate(reqs):
            algo = ot.OT_BKM if i % 3 == 0 else ot.OT_KM
            tickets.append((ot.ot_assign_submit(served, torch.from_numpy(C), algo), algo, C))
        outs = {}
        pending = list(tickets)
        import time
        t0 = time.time()
        while pending and time.time() - t0 < 300:
            rest = []
            for t, algo, C in pending:
                n, m = C.shape
                o = (torch.empty(n, dtype=torch.int32), torch.empty(1, dtype=torch.int64),
                     torch.empty(n, dtype=torch.int64), torch.empty(m, dtype=torch.int64))
                if ot.ot_assign_poll(served, t, o) == ot.OT_OK:
                    outs[t] = o
                else:
                    rest.append((t, algo, C))
            pending = rest
        assert not pending
        cnt = ot.ot_serving_counters(served)
        assert cnt["completed"] == len(reqs) and cnt["waves"] >= 1
        for t, algo, C in tickets:
            r, c, u, v = outs[t]
            rs, cs, us, vs = gpu_solve(ctx, C, algo)
            assert int(c.item()) == cs
            np.testing.assert_array_equal(r.numpy(), rs)
            np.testing.assert_array_equal(u.numpy(), us)
            np.testing.assert_array_equal(v.numpy(), vs)
            if algo == ot.OT_KM and C.shape[0] <= 300:
                assert oracle_mod.km(C)[1] == cs
    finally:
        served.close()


def test_serving_budget_refusal(ctx):
    served = ot.Context(hbm_budget_bytes=1 << 20)
    try:
        C = torch.from_numpy(W.pixel_sqdist(600, seed=1))  # 1.44 MB > budget
        with pytest.raises(ot.OtError) as e:
            ot.ot_assign_submit(served, C, ot.OT_KM)
        assert e.value.code == ot.OT_ERR_BUDGET
        with pytest.raises(ot.OtError) as e:
            ot.ot_assign_poll(served, 12345, (None, None, None, None))
        assert e.value.code == ot.OT_ERR_TICKET
    finally:
        served.close()


def test_autotune_keeps_results(oracle_mod, ctx):
    Cs = _batch(200, 20, 260, 5)
    dev = [torch.from_numpy(C).cuda() for C in Cs]
    for algo in (ot.OT_KM, ot.OT_BKM):
        ot.ot_autotune(ctx, dev, algo, repeats=1)
        for m in (64, 128, 256, 512):
            t, k = ot.ot_tune_lookup(ctx, algo, m)
            assert t * k >= m
        a = ot.ot_assign_solve_batched(ctx, dev, algo)
        torch.cuda.synchronize()
        for t in range(0, 200, 9):
            C = Cs[t]
            r, u, v = (x.cpu().numpy() for x in a.outs[t])
            assert oracle_mod.check_certificate(C, r, u, v, int(a.cost[t])) == 0


def test_auto_algorithm_per_bucket(oracle_mod, ctx):
    """OT_AUTO resolves per size bucket to KM or batched KM (both exact)."""
    Cs = _batch(120, 16, 700, 77)
    dev = [torch.from_numpy(C).cuda() for C in Cs]
    for choice in (ot.OT_KM, ot.OT_BKM):
        for m in (32, 64, 128, 256, 512, 1024):
            ot.ot_tune_set(ctx, ot.OT_AUTO, m, choice, 0)
        a = ot.ot_assign_solve_batched(ctx, dev, ot.OT_AUTO)
        torch.cuda.synchronize()
        for t, C in enumerate(Cs):
            r, u, v = (x.cpu().numpy() for x in a.outs[t])
            if choice == ot.OT_KM:
                a0, c0, u0, v0 = oracle_mod.km(C)
                np.testing.assert_array_equal(r, a0)
                np.testing.assert_array_equal(u, u0)
            assert oracle_mod.check_certificate(C, r, u, v, int(a.cost[t])) == 0
    ot.ot_autotune(ctx, dev, ot.OT_AUTO, repeats=1)
    a = ot.ot_assign_solve_batched(ctx, dev, ot.OT_AUTO)
    torch.cuda.synchronize()
    for t, C in enumerate(Cs):
        r, u, v = (x.cpu().numpy() for x in a.outs[t])
        assert oracle_mod.check_certificate(C, r, u, v, int(a.cost[t])) == 0
    for m in (32, 64, 128, 256, 512, 1024):
        ot.ot_tune_set(ctx, ot.OT_AUTO, m, ot.OT_KM if m <= 256 else ot.OT_BKM, 0)
