"""GPU parity of the cluster engine (instances wider than one CTA, m > 4096,
and smaller buckets routed to it on purpose) against the CPU oracle."""
import os

import numpy as np
import pytest
import torch

from paper_2005_01182_gb300 import otassign as ot
from paper_2005_01182_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEFAULT = [(32, 1), (32, 2), (32, 4), (32, 8), (128, 4), (256, 4), (512, 4), (1024, 4)]
BUCKET_M = [32, 64, 128, 256, 512, 1024, 2048, 4096]


@pytest.fixture()
def large_ctx(ctx):
    for algo in (0, 1):
        for m in BUCKET_M:
            ot.ot_tune_set(ctx, algo, m, 0, 0)
    yield ctx
    for algo in (0, 1):
        for m, (t, k) in zip(BUCKET_M, DEFAULT):
            ot.ot_tune_set(ctx, algo, m, t, k)


def solve(ctx, C, algo):
    r, c, u, v, st = ot.ot_assign_solve_stats(ctx, torch.from_numpy(np.ascontiguousarray(C)).cuda(), algo)
    return r.cpu().numpy(), int(c.item()), u.cpu().numpy(), v.cpu().numpy(), st


def test_lookup_reports_cluster_engine(large_ctx):
    assert ot.ot_tune_lookup(large_ctx, ot.OT_KM, 100) == (0, 0)
    assert ot.ot_tune_lookup(large_ctx, ot.OT_BKM, 9000) == (0, 0)


@pytest.mark.parametrize("kind", ["pixel", "uniform", "embed", "negative"])
def test_cluster_engine_small_sizes(oracle_mod, large_ctx, kind):
    rng = np.random.default_rng(len(kind))
    for n, m in [(1, 1), (2, 3), (31, 31), (100, 100), (257, 300), (700, 700), (1500, 1531)]:
        seed = int(rng.integers(1 << 30))
        if kind == "pixel":
            C = W.pixel_sqdist(n, m, seed=seed)
        elif kind == "uniform":
            C = W.uniform_costs(n, m, seed=seed)
        elif kind == "embed":
            C = W.embedding_costs(n, seed=seed)[:, :m] if m == n else W.uniform_costs(n, m, hi=50, seed=seed)
        else:
            C = rng.integers(-(1 << 30), 1 << 30, size=(n, m)).astype(np.int32)
        a0, c0, u0, v0, st0 = oracle_mod.km(C, stats=True)
        a, c, u, v, st = solve(large_ctx, C, ot.OT_KM)
        assert c == c0
        np.testing.assert_array_equal(a, a0)
        np.testing.assert_array_equal(u, u0)
        np.testing.assert_array_equal(v, v0)
        assert st["steps"] == st0["steps"] and st["cost_bytes"] == st0["bytes"]
        a, c, u, v, st = solve(large_ctx, C, ot.OT_BKM)
        assert c == c0
        assert oracle_mod.check_certificate(C, a, u, v, c) == 0
        assert (v <= 0).all()


def test_cluster_engine_degenerate(oracle_mod, large_ctx):
    for C in [np.zeros((40, 50), np.int32), np.full((64, 64), 9, np.int32)]:
        for algo in (ot.OT_KM, ot.OT_BKM):
            a, c, u, v, _ = solve(large_ctx, C, algo)
            assert c == oracle_mod.km(C)[1]
            assert oracle_mod.check_certificate(C, a, u, v, c) == 0


def test_wide_instances(oracle_mod, ctx):
    """m > 4096 goes to the cluster engine without any forcing."""
    C = W.uniform_costs(4100, seed=3)
    a0, c0, u0, v0 = oracle_mod.km(C)
    a, c, u, v, _ = solve(ctx, C, ot.OT_KM)
    assert c == c0
    np.testing.assert_array_equal(a, a0)
    np.testing.assert_array_equal(v, v0)
    a, c, u, v, _ = solve(ctx, C, ot.OT_BKM)
    assert c == c0 and oracle_mod.check_certificate(C, a, u, v, c) == 0
    C = W.pixel_sqdist(2500, 5000, seed=4)
    a, c, u, v, _ = solve(ctx, C, ot.OT_BKM)
    assert oracle_mod.check_certificate(C, a, u, v, c) == 0
    assert c == oracle_mod.km(C)[1]


def oracle_cost(name):
    """The CPU oracle's optimal cost of a named workload, stored by
    tests/golden/make_oracle_costs.py (None when not stored)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_costs.txt")
    if os.path.exists(path):
        for line in open(path):
            f = line.split()
            if f and not line.startswith("#") and f[0] == name:
                return int(f[1])
    return None


def test_single_16384(oracle_mod, ctx):
    """n = m = 16384 on a 1024 x 1024 grid: batched KM certified on the host
    (O(n^2) dual check), equal to the cluster engine's KM cost and to the
    oracle's stored optimum."""
    C = W.single_16384()
    a, c, u, v, st = solve(ctx, C, ot.OT_BKM)
    assert oracle_mod.check_certificate(C, a, u, v, c) == 0
    assert st["augmentations"] == 16384
    a2, c2, u2, v2, _ = solve(ctx, C, ot.OT_KM)
    assert c2 == c
    assert oracle_mod.check_certificate(C, a2, u2, v2, c2) == 0
    stored = oracle_cost("single_16384_grid")
    assert stored is None or stored == c


@pytest.mark.parametrize("kind", ["circle-square", "circle-triangle", "uniform"])
def test_single_4096_matches_stored_oracle_cost(ctx, kind):
    """n = 4096 single solves (both engines, KM and batched KM) against the
    oracle's stored optimum."""
    stored = oracle_cost("single_4096_" + kind.replace("-", "_"))
    if stored is None:
        pytest.skip("no stored oracle cost")
    C = W.single_4096(kind)
    for algo in (ot.OT_KM, ot.OT_BKM, ot.OT_AUCTION):
        _, c, _, _, _ = solve(ctx, C, algo)
        assert c == stored


def test_wide_single_batched_km_takes_the_cluster_engine(oracle_mod):
    """With an untuned table, a single batched-KM instance wider than 1024
    columns (ot_assign_solve) runs on the cluster engine, while the batched
    entry point keeps the group engine; both give certified optima."""
    fresh = ot.Context()
    try:
        for n in (1100, 2047):
            C = W.uniform_costs(n, n + 4, seed=n)
            a, c, u, v = gpu_solve_on(fresh, C, ot.OT_BKM)
            assert oracle_mod.check_certificate(C, a, u, v, c) == 0
            assert c == oracle_mod.km(C)[1]
        many = [W.pixel_sqdist(1030 + 7 * i, seed=i) for i in range(3)]
        b = ot.ot_assign_solve_batched(fresh, [torch.from_numpy(C).cuda() for C in many], ot.OT_BKM)
        torch.cuda.synchronize()
        for t, C in enumerate(many):
            r, u, v = (x.cpu().numpy() for x in b.outs[t])
            assert oracle_mod.check_certificate(C, r, u, v, int(b.cost[t])) == 0
    finally:
        fresh.close()


def gpu_solve_on(c, C, algo):
    r, cost, u, v = ot.ot_assign_solve(c, torch.from_numpy(np.ascontiguousarray(C)).cuda(), algo)
    torch.cuda.synchronize()
    return r.cpu().numpy(), int(cost.item()), u.cpu().numpy(), v.cpu().numpy()


def test_widest_instances(oracle_mod, ctx):
    """Few rows, very many columns: m = 30000 on the cluster engine (each
    thread owns several columns), and a width beyond what the engine holds
    (m = 65537) refused with OT_ERR_UNSUPPORTED before any launch."""
    C = W.uniform_costs(3, 30000, seed=41)
    a0, c0, u0, v0 = oracle_mod.km(C)
    for algo in (ot.OT_KM, ot.OT_BKM):
        a, c, u, v, _ = solve(ctx, C, algo)
        assert c == c0
        assert oracle_mod.check_certificate(C, a, u, v, c) == 0
    too_wide = torch.zeros((2, 65537), dtype=torch.int32, device="cuda")
    with pytest.raises(ot.OtError) as e:
        ot.ot_assign_solve(ctx, too_wide, ot.OT_KM)
    assert e.value.code == ot.OT_ERR_UNSUPPORTED
