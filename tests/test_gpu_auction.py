"""GPU auction engine (OT_AUCTION: the auction algorithm with epsilon-scaling,
Sec. 2.3.3 and Sec. 4.1 "Auction") against the CPU oracle's auction: the
rounds are deterministic, so assignment, cost and counters must agree
exactly; the cost must also equal the KM optimum."""
import numpy as np
import pytest
import torch

from paper_2005_01182_gb300 import otassign as ot
from paper_2005_01182_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def gpu_auction(ctx, C):
    r, c, u, v, st = ot.ot_assign_solve_stats(ctx, torch.from_numpy(np.ascontiguousarray(C)).cuda(), ot.OT_AUCTION)
    return r.cpu().numpy(), int(c.item()), u.cpu().numpy(), v.cpu().numpy(), st


def check(oracle_mod, ctx, C):
    n, m = C.shape
    a0, c0, _, st0 = oracle_mod.auction(C, stats=True)
    a, c, u, v, st = gpu_auction(ctx, C)
    assert c == c0
    np.testing.assert_array_equal(a, a0)
    assert st["steps"] == st0["rounds"]
    assert st["rows_scanned"] == st0["bids"]
    assert st["phases"] == st0["stages"]
    assert st["cost_bytes"] == 4 * m * st0["real_bids"]
    assert st["init_bytes"] == 4 * n * m
    assert (u == 0).all() and (v == 0).all()
    return c


CASES = [
    ("uniform", lambda s: W.uniform_costs(100, seed=s)),
    ("uniform_rect", lambda s: W.uniform_costs(70, 97, seed=s)),
    ("pixel_ties", lambda s: W.pixel_sqdist(120, seed=s)),
    ("embed", lambda s: W.embedding_costs(64, seed=s)),
    ("grid", lambda s: W.grid_sqdist(256, seed=s)),
    ("negative_wide_range",
     lambda s: np.random.default_rng(s).integers(-(1 << 30), 1 << 30, size=(50, 60)).astype(np.int32)),
    ("tiny", lambda s: np.random.default_rng(s).integers(0, 4, size=(3, 3)).astype(np.int32)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_auction_matches_oracle(oracle_mod, ctx, name, make):
    for s in range(3):
        C = make(s)
        c = check(oracle_mod, ctx, C)
        assert c == oracle_mod.km(C)[1]


def test_auction_degenerate(oracle_mod, ctx):
    for C in [np.array([[5]], np.int32), np.array([[3, 1, 2, 7]], np.int32), np.zeros((17, 33), np.int32),
              np.full((40, 40), 9, np.int32), np.arange(64, dtype=np.int32).reshape(8, 8)]:
        check(oracle_mod, ctx, C)


def test_auction_every_shape(oracle_mod, ctx):
    """One size per thread count of the auction engine (32 .. 512 threads).
    Near-square: many more columns than rows make the zero-cost padding rows
    bid against one another for many rounds (slow, still exact)."""
    for n, m in [(60, 64), (120, 128), (250, 256), (1000, 1024), (1500, 1500)]:
        check(oracle_mod, ctx, W.uniform_costs(n, m, seed=n))


def test_auction_batched(oracle_mod, ctx):
    rng = np.random.default_rng(11)
    mats = []
    for t in range(60):
        n = int(rng.integers(1, 300))
        m = n + int(rng.integers(0, 20))
        mats.append(W.uniform_costs(n, m, hi=1000, seed=t) if t % 2 else W.pixel_sqdist(n, m, seed=t))
    b = ot.ot_assign_solve_batched(ctx, [torch.from_numpy(C).cuda() for C in mats], ot.OT_AUCTION)
    torch.cuda.synchronize()
    assert (b.status.cpu().numpy() == 0).all()
    for t, C in enumerate(mats):
        a0, c0, _ = oracle_mod.auction(C)
        assert int(b.cost[t]) == c0
        np.testing.assert_array_equal(b.outs[t][0].cpu().numpy(), a0)


def test_auction_4096(oracle_mod, ctx):
    C = W.uniform_costs(4096, seed=21, hi=1 << 16)
    a0, c0, _ = oracle_mod.auction(C)
    a, c, _, _, _ = gpu_auction(ctx, C)
    assert c == c0
    np.testing.assert_array_equal(a, a0)


def test_auction_too_wide(ctx):
    C = torch.zeros((10, 4097), dtype=torch.int32, device="cuda")
    with pytest.raises(ot.OtError):
        ot.ot_assign_solve(ctx, C, ot.OT_AUCTION)
        torch.cuda.synchronize()
