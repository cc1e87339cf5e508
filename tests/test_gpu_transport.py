"""GPU integer-supply transport (vertex replication) against an LP optimum."""
import numpy as np
import pytest
import torch

from paper_2005_01182_gb300 import otassign as ot
from paper_2005_01182_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _lp(C, r, c):
    from scipy.optimize import linprog
    n, m = C.shape
    A_eq = np.zeros((n, n * m))
    for i in range(n):
        A_eq[i, i * m:(i + 1) * m] = 1
    A_ub = np.zeros((m, n * m))
    for j in range(m):
        A_ub[j, j::m] = 1
    res = linprog(C.astype(np.float64).ravel(), A_ub=A_ub, b_ub=c, A_eq=A_eq, b_eq=r, bounds=(0, None),
                  method="highs")
    return int(round(res.fun))


@pytest.mark.parametrize("algo", [ot.OT_KM, ot.OT_BKM, ot.OT_AUTO])
def test_transport_matches_lp(ctx, algo):
    rng = np.random.default_rng(7 + algo)
    for trial in range(12):
        n, m = int(rng.integers(1, 15)), int(rng.integers(1, 15))
        r = rng.integers(0, 12, n)
        c = rng.integers(0, 14, m)
        if r.sum() > c.sum():
            c[-1] += r.sum() - c.sum()
        C = rng.integers(0, 500, size=(n, m)).astype(np.int32)
        for dev in (True, False):
            Ct = torch.from_numpy(C).cuda() if dev else torch.from_numpy(C)
            flow, cost = ot.ot_transport_solve(ctx, Ct, r, c, algo)
            X = flow.cpu().numpy().astype(np.int64)
            assert (X >= 0).all()
            np.testing.assert_array_equal(X.sum(1), r)
            assert (X.sum(0) <= c).all()
            assert int((X * C).sum()) == cost
            assert cost == _lp(C, r, c)


def test_transport_mnist_like(ctx):
    """Two 'images': pixel positions on a 28 x 28 grid with small integer
    intensities as supplies/demands, squared-distance costs."""
    rng = np.random.default_rng(3)
    pa = rng.choice(784, 40, replace=False)
    pb = rng.choice(784, 45, replace=False)
    r = rng.integers(1, 8, 40)
    c = rng.integers(1, 8, 45)
    c[0] += max(0, r.sum() - c.sum())
    a = np.stack([pa // 28, pa % 28], 1)
    b = np.stack([pb // 28, pb % 28], 1)
    C = ((a[:, None, :] - b[None, :, :]) ** 2).sum(-1).astype(np.int32)
    flow, cost = ot.ot_transport_solve(ctx, torch.from_numpy(C).cuda(), r, c)
    X = flow.cpu().numpy()
    np.testing.assert_array_equal(X.sum(1), r)
    assert cost == _lp(C, r, c)


def test_transport_km_flow_matches_oracle(ctx, oracle_mod):
    """Through KM on the replicated matrix (rows and columns repeated in
    index order on both sides) the flow is the oracle's, entry for entry;
    batched KM and the automatic choice reach the same cost."""
    cases = [W.mnist_transport(40, 45, 300, seed=5), W.mnist_transport(116, 169, 700, seed=6)]
    rng = np.random.default_rng(17)
    for _ in range(4):
        n, m = int(rng.integers(1, 30)), int(rng.integers(1, 30))
        r = rng.integers(0, 9, n).astype(np.int32)
        c = rng.integers(0, 11, m).astype(np.int32)
        if r.sum() > c.sum():
            c[-1] += r.sum() - c.sum()
        cases.append((rng.integers(-300, 300, size=(n, m)).astype(np.int32), r, c))
    for C, r, c in cases:
        f0, c0 = oracle_mod.transport(C, r, c)
        Cd = torch.from_numpy(C).cuda()
        flow, cost = ot.ot_transport_solve(ctx, Cd, r, c, ot.OT_KM)
        assert cost == c0
        np.testing.assert_array_equal(flow.cpu().numpy(), f0)
        for algo in (ot.OT_BKM, ot.OT_AUTO):
            flow, cost = ot.ot_transport_solve(ctx, Cd, r, c, algo)
            X = flow.cpu().numpy().astype(np.int64)
            assert cost == c0 and int((X * C).sum()) == c0
            np.testing.assert_array_equal(X.sum(1), r)
            assert (X.sum(0) <= c).all()


def test_transport_degenerate_and_limits(ctx, oracle_mod):
    """No supply (zero flow, zero cost, host or device C); one unit; the
    argument checks (supply above demand, negative entries) and the size
    limit of replication, all reported as error codes."""
    C = np.arange(12, dtype=np.int32).reshape(3, 4)
    for dev in (True, False):
        Ct = torch.from_numpy(C).cuda() if dev else torch.from_numpy(C)
        flow, cost = ot.ot_transport_solve(ctx, Ct, [0, 0, 0], [1, 0, 2, 0])
        assert cost == 0 and not flow.cpu().numpy().any()
    flow, cost = ot.ot_transport_solve(ctx, torch.from_numpy(C).cuda(), [0, 1, 0], [0, 0, 3, 1], ot.OT_KM)
    f0, c0 = oracle_mod.transport(C, [0, 1, 0], [0, 0, 3, 1])
    assert cost == c0 == 6 and np.array_equal(flow.cpu().numpy(), f0)
    for sup, dem, code in [([2, 2, 2], [1, 1, 1, 1], ot.OT_ERR_ARG), ([1, -1, 1], [1, 1, 1, 1], ot.OT_ERR_ARG),
                           ([1, 0, 0], [1, -2, 1, 1], ot.OT_ERR_ARG),
                           ([1, 0, 0], [70000, 0, 0, 0], ot.OT_ERR_UNSUPPORTED)]:
        with pytest.raises(ot.OtError) as e:
            ot.ot_transport_solve(ctx, torch.from_numpy(C).cuda(), sup, dem)
        assert e.value.code == code
