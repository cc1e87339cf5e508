"""The sparse-list batched-KM engine against the dense cluster engine and the
CPU oracle.

Both engines run the same multi-source search with the same tie-breaks; the
sparse engine only takes its reduced costs from per-row candidate lists while
they are provably complete, so assignment, duals and the counters of levels
and phases must be identical bit for bit.  Against the oracle: optimal cost
and a valid dual certificate.
"""
import numpy as np
import pytest
import torch

from paper_2005_01182_gb300 import otassign as ot
from paper_2005_01182_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dense_ctx(lib_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = ot.Context(flags=ot.OT_CFG_DENSE_WIDE)
    yield c
    c.close()


@pytest.fixture(scope="module")
def sparse_ctx(lib_path):
    """A context of its own: an untuned table routes single batched-KM
    solves wider than 1024 columns to the wide engines."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = ot.Context()
    yield c
    c.close()


def solve(ctx, C, algo=ot.OT_BKM):
    r, c, u, v, st = ot.ot_assign_solve_stats(ctx, torch.from_numpy(np.ascontiguousarray(C)).cuda(), algo)
    return r.cpu().numpy(), int(c.item()), u.cpu().numpy(), v.cpu().numpy(), st


CASES = [
    ("grid", 1100, 1100), ("grid", 3000, 3000), ("grid", 2500, 2600),
    ("pixel", 1500, 1500), ("pixel", 1200, 2100),
    ("uniform", 2048, 2048), ("shapes", 2048, 2048), ("negative", 1300, 1333),
]


def make(kind, n, m, seed):
    if kind == "grid":
        return W.grid_sqdist(n, m, grid=int((n * 64) ** 0.5), seed=seed)
    if kind == "pixel":
        return W.pixel_sqdist(n, m, seed=seed)
    if kind == "uniform":
        return W.uniform_costs(n, m, seed=seed)
    if kind == "shapes":
        return W.shapes_sqdist(n, seed=seed)
    rng = np.random.default_rng(seed)
    return rng.integers(-(1 << 30), 1 << 30, size=(n, m)).astype(np.int32)


@pytest.mark.parametrize("kind,n,m", CASES)
def test_sparse_equals_dense_engine(oracle_mod, sparse_ctx, dense_ctx, kind, n, m):
    C = make(kind, n, m, seed=n + m)
    a, c, u, v, st = solve(sparse_ctx, C)
    a2, c2, u2, v2, st2 = solve(dense_ctx, C)
    assert c == c2
    np.testing.assert_array_equal(a, a2)
    np.testing.assert_array_equal(u, u2)
    np.testing.assert_array_equal(v, v2)
    assert st["steps"] == st2["steps"] and st["phases"] == st2["phases"]
    assert st["augmentations"] == n
    assert oracle_mod.check_certificate(C, a, u, v, c) == 0
    # the sparse engine reads far less than the dense one
    assert st["cost_bytes"] < st2["cost_bytes"]


def test_sparse_small_and_degenerate(oracle_mod, sparse_ctx):
    """Rows and columns of one, all-equal and all-zero costs, very few rows
    against many columns; optimum and certificate against the oracle."""
    cases = [np.zeros((1, 1), np.int32), np.array([[5, 3, 9]], np.int32),
             np.zeros((40, 1500), np.int32), np.full((1200, 1200), 7, np.int32),
             W.uniform_costs(3, 16384, seed=9), W.pixel_sqdist(1025, 1030, seed=3)]
    for C in cases:
        a, c, u, v, _ = solve(sparse_ctx, C)
        assert c == oracle_mod.km(C)[1]
        assert oracle_mod.check_certificate(C, a, u, v, c) == 0


def test_sparse_width_limit_falls_back_to_cluster_engine(oracle_mod, sparse_ctx):
    """Batched KM wider than 16384 columns stays on the cluster engine."""
    C = W.uniform_costs(5, 16390, seed=4)
    a, c, u, v, _ = solve(sparse_ctx, C)
    assert c == oracle_mod.km(C)[1]
    assert oracle_mod.check_certificate(C, a, u, v, c) == 0
