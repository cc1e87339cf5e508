"""The seeded input generators: shapes, value ranges and structure of the
stand-ins for the paper's workloads (Sec. 3.2, Table 1), and determinism."""
import numpy as np

from paper_2005_01182_gb300 import workloads as W


def test_deterministic_by_seed():
    a = W.embedding_costs(40, seed=11)
    assert np.array_equal(a, W.embedding_costs(40, seed=11))
    assert not np.array_equal(a, W.embedding_costs(40, seed=12))
    assert np.array_equal(W.pixel_sqdist(30, 35, seed=3), W.pixel_sqdist(30, 35, seed=3))


def test_value_ranges():
    g = W.grid_sqdist(200, grid=64, seed=1)
    assert g.dtype == np.int32 and g.min() >= 0 and g.max() <= 2 * 63 * 63
    p = W.pixel_sqdist(100, 120, seed=2)
    assert p.shape == (100, 120) and p.max() <= 2 * 27 * 27
    e = W.embedding_costs(64, seed=4)
    # unit vectors: distances in [0, 2], costs round(1e4 * distance)
    assert e.min() >= 0 and e.max() <= 20000
    u = W.uniform_costs(50, 60, seed=5)
    assert u.min() >= 0 and u.max() < (1 << 20)


def test_batch_sizes_span_the_range():
    s = W.batch_sizes(4096)
    assert s.min() >= 32 and s.max() <= 256 and len(s) == 4096
    assert len(np.unique(s)) > 200


def test_mnist_transport_totals_and_pixels():
    for n, m, total in [(116, 169, 2048), (12, 15, 40), (5, 5, 5)]:
        C, r, c = W.mnist_transport(n, m, total, seed=n)
        assert C.shape == (n, m) and C.dtype == np.int32 and C.max() <= 2 * 27 * 27
        assert r.sum() == total and c.sum() == total
        assert (r >= 1).all() and (c >= 1).all()
    # distinct pixels per image: two pixels of one image at the same place
    # would give two identical rows (or columns) of distances
    C, _, _ = W.mnist_transport(116, 169, 2048, seed=9)
    assert np.unique(C, axis=0).shape[0] == 116 and np.unique(C, axis=1).shape[1] == 169
