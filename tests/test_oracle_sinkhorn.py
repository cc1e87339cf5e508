"""Pins of the oracle's log-domain Sinkhorn (Sec. 2.2 "Matrix Scaling",
Sec. 2.2.1 "Sinkhorn", Sec. 4.1 "Sinkhorn").

What fixes the result independently of the oracle's code:
  * closed forms: a constant cost and a rank-one cost C_ij = a_i + b_j make
    exp(-eta C) rank one, so one row-and-column scaling reaches
    X = r c^T / sum(r) exactly;
  * a permuted zero pattern C = K (1 - P), whose Sinkhorn solution has a
    closed form for every eta;
  * the limit eta -> infinity: the transport cost approaches the assignment
    optimum (brute force over permutations), within the entropy bound
    n log(m) / eta;
  * the textbook matrix-scaling form (Sinkhorn-Knopp on K = exp(-eta C),
    u = r / (K v), v = c / (K^T u)) runs the same sequence in the plain
    domain: f = log u, g = log v after every iteration;
  * at convergence the residue computed here from (f, g) is below the
    threshold and the column sums equal c.
A mutation test plants mistakes into a copy of the oracle.
"""
import importlib.util
import itertools
import os
import shutil
import tempfile

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "sinkhorn.py")


@pytest.fixture(scope="module")
def sk():
    import oracle.sinkhorn as mod
    return mod


def pin_constant(sk):
    n, m, kappa, eta = 5, 8, 7.0, 0.3
    C = np.full((n, m), kappa)
    f, g, cost, it, res = sk.sinkhorn(C, eta, eps_rel=1e-12, max_iter=50)
    # f_i = log r_i - log sum_j exp(-eta kappa) = eta kappa - log m; g_j = 0
    assert it == 1
    np.testing.assert_allclose(f, eta * kappa - np.log(m), rtol=0, atol=1e-12)
    np.testing.assert_allclose(g, 0.0, rtol=0, atol=1e-12)
    assert abs(cost - kappa * n) < 1e-9


def pin_rank_one(sk):
    rng = np.random.default_rng(3)
    n, m, eta = 6, 9, 0.7
    a, b = rng.uniform(0, 5, n), rng.uniform(0, 5, m)
    r, c = rng.uniform(0.5, 2, n), rng.uniform(0.5, 2, m)
    c *= r.sum() / c.sum()
    C = a[:, None] + b[None, :]
    f, g, cost, it, res = sk.sinkhorn(C, eta, eps_rel=1e-12, max_iter=50, r=r, c=c)
    assert it == 1
    X = np.exp(-eta * C + f[:, None] + g[None, :])
    np.testing.assert_allclose(X, np.outer(r, c) / r.sum(), rtol=1e-10)
    assert abs(cost - ((a * r).sum() + (b * c).sum())) < 1e-9 * cost


def pin_large_eta_reaches_assignment_optimum(sk):
    """<X, C> - h(X)/eta is minimal at X, so <X, C> <= OPT + (h(X) - h(P))/eta
    <= OPT + n log(m)/eta for an optimal permutation matrix P; X is feasible
    up to the residue, which moves the cost by at most residue * max C."""
    rng = np.random.default_rng(5)
    for _ in range(4):
        n = 4
        C = rng.integers(0, 10, size=(n, n)).astype(np.float64)
        opt = min(sum(C[i, p[i]] for i in range(n)) for p in itertools.permutations(range(n)))
        gaps = []
        for eta in (1.0, 3.0):
            f, g, cost, it, res = sk.sinkhorn(C, eta, eps_rel=1e-6, max_iter=4000)
            slack = res * C.max()
            assert opt - slack - 1e-9 <= cost <= opt + n * np.log(n) / eta + slack + 1e-9
            gaps.append(cost - opt)
        assert gaps[1] < gaps[0]


def pin_permuted_zero_closed_form(sk):
    """C = K (1 - P) for a permutation P: exp(-eta C) = (1 - t) P + t J with
    t = exp(-eta K), whose rows and columns all sum to 1 + (n - 1) t, so one
    iteration gives X = ((1 - t) P + t J) / (1 + (n - 1) t) and
    <C, X> = K n (n - 1) t / (1 + (n - 1) t), for every eta."""
    n, K = 7, 5.0
    P = np.eye(n)[np.random.default_rng(2).permutation(n)]
    C = K * (1 - P)
    for eta in (0.1, 1.0, 4.0):
        t = np.exp(-eta * K)
        f, g, cost, it, res = sk.sinkhorn(C, eta, eps_rel=1e-12, max_iter=20)
        assert it == 1
        X = np.exp(-eta * C + f[:, None] + g[None, :])
        np.testing.assert_allclose(X, ((1 - t) * P + t) / (1 + (n - 1) * t), rtol=1e-12, atol=1e-300)
        assert abs(cost - K * n * (n - 1) * t / (1 + (n - 1) * t)) <= 1e-12 * max(1.0, cost)


def pin_plain_domain_equivalence(sk):
    rng = np.random.default_rng(7)
    n, m, eta = 12, 15, 0.05
    C = rng.integers(0, 60, size=(n, m)).astype(np.float64)
    r, c = sk.default_marginals(n, m)
    K = np.exp(-eta * C)
    v = np.ones(m)
    for k in range(1, 8):
        u = r / (K @ v)
        v = c / (K.T @ u)
        f, g, _, it, _ = sk.sinkhorn(C, eta, max_iter=k, check=False)
        assert it == k
        np.testing.assert_allclose(f, np.log(u), rtol=1e-11, atol=1e-11)
        np.testing.assert_allclose(g, np.log(v), rtol=1e-11, atol=1e-11)


def pin_converged_marginals(sk):
    rng = np.random.default_rng(9)
    n, m, eta = 20, 30, 0.02
    C = rng.integers(0, 200, size=(n, m)).astype(np.float64)
    r = rng.uniform(0.5, 2.0, n)
    c = rng.uniform(0.5, 2.0, m)
    c *= r.sum() / c.sum()
    f, g, cost, it, res = sk.sinkhorn(C, eta, eps_rel=1e-6, max_iter=5000, r=r, c=c)
    X = np.exp(-eta * C + f[:, None] + g[None, :])
    assert np.abs(r - X.sum(1)).sum() + np.abs(c - X.sum(0)).sum() <= 1e-6 * r.sum()
    np.testing.assert_allclose(X.sum(0), c, rtol=1e-12)
    assert abs(cost - (C * X).sum()) < 1e-9 * cost
    assert it > 1


PINS = [pin_constant, pin_rank_one, pin_permuted_zero_closed_form, pin_large_eta_reaches_assignment_optimum,
        pin_plain_domain_equivalence, pin_converged_marginals]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pins(sk, pin):
    pin(sk)


def test_fixed_iteration_count(sk):
    C = np.arange(12.0).reshape(3, 4)
    f, g, cost, it, res = sk.sinkhorn(C, 0.1, max_iter=4, check=False)
    assert it == 4 and np.isfinite(res)


MUTANTS = [
    ("K = -eta * C", "K = eta * C"),                                                   # wrong sign
    ("g = logc - logsumexp(K + f[:, None], axis=0)", "g = logc - logsumexp(K, axis=0)"),  # dropped term
    ("f = logr - logsumexp(K + g[None, :], axis=1)", "f = -logsumexp(K + g[None, :], axis=1)"),  # dropped log r
    ("if res <= threshold:", "if res <= 100 * threshold:"),                            # early stop
    ("X = np.exp(-eta * C + np.asarray(f, np.float64)[:, None]", "X = np.exp(-eta * C.T.T + np.asarray(f, np.float64)[:, None] * 0"),
]


@pytest.mark.parametrize("idx", range(len(MUTANTS)))
def test_pins_catch_planted_mistakes(idx):
    src = open(SRC).read()
    old, new = MUTANTS[idx]
    assert old in src, old
    d = tempfile.mkdtemp()
    path = os.path.join(d, "sk_mutant.py")
    open(path, "w").write(src.replace(old, new, 1))
    spec = importlib.util.spec_from_file_location("sk_mutant", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    caught = False
    for pin in PINS:
        try:
            with np.errstate(all="ignore"):
                pin(mod)
        except (AssertionError, FloatingPointError, ValueError):
            caught = True
            break
    shutil.rmtree(d)
    assert caught, f"mutant {idx} survived the pins"
