"""Pins of the CPU oracle against things other than itself (CPU only).

What fixes the answer of the assignment problem (paper Sec. 1, Eq. 1 with
all-ones supplies and demands) independently of any implementation:
  * brute force over every injective row->column map (plain definition),
  * closed forms (rank-one costs, dominant diagonal, permuted zero pattern,
    1-D convex costs where the sorted matching is optimal),
  * LP duality (a feasible dual with equal objective proves optimality),
  * scipy's linear_sum_assignment (an independent library routine),
  * hand-solved fixtures under tests/golden/.
A mutation test plants mistakes into a copy of the oracle and checks that
these pins catch them.
"""
import itertools
import os
import re
import shutil
import subprocess
import sys
import tempfile

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def py_brute(C):
    n, m = C.shape
    best = None
    for cols in itertools.permutations(range(m), n):
        s = int(sum(int(C[i, cols[i]]) for i in range(n)))
        if best is None or s < best:
            best = s
    return 0 if best is None else best


def rand_instance(r, n, m, lo, hi):
    return r.integers(lo, hi, size=(n, m)).astype(np.int32)


def check_all(oracle, C, expect_cost):
    for algo in (oracle.km, oracle.bkm):
        a, cost, u, v = algo(C)
        assert cost == expect_cost, (algo.__name__, C, cost, expect_cost)
        assert oracle.check_certificate(C, a, u, v, cost) == 0
        assert len(set(a.tolist())) == C.shape[0]
        assert (v <= 0).all()


def load_golden(name):
    lines = [l for l in open(os.path.join(HERE, "golden", name)) if not l.startswith("#")]
    cost = int(lines[0].split()[1])
    assign = [int(x) for x in lines[1].split()[1:]]
    mat = np.array([[int(x) for x in l.split()] for l in lines[3:] if l.strip()], np.int32)
    return mat, cost, assign


@pytest.mark.parametrize("name", ["hand_3x3.txt", "hand_2x4_negative.txt"])
def test_hand_solved(oracle_mod, name):
    C, cost, assign = load_golden(name)
    check_all(oracle_mod, C, cost)
    a, c, _, _ = oracle_mod.km(C)
    assert a.tolist() == assign  # unique optimum
    a, c, _, _ = oracle_mod.bkm(C)
    assert a.tolist() == assign
    assert py_brute(C) == cost


def test_c_brute_force_matches_python(oracle_mod):
    r = np.random.default_rng(1)
    for _ in range(200):
        n = int(r.integers(0, 6))
        m = int(r.integers(n, 7)) if n < 7 else n
        C = rand_instance(r, n, max(m, n), -20, 20)
        _, c = oracle_mod.brute_force(C)
        assert c == py_brute(C)


@pytest.mark.parametrize("lo,hi", [(0, 3), (0, 100), (-50, 50), (0, 1 << 20), (-(1 << 31), (1 << 31) - 1)])
def test_km_bkm_vs_brute_force(oracle_mod, lo, hi):
    r = np.random.default_rng(hi & 0xffff)
    for trial in range(600):
        n = int(r.integers(1, 9))
        m = n + int(r.integers(0, 3)) if n <= 8 else n
        m = min(m, 10)
        C = r.integers(lo, hi, size=(n, m), dtype=np.int64).astype(np.int32)
        _, best = oracle_mod.brute_force(C)
        check_all(oracle_mod, C, best)


def test_degenerate(oracle_mod):
    # empty, 1 x 1, 1 x m, all-equal, all-zero (KM's tie-breaks give identity)
    for C in [np.zeros((0, 0), np.int32), np.zeros((0, 5), np.int32)]:
        a, c, u, v = oracle_mod.km(C)
        assert c == 0 and a.size == 0 and (v == 0).all()
    C = np.array([[-7]], np.int32)
    check_all(oracle_mod, C, -7)
    C = np.array([[5, 3, 3, 9]], np.int32)
    check_all(oracle_mod, C, 3)
    a, *_ = oracle_mod.km(C)
    assert a.tolist() == [1]  # lowest column on ties
    C = np.full((6, 6), 4, np.int32)
    check_all(oracle_mod, C, 24)
    a, *_ = oracle_mod.km(np.zeros((7, 9), np.int32))
    assert a.tolist() == list(range(7))


def test_rank_one_closed_form(oracle_mod):
    # c_ij = a_i + b_j: every perfect matching costs sum(a) + sum(b)
    r = np.random.default_rng(3)
    for n in (1, 5, 40, 200):
        a = r.integers(-1000, 1000, n)
        b = r.integers(-1000, 1000, n)
        C = (a[:, None] + b[None, :]).astype(np.int32)
        check_all(oracle_mod, C, int(a.sum() + b.sum()))


def test_dominant_diagonal_closed_form(oracle_mod):
    # c_ii << c_ij: the identity is the unique optimum, cost = trace
    r = np.random.default_rng(4)
    for n in (2, 17, 150):
        C = r.integers(1000, 2000, size=(n, n)).astype(np.int32)
        d = r.integers(0, 10, n)
        C[np.arange(n), np.arange(n)] = d
        check_all(oracle_mod, C, int(d.sum()))
        for algo in (oracle_mod.km, oracle_mod.bkm):
            assert algo(C)[0].tolist() == list(range(n))


def test_permuted_zero_pattern(oracle_mod):
    # C = K * (1 - P) with P a permutation matrix: cost 0, assignment = P
    r = np.random.default_rng(5)
    for n in (3, 33, 120):
        p = r.permutation(n)
        C = r.integers(1, 500, size=(n, n)).astype(np.int32)
        C[np.arange(n), p] = 0
        check_all(oracle_mod, C, 0)
        for algo in (oracle_mod.km, oracle_mod.bkm):
            assert algo(C)[0].tolist() == p.tolist()


def test_one_dimensional_convex(oracle_mod):
    # points on a line, c = (x_i - y_j)^2 (convex): sorted-to-sorted is optimal
    r = np.random.default_rng(6)
    for n in (4, 50, 300):
        x = r.integers(0, 1000, n)
        y = r.integers(0, 1000, n)
        C = ((x[:, None] - y[None, :]) ** 2).astype(np.int32)
        expect = int(((np.sort(x) - np.sort(y)) ** 2).sum())
        check_all(oracle_mod, C, expect)


def test_vs_scipy(oracle_mod):
    from scipy.optimize import linear_sum_assignment
    from paper_2005_01182_gb300 import workloads as W
    r = np.random.default_rng(7)
    cases = [W.single_256(), W.embedding_costs(100, seed=11), W.pixel_sqdist(150, 170, seed=12),
             W.uniform_costs(90, 130, seed=13), W.shapes_sqdist(200, "circle-triangle", seed=14)]
    for _ in range(20):
        n = int(r.integers(1, 60))
        m = n + int(r.integers(0, 20))
        cases.append(rand_instance(r, n, m, -1000, 1000))
    for C in cases:
        ri, ci = linear_sum_assignment(C.astype(np.float64))
        check_all(oracle_mod, C, int(C[ri, ci].astype(np.int64).sum()))


def test_km_stats_bytes(oracle_mod):
    # the byte counter is 4 bytes per reduced cost evaluated; on a dominant
    # diagonal every row is matched in one step scanning all m columns
    n = 20
    C = np.full((n, n), 100, np.int32)
    C[np.arange(n), np.arange(n)] = 0
    *_, st = oracle_mod.km(C, stats=True)
    assert st["steps"] == n and st["bytes"] == 4 * n * n and st["augmentations"] == n


def test_km_counters_closed_form_all_ties(oracle_mod):
    """All costs equal: in the phase of row r every slack is 0, so the lowest
    column wins each step (0, 1, ..., r) and only column r is free; the
    strict < keeps every predecessor at the root, so row r takes column r.
    Phase r has r + 1 steps scanning m, m - 1, ..., m - r columns."""
    for n, m in [(6, 6), (5, 9), (30, 30)]:
        a, c, u, v, st = oracle_mod.km(np.zeros((n, m), np.int32), stats=True)
        assert a.tolist() == list(range(n)) and c == 0
        assert not u.any() and not v.any()
        assert st["steps"] == n * (n + 1) // 2
        assert st["bytes"] == 4 * sum((r + 1) * m - r * (r + 1) // 2 for r in range(n))


def test_certificate_rejects_planted_errors(oracle_mod):
    from paper_2005_01182_gb300 import workloads as W
    C = W.pixel_sqdist(40, 45, seed=3)
    a, cost, u, v = oracle_mod.km(C)
    assert oracle_mod.check_certificate(C, a, u, v, cost) == 0
    bad = a.copy(); bad[0], bad[1] = bad[1], bad[0]
    assert oracle_mod.check_certificate(C, bad, u, v, cost) != 0
    bad = a.copy(); bad[1] = bad[0]
    assert oracle_mod.check_certificate(C, bad, u, v, cost) == 2
    u2 = u.copy(); u2[3] += 1
    assert oracle_mod.check_certificate(C, a, u2, v, cost) != 0
    v2 = v.copy(); v2[:] = 0
    assert oracle_mod.check_certificate(C, a, u, v2, cost) != 0
    assert oracle_mod.check_certificate(C, a, u, v, cost + 1) == 6
    unmatched = sorted(set(range(45)) - set(a.tolist()))
    v3 = v.copy(); v3[unmatched[0]] = -1  # still feasible, but an unmatched column is priced
    assert oracle_mod.check_certificate(C, a, u, v3, cost) == 5


MUTANTS = [
    ("km", "u[r] += delta;", "u[r] += delta + 1;"),                      # extra term
    ("km", "v[j] -= delta; }", "v[j] += delta; }"),                       # wrong sign
    ("km", "int64_t rc = AT(C, ldc, i, j) - u[i] - v[j];\n        bytes += 4;",
     "int64_t rc = AT(C, ldc, j % n, i) - u[i] - v[j];\n        bytes += 4;"),  # transposed operand
    ("km", "else slack[j] -= delta;", "else slack[j] -= 0;"),            # dropped term
    ("km", "if (rc < slack[j]) { slack[j] = rc; pred[j] = i; }",
     "if (rc <= slack[j]) { slack[j] = rc; pred[j] = i; }"),              # tie-break: latest predecessor
    ("km", "if (!in_tree[j] && slack[j] < delta) { delta = slack[j]; jstar = j; }",
     "if (!in_tree[j] && slack[j] <= delta) { delta = slack[j]; jstar = j; }"),  # tie-break: highest column
    ("bkm", "if (rc < delta) delta = rc;", "if (rc < delta) delta = rc + 1;"),   # off-by-one step
    ("bkm", "for (int j = 0; j < m; ++j) { int64_t c = AT(C, ldc, i, j); if (c < mn) mn = c; }",
     "for (int j = 1; j < m; ++j) { int64_t c = AT(C, ldc, i, j); if (c < mn) mn = c; }"),  # wrong index
]


def _mutant_check(so, fn_name, seed):
    """Run in a child process: exit 0 if the mutant survives every pin."""
    import ctypes
    sys.path.insert(0, os.path.dirname(HERE))
    import oracle
    lib = ctypes.CDLL(so)
    fn = getattr(lib, fn_name)
    fn.restype = ctypes.c_int64
    r = np.random.default_rng(seed)
    P = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    for _ in range(300):
        n = int(r.integers(2, 7))
        C = r.integers(-30, 30, size=(n, n + int(r.integers(0, 2)))).astype(np.int32)
        n, m = C.shape
        a = np.zeros(n, np.int32); u = np.zeros(n, np.int64); v = np.zeros(m, np.int64)
        st = np.zeros(4, np.int64)
        cost = fn(P(C), ctypes.c_int64(m), n, m, P(a), P(u), P(v), P(st))
        if cost != py_brute(C) or oracle.check_certificate(C, a, u, v, cost) != 0:
            sys.exit(3)
    if fn_name == "oracle_km":
        # the tie-break rules, through the all-ties closed form
        # (test_km_counters_closed_form_all_ties)
        for n, m in [(6, 6), (5, 9)]:
            C = np.zeros((n, m), np.int32)
            a = np.zeros(n, np.int32); u = np.zeros(n, np.int64); v = np.zeros(m, np.int64)
            st = np.zeros(4, np.int64)
            fn(P(C), ctypes.c_int64(m), n, m, P(a), P(u), P(v), P(st))
            if a.tolist() != list(range(n)) or st[0] != n * (n + 1) // 2:
                sys.exit(4)
    sys.exit(0)


@pytest.mark.parametrize("idx", range(len(MUTANTS)))
def test_pins_catch_planted_mistakes(oracle_mod, idx):
    """Compile a mutated copy of the oracle (CPU only) and check that the
    brute-force / certificate pins reject it (a hang counts as caught)."""
    src = open(os.path.join(os.path.dirname(HERE), "oracle", "ot_oracle.c")).read()
    which, old, new = MUTANTS[idx]
    assert old in src, old
    d = tempfile.mkdtemp()
    try:
        so = os.path.join(d, "m.so")
        cfile = os.path.join(d, "m.c")
        open(cfile, "w").write(src.replace(old, new, 1))
        subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-o", so, cfile],
                              stderr=subprocess.DEVNULL)
        try:
            r = subprocess.run([sys.executable, __file__, "--mutant-check", so, "oracle_" + which, str(idx)],
                               timeout=60, capture_output=True)
            survived = r.returncode == 0
        except subprocess.TimeoutExpired:
            survived = False
        assert not survived, f"mutant {idx} survived the pins"
    finally:
        shutil.rmtree(d)


if __name__ == "__main__" and len(sys.argv) == 5 and sys.argv[1] == "--mutant-check":
    _mutant_check(sys.argv[2], sys.argv[3], int(sys.argv[4]))


def test_single_scaling_factor_bound(oracle_mod):
    """The paper's approximate batched KM solves floor(C/s) exactly; with
    c = s*floor(c/s) + r, 0 <= r <= s-1, the assignment it returns costs at
    most OPT + n*(s-1) under C.  Checked against brute force."""
    r = np.random.default_rng(21)
    for trial in range(300):
        n = int(r.integers(1, 7))
        m = n + int(r.integers(0, 2))
        C = r.integers(-500, 5000, size=(n, m)).astype(np.int32)
        _, opt = oracle_mod.brute_force(C)
        for s in (1, 2, 7, 100, 4096):
            Cs = np.floor_divide(C, s).astype(np.int32)
            a, cs, u, v = oracle_mod.bkm(Cs)
            true = int(C[np.arange(n), a].astype(np.int64).sum())
            assert cs == oracle_mod.brute_force(Cs)[1]
            assert opt <= true <= opt + n * (s - 1)
            if s == 1:
                assert true == opt


def _transport_lp(C, r, c):
    """Optimal value of min <C, X>, X 1 = r, X^T 1 <= c, X >= 0 (scipy LP;
    integral at the optimum for integer r, c)."""
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
    assert res.status == 0
    return int(round(res.fun))


def _check_flow(C, r, c, flow, cost):
    assert (flow >= 0).all()
    np.testing.assert_array_equal(flow.sum(1), r)
    assert (flow.sum(0) <= c).all()
    assert int((flow * C.astype(np.int64)).sum()) == cost


def _pin_transport_lp(transport):
    """Vertex replication turns integer-supply transport (Eq. 1) into an
    assignment problem with the same optimum: the folded flow is feasible,
    costs what the oracle reports, and that cost equals an LP optimum."""
    rng = np.random.default_rng(31)
    for trial in range(40):
        n, m = int(rng.integers(1, 6)), int(rng.integers(1, 7))
        r = rng.integers(0, 5, n)
        c = rng.integers(0, 6, m)
        if r.sum() > c.sum():
            c[0] += r.sum() - c.sum()
        C = rng.integers(-20, 100, size=(n, m)).astype(np.int32)
        flow, cost = transport(C, r, c)
        _check_flow(C, r, c, flow, cost)
        if r.sum() > 0:
            assert cost == _transport_lp(C, r, c)
        else:
            assert cost == 0 and not flow.any()


def _pin_transport_closed_forms(transport, brute_force):
    """One source fills the cheapest columns first (a greedy optimum); one
    sink takes every unit; unit supplies and demands give the assignment."""
    rng = np.random.default_rng(37)
    for trial in range(30):
        m = int(rng.integers(1, 9))
        C = rng.integers(0, 50, size=(1, m)).astype(np.int32)
        c = rng.integers(0, 4, m)
        s = int(rng.integers(0, c.sum() + 1))
        left, best = s, 0
        for j in np.argsort(C[0], kind="stable"):
            take = min(left, int(c[j]))
            best += take * int(C[0, j])
            left -= take
        flow, cost = transport(C, [s], c)
        _check_flow(C, [s], c, flow, cost)
        assert cost == best
        n = int(rng.integers(1, 6))
        C1 = rng.integers(-30, 30, size=(n, 1)).astype(np.int32)
        r1 = rng.integers(0, 4, n)
        d1 = [int(r1.sum()) + int(rng.integers(0, 3))]
        flow, cost = transport(C1, r1, d1)
        _check_flow(C1, r1, d1, flow, cost)
        assert cost == int((C1[:, 0].astype(np.int64) * r1).sum())
        k = int(rng.integers(1, 7))
        Ck = rng.integers(0, 100, size=(k, k + 1)).astype(np.int32)
        flow, cost = transport(Ck, np.ones(k, int), np.ones(k + 1, int))
        _check_flow(Ck, np.ones(k, int), np.ones(k + 1, int), flow, cost)
        assert cost == brute_force(Ck)[1]


def test_transport_by_replication(oracle_mod):
    _pin_transport_lp(oracle_mod.transport)


def test_transport_closed_forms(oracle_mod):
    _pin_transport_closed_forms(oracle_mod.transport, oracle_mod.brute_force)


TRANSPORT_MUTANTS = [
    ("np.add.at(flow, (rows, cols[a]), 1)", "np.add.at(flow, (rows, a % m), 1)"),  # column copies not folded
    ("rows = np.repeat(np.arange(n), r)", "rows = np.repeat(np.arange(n), np.minimum(r, 1))"),  # supply dropped
    ("cols = np.repeat(np.arange(m), c)", "cols = np.repeat(np.arange(m), c + 1)"),  # demand ignored
    ("km(C[np.ix_(rows, cols)])", "km(-C[np.ix_(rows, cols)])"),  # wrong sign
    ("return flow, int(cost)", "return flow, int(cost) - int(len(rows) > 1)"),  # cost off the flow's
]


@pytest.mark.parametrize("idx", range(len(TRANSPORT_MUTANTS)))
def test_transport_pins_catch_planted_mistakes(oracle_mod, idx):
    import inspect
    src = inspect.getsource(oracle_mod.transport)
    old, new = TRANSPORT_MUTANTS[idx]
    assert old in src, old
    ns = dict(vars(oracle_mod))
    exec(src.replace(old, new, 1), ns)
    caught = False
    for pin in (lambda t: _pin_transport_lp(t), lambda t: _pin_transport_closed_forms(t, oracle_mod.brute_force)):
        try:
            pin(ns["transport"])
        except (AssertionError, ValueError, IndexError):
            caught = True
            break
    assert caught, f"transport mutant {idx} survived the pins"


def test_stored_oracle_costs_reproduce(oracle_mod):
    """tests/golden/oracle_costs.txt holds the oracle's optima of the large
    named workloads (written by tests/golden/make_oracle_costs.py); the
    cheapest entry is recomputed here, so the file cannot drift from the
    oracle unnoticed."""
    from paper_2005_01182_gb300 import workloads as W
    stored = {}
    for line in open(os.path.join(HERE, "golden", "oracle_costs.txt")):
        f = line.split()
        if f and not line.startswith("#"):
            stored[f[0]] = int(f[1])
    assert set(stored) == {"single_4096_circle_square", "single_4096_circle_triangle", "single_4096_uniform",
                           "single_16384_grid"}
    assert oracle_mod.km(W.single_4096("uniform"))[1] == stored["single_4096_uniform"]
