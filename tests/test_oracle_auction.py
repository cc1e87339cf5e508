"""Pins of the oracle's auction algorithm with epsilon-scaling (paper,
Sec. 2.3.3 "The auction algorithm" and Sec. 4.1 "Auction").

What fixes the result independently of the oracle's code:
  * two instances traced by hand (tests/golden/auction_*.txt): every bid,
    price and counter of the rounds;
  * the optimum itself: brute force over permutations on tiny instances and
    scipy's linear_sum_assignment on larger ones (the auction is exact for
    integer costs once epsilon < 1/n, here through the N + 1 cost scaling);
  * epsilon-complementary slackness at the end of the last stage: every
    bidder holds an object within epsilon = 1 of its best value under the
    final prices.
A mutation test plants mistakes into a copy of the oracle (CPU only).
"""
import os
import shutil
import subprocess
import sys
import tempfile

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def load_trace(name):
    d = {}
    rows = []
    in_matrix = False
    for line in open(os.path.join(HERE, "golden", name)):
        if line.startswith("#") or not line.strip():
            continue
        tok = line.split()
        if in_matrix:
            rows.append([int(x) for x in tok])
        elif tok[0] == "matrix":
            in_matrix = True
        elif tok[0] == "stats":
            d["stats"] = {tok[k]: int(tok[k + 1]) for k in range(1, len(tok), 2)}
        else:
            d[tok[0]] = [int(x) for x in tok[1:]]
    return np.array(rows, np.int32), d


TRACES = ["auction_2x2_one_stage.txt", "auction_2x2_two_stages.txt", "auction_2x2_tied_bids.txt"]


@pytest.mark.parametrize("name", TRACES)
def test_hand_traces(oracle_mod, name):
    C, d = load_trace(name)
    a, cost, p, st = oracle_mod.auction(C, stats=True)
    assert cost == d["cost"][0]
    assert a.tolist() == d["assignment"]
    assert p.tolist() == d["prices"]
    for k, v in d["stats"].items():
        assert st[k] == v, k


def brute(C):
    import itertools
    n, m = C.shape
    return min(sum(int(C[i, c[i]]) for i in range(n)) for c in itertools.permutations(range(m), n))


@pytest.mark.parametrize("lo,hi", [(-40, 40), (0, 3), (0, 1000000), (-(1 << 30), 1 << 30)])
def test_exact_vs_brute_force(oracle_mod, lo, hi):
    r = np.random.default_rng(hi)
    for _ in range(150):
        n = int(r.integers(1, 7))
        m = n + int(r.integers(0, 3))
        C = r.integers(lo, hi, size=(n, m)).astype(np.int32)
        a, cost, _ = oracle_mod.auction(C)
        assert cost == brute(C)
        assert len(set(a.tolist())) == n and a.min() >= 0 and a.max() < m
        assert cost == int(C[np.arange(n), a].sum())


def test_exact_vs_scipy(oracle_mod):
    from scipy.optimize import linear_sum_assignment
    from paper_2005_01182_gb300 import workloads as W
    cases = [W.uniform_costs(120, seed=1), W.uniform_costs(90, 130, seed=2),
             W.pixel_sqdist(150, seed=3), W.embedding_costs(100, seed=4),
             W.grid_sqdist(200, seed=5), np.zeros((30, 40), np.int32)]
    for C in cases:
        r, c = linear_sum_assignment(C)
        a, cost, _ = oracle_mod.auction(C)
        assert cost == int(C[r, c].sum())


def test_epsilon_complementary_slackness(oracle_mod):
    """At the end of the eps = 1 stage each bidder's object is within 1 of
    its best value w_ij = C'[i][j] + p_j (scaled costs, dummy rows 0)."""
    from paper_2005_01182_gb300 import workloads as W
    for C in [W.uniform_costs(60, 75, seed=7), W.pixel_sqdist(80, seed=8)]:
        n, m = C.shape
        a, cost, p = oracle_mod.auction(C)
        S = (C.astype(np.int64) - C.min()) * (m + 1)
        W_ = S + p[None, :]
        held = W_[np.arange(n), a]
        assert (held <= W_.min(axis=1) + 1).all()
        # dummy bidders hold the remaining objects, each within 1 of min p
        rest = sorted(set(range(m)) - set(a.tolist()))
        assert (p[rest] <= p.min() + 1).all()


def test_degenerate(oracle_mod):
    a, cost, p = oracle_mod.auction(np.zeros((0, 5), np.int32))
    assert cost == 0 and len(a) == 0
    a, cost, p = oracle_mod.auction(np.array([[7]], np.int32))
    assert cost == 7 and a.tolist() == [0]
    a, cost, p = oracle_mod.auction(np.full((6, 6), 4, np.int32))
    assert cost == 24 and sorted(a.tolist()) == list(range(6))


MUTANTS = [
    ("if (eps == 1) break;", "if (eps <= 4) break;"),                 # stops before eps = 1
    ("bid_amt[i] = p[j1] + (w2 - w1) + eps;", "bid_amt[i] = p[j1] + eps;"),  # dropped term
    ("const int64_t w = c + p[j];", "const int64_t w = c - p[j];"),     # wrong sign
    ("if (j >= 0 && (win[j] < 0 || bid_amt[i] > bid_amt[win[j]])) win[j] = i;",
     "if (j >= 0 && (win[j] < 0 || bid_amt[i] >= bid_amt[win[j]])) win[j] = i;"),  # tie-break
    ("const int64_t scale = (int64_t)N + 1;", "const int64_t scale = 1;"),          # no exactness scaling
]


def _mutant_check(so, seed):
    import ctypes
    lib = ctypes.CDLL(so)
    fn = lib.oracle_auction
    fn.restype = ctypes.c_int64
    P = lambda x: x.ctypes.data_as(ctypes.c_void_p)

    def run(C):
        n, m = C.shape
        a = np.zeros(n, np.int32); p = np.zeros(m, np.int64); st = np.zeros(4, np.int64)
        cost = fn(P(C), ctypes.c_int64(m), n, m, P(a), P(p), P(st))
        return a, cost, p, st
    for name in TRACES:
        C, d = load_trace(name)
        a, cost, p, st = run(C)
        if (cost != d["cost"][0] or a.tolist() != d["assignment"] or p.tolist() != d["prices"]
                or int(st[2]) != d["stats"]["bids"]):
            sys.exit(3)
    r = np.random.default_rng(seed)
    for _ in range(300):
        n = int(r.integers(2, 7))
        C = r.integers(-30, 30, size=(n, n + int(r.integers(0, 2)))).astype(np.int32)
        a, cost, p, st = run(C)
        if cost != brute(C):
            sys.exit(3)
    sys.exit(0)


@pytest.mark.parametrize("idx", range(len(MUTANTS)))
def test_pins_catch_planted_mistakes(oracle_mod, idx):
    src = open(os.path.join(os.path.dirname(HERE), "oracle", "ot_oracle.c")).read()
    old, new = MUTANTS[idx]
    assert old in src, old
    d = tempfile.mkdtemp()
    try:
        so = os.path.join(d, "m.so")
        cfile = os.path.join(d, "m.c")
        open(cfile, "w").write(src.replace(old, new, 1))
        subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-o", so, cfile], stderr=subprocess.DEVNULL)
        try:
            r = subprocess.run([sys.executable, __file__, "--mutant-check", so, str(idx)],
                               timeout=60, capture_output=True)
            survived = r.returncode == 0
        except subprocess.TimeoutExpired:
            survived = False
        assert not survived, f"mutant {idx} survived the pins"
    finally:
        shutil.rmtree(d)


if __name__ == "__main__" and len(sys.argv) == 4 and sys.argv[1] == "--mutant-check":
    _mutant_check(sys.argv[2], int(sys.argv[3]))
