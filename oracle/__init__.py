"""CPU oracle for the exact assignment problem -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this package.  The product
library never calls it and shares no code with it.

The arithmetic lives in ``ot_oracle.c`` (plain C, single-threaded, int64
duals); this module only compiles it with gcc and marshals numpy arrays.

What each function follows in the paper:
  * ``brute_force``  -- the plain definition of the assignment problem
    (Sec. 1, Eq. 1 with all-ones supplies and demands).
  * ``km``           -- the exact Kuhn-Munkres algorithm (Sec. 2.3, Sec. 4.1
    "KM and variants").
  * ``bkm``          -- batched KM, exact mode (Sec. 2.3 "Batched KM").
  * ``check_certificate`` -- LP duality for Eq. 1 (weak duality makes a
    feasible dual with equal objective a proof of optimality).
  * ``transport``    -- integer-supply transport (Eq. 1, Sec. 1) by vertex
    replication onto ``km``.
  * ``auction``      -- the auction algorithm with epsilon-scaling in
    parallel (Jacobi) rounds (Sec. 2.3.3 "The auction algorithm", Sec. 4.1
    "Auction"), exact for integer costs by scaling them by N + 1 and
    finishing at epsilon = 1.

``oracle.sinkhorn`` (numpy, float64) holds the log-domain Sinkhorn of
Sec. 2.2.1, pinned in ``tests/test_oracle_sinkhorn.py``.

Parity is pinned for every function (brute force over permutations, closed
forms, scipy's ``linear_sum_assignment``, the certificate); see
``tests/test_oracle.py``.  bKM's intermediate round structure (how many
dual adjustments, phases) is "parity unpinned": the paper prints no counts.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ot_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

_lib = None

CERT_CODES = {
    0: "ok",
    1: "assignment out of range",
    2: "column used twice",
    3: "dual infeasible",
    4: "matched pair not tight",
    5: "column dual positive or nonzero on an unmatched column",
    6: "cost differs from matched sum",
    7: "cost differs from dual objective",
    8: "bad sizes",
}


def build(force: bool = False) -> str:
    """Compile ot_oracle.c into a shared object (gcc -O2, no arch flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        for name in ("oracle_km", "oracle_bkm"):
            f = getattr(lib, name)
            f.restype = ctypes.c_int64
            f.argtypes = [i32p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, i32p, i64p, i64p, i64p]
        lib.oracle_brute_force.restype = ctypes.c_int64
        lib.oracle_brute_force.argtypes = [i32p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, i32p]
        lib.oracle_auction.restype = ctypes.c_int64
        lib.oracle_auction.argtypes = [i32p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, i32p, i64p, i64p]
        lib.oracle_check_certificate.restype = ctypes.c_int
        lib.oracle_check_certificate.argtypes = [i32p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                                 i32p, i64p, i64p, ctypes.c_int64]
        _lib = lib
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _as_cost(C):
    C = np.ascontiguousarray(C, dtype=np.int32)
    if C.ndim != 2:
        raise ValueError("cost matrix must be 2-D")
    n, m = C.shape
    if n > m:
        raise ValueError("need n <= m")
    return C, n, m


def km(C, stats: bool = False):
    """Exact Kuhn-Munkres.  Returns (row_to_col int32[n], cost, u int64[n],
    v int64[m]) and, with ``stats``, {steps, bytes, augmentations}."""
    C, n, m = _as_cost(C)
    a = np.empty(n, np.int32)
    u = np.empty(n, np.int64)
    v = np.empty(m, np.int64)
    st = np.zeros(4, np.int64)
    cost = _load().oracle_km(_p(C, ctypes.c_int32), m, n, m, _p(a, ctypes.c_int32),
                             _p(u, ctypes.c_int64), _p(v, ctypes.c_int64), _p(st, ctypes.c_int64))
    if cost == np.iinfo(np.int64).min:
        raise MemoryError("oracle_km failed")
    out = (a, int(cost), u, v)
    if stats:
        return out + ({"steps": int(st[0]), "bytes": int(st[1]), "augmentations": int(st[2])},)
    return out


def bkm(C, stats: bool = False):
    """Exact batched KM (scaling factor 1).  Same returns as ``km``; stats are
    {rounds, phases, augmentations, bytes}."""
    C, n, m = _as_cost(C)
    a = np.empty(n, np.int32)
    u = np.empty(n, np.int64)
    v = np.empty(m, np.int64)
    st = np.zeros(4, np.int64)
    cost = _load().oracle_bkm(_p(C, ctypes.c_int32), m, n, m, _p(a, ctypes.c_int32),
                              _p(u, ctypes.c_int64), _p(v, ctypes.c_int64), _p(st, ctypes.c_int64))
    if cost == np.iinfo(np.int64).min:
        raise MemoryError("oracle_bkm failed")
    out = (a, int(cost), u, v)
    if stats:
        return out + ({"rounds": int(st[0]), "phases": int(st[1]), "augmentations": int(st[2]),
                       "bytes": int(st[3])},)
    return out


def auction(C, stats: bool = False):
    """Exact auction with epsilon-scaling.  Returns (row_to_col int32[n],
    cost, prices int64[m] in scaled units) and, with ``stats``, {stages,
    rounds, bids, real_bids}."""
    C, n, m = _as_cost(C)
    a = np.empty(n, np.int32)
    p = np.zeros(m, np.int64)
    st = np.zeros(4, np.int64)
    cost = _load().oracle_auction(_p(C, ctypes.c_int32), m, n, m, _p(a, ctypes.c_int32),
                                  _p(p, ctypes.c_int64), _p(st, ctypes.c_int64))
    if cost == np.iinfo(np.int64).min:
        raise ValueError("oracle_auction failed (allocation or scaled range above 2^50)")
    out = (a, int(cost), p)
    if stats:
        return out + ({"stages": int(st[0]), "rounds": int(st[1]), "bids": int(st[2]),
                       "real_bids": int(st[3])},)
    return out


def transport(C, supply, demand):
    """Integer-supply transport (Eq. 1 with integer r and c, the
    Hitchcock-Koopmans case of Sec. 1) by vertex replication: row i is
    repeated supply[i] times and column j demand[j] times, in index order,
    ``km`` solves the replicated assignment problem, and the flow counts the
    copies of row i matched to copies of column j.  Demands are capacities:
    sum(supply) <= sum(demand).  Returns (flow int64 n x m, cost)."""
    C = np.ascontiguousarray(C, dtype=np.int32)
    r = np.asarray(supply, dtype=np.int64)
    c = np.asarray(demand, dtype=np.int64)
    n, m = C.shape
    if r.shape != (n,) or c.shape != (m,) or (r < 0).any() or (c < 0).any() or r.sum() > c.sum():
        raise ValueError("need nonnegative supplies and demands with sum(supply) <= sum(demand)")
    rows = np.repeat(np.arange(n), r)
    cols = np.repeat(np.arange(m), c)
    flow = np.zeros((n, m), np.int64)
    if len(rows) == 0:
        return flow, 0
    a, cost, _, _ = km(C[np.ix_(rows, cols)])
    np.add.at(flow, (rows, cols[a]), 1)
    return flow, int(cost)


def brute_force(C):
    """OPT by enumerating every injective row->column map (n <= 8, m <= 10)."""
    C, n, m = _as_cost(C)
    if n > 8 or m > 10:
        raise ValueError("brute force limited to n <= 8, m <= 10")
    a = np.zeros(max(n, 1), np.int32)
    cost = _load().oracle_brute_force(_p(C, ctypes.c_int32), m, n, m, _p(a, ctypes.c_int32))
    return a[:n], int(cost)


def check_certificate(C, row_to_col, u, v, cost) -> int:
    """0 if (row_to_col, u, v, cost) is a certified optimum, else a code from
    ``CERT_CODES``."""
    C, n, m = _as_cost(C)
    a = np.ascontiguousarray(row_to_col, dtype=np.int32)
    u = np.ascontiguousarray(u, dtype=np.int64)
    v = np.ascontiguousarray(v, dtype=np.int64)
    if a.shape != (n,) or u.shape != (n,) or v.shape != (m,):
        return 8
    return int(_load().oracle_check_certificate(_p(C, ctypes.c_int32), m, n, m, _p(a, ctypes.c_int32),
                                                _p(u, ctypes.c_int64), _p(v, ctypes.c_int64),
                                                int(cost)))
