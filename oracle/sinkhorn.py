"""Log-domain Sinkhorn for entropic optimal transport -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module; the product library never calls it and shares
no code with it.  Plain numpy in float64; ``scipy.special.logsumexp`` is the
only library step.

What it follows in the paper:
  * Sec. 2.2.1 "Sinkhorn": the entropic problem min <X, C> - h(X)/eta over
    X 1 = r, X^T 1 = c has the solution X = D1 exp(-eta C) D2; it is found
    by scaling all rows and then all columns of exp(-eta C), alternately,
    until the residue ||r - X 1||_1 + ||c - X^T 1||_1 drops below a
    threshold epsilon.
  * Sec. 2.2 "Matrix Scaling": the logarithms of the scalings are tracked
    instead of the scalings (the log domain), against under- and overflow.
    Here X_ij = exp(f_i + g_j - eta C_ij).
  * Sec. 4.1 "Sinkhorn": the stopping threshold is 10^-3 times the summed
    demand, and the flow is not rounded; the reported cost is <C, X> of the unrounded X.

Readings where the paper is silent:
  * start from f = g = 0; one iteration scales the rows (f) and then the
    columns (g) with the new f; the residue is checked after every
    iteration and the first iterate at or below the threshold is returned;
  * unit supplies and demands (the assignment setting): r = 1 (n entries)
    and c = n/m (m entries), so that both sides carry the same total mass.
"""
from __future__ import annotations

import numpy as np
from scipy.special import logsumexp


def marginals(C, eta, f, g):
    """Row and column sums of X = exp(f_i + g_j - eta C_ij)."""
    logX = -eta * np.asarray(C, np.float64) + np.asarray(f, np.float64)[:, None] + np.asarray(g, np.float64)[None, :]
    return np.exp(logsumexp(logX, axis=1)), np.exp(logsumexp(logX, axis=0))


def transport_cost(C, eta, f, g):
    """<C, X> for X = exp(f_i + g_j - eta C_ij)."""
    C = np.asarray(C, np.float64)
    X = np.exp(-eta * C + np.asarray(f, np.float64)[:, None] + np.asarray(g, np.float64)[None, :])
    return float((C * X).sum())


def default_marginals(n: int, m: int):
    return np.ones(n), np.full(m, n / m)


def sinkhorn(C, eta: float, eps_rel: float = 1e-3, max_iter: int = 1000, r=None, c=None,
             check: bool = True):
    """Returns (f, g, cost, iterations, residue).  With ``check`` False the
    residue test is skipped and exactly ``max_iter`` iterations run."""
    C = np.asarray(C, np.float64)
    n, m = C.shape
    r0, c0 = default_marginals(n, m)
    r = r0 if r is None else np.asarray(r, np.float64)
    c = c0 if c is None else np.asarray(c, np.float64)
    logr, logc = np.log(r), np.log(c)
    K = -eta * C  # log of the Gibbs kernel exp(-eta C)
    f = np.zeros(n)
    g = np.zeros(m)
    threshold = eps_rel * r.sum()
    res = np.inf
    it = 0
    for it in range(1, max_iter + 1):
        f = logr - logsumexp(K + g[None, :], axis=1)  # every row sums to r_i
        g = logc - logsumexp(K + f[:, None], axis=0)  # every column sums to c_j
        if check:
            rows, cols = marginals(C, eta, f, g)
            res = np.abs(r - rows).sum() + np.abs(c - cols).sum()
            if res <= threshold:
                break
    if not check:
        rows, cols = marginals(C, eta, f, g)
        res = np.abs(r - rows).sum() + np.abs(c - cols).sum()
    return f, g, transport_cost(C, eta, f, g), it, float(res)
