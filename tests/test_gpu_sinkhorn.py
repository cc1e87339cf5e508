"""GPU log-domain Sinkhorn (ot_sinkhorn_solve) against the float64 oracle.

Tolerance, derived from the arithmetic: one log-sum-exp on the GPU rounds
the exponent argument (int -> float conversion and one FMA: <= 2u|x|), the
exponential (__expf on arguments <= 0: a few ulp, counted as 2u|x| + 4u),
the float32 sums (a lane adds up to m/32 terms, then 5 shuffle levels:
(m/32 + 5) u) and the log (u |L|), with u = 2^-24 and |x| <= A = eta max|C|
+ max|f|, |g|.  So one dual update errs by at most
delta = u (4A + m/32 + 16).  The log-sum-exp is 1-Lipschitz in the maximum
norm, so errors add along the iterations: after K iterations (2K dual
updates) |f - f_oracle|, |g - g_oracle| <= 2 K delta, and <C, X> is off by a
relative 4 K delta at most (X_ij = exp(f_i + g_j - eta C_ij))."""
import numpy as np
import pytest
import torch

from paper_2005_01182_gb300 import otassign as ot
from paper_2005_01182_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


def dual_tol(C, eta, f, g, K):
    A = eta * float(np.abs(C).max()) + max(float(np.abs(f).max()), float(np.abs(g).max()))
    delta = U * (4 * A + max(C.shape) / 32 + 16)
    return 2 * K * delta


@pytest.fixture(scope="module")
def sk():
    import oracle.sinkhorn as mod
    return mod


def gpu(ctx, C, eta, **kw):
    Cd = torch.from_numpy(np.ascontiguousarray(C)).cuda()
    f, g, (cost, res, it) = ot.ot_sinkhorn_solve(ctx, Cd, eta, **kw)
    return f.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64), cost, res, it


CASES = [
    ("uniform", lambda: W.uniform_costs(300, hi=1000, seed=1), 0.02),
    ("rect", lambda: W.uniform_costs(200, 333, hi=500, seed=2), 0.05),
    ("pixel_ties", lambda: W.pixel_sqdist(256, seed=3), 0.05),
    ("embed", lambda: W.embedding_costs(128, seed=4), 0.002),
    ("wide_tiles", lambda: W.uniform_costs(97, 2500, hi=100, seed=5), 0.2),
    ("odd_m", lambda: W.uniform_costs(130, 131, hi=300, seed=6), 0.05),
    ("negative", lambda: np.random.default_rng(7).integers(-500, 500, size=(64, 80)).astype(np.int32), 0.01),
]


@pytest.mark.parametrize("name,make,eta", CASES, ids=[c[0] for c in CASES])
def test_fixed_iterations_match_oracle(sk, ctx, name, make, eta):
    C = make()
    K = 10
    f0, g0, c0, it0, _ = sk.sinkhorn(C, eta, max_iter=K, check=False)
    f, g, cost, res, it = gpu(ctx, C, eta, eps_rel=0.0, max_iter=K)
    assert it == K == it0
    tol = dual_tol(C, eta, f0, g0, K)
    assert np.abs(f - f0).max() <= tol
    assert np.abs(g - g0).max() <= tol
    assert abs(cost - c0) <= 2 * tol * abs(c0) + 1e-9


def test_strided_rows_scalar_path(sk, ctx):
    """ldc > m and not a multiple of 4: the unvectorised loads."""
    base = W.uniform_costs(90, 123, hi=400, seed=8)
    big = np.zeros((90, 127), np.int32)
    big[:, :123] = base
    Cd = torch.from_numpy(big).cuda()[:, :123]
    f, g, (cost, res, it) = ot.ot_sinkhorn_solve(ctx, Cd, 0.03, eps_rel=0.0, max_iter=6)
    f0, g0, c0, _, _ = sk.sinkhorn(base, 0.03, max_iter=6, check=False)
    tol = dual_tol(base, 0.03, f0, g0, 6)
    assert np.abs(f.cpu().numpy() - f0).max() <= tol
    assert np.abs(g.cpu().numpy() - g0).max() <= tol


def test_marginals_given(sk, ctx):
    rng = np.random.default_rng(9)
    C = W.uniform_costs(150, 170, hi=300, seed=9)
    r = rng.uniform(0.5, 2.0, 150)
    c = rng.uniform(0.5, 2.0, 170)
    c *= r.sum() / c.sum()
    f0, g0, c0, _, _ = sk.sinkhorn(C, 0.05, max_iter=8, check=False, r=r, c=c)
    f, g, cost, res, it = gpu(ctx, C, 0.05, eps_rel=0.0, max_iter=8, r=r, c=c)
    tol = dual_tol(C, 0.05, f0, g0, 8)
    assert np.abs(f - f0).max() <= tol and np.abs(g - g0).max() <= tol


def test_convergence(sk, ctx):
    """The stopping iteration is a float decision: the GPU's may differ from
    the oracle's by one; the iterate it returns must meet the threshold
    (checked in float64 from its own f, g, with a 10% float32 margin)."""
    for C, eta in [(W.uniform_costs(200, hi=1000, seed=10), 0.1), (W.pixel_sqdist(300, seed=11), 0.05)]:
        n, m = C.shape
        f0, g0, c0, it0, res0 = sk.sinkhorn(C, eta, eps_rel=1e-3, max_iter=2000)
        f, g, cost, res, it = gpu(ctx, C, eta, eps_rel=1e-3, max_iter=2000)
        assert abs(it - it0) <= 1
        r, cc = sk.default_marginals(n, m)
        rows, cols = sk.marginals(C, eta, f, g)
        assert np.abs(r - rows).sum() <= 1.1e-3 * n
        assert abs(cost - sk.transport_cost(C, eta, f, g)) <= 1e-4 * abs(cost)
        assert abs(res - np.abs(r - rows).sum()) <= 1e-4 * n


def test_sinkhorn_approaches_assignment_optimum(oracle_mod, ctx):
    """Larger eta: the entropic cost is within n log(m)/eta + residue * max C
    of the assignment optimum (Sec. 4.1 picks eta for a 1.1-approximation)."""
    C = W.embedding_costs(96, seed=12)
    opt = oracle_mod.km(C)[1]
    eta = 0.01
    f, g, cost, res, it = gpu(ctx, C, eta, eps_rel=1e-3, max_iter=5000)
    assert opt - res * C.max() - 1e-6 * opt <= cost <= opt + 96 * np.log(96) / eta + res * C.max()


def test_max_iter_one_and_tiny(sk, ctx):
    C = np.array([[3]], np.int32)
    f, g, cost, res, it = gpu(ctx, C, 0.5, eps_rel=1e-3, max_iter=1)
    assert it == 1 and abs(cost - 3.0) < 1e-5
    C = W.uniform_costs(5, 9, hi=10, seed=13)
    f0, g0, c0, it0, _ = sk.sinkhorn(C, 0.3, max_iter=1, check=False)
    f, g, cost, res, it = gpu(ctx, C, 0.3, eps_rel=0.0, max_iter=1)
    assert it == 1 and np.abs(f - f0).max() <= dual_tol(C, 0.3, f0, g0, 1)


def test_bad_arguments(ctx):
    C = torch.zeros((4, 4), dtype=torch.int32, device="cuda")
    for kw in [dict(eta=0.0), dict(eta=-1.0), dict(eta=1.0, max_iter=0),
               dict(eta=1.0, r=[1, 1, 1, 1], c=[1, 1, 1, 2]), dict(eta=1.0, r=[1, 0, 1, 1], c=[1, 1, 1, 0])]:
        with pytest.raises(ot.OtError):
            ot.ot_sinkhorn_solve(ctx, C, **kw)
    with pytest.raises(ot.OtError):
        ot.ot_sinkhorn_solve(ctx, C.cpu(), 1.0)


def test_large_fixed_iterations(sk, ctx):
    """n = m = 4096 (a 64 MiB cost matrix), 3 iterations."""
    C = W.shapes_sqdist(4096)
    eta = 2e-3
    f0, g0, c0, _, _ = sk.sinkhorn(C, eta, max_iter=3, check=False)
    f, g, cost, res, it = gpu(ctx, C, eta, eps_rel=0.0, max_iter=3)
    tol = dual_tol(C, eta, f0, g0, 3)
    assert np.abs(f - f0).max() <= tol and np.abs(g - g0).max() <= tol
    assert abs(cost - c0) <= 2 * tol * c0


def test_host_outputs_and_default_stream(sk, ctx):
    """f and g may be host arrays (raw C-ABI call); the NULL stream is the
    caller's default stream."""
    import ctypes
    C = W.uniform_costs(64, 80, hi=200, seed=14)
    Cd = torch.from_numpy(C).cuda()
    f = np.zeros(64, np.float32)
    g = np.zeros(80, np.float32)
    cost, res, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    P = lambda a: ctypes.c_void_p(a.ctypes.data)
    rc = ctx.lib.ot_sinkhorn_solve(ctx.h, ctypes.c_void_p(Cd.data_ptr()), 80, 64, 80, None, None, 0.05, 0.0, 7,
                                   P(f), P(g), ctypes.byref(cost), ctypes.byref(res), ctypes.byref(it), None)
    assert rc == 0 and it.value == 7
    f0, g0, c0, _, _ = sk.sinkhorn(C, 0.05, max_iter=7, check=False)
    tol = dual_tol(C, 0.05, f0, g0, 7)
    assert np.abs(f - f0).max() <= tol and np.abs(g - g0).max() <= tol
    assert abs(cost.value - c0) <= 2 * tol * c0


def test_batched_fixed_iterations(sk, ctx):
    """ot_sinkhorn_solve_batched: each instance equals the float64 oracle
    within the same bound, sizes 1 x 1 to 300 x 333 in one call."""
    rng = np.random.default_rng(15)
    shapes = [(1, 1), (1, 5), (7, 7), (33, 40), (100, 100), (128, 200), (256, 256), (300, 333)]
    mats = [W.uniform_costs(n, m, hi=400, seed=int(rng.integers(1 << 20))) for n, m in shapes]
    eta, K = 0.03, 6
    b = ot.ot_sinkhorn_solve_batched(ctx, [torch.from_numpy(C).cuda() for C in mats], eta, eps_rel=0.0, max_iter=K)
    torch.cuda.synchronize()
    its = b.iterations.cpu().numpy()
    costs = b.cost.cpu().numpy()
    for t, C in enumerate(mats):
        f0, g0, c0, _, _ = sk.sinkhorn(C, eta, max_iter=K, check=False)
        tol = dual_tol(C, eta, f0, g0, K)
        assert its[t] == K
        assert np.abs(b.f[t].cpu().numpy() - f0).max() <= tol
        assert np.abs(b.g[t].cpu().numpy() - g0).max() <= tol
        assert abs(costs[t] - c0) <= 2 * tol * abs(c0) + 1e-9


def test_batched_convergence(sk, ctx):
    mats = [W.uniform_costs(n, hi=1000, seed=n) for n in (40, 90, 200)] + [W.pixel_sqdist(150, seed=3)]
    eta = 0.05
    b = ot.ot_sinkhorn_solve_batched(ctx, [torch.from_numpy(C).cuda() for C in mats], eta, eps_rel=1e-3, max_iter=3000)
    torch.cuda.synchronize()
    for t, C in enumerate(mats):
        n, m = C.shape
        f0, g0, c0, it0, _ = sk.sinkhorn(C, eta, eps_rel=1e-3, max_iter=3000)
        it = int(b.iterations[t])
        assert abs(it - it0) <= 1
        f = b.f[t].cpu().numpy().astype(np.float64)
        g = b.g[t].cpu().numpy().astype(np.float64)
        r, _ = sk.default_marginals(n, m)
        rows, _ = sk.marginals(C, eta, f, g)
        assert np.abs(r - rows).sum() <= 1.1e-3 * n
        assert abs(float(b.cost[t]) - sk.transport_cost(C, eta, f, g)) <= 1e-4 * abs(float(b.cost[t]))


def test_batched_limits(ctx):
    big = torch.zeros((4097, 4097), dtype=torch.int32, device="cuda")
    with pytest.raises(ot.OtError) as e:
        ot.ot_sinkhorn_solve_batched(ctx, [big], 1.0)
    assert e.value.code == ot.OT_ERR_UNSUPPORTED
    with pytest.raises(ot.OtError):
        ot.ot_sinkhorn_solve_batched(ctx, [big[:4, :4].contiguous()], 0.0)
