"""Serving (continuous batching) at the request sizes of the served workload,
ticket cancellation, and the step cap that makes one instance's bounded
device loop run out.

The served workload draws n log-uniform on [16, 2048] with MNIST-like pixel
costs (many ties).  Every KM result must equal the CPU oracle's KM bit for bit
(assignment, cost, both duals); every batched-KM result must carry a valid
dual certificate and the oracle's optimal cost.
"""
import time

import numpy as np
import pytest
import torch

from paper_2005_01182_gb300 import otassign as ot
from paper_2005_01182_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _host_out(n, m):
    return (torch.empty(n, dtype=torch.int32), torch.empty(1, dtype=torch.int64),
            torch.empty(n, dtype=torch.int64), torch.empty(m, dtype=torch.int64))


def _poll_all(served, pending, outs, limit_s=600):
    t0 = time.time()
    while pending and time.time() - t0 < limit_s:
        rest = []
        for t, C in pending:
            o = _host_out(*C.shape)
            if ot.ot_assign_poll(served, t, o) == ot.OT_OK:
                outs[t] = o
            else:
                rest.append((t, C))
        pending[:] = rest
        if rest:
            time.sleep(0.0005)
    return not pending


def test_serving_full_size_range_against_oracle(oracle_mod, lib_path):
    """48 requests, n log-uniform on [16, 2048], submitted in four bursts so
    that later requests arrive while earlier waves still run; KM and batched
    KM alternate; every result is checked against the oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    reqs = W.served_requests(48, rate_per_s=1e9, lo=16, hi=2048, seed=2024)
    sizes = [C.shape[0] for _, C in reqs]
    assert max(sizes) >= 1024 and min(sizes) <= 64  # the draw spans the range
    served = ot.Context(hbm_budget_bytes=256 << 20, wave_streams=4)
    try:
        tickets = []
        outs = {}
        pending = []
        for burst in range(4):
            for i in range(burst * 12, burst * 12 + 12):
                C = reqs[i][1]
                algo = ot.OT_BKM if i % 2 else ot.OT_KM
                t = ot.ot_assign_submit(served, torch.from_numpy(C), algo)
                tickets.append((t, algo, C))
                pending.append((t, C))
            # collect whatever finished, leave the rest running
            deadline = time.time() + 0.02
            while time.time() < deadline:
                _poll_all(served, pending, outs, limit_s=0)
        assert _poll_all(served, pending, outs)
        cnt = ot.ot_serving_counters(served)
        assert cnt["completed"] == len(reqs)
        assert cnt["waves"] >= 1  # grid launches (requests of m <= 2048 join the resident grid)
        assert cnt["bytes_resident"] == 0
        for t, algo, C in tickets:
            r, c, u, v = (x.numpy() for x in outs[t])
            a0, c0, u0, v0 = oracle_mod.km(C)
            assert int(c[0]) == c0
            if algo == ot.OT_KM:
                np.testing.assert_array_equal(r, a0)
                np.testing.assert_array_equal(u, u0)
                np.testing.assert_array_equal(v, v0)
            else:
                assert oracle_mod.check_certificate(C, r, u, v, int(c[0])) == 0
    finally:
        served.close()


def test_cancel_waiting_running_and_unknown(lib_path):
    """Cancel a request that waits for admission (dropped at once), one that
    runs (discarded; its arena block comes back once the solver ends), and
    an unknown ticket (OT_ERR_TICKET); the queue keeps serving."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    big = W.pixel_sqdist(1500, seed=5)
    small = W.pixel_sqdist(300, seed=6)
    one = 4 * 1500 * 1500 + (1 << 16)
    # room for one large request: the second waits in the host queue
    served = ot.Context(hbm_budget_bytes=one + (1 << 20), wave_streams=2)
    try:
        t_run = ot.ot_assign_submit(served, torch.from_numpy(big), ot.OT_KM)
        t_wait = ot.ot_assign_submit(served, torch.from_numpy(big), ot.OT_KM)
        ot.ot_assign_cancel(served, t_wait)
        with pytest.raises(ot.OtError) as e:
            ot.ot_assign_poll(served, t_wait, _host_out(1500, 1500))
        assert e.value.code == ot.OT_ERR_TICKET
        with pytest.raises(ot.OtError) as e:
            ot.ot_assign_cancel(served, t_wait)
        assert e.value.code == ot.OT_ERR_TICKET
        ot.ot_assign_cancel(served, t_run)
        with pytest.raises(ot.OtError) as e:
            ot.ot_assign_poll(served, t_run, _host_out(1500, 1500))
        assert e.value.code == ot.OT_ERR_TICKET
        with pytest.raises(ot.OtError) as e:
            ot.ot_assign_cancel(served, 987654321)
        assert e.value.code == ot.OT_ERR_TICKET
        # the cancelled running request gives its block back once it ends
        t0 = time.time()
        while ot.ot_serving_counters(served)["bytes_resident"] != 0 and time.time() - t0 < 120:
            time.sleep(0.005)
        assert ot.ot_serving_counters(served)["bytes_resident"] == 0
        # and the queue still serves: a fresh large request fits and solves
        t_new = ot.ot_assign_submit(served, torch.from_numpy(big), ot.OT_KM)
        t_small = ot.ot_assign_submit(served, torch.from_numpy(small), ot.OT_KM)
        outs = {}
        assert _poll_all(served, [(t_new, big), (t_small, small)], outs, limit_s=300)
        ref = ot.Context()
        try:
            for t, C in ((t_new, big), (t_small, small)):
                r, c, u, v = ot.ot_assign_solve(ref, torch.from_numpy(C).cuda(), ot.OT_KM)
                torch.cuda.synchronize()
                assert int(outs[t][1][0]) == int(c.item())
                np.testing.assert_array_equal(outs[t][0].numpy(), r.cpu().numpy())
        finally:
            ref.close()
    finally:
        served.close()


def test_step_cap_times_out_one_instance(oracle_mod, lib_path):
    """A context whose step cap lies below what one instance of a batch needs:
    that instance reports OT_ERR_TIMEOUT, every other instance equals the
    oracle bit for bit, and the same context then solves a fresh batch."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mats = [W.embedding_costs(n, seed=100 + n) for n in (20, 40, 60, 90, 200, 61)]
    steps = [oracle_mod.km(C, stats=True)[4]["steps"] for C in mats]
    hard = int(np.argmax(steps))
    cap = max(s for t, s in enumerate(steps) if t != hard)
    assert steps[hard] > cap
    ctx = ot.Context(step_limit=cap)
    try:
        dev = [torch.from_numpy(C).cuda() for C in mats]
        b = ot.ot_assign_solve_batched(ctx, dev, ot.OT_KM)
        torch.cuda.synchronize()
        status = b.status.cpu().numpy()
        assert status[hard] == ot.OT_ERR_TIMEOUT
        for t, C in enumerate(mats):
            if t == hard:
                continue
            assert status[t] == ot.OT_OK
            a0, c0, u0, v0 = oracle_mod.km(C)
            assert int(b.cost[t]) == c0
            np.testing.assert_array_equal(b.outs[t][0].cpu().numpy(), a0)
            np.testing.assert_array_equal(b.outs[t][1].cpu().numpy(), u0)
            np.testing.assert_array_equal(b.outs[t][2].cpu().numpy(), v0)
        # the context stays usable: a fresh batch within the cap
        fresh = [W.embedding_costs(n, seed=300 + n) for n in (16, 30, 45)]
        fresh = [C for C in fresh if oracle_mod.km(C, stats=True)[4]["steps"] <= cap]
        assert fresh
        b2 = ot.ot_assign_solve_batched(ctx, [torch.from_numpy(C).cuda() for C in fresh], ot.OT_KM)
        torch.cuda.synchronize()
        assert (b2.status.cpu().numpy() == 0).all()
        for t, C in enumerate(fresh):
            assert int(b2.cost[t]) == oracle_mod.km(C)[1]
        # a single solve that runs out reports the code through the API
        with pytest.raises(ot.OtError) as e:
            ot.ot_assign_solve_stats(ctx, dev[hard], ot.OT_KM)
        assert e.value.code == ot.OT_ERR_TIMEOUT
    finally:
        ctx.close()


def test_serving_grid_relaunch_and_wide_requests(lib_path):
    """Requests of m <= 2048 run on the resident serving grid, which leaves
    after a spell without work and is launched again for later requests;
    a request wider than 2048 columns takes a wave beside it.  Every result
    equals the solo solve."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    first = [W.pixel_sqdist(n, seed=n) for n in (20, 130, 700)]
    later = [W.pixel_sqdist(n, seed=n) for n in (45, 999)] + [W.pixel_sqdist(2100, 2150, seed=7)]
    served = ot.Context(hbm_budget_bytes=512 << 20)
    try:
        outs = {}
        pend = [(ot.ot_assign_submit(served, torch.from_numpy(C), ot.OT_KM), C) for C in first]
        assert _poll_all(served, list(pend), outs, limit_s=120)
        launches = ot.ot_serving_counters(served)["waves"]
        time.sleep(1.0)  # long past the grid's idle limit: it has left
        pend2 = [(ot.ot_assign_submit(served, torch.from_numpy(C), ot.OT_KM), C) for C in later]
        assert _poll_all(served, list(pend2), outs, limit_s=300)
        cnt = ot.ot_serving_counters(served)
        assert cnt["waves"] >= launches + 2  # the grid again, and a wave for the wide request
        assert cnt["completed"] == len(first) + len(later)
        ref = ot.Context()
        try:
            for t, C in pend + pend2:
                r, c, u, v = ot.ot_assign_solve(ref, torch.from_numpy(C).cuda(), ot.OT_KM)
                torch.cuda.synchronize()
                assert int(outs[t][1][0]) == int(c.item())
                np.testing.assert_array_equal(outs[t][0].numpy(), r.cpu().numpy())
                np.testing.assert_array_equal(outs[t][2].numpy(), u.cpu().numpy())
        finally:
            ref.close()
    finally:
        served.close()


def test_serving_result_paths_and_destinations(lib_path):
    """Requests on the resident grid write their results into mapped host
    slots (1024 of them); once every slot is held by an uncollected request
    the next ones write into their device blocks instead.  1100 small
    requests are submitted before any is polled, so both paths run; they are
    polled into device, pinned and pageable tensors in turn, beside a request
    wider than 2048 columns (a wave).  Every result equals the batched solo
    solve bit for bit."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(77)
    mats = [W.pixel_sqdist(int(n), seed=int(s)) for n, s in zip(rng.integers(16, 41, size=1100), range(1100))]
    mats.append(W.pixel_sqdist(2060, 2100, seed=5))
    served = ot.Context(hbm_budget_bytes=1 << 30)
    ref = ot.Context()
    try:
        tickets = [ot.ot_assign_submit(served, torch.from_numpy(C), ot.OT_KM) for C in mats]
        b = ot.ot_assign_solve_batched(ref, [torch.from_numpy(C).cuda() for C in mats], ot.OT_KM)
        torch.cuda.synchronize()
        assert (b.status.cpu().numpy() == 0).all()
        kinds = ("cuda", "pinned", "pageable")
        pending = list(range(len(mats)))
        got = {}
        t0 = time.time()
        while pending and time.time() - t0 < 300:
            rest = []
            for q in pending:
                n, m = mats[q].shape
                kind = kinds[q % 3]
                o = [torch.empty(n, dtype=torch.int32), torch.empty(1, dtype=torch.int64),
                     torch.empty(n, dtype=torch.int64), torch.empty(m, dtype=torch.int64)]
                if kind == "cuda":
                    o = [x.cuda() for x in o]
                elif kind == "pinned":
                    o = [x.pin_memory() for x in o]
                if ot.ot_assign_poll(served, tickets[q], tuple(o)) == ot.OT_OK:
                    got[q] = o
                else:
                    rest.append(q)
            pending = rest
            if pending:
                time.sleep(0.001)
        assert not pending
        torch.cuda.synchronize()
        for q in range(len(mats)):
            r, c, u, v = (x.cpu().numpy() for x in got[q])
            assert int(c[0]) == int(b.cost[q])
            np.testing.assert_array_equal(r, b.outs[q][0].cpu().numpy())
            np.testing.assert_array_equal(u, b.outs[q][1].cpu().numpy())
            np.testing.assert_array_equal(v, b.outs[q][2].cpu().numpy())
        assert ot.ot_serving_counters(served)["completed"] == len(mats)
    finally:
        served.close()
        ref.close()


def test_completion_query_returns_each_request_once(oracle_mod, lib_path):
    """ot_assign_completed returns every finished request exactly once (three
    at most per call here), never a cancelled one, then nothing; results
    collected through it equal the oracle's KM (small requests) or the solo
    solve (the rest, a wave-sized one included) bit for bit."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sizes = (16, 33, 70, 150, 300, 700, 1200, 2100)
    mats = [W.pixel_sqdist(n, seed=400 + n) for n in sizes]
    served = ot.Context(hbm_budget_bytes=512 << 20)
    ref = ot.Context()
    try:
        tickets = [ot.ot_assign_submit(served, torch.from_numpy(C), ot.OT_KM) for C in mats]
        gone = ot.ot_assign_submit(served, torch.from_numpy(W.pixel_sqdist(500, seed=1)), ot.OT_KM)
        ot.ot_assign_cancel(served, gone)
        seen, outs = [], {}
        t0 = time.time()
        while len(seen) < len(mats) and time.time() - t0 < 300:
            got = ot.ot_assign_completed(served, 3)
            assert len(got) <= 3
            for tk in got:
                q = tickets.index(tk)
                n, m = mats[q].shape
                o = _host_out(n, m)
                assert ot.ot_assign_poll(served, tk, o) == ot.OT_OK
                seen.append(tk)
                outs[q] = o
            if not got:
                time.sleep(0.001)
        assert sorted(seen) == sorted(tickets) and len(set(seen)) == len(seen)
        assert gone not in seen
        assert ot.ot_assign_completed(served) == []
        for q, C in enumerate(mats):
            r, c, u, v = (x.numpy() for x in outs[q])
            if C.shape[0] <= 300:
                a0, c0, u0, v0 = oracle_mod.km(C)
            else:
                a0, c0, u0, v0 = (x.cpu().numpy() if hasattr(x, "cpu") else x
                                  for x in ot.ot_assign_solve(ref, torch.from_numpy(C).cuda(), ot.OT_KM))
                c0 = int(np.asarray(c0).reshape(-1)[0])
            assert int(c[0]) == c0
            np.testing.assert_array_equal(r, a0)
            np.testing.assert_array_equal(u, u0)
            np.testing.assert_array_equal(v, v0)
    finally:
        served.close()
        ref.close()


def test_native_client_replay_matches_solo(lib_path):
    """The native serving client (lib/libotclient.so) replays a stream through
    submit / completed / poll: at once with a window of 8 outstanding
    requests, then on Poisson arrival times; every collected cost equals the
    matrix's solo solve and every request completes after it arrives."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes
    from paper_2005_01182_gb300 import build
    client = ctypes.CDLL(build.CLIENT_LIB)
    client.otc_replay.restype = ctypes.c_int
    client.otc_replay.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                  ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    reqs = W.served_requests(12, rate_per_s=1.0, lo=16, hi=600, seed=31)
    mats = [torch.from_numpy(C).pin_memory() for _, C in reqs]
    nreq = len(mats)
    ref = ot.Context()
    try:
        b = ot.ot_assign_solve_batched(ref, [m.cuda() for m in mats], ot.OT_KM)
        torch.cuda.synchronize()
        solo = b.cost.cpu().numpy()
    finally:
        ref.close()
    cptr = (ctypes.c_void_p * nreq)(*[m.data_ptr() for m in mats])
    n_arr = np.array([m.shape[0] for m in mats], dtype=np.int32)
    m_arr = np.array([m.shape[1] for m in mats], dtype=np.int32)
    nstream = 40
    for arrivals, window in ((np.zeros(nstream), 8), (np.cumsum(np.full(nstream, 2e-4)), nstream)):
        arrivals = np.ascontiguousarray(arrivals, dtype=np.float64)
        served = ot.Context(hbm_budget_bytes=256 << 20)
        try:
            done = np.zeros(nstream, dtype=np.float64)
            cost = np.zeros(nstream, dtype=np.int64)
            total = ctypes.c_double()
            rc = client.otc_replay(served.h, nreq, cptr, n_arr.ctypes.data, m_arr.ctypes.data, nstream,
                                   arrivals.ctypes.data, window, ot.OT_KM, done.ctypes.data, cost.ctypes.data,
                                   ctypes.byref(total))
            assert rc == 0
            np.testing.assert_array_equal(cost, solo[np.arange(nstream) % nreq])
            assert (done >= arrivals).all() and total.value >= done.max()
            assert ot.ot_serving_counters(served)["completed"] == nstream
        finally:
            served.close()
