"""Benchmark: exact assignment solves/s on GB300 through libotassign's C-ABI.

Default workload (one "step" = one pass of the whole hot path over one
batch): 4096 independent instances, n = m ~ U{32..256}, costs =
round(1e4 * Euclidean distance) between unit-normalised 300-d Gaussian
vectors (token-embedding-like), solved in one ot_assign_solve_batched call.
`value` = instances solved per second with the cost matrices resident in
HBM; `e2e` = the same metric through the C-ABI with pinned host buffers
(host->device copy of every matrix and device->host copy of every result
inside the timed region).  Side measurements in the same line: the plain
one-instance-per-launch GPU KM on the same instances, the epsilon-scaling
auction on the same batch, the served (continuous batching) p50/p99
latency, the n = 4096 and n = 16384 single solves, and log-domain Sinkhorn
(per-iteration bandwidth at n = 16384; the paper's 1.1-approximation
protocol at n = 4096 and on the 4096-instance batch).

Under torchrun each rank solves its own 4096 instances (weak scaling, no
collective on the data path); rank 0 prints the JSON line.
`--impl reference` times the CPU oracle on bounded samples of the same
workload instead (host cores, single-threaded per solve).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2005_01182_gb300 import workloads as W  # noqa: E402

METRIC = "assignment solves/s (4096-instance batch, n~U{32..256}, exact)"
UNIT = "solves/s"


KERNEL_SOURCES = ["ot_group.cuh", "ot_group_km.cu", "ot_group_bkm.cu", "ot_group_launch.inc", "ot_shapes.h",
                  "ot_internal.h", "ot_pack.cu"]


def code_text(src: str) -> str:
    """C/CUDA source with comments removed and whitespace collapsed: what the
    compiler sees (comment edits do not count as kernel changes)."""
    import re
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def kernel_source_hash(read=None) -> str:
    """sha256 over the code (comments stripped) of the sources that define
    the group-engine kernels; `read(name)` returns a source's text."""
    import hashlib
    if read is None:
        def read(f):
            return open(os.path.join(ROOT, "paper_2005_01182_gb300", "csrc", f)).read()
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(code_text(read(f)).encode())
    return h.hexdigest()


def measured_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` ("<name> instances <count>": the
    launch and the instance set it ran) from the committed ncu summary, if
    it was taken on the kernel sources as they are now (else None).  Lines:
    `traffic <name> instances <count> <bytes per launch> source <sha256>`."""
    p = os.path.join(ROOT, "profiles", "batch4096_embed_traffic.md")
    if not os.path.exists(p):
        return None
    digest = kernel_source_hash()
    for line in open(p):
        tok = line.strip().strip("`").split()
        if len(tok) >= 5 and tok[0] == "traffic" and tok[-2] == "source":
            name = " ".join(tok[1:-3])
            if name == kernel and tok[-1] == digest:
                return int(tok[-3])
    return None


def measured_instructions(kernel: str):
    """Warp instructions per launch of `kernel` ("<name> instances <count>")
    (ncu smsp__inst_executed.sum) from the committed summary, if taken on the
    kernel sources as they are now (else None).  Lines: `issue <name>
    instances <count> <instructions per launch> source <sha256>`."""
    p = os.path.join(ROOT, "profiles", "batch4096_embed_traffic.md")
    if not os.path.exists(p):
        return None
    digest = kernel_source_hash()
    for line in open(p):
        tok = line.strip().strip("`").split()
        if len(tok) >= 5 and tok[0] == "issue" and tok[-2] == "source":
            name = " ".join(tok[1:-3])
            if name == kernel and tok[-1] == digest:
                return int(tok[-3])
    return None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """Sample SM clocks and throttle reasons with nvidia-smi during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def rank_seed(rank: int) -> int:
    """Base seed of rank r's batch: every rank solves its own instances."""
    return W.BASE_SEED + 1_000_003 * rank


def batch_for_rank(rank: int, k: int):
    return W.batch_embeddings(k, seed=rank_seed(rank))


def job_throughput(local_ms: float, k: int, steps: int, world: int, dist=None, device=None) -> tuple[float, float]:
    """Whole-job solves/s: every rank solved k instances per step; the job
    took as long as the slowest rank (max over ranks of the timed region)."""
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return world * k * steps / (ms / 1000.0), ms


def cpu_oracle_rate(Cs, budget_s: float):
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    done = 0
    while time.perf_counter() - t0 < budget_s and done < len(Cs):
        oracle.km(Cs[done])
        done += 1
    dt = time.perf_counter() - t0
    return done / dt, done, dt


def cpu_oracle_rate_threads(Cs, budget_s: float, threads: int):
    """The oracle as it stands, one instance per call, on `threads` host
    threads at once (ctypes releases the GIL inside each call)."""
    import oracle
    oracle.build()
    oracle.km(Cs[0])  # load the library before the threads start
    nxt = [0]
    done = [0]
    lock = threading.Lock()
    t0 = time.perf_counter()

    def work():
        while time.perf_counter() - t0 < budget_s:
            with lock:
                t = nxt[0]
                if t >= len(Cs):
                    return
                nxt[0] = t + 1
            oracle.km(Cs[t])
            with lock:
                done[0] += 1

    ts = [threading.Thread(target=work) for _ in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    dt = time.perf_counter() - t0
    return done[0] / dt, done[0], dt


def host_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    Cs = batch_for_rank(0, 4096)
    rates = []
    cores = host_threads()
    per_step = max(8, min(4096, args.sample * cores))
    for s in range(args.warmup + args.steps):
        sample = [Cs[(s * per_step + t) % len(Cs)] for t in range(per_step)]
        r, done, dt = cpu_oracle_rate_threads(sample, 1e9, cores)
        if s >= args.warmup:
            rates.append((done, dt))
    n = sum(d for d, _ in rates)
    t = sum(dt for _, dt in rates)
    v = n / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": "batch4096_embed300_n32-256", "sample_per_step": per_step},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} instances per step of the 4096-instance batch, oracle KM, "
                                       f"one instance per thread on {cores} host threads"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure_single_4096(stream, ot, torch):
    """Single solves: n = m = 4096 (circle/square shapes and uniform costs)
    and n = m = 256 (integer points on a 64 x 64 grid): KM on one CTA vs
    batched KM (routed to the cluster engine above 1024 columns) vs the
    epsilon-scaling auction on one CTA, s/solve; on circle/square also the
    single-scaling-factor variant (s = 16) and the oracle's KM and scaled
    batched KM beside them."""
    out = {}
    ctx = ot.Context()
    for kind in ("circle-square", "uniform", "grid256"):
        Cd = torch.from_numpy(W.single_256() if kind == "grid256" else W.single_4096(kind)).cuda()
        torch.cuda.synchronize()
        res = {}
        for name, algo in (("km", ot.OT_KM), ("batched_km", ot.OT_BKM), ("auction", ot.OT_AUCTION)):
            best = None
            for _ in range(2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r, c, u, v, st = ot.ot_assign_solve_stats(ctx, Cd, algo, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1) / 1000.0
                best = t if best is None else min(best, t)
            res[name] = {"s_per_solve": best, "cost": int(c.item()), "steps": st["steps"]}
        if kind == "circle-square":
            # the single-scaling-factor variant (s = 16) and the oracle beside both
            import oracle
            C = Cd.cpu().numpy()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r, c, bound = ot.ot_assign_solve_scaled(ctx, Cd, 16, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            res["scaled_batched_km_s16"] = {"s_per_solve": e0.elapsed_time(e1) / 1000.0, "cost": int(c.item()),
                                            "bound": bound}
            t0 = time.perf_counter()
            _, c_km, _, _ = oracle.km(C)
            t_km = time.perf_counter() - t0
            t0 = time.perf_counter()
            oracle.bkm(np.floor_divide(C, 16).astype(np.int32))
            t_sc = time.perf_counter() - t0
            res["cpu_oracle"] = {"km_s_per_solve": t_km, "cost": c_km, "scaled_batched_km_s16_s_per_solve": t_sc,
                                 "cores": 1, "kind": "oracle", "sample": "one solve each, single thread"}
        out[kind] = res
    ctx.close()
    return out


def measure_single_16384(ctx, stream, ot, torch):
    """n = m = 16384 (1024 x 1024 grid, squared distances, 1 GiB int32):
    batched KM solve time and effective cost-matrix bandwidth."""
    C = W.single_16384()
    Cd = torch.from_numpy(C).cuda()
    C_shape = C.shape
    del C
    torch.cuda.synchronize()
    peak, kind = _peaks()
    best = None
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r, c, u, v, st = ot.ot_assign_solve_stats(ctx, Cd, ot.OT_BKM, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1000.0
        if best is None or t < best[0]:
            best = (t, st, int(c.item()))
    t, st, cost = best
    alg = st["cost_bytes"] + st["init_bytes"]
    # the same solve on the dense cluster engine (every row of a tree scanned
    # in full): the comparison point of the sparse-list engine above
    dctx = ot.Context(flags=ot.OT_CFG_DENSE_WIDE)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r, c, u, v, dst = ot.ot_assign_solve_stats(dctx, Cd, ot.OT_BKM, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    dctx.close()
    dt = e0.elapsed_time(e1) / 1000.0
    dalg = dst["cost_bytes"] + dst["init_bytes"]
    assert int(c.item()) == cost, "dense and sparse engines disagree"
    dense = {"s_per_solve": dt, "algorithmic_bytes": dalg, "achieved_gbs": dalg / dt / 1e9,
             "hbm_frac": dalg / dt / 1e9 / peak, "steps": dst["steps"], "phases": dst["phases"],
             "note": "cluster engine: the rows of every tree scanned in full at each level"}
    # the paper's approximate variant: one scaling factor s (s = 16 keeps the
    # a-priori bound n*(s-1) within 10 % of the optimum here)
    scaled = {}
    for sc in (16, 64):
        ot.ot_assign_solve_scaled(ctx, Cd, sc, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r2, c2, bnd = ot.ot_assign_solve_scaled(ctx, Cd, sc, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        scaled[str(sc)] = {"s_per_solve": e0.elapsed_time(e1) / 1000.0, "cost": int(c2.item()),
                           "ratio_to_opt": int(c2.item()) / cost, "bound": bnd, "bound_ratio": 1 + bnd / cost}
    # log-domain Sinkhorn on the same matrix: the cost of one iteration (a row
    # pass and a column pass, each reading the 1 GiB matrix once), from the
    # difference of a 12- and a 2-iteration run
    sk_t = {}
    for K in (2, 12):
        ot.ot_sinkhorn_solve(ctx, Cd, 2.0, eps_rel=0.0, max_iter=K, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ot.ot_sinkhorn_solve(ctx, Cd, 2.0, eps_rel=0.0, max_iter=K, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        sk_t[K] = e0.elapsed_time(e1) / 1000.0
    per_it = (sk_t[12] - sk_t[2]) / 10
    sk_bytes = 2 * 4 * C_shape[0] * C_shape[1]
    sinkhorn = {"s_per_iteration": per_it, "bytes_per_iteration": sk_bytes,
                "achieved_gbs": sk_bytes / per_it / 1e9, "hbm_frac": sk_bytes / per_it / 1e9 / peak,
                "hbm_frac_vs_8tbs": sk_bytes / per_it / 1e9 / 8000.0, "eta": 2.0,
                "note": "log-domain Sinkhorn, fixed iterations; (t(12) - t(2)) / 10"}
    del Cd
    torch.cuda.empty_cache()
    return {"algo": "batched KM, sparse-list engine", "s_per_solve": t, "solves_per_s": 1.0 / t, "cost": cost,
            "sinkhorn": sinkhorn, "algorithmic_bytes": alg, "achieved_gbs": alg / t / 1e9,
            "hbm_frac": alg / t / 1e9 / peak, "peak_gbs": peak, "peak_kind": kind,
            "hbm_frac_vs_8tbs": alg / t / 1e9 / 8000.0,
            "dense_equivalent_gbs": dalg / t / 1e9,
            "note": "algorithmic bytes: dense cost rows read (row reduction, list rebuilds) plus 8 per list "
                    "entry relaxed; dense_equivalent_gbs divides the dense engine's reduced-cost bytes by "
                    "this solve time; the solve is bound by the latency of its dependent levels",
            "steps": st["steps"], "phases": st["phases"], "rows_scanned": st["rows_scanned"],
            "dense_engine": dense, "scaled_batched_km": scaled}


def measure_sinkhorn_4096(stream, ot, torch):
    """Log-domain Sinkhorn on the n = 4096 circle/square instance with the
    paper's stopping rule (Sec. 4.1: residue at most 10^-3 of the summed
    demand, no rounding) at one fixed eta = 0.3 (the smallest eta whose cost
    stays within 1.1 x the optimum here; choosing eta is not part of the
    solver): time to convergence, iterations and cost over the exact
    optimum (batched KM)."""
    ctx = ot.Context()
    Cd = torch.from_numpy(W.single_4096("circle-square")).cuda()
    _, c, _, _ = ot.ot_assign_solve(ctx, Cd, ot.OT_BKM, stream)
    torch.cuda.synchronize()
    opt = int(c.item())
    eta = 0.3
    ot.ot_sinkhorn_solve(ctx, Cd, eta, eps_rel=1e-3, max_iter=20000, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    f, g, (cost, res, it) = ot.ot_sinkhorn_solve(ctx, Cd, eta, eps_rel=1e-3, max_iter=20000, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1000.0
    ctx.close()
    # the float64 oracle's cost per iteration at this size (2 iterations)
    import oracle.sinkhorn as sko
    C = Cd.cpu().numpy()
    t0 = time.perf_counter()
    sko.sinkhorn(C, eta, max_iter=2, check=False)
    oracle_it = (time.perf_counter() - t0) / 2
    del Cd
    torch.cuda.empty_cache()
    return {"opt": opt, "epsilon_rel": 1e-3, "eta": eta, "iterations": it, "s": secs,
            "cost_over_opt": cost / opt, "residue_over_total": res / 4096,
            "gpu_s_per_iteration": secs / max(1, it),
            "cpu_oracle": {"s_per_iteration": oracle_it, "cores": 1, "kind": "oracle",
                           "sample": "2 iterations of the numpy float64 oracle at n = 4096"}}


def measure_transport(stream, ot, torch):
    """Integer-supply transport (Eq. 1 with integer r, c) by vertex
    replication: two MNIST-like images (116 and 169 nonzero pixels of a
    28 x 28 grid, the sizes of Table 1's mnist0) with intensities scaled to
    a total of 2048 units (the paper's totals of ~10^6 are beyond
    replication), i.e. a 2048 x 2048 replicated assignment problem.  GPU
    s/solve per algorithm (matrix resident, flow and cost returned) beside
    the oracle (replication + KM, one host thread)."""
    ctx = ot.Context()
    C, r, c = W.mnist_transport(116, 169, 2048)
    Cd = torch.from_numpy(C).cuda()
    res = {}
    for name, algo in (("km", ot.OT_KM), ("batched_km", ot.OT_BKM), ("auto", ot.OT_AUTO)):
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            flow, cost = ot.ot_transport_solve(ctx, Cd, r, c, algo, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1000.0
            best = t if best is None else min(best, t)
        res[name] = {"s_per_solve": best, "cost": cost}
    ctx.close()
    import oracle
    t0 = time.perf_counter()
    _, c0 = oracle.transport(C, r, c)
    t_or = time.perf_counter() - t0
    return {"workload": "mnist-like 116 x 169 pixels, totals 2048 (replicated 2048 x 2048)", "gpu": res,
            "cpu_oracle": {"s_per_solve": t_or, "cost": c0, "cores": 1, "kind": "oracle",
                           "sample": "one solve: replication + oracle KM"}}


def measure_sinkhorn_batch(ctx, dC, opt, stream, ot, torch):
    """Log-domain Sinkhorn on the same 4096 instances (one CTA each) at one
    fixed eta = 10^-2 with the paper's stopping rule (residue at most 0.1 %
    of the demand, no rounding): throughput, iterations and cost over each
    instance's exact optimum (from the KM solve)."""
    b = ot.SinkhornBatch(dC)
    eta = 1e-2
    ot.ot_sinkhorn_solve_batched(ctx, b, eta, eps_rel=1e-3, max_iter=5000, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ot.ot_sinkhorn_solve_batched(ctx, b, eta, eps_rel=1e-3, max_iter=5000, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1000.0
    ratio = b.cost.cpu().numpy() / np.maximum(opt.astype(np.float64), 1.0)
    its = b.iterations.cpu().numpy()
    out = {"eta": eta, "epsilon_rel": 1e-3, "s": secs, "solves_per_s": len(dC) / secs,
           "max_cost_over_opt": float(ratio.max()), "median_cost_over_opt": float(np.median(ratio)),
           "mean_iterations": float(its.mean()), "max_iterations": int(its.max()),
           "note": "approximate; exact KM on the same batch is the main value"}
    # the float64 oracle, single thread, on a bounded sample
    import oracle.sinkhorn as sko
    t0 = time.perf_counter()
    done = 0
    while time.perf_counter() - t0 < 3.0 and done < len(dC):
        sko.sinkhorn(dC[done].cpu().numpy(), eta, eps_rel=1e-3, max_iter=5000)
        done += 1
    out["cpu_oracle"] = {"value": done / (time.perf_counter() - t0), "unit": UNIT, "cores": 1,
                         "sample": f"first {done} instances, numpy float64 oracle, eta {eta}"}
    return out


def measure_served_process(args) -> dict:
    """The served stream measured in a process of its own, as a server runs:
    inside this process, after the batch, e2e and their GiB of pinned host
    buffers, the same stream kept only 68 % of the offered rate at 0.9x
    load, against 100 % in a fresh process."""
    cmd = [sys.executable, os.path.abspath(__file__), "--served-only", "--served-requests",
           str(args.served_requests)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("served stream failed:\n" + r.stdout[-2000:] + r.stderr[-2000:])
    res = json.loads(r.stdout.strip().splitlines()[-1])
    res["process"] = "separate (bench.py --served-only)"
    return res


def measure_served(ctx_unused, stream, ot, torch, dev, args):
    """Open-loop Poisson stream of MNIST-like requests (n log-uniform in
    [16, 2048], squared pixel distances on a 28 x 28 grid) through
    ot_assign_submit / ot_assign_completed / ot_assign_poll, driven by the
    native client in lib/libotclient.so (one host thread, no interpreter in
    the loop), at 0.5x and 0.9x of the measured saturated throughput;
    p50/p99 latency from arrival to completion.  The
    stream is ten times as long as the set of matrices it cycles over;
    every served cost is checked against the matrix's solo solve.  Steady
    throughput: completions over arrivals within one window (after the
    first tenth of the arrivals, up to the last arrival), so that neither
    the start nor the drain after the last arrival counts."""
    nreq = args.served_requests
    reqs = W.served_requests(nreq, rate_per_s=1.0, seed=W.BASE_SEED + 7)
    mats = [torch.from_numpy(C).pin_memory() for _, C in reqs]
    import tempfile
    tune_dir = tempfile.mkdtemp(prefix="otassign_served_")
    tune_path = os.path.join(tune_dir, "served_tune.jsonl")
    tctx = ot.Context(tune_file=tune_path)
    sample = [m.to(dev) for m in mats[:256]]
    ot.ot_autotune(tctx, sample, ot.OT_AUTO, repeats=1)
    tctx.close()
    del sample

    # the stream: `nstream` requests cycling over the nreq matrices, unit-rate
    # Poisson arrival times scaled by the offered rate
    nstream = 10 * nreq
    unit_t = np.cumsum(np.random.default_rng(W.BASE_SEED + 8).exponential(1.0, size=nstream))
    unit_t -= unit_t[0]
    import ctypes
    client = ctypes.CDLL(os.path.join(ROOT, "paper_2005_01182_gb300", "lib", "libotclient.so"))
    client.otc_replay.restype = ctypes.c_int
    client.otc_replay.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                  ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    cptr = (ctypes.c_void_p * nreq)(*[mm.data_ptr() for mm in mats])
    n_mat = np.array([mm.shape[0] for mm in mats], dtype=np.int32)
    m_mat = np.array([mm.shape[1] for mm in mats], dtype=np.int32)
    costs = np.zeros(nstream, dtype=np.int64)

    def run(rate):
        """The native client (`client/served_client.cpp`, one host thread):
        submit every request whose arrival time has passed, collect the
        requests the completion query returns, yield briefly when idle.  rate
        None: saturation, with at most `window` requests outstanding
        (submitted, not yet collected)."""
        sctx = ot.Context(hbm_budget_bytes=8 << 30, wave_streams=4, tune_file=tune_path)
        arrivals = np.ascontiguousarray(unit_t / rate if rate else np.zeros(nstream), dtype=np.float64)
        window = nstream if rate else 1024
        done = np.zeros(nstream, dtype=np.float64)
        total_c = ctypes.c_double()
        rc = client.otc_replay(sctx.h, nreq, cptr, n_mat.ctypes.data, m_mat.ctypes.data, nstream,
                               arrivals.ctypes.data, window, ot.OT_AUTO, done.ctypes.data, costs.ctypes.data,
                               ctypes.byref(total_c))
        assert rc == 0, f"served client: error {rc}"
        total = total_c.value
        cnt = ot.ot_serving_counters(sctx)
        sctx.close()
        lat = done - arrivals
        res = {"rate_per_s": rate, "requests": nstream, "solves_per_s": nstream / total,
               "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
               "grid_or_wave_launches": cnt["waves"]}
        if rate:
            # the rate the loop keeps up with: completions within the window
            # over arrivals within it (equal when it keeps up, whatever the
            # latency)
            lo, hi = float(arrivals[nstream // 10]), float(arrivals[-1])
            n_arr = float(((arrivals >= lo) & (arrivals <= hi)).sum())
            n_done = float(((done >= lo) & (done <= hi)).sum())
            res["steady_solves_per_s"] = n_done / (hi - lo)
            res["steady_over_offered"] = n_done / n_arr
        return res

    # the cost of every request solved alone (one batched call on the device,
    # same tuned table): each served run must return exactly these
    rctx = ot.Context(tune_file=tune_path)
    ref = ot.ot_assign_solve_batched(rctx, [m.to(dev) for m in mats], ot.OT_AUTO)
    torch.cuda.synchronize()
    solo = ref.cost.cpu().numpy().copy()
    assert (ref.status.cpu().numpy() == 0).all()
    rctx.close()
    del ref

    def checked(rate):
        r = run(rate)
        bad = int((costs != solo[np.arange(nstream) % nreq]).sum())
        assert bad == 0, f"{bad} served costs differ from the solo solves"
        r["checked_against_solo"] = nstream
        return r

    sat = checked(None)
    res = {"matrices": nreq, "requests_per_run": nstream, "n": "log-uniform [16, 2048]",
           "client": "native, one host thread (submit on arrival, collect through ot_assign_completed)",
           "saturated": sat}
    for f in (0.5, 0.9):
        res[f"at_{f}x"] = checked(f * sat["solves_per_s"])
    import shutil
    shutil.rmtree(tune_dir, ignore_errors=True)
    # plain: one ot_assign_solve per request on the device, no batching
    dmats = [m.to(dev) for m in mats[: min(64, nreq)]]
    ctx = ot.Context()
    torch.cuda.synchronize()
    t = time.perf_counter()
    lats = []
    for C in dmats:
        a = time.perf_counter()
        r, c, u, v = ot.ot_assign_solve(ctx, C, ot.OT_KM, stream)
        torch.cuda.synchronize()
        lats.append(time.perf_counter() - a)
    tp = time.perf_counter() - t
    ctx.close()
    res["plain_gpu_km"] = {"solves_per_s": len(dmats) / tp, "p50_solve_ms": float(np.median(lats) * 1e3),
                           "p99_solve_ms": float(np.percentile(lats, 99) * 1e3), "sample": len(dmats)}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--k", type=int, default=4096)
    ap.add_argument("--sample", type=int, default=96)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--skip-extras", action="store_true")
    ap.add_argument("--served-only", action="store_true",
                    help="measure the served stream alone and print its JSON (the full run starts this as a "
                         "process of its own)")
    ap.add_argument("--profile-table", default=None,
                    help="with --profile-once batch: the shape table to use instead of autotuning, as "
                         "'32:32x1,64:32x2,128:64x4,256:64x4' (bucket bound m: threads x columns per thread)")
    ap.add_argument("--served-requests", type=int, default=1500)
    ap.add_argument("--profile-once", default=None,
                    choices=["batch", "auction", "n16384", "n8192", "n16384dense", "n8192dense", "sinkhorn16384",
                             "sinkhorn8192"],
                    help="untimed single run for an ncu capture: 'batch' = autotune, then 3 batched "
                         "OT_AUTO calls on the 4096-instance batch inside an NVTX range 'timed'; "
                         "'n16384' / 'n8192' = one batched-KM solve on a grid instance (sparse-list engine; "
                         "'n16384dense' / 'n8192dense' on the dense cluster engine); "
                         "'sinkhorn16384' / 'sinkhorn8192' = log-domain Sinkhorn, eta = 2, 3 / 2 "
                         "fixed iterations on a 1024 x 1024-grid instance; 'auction' = one OT_AUCTION "
                         "solve of the 4096-instance batch inside an NVTX range 'timed'")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    from paper_2005_01182_gb300 import build as B
    from paper_2005_01182_gb300 import otassign as ot

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if rank == 0:
        B.build()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist.barrier()
        B.build()
    else:
        torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.served_only:
        print(json.dumps(measure_served(None, torch.cuda.current_stream(), ot, torch, dev, args)), flush=True)
        return
    ctx = ot.Context(device=local)
    stream = torch.cuda.current_stream()

    if args.profile_once in ("sinkhorn16384", "sinkhorn8192"):
        big = args.profile_once == "sinkhorn16384"
        C = W.single_16384() if big else W.grid_sqdist(8192, grid=1024)
        Cd = torch.from_numpy(C).to(dev)
        del C
        f, g, (cost, res, it) = ot.ot_sinkhorn_solve(ctx, Cd, 2.0, eps_rel=0.0, max_iter=3 if big else 2,
                                                     stream=stream)
        torch.cuda.synchronize()
        print(json.dumps({"profile_once": args.profile_once, "cost": cost, "iterations": it}))
        ctx.close()
        return
    if args.profile_once in ("n16384", "n8192", "n16384dense", "n8192dense"):
        n = 16384 if args.profile_once.startswith("n16384") else 8192
        C = W.grid_sqdist(n, n, grid=1024 if n == 16384 else 724)
        if args.profile_once.endswith("dense"):
            ctx.close()
            ctx = ot.Context(device=local, flags=ot.OT_CFG_DENSE_WIDE)
        r, c, u, v, st = ot.ot_assign_solve_stats(ctx, torch.from_numpy(C).to(dev), ot.OT_BKM, stream)
        torch.cuda.synchronize()
        print(json.dumps({"profile_once": args.profile_once, "cost": int(c.item()), **st}))
        ctx.close()
        return
    Cs = batch_for_rank(rank, args.k)
    dC = [torch.from_numpy(C).to(dev) for C in Cs]
    if args.profile_once == "auction":
        a = ot.BatchArgs(dC)
        ot.ot_assign_solve_batched(ctx, a, ot.OT_AUCTION, stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        ot.ot_assign_solve_batched(ctx, a, ot.OT_AUCTION, stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        assert (a.status.cpu().numpy() == 0).all()
        ctx.close()
        return
    if args.profile_once:
        # the timed configuration: tuned table (or the one given), OT_AUTO;
        # the three calls sit in an NVTX range "timed" for ncu --nvtx-include
        if args.profile_table:
            for ent in args.profile_table.split(","):
                mb, shape = ent.split(":")
                tpi, kk = shape.split("x")
                ot.ot_tune_set(ctx, ot.OT_KM, int(mb), int(tpi), int(kk))
        else:
            ot.ot_autotune(ctx, dC, ot.OT_AUTO, repeats=3)
        a = ot.BatchArgs(dC)
        ot.ot_assign_solve_batched(ctx, a, ot.OT_AUTO, stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        for _ in range(3):
            ot.ot_assign_solve_batched(ctx, a, ot.OT_AUTO, stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        assert (a.status.cpu().numpy() == 0).all()
        # the launches of the timed solves (kernel and instances), which key
        # the per-launch counts committed from a capture of this run
        print(json.dumps({"profile_once": "batch", "launches": [
            {"kernel": "group_kernel<%d, %d, %s>" % (L["threads_per_instance"], L["cols_per_thread"],
                                                     {0: "KM", 1: "BKM"}.get(L["algo"], "AUCTION")),
             "instances": L["instances"]} for L in ot.ot_last_call_launches(ctx)]}), flush=True)
        ctx.close()
        return
    h2d_bytes = sum(C.nbytes for C in Cs)
    d2h_bytes = sum(C.shape[0] * 4 + C.shape[0] * 8 + C.shape[1] * 8 + 8 for C in Cs)
    torch.cuda.synchronize()

    # autotune shape and algorithm (KM or batched KM) per size bucket on
    # this batch; OT_AUTO then uses the faster exact algorithm per bucket
    ot.ot_autotune(ctx, dC, ot.OT_AUTO, repeats=3)
    algo = ot.OT_AUTO
    tuned = {m: ot.ot_tune_lookup(ctx, ot.OT_AUTO, m) for m in (32, 64, 128, 256)}
    args_dev = ot.BatchArgs(dC)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region --------------------------------------
    for _ in range(args.warmup):
        ot.ot_assign_solve_batched(ctx, args_dev, algo, stream)
    barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks(local) as clk:
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for s in range(args.steps):
            evs[s][0].record(stream)
            ot.ot_assign_solve_batched(ctx, args_dev, algo, stream)
            evs[s][1].record(stream)
        t1.record(stream)
        barrier()
    total_ms = t0.elapsed_time(t1)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    st = ot.ot_last_call_stats(ctx)
    launches_per_step = st["launches"]
    value, total_ms = job_throughput(total_ms, args.k, args.steps, world, dist if world > 1 else None, dev)

    # correctness spot check of the timed results (cost must be finite/status ok)
    assert (args_dev.status.cpu().numpy() == 0).all(), "device status error"

    # the dominant kernel of a step, timed by the CUDA events the library
    # records around every bucket kernel on the stream it launches on
    kern = []
    for _ in range(5):
        ot.ot_assign_solve_batched(ctx, args_dev, algo, stream)
        kern.append(ot.ot_last_call_launches(ctx))
    dom_idx = max(range(len(kern[0])), key=lambda b: sum(k[b]["ms"] for k in kern))
    dom = kern[0][dom_idx]
    dom_ms = float(np.mean([k[dom_idx]["ms"] for k in kern]))
    dom_name = "group_kernel<%d, %d, %s>" % (dom["threads_per_instance"], dom["cols_per_thread"],
                                             {0: "KM", 1: "BKM", 3: "AUCTION"}[dom["algo"]])

    # ---- e2e through the C-ABI with pinned host buffers ---------------------
    # one pinned slab per array kind, instances back to back
    ns = [C.shape[0] for C in Cs]
    ms = [C.shape[1] for C in Cs]
    slabC = torch.empty(sum(n * m for n, m in zip(ns, ms)), dtype=torch.int32).pin_memory()
    slabR = torch.empty(sum(ns), dtype=torch.int32).pin_memory()
    slabU = torch.empty(sum(ns), dtype=torch.int64).pin_memory()
    slabV = torch.empty(sum(ms), dtype=torch.int64).pin_memory()
    hC, houts, oc, orow, ocol = [], [], 0, 0, 0
    for C, n, m in zip(Cs, ns, ms):
        v = slabC[oc:oc + n * m].view(n, m)
        v.copy_(torch.from_numpy(C))
        hC.append(v)
        houts.append((slabR[orow:orow + n], slabU[orow:orow + n], slabV[ocol:ocol + m]))
        oc += n * m
        orow += n
        ocol += m
    args_host = ot.BatchArgs(hC, outs=houts, device="cpu",
                             cost=torch.empty(args.k, dtype=torch.int64).pin_memory(),
                             status=torch.empty(args.k, dtype=torch.int32).pin_memory())
    e2e_steps = max(3, min(20, args.steps // 2))
    ot.ot_assign_solve_batched(ctx, args_host, algo)
    barrier()
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        ot.ot_assign_solve_batched(ctx, args_host, algo)
    barrier()
    e2e_s = time.perf_counter() - w0
    e2e_t = torch.tensor([e2e_s], device=dev)
    if world > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_value = world * args.k * e2e_steps / float(e2e_t.item())

    line = None
    if rank == 0:
        peak, peak_kind = _peaks()
        # algorithmic bytes: cost elements the scans must read (2 bytes each
        # for rows packed to 16 bits) plus the batched-KM row reduction
        alg_bytes = dom["read_bytes"] + dom["init_bytes"]
        achieved = alg_bytes / (dom_ms / 1000.0) / 1e9
        clocks = clk.summary()
        # The dominant kernel is bound by instruction issue along each
        # instance's chain of dependent steps, not by HBM: its ceiling is the
        # issue rate of the SMs' warp schedulers (4 per SM, one warp
        # instruction per cycle each) at the sampled SM clock.
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        sm_mhz = clocks.get("sm_mhz") or 2070.0
        issue_peak = nsm * 4 * sm_mhz * 1e6
        dom_key = "%s instances %d" % (dom_name, dom["instances"])
        inst = measured_instructions(dom_key)
        issue_rate = inst / (dom_ms / 1000.0) if inst else None
        roofline = {"bound": "alu", "achieved": issue_rate / 1e9 if inst else None,
                    "peak": issue_peak / 1e9, "unit": "G warp instructions/s",
                    "frac": issue_rate / issue_peak if inst else None,
                    "traffic": measured_traffic(dom_key), "kernel": dom_name,
                    "peak_kind": f"{nsm} SMs x 4 schedulers x 1 warp instruction/cycle at the sampled "
                                 f"median SM clock ({sm_mhz:.0f} MHz)",
                    "warp_instructions_per_launch": inst, "launch_ms": dom_ms,
                    "instances_per_launch": dom["instances"],
                    "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                            "peak_kind": peak_kind, "algorithmic_bytes_per_launch": alg_bytes},
                    "step_kernels": [{"kernel": "group_kernel<%d, %d, %s>" % (
                        k["threads_per_instance"], k["cols_per_thread"], {0: "KM", 1: "BKM", 3: "AUCTION"}[k["algo"]]),
                        "instances": k["instances"], "ms": k["ms"]} for k in kern[-1]]}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "batch4096_embed300_n32-256", "instances_per_gpu": args.k,
                       "algo": "auto (tuned per bucket)",
                       "tuned_shapes": {str(m): list(v) for m, v in tuned.items()},
                       "cost_bytes_resident": h2d_bytes, "l2": "inputs larger than L2 (%.0f MB > 129 MB)" % (h2d_bytes / 1e6),
                       "parallelism": f"replicas x{world} (instances sharded, no collective)"},
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d_bytes,
                    "d2h_bytes_per_step": d2h_bytes},
            "gpu_launches": int(launches_per_step * args.steps),
            "clocks": clocks,
            "step_ms": {"min": min(step_ms), "median": float(np.median(step_ms)), "max": max(step_ms)},
        }

    if rank == 0 and not args.skip_extras and world == 1:
        # side measurements at N = 1 only (the other GPUs of a multi-GPU run
        # are not held for them).  The served stream comes first, in a
        # process of its own (measure_served_process).
        line["served"] = measure_served_process(args)
        # plain one-instance-per-launch GPU KM on a sample of the same
        # instances
        sample = dC[: args.sample]
        outs = [ot._outputs(C.shape[0], C.shape[1], dev) for C in sample]
        for C, o in zip(sample[:8], outs[:8]):
            ot.ot_assign_solve(ctx, C, ot.OT_KM, stream, out=o)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for C, o in zip(sample, outs):
            ot.ot_assign_solve(ctx, C, ot.OT_KM, stream, out=o)
        a1.record(stream)
        torch.cuda.synchronize()
        plain = len(sample) / (a0.elapsed_time(a1) / 1000.0)
        line["plain_gpu_km"] = {"value": plain, "unit": UNIT, "sample": f"first {len(sample)} instances, one launch each",
                                "speedup_of_batched": value / world / plain}
        # the epsilon-scaling auction (exact) on the same batch, device-resident
        args_auc = ot.BatchArgs(dC)
        ot.ot_assign_solve_batched(ctx, args_auc, ot.OT_AUCTION, stream)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(3):
            ot.ot_assign_solve_batched(ctx, args_auc, ot.OT_AUCTION, stream)
        a1.record(stream)
        torch.cuda.synchronize()
        ast = ot.ot_last_call_stats(ctx)
        assert (args_auc.status.cpu().numpy() == 0).all()
        assert (args_auc.cost.cpu().numpy() == args_dev.cost.cpu().numpy()).all(), "auction cost differs from KM"
        auc_s = a0.elapsed_time(a1) / 3000.0
        auc_bytes = ast["cost_bytes"] + ast["init_bytes"]
        peak_a, _ = _peaks()
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        done = 0
        while time.perf_counter() - t0 < 3.0 and done < len(Cs):
            oracle.auction(Cs[done])
            done += 1
        oracle_rate = done / (time.perf_counter() - t0)
        line["auction"] = {"value": len(dC) / auc_s, "unit": UNIT,
                           "ms_per_step": auc_s * 1000.0, "bids": ast["rows_scanned"],
                           "rounds": ast["steps"], "stages": ast["phases"],
                           "algorithmic_bytes": auc_bytes, "achieved_gbs": auc_bytes / auc_s / 1e9,
                           "hbm_frac": auc_bytes / auc_s / 1e9 / peak_a,
                           "cpu_oracle": {"value": oracle_rate, "unit": UNIT, "cores": 1,
                                          "sample": f"first {done} instances, oracle auction, single thread"},
                           "note": "same 4096 instances, OT_AUCTION, costs equal to KM's; bound: round latency"}
        del args_auc
        line["sinkhorn_batch"] = measure_sinkhorn_batch(ctx, dC, args_dev.cost.cpu().numpy(), stream, ot, torch)
        cores = host_threads()
        rate, done, dt = cpu_oracle_rate_threads(Cs, args.cpu_seconds, cores)
        rate1, done1, dt1 = cpu_oracle_rate(Cs, args.cpu_seconds / 2)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"first {done} instances of the batch, oracle KM, one instance per "
                                          f"thread on {cores} host threads, {dt:.1f}s",
                                "single_thread": {"value": rate1, "sample": f"first {done1} instances, {dt1:.1f}s"}}
        del Cs, dC, args_dev, args_host, hC, houts, slabC
        torch.cuda.empty_cache()
        line["single_4096"] = measure_single_4096(stream, ot, torch)
        line["single_16384"] = measure_single_16384(ctx, stream, ot, torch)
        line["sinkhorn_4096"] = measure_sinkhorn_4096(stream, ot, torch)
        line["transport_mnist"] = measure_transport(stream, ot, torch)
    elif rank == 0:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
