"""Thin ctypes binding of libotassign.so (argument marshalling only).

Every function here has the name of the C entry point it calls
(``include/otassign.h``); all arithmetic of the assignment solvers runs in
the library's CUDA kernels.  Tensors are passed by pointer: device tensors
stay on the device, host tensors (pinned or not) are staged by the library.
If the shared library has not been built this module raises on import of a
solver call -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libotassign.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "otassign.h")

OT_OK = 0
OT_PENDING = 1
OT_ERR_ARG = -1
OT_ERR_OOM = -2
OT_ERR_BUDGET = -3
OT_ERR_TIMEOUT = -4
OT_ERR_CUDA = -5
OT_ERR_OVERFLOW = -6
OT_ERR_UNSUPPORTED = -7
OT_ERR_TICKET = -8
OT_KM = 0
OT_BKM = 1
OT_AUTO = 2
OT_AUCTION = 3

_lib = None


class OtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"otassign error {code}: {msg}")
        self.code = code


class ot_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("rows_scanned", ctypes.c_int64),
                ("cost_bytes", ctypes.c_int64), ("phases", ctypes.c_int64),
                ("augmentations", ctypes.c_int64), ("init_bytes", ctypes.c_int64),
                ("reserved", ctypes.c_int64 * 2)]


class ot_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_int64),
                ("max_inflight", ctypes.c_int32), ("wave_streams", ctypes.c_int32),
                ("tune_file", ctypes.c_char_p), ("flags", ctypes.c_uint32),
                ("max_group_ctas", ctypes.c_int32), ("step_limit", ctypes.c_int64)]


OT_CFG_NO_ROW_PACKING = 1
OT_CFG_DENSE_WIDE = 2


def declared_symbols() -> list[str]:
    """Function names declared in include/otassign.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ot_[a-z_0-9]+)\s*\(", text)))


def load(path: str | None = None):
    """Load the shared library (built by ``build.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"{p} not found: build the CUDA library first (paper_2005_01182_gb300.build)")
    lib = ctypes.CDLL(p)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "ot_ctx_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(ot_config)]),
        "ot_ctx_destroy": (None, [vp]),
        "ot_last_error_string": (ctypes.c_char_p, [vp]),
        "ot_assign_solve": (ctypes.c_int, [vp, vp, i64, i32, i32, i32, vp, vp, vp, vp, vp]),
        "ot_assign_solve_stats": (ctypes.c_int, [vp, vp, i64, i32, i32, i32, vp, vp, vp, vp,
                                                 ctypes.POINTER(ot_stats), vp]),
        "ot_assign_solve_batched": (ctypes.c_int, [vp, i32, pp, ctypes.POINTER(i64),
                                                   ctypes.POINTER(i32), ctypes.POINTER(i32), i32,
                                                   pp, vp, pp, pp, vp, vp]),
        "ot_assign_submit": (ctypes.c_int, [vp, vp, i64, i32, i32, i32, ctypes.POINTER(ctypes.c_uint64)]),
        "ot_assign_poll": (ctypes.c_int, [vp, ctypes.c_uint64, vp, vp, vp, vp]),
        "ot_assign_drain": (ctypes.c_int, [vp]),
        "ot_assign_cancel": (ctypes.c_int, [vp, ctypes.c_uint64]),
        "ot_assign_completed": (ctypes.c_int, [vp, vp, ctypes.c_int32, vp]),
        "ot_serving_counters": (ctypes.c_int, [vp, ctypes.POINTER(i64)]),
        "ot_autotune": (ctypes.c_int, [vp, i32, pp, ctypes.POINTER(i64), ctypes.POINTER(i32),
                                       ctypes.POINTER(i32), i32, i32]),
        "ot_tune_lookup": (ctypes.c_int, [vp, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "ot_tune_set": (ctypes.c_int, [vp, i32, i32, i32, i32]),
        "ot_last_call_stats": (ctypes.c_int, [vp, ctypes.POINTER(ot_stats)]),
        "ot_assign_solve_batched_noalloc": (ctypes.c_int, [i32, pp, ctypes.POINTER(i64),
                                                           ctypes.POINTER(i32), ctypes.POINTER(i32), i32,
                                                           pp, vp, pp, pp, vp, vp]),
        "ot_assign_solve_scaled": (ctypes.c_int, [vp, vp, i64, i32, i32, i32, vp, vp, vp, vp]),
        "ot_transport_solve": (ctypes.c_int, [vp, vp, i64, i32, i32, vp, vp, i32, vp, vp, vp]),
        "ot_sinkhorn_solve": (ctypes.c_int, [vp, vp, i64, i32, i32, vp, vp, ctypes.c_double, ctypes.c_double,
                                             i32, vp, vp, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32), vp]),
        "ot_last_call_launches": (ctypes.c_int, [vp, vp, i32, ctypes.POINTER(i32)]),
        "ot_sinkhorn_solve_batched": (ctypes.c_int, [vp, i32, pp, ctypes.POINTER(i64), ctypes.POINTER(i32),
                                                     ctypes.POINTER(i32), ctypes.c_double, ctypes.c_double, i32,
                                                     pp, pp, vp, vp, vp, vp]),
        "ot_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream_handle(stream) -> ctypes.c_void_p | None:
    """The stream a call is issued on: the given one, else torch's current
    stream (handle 0, the default stream, is ordered by the library)."""
    if stream is None:
        if not torch.cuda.is_available():
            return None
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _check_cost(C: torch.Tensor):
    if C.dtype != torch.int32 or C.dim() != 2 or (C.shape[0] > 0 and C.stride(1) != 1):
        raise ValueError("cost matrix must be a 2-D int32 tensor with unit column stride")
    n, m = C.shape
    ldc = C.stride(0) if n > 1 else m
    return n, m, max(ldc, m)


class Context:
    """Owns one ot_ctx (device buffers, streams, serving thread)."""

    def __init__(self, device: int = -1, hbm_budget_bytes: int = 0, max_inflight: int = 0,
                 wave_streams: int = 0, tune_file: str | None = None, flags: int = 0,
                 max_group_ctas: int = 0, step_limit: int = 0):
        lib = load()
        cfg = ot_config(device, hbm_budget_bytes, max_inflight, wave_streams,
                        tune_file.encode() if tune_file else None, flags, max_group_ctas, step_limit)
        h = ctypes.c_void_p()
        rc = lib.ot_ctx_create(ctypes.byref(h), ctypes.byref(cfg))
        if rc != OT_OK:
            raise OtError(rc, "ot_ctx_create failed")
        self.h = h
        self.lib = lib

    def close(self):
        if getattr(self, "h", None):
            self.lib.ot_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def error(self) -> str:
        return self.lib.ot_last_error_string(self.h).decode()

    def _raise(self, rc: int, what: str):
        if rc != OT_OK:
            raise OtError(rc, f"{what}: {self.error()}")


def ot_ctx_create(**kw) -> Context:
    return Context(**kw)


def ot_ctx_destroy(ctx: Context):
    ctx.close()


def ot_last_error_string(ctx: Context) -> str:
    return ctx.error()


def _outputs(n, m, device, pin=False):
    kw = dict(device=device)
    r = torch.empty(n, dtype=torch.int32, **kw)
    c = torch.empty(1, dtype=torch.int64, **kw)
    u = torch.empty(n, dtype=torch.int64, **kw)
    v = torch.empty(m, dtype=torch.int64, **kw)
    if pin and device == "cpu":
        r, c, u, v = (x.pin_memory() for x in (r, c, u, v))
    return r, c, u, v


def ot_assign_solve(ctx: Context, C: torch.Tensor, algo: int = OT_KM, stream=None, out=None,
                    duals: bool = True):
    """Solve one instance.  Returns (row_to_col, cost[1], u, v) on C's device."""
    n, m, ldc = _check_cost(C)
    r, c, u, v = out if out is not None else _outputs(n, m, C.device)
    rc = ctx.lib.ot_assign_solve(ctx.h, _ptr(C), ldc, n, m, algo, _ptr(r), _ptr(c),
                                 _ptr(u) if duals else None, _ptr(v) if duals else None,
                                 _stream_handle(stream))
    ctx._raise(rc, "ot_assign_solve")
    return r, c, u, v


def ot_assign_solve_stats(ctx: Context, C: torch.Tensor, algo: int = OT_KM, stream=None):
    """Solve one instance synchronously; also returns the device counters."""
    n, m, ldc = _check_cost(C)
    r, c, u, v = _outputs(n, m, C.device)
    st = ot_stats()
    rc = ctx.lib.ot_assign_solve_stats(ctx.h, _ptr(C), ldc, n, m, algo, _ptr(r), _ptr(c), _ptr(u),
                                       _ptr(v), ctypes.byref(st), _stream_handle(stream))
    ctx._raise(rc, "ot_assign_solve_stats")
    stats = {f: getattr(st, f) for f, _ in ot_stats._fields_ if f != "reserved"}
    stats["read_bytes"] = st.reserved[1]
    return r, c, u, v, stats


class BatchArgs:
    """Pre-marshalled pointer arrays for ot_assign_solve_batched, so that a
    timed loop re-issues the call without rebuilding them."""

    def __init__(self, Cs, outs=None, device=None, cost=None, status=None):
        k = len(Cs)
        self.k = k
        self.Cs = Cs
        dev = device if device is not None else (Cs[0].device if k else "cpu")
        sizes = [_check_cost(C) for C in Cs]
        self.n = (ctypes.c_int32 * k)(*[s[0] for s in sizes])
        self.m = (ctypes.c_int32 * k)(*[s[1] for s in sizes])
        self.ldc = (ctypes.c_int64 * k)(*[s[2] for s in sizes])
        self.cp = (ctypes.c_void_p * k)(*[C.data_ptr() for C in Cs])
        if outs is None:
            outs = [(torch.empty(s[0], dtype=torch.int32, device=dev),
                     torch.empty(s[0], dtype=torch.int64, device=dev),
                     torch.empty(s[1], dtype=torch.int64, device=dev)) for s in sizes]
        self.outs = outs
        self.rp = (ctypes.c_void_p * k)(*[o[0].data_ptr() for o in outs])
        self.up = (ctypes.c_void_p * k)(*[o[1].data_ptr() for o in outs])
        self.vp = (ctypes.c_void_p * k)(*[o[2].data_ptr() for o in outs])
        self.cost = cost if cost is not None else torch.empty(k, dtype=torch.int64, device=dev)
        self.status = status if status is not None else torch.empty(k, dtype=torch.int32, device=dev)


def ot_assign_solve_batched(ctx: Context, Cs_or_args, algo: int = OT_KM, stream=None):
    """Solve many instances in one launch set.  Accepts a list of cost
    tensors (all on one device, or all on the host) or a ``BatchArgs``.
    Returns the BatchArgs holding (row_to_col, u, v) per instance, cost[k]
    and status[k]."""
    a = Cs_or_args if isinstance(Cs_or_args, BatchArgs) else BatchArgs(Cs_or_args)
    P = ctypes.cast
    pp = ctypes.POINTER(ctypes.c_void_p)
    rc = ctx.lib.ot_assign_solve_batched(ctx.h, a.k, P(a.cp, pp), a.ldc, a.n, a.m, algo,
                                         P(a.rp, pp), _ptr(a.cost), P(a.up, pp), P(a.vp, pp),
                                         _ptr(a.status), _stream_handle(stream))
    ctx._raise(rc, "ot_assign_solve_batched")
    return a


def ot_assign_solve_scaled(ctx: Context, C: torch.Tensor, scale: int, stream=None):
    """Batched KM on floor(C / scale): returns (row_to_col, cost under C,
    a-priori bound n*(scale-1) on cost - OPT)."""
    n, m, ldc = _check_cost(C)
    r = torch.empty(n, dtype=torch.int32, device=C.device)
    c = torch.empty(1, dtype=torch.int64, device=C.device)
    b = torch.empty(1, dtype=torch.int64)
    rc = ctx.lib.ot_assign_solve_scaled(ctx.h, _ptr(C), ldc, n, m, scale, _ptr(r), _ptr(c), _ptr(b),
                                        _stream_handle(stream))
    ctx._raise(rc, "ot_assign_solve_scaled")
    return r, c, int(b.item())


def ot_transport_solve(ctx: Context, C: torch.Tensor, supply, demand, algo: int = OT_AUTO, stream=None):
    """Integer-supply transport by vertex replication: returns (flow n x m
    int32 on C's device, cost)."""
    import numpy as np
    n, m, ldc = _check_cost(C)
    sp = np.ascontiguousarray(supply, dtype=np.int32)
    dm = np.ascontiguousarray(demand, dtype=np.int32)
    flow = torch.empty((n, m), dtype=torch.int32, device=C.device)
    c = torch.empty(1, dtype=torch.int64)
    rc = ctx.lib.ot_transport_solve(ctx.h, _ptr(C), ldc, n, m, ctypes.c_void_p(sp.ctypes.data),
                                    ctypes.c_void_p(dm.ctypes.data), algo, _ptr(c), _ptr(flow),
                                    _stream_handle(stream))
    ctx._raise(rc, "ot_transport_solve")
    return flow, int(c.item())


class SinkhornBatch:
    """Pre-marshalled arguments of ot_sinkhorn_solve_batched (device cost
    matrices); outputs f[t], g[t] (float32), cost, residue, iterations."""

    def __init__(self, Cs):
        k = len(Cs)
        self.k = k
        self.Cs = Cs
        sizes = [_check_cost(C) for C in Cs]
        dev = Cs[0].device
        self.n = (ctypes.c_int32 * k)(*[s[0] for s in sizes])
        self.m = (ctypes.c_int32 * k)(*[s[1] for s in sizes])
        self.ldc = (ctypes.c_int64 * k)(*[s[2] for s in sizes])
        self.cp = (ctypes.c_void_p * k)(*[C.data_ptr() for C in Cs])
        self.f = [torch.empty(s[0], dtype=torch.float32, device=dev) for s in sizes]
        self.g = [torch.empty(s[1], dtype=torch.float32, device=dev) for s in sizes]
        self.fp = (ctypes.c_void_p * k)(*[x.data_ptr() for x in self.f])
        self.gp = (ctypes.c_void_p * k)(*[x.data_ptr() for x in self.g])
        self.cost = torch.empty(k, dtype=torch.float64, device=dev)
        self.residue = torch.empty(k, dtype=torch.float64, device=dev)
        self.iterations = torch.empty(k, dtype=torch.int32, device=dev)


def ot_sinkhorn_solve_batched(ctx: Context, Cs_or_batch, eta: float, eps_rel: float = 1e-3,
                              max_iter: int = 1000, stream=None):
    """Log-domain Sinkhorn on many device instances, one CTA each; returns
    the SinkhornBatch holding f, g, cost, residue, iterations."""
    b = Cs_or_batch if isinstance(Cs_or_batch, SinkhornBatch) else SinkhornBatch(Cs_or_batch)
    P = ctypes.cast
    pp = ctypes.POINTER(ctypes.c_void_p)
    rc = ctx.lib.ot_sinkhorn_solve_batched(ctx.h, b.k, P(b.cp, pp), b.ldc, b.n, b.m, float(eta), float(eps_rel),
                                           int(max_iter), P(b.fp, pp), P(b.gp, pp), _ptr(b.cost), _ptr(b.residue),
                                           _ptr(b.iterations), _stream_handle(stream))
    ctx._raise(rc, "ot_sinkhorn_solve_batched")
    return b


class ot_launch_info(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("threads_per_instance", ctypes.c_int32),
                ("cols_per_thread", ctypes.c_int32), ("instances", ctypes.c_int32), ("ms", ctypes.c_float),
                ("reserved", ctypes.c_int32), ("read_bytes", ctypes.c_int64), ("init_bytes", ctypes.c_int64)]


def ot_last_call_launches(ctx: Context) -> list:
    """Per-launch description of the most recent solve call (synchronises):
    algorithm, shape, instances, device ms and bytes of each bucket kernel."""
    buf = (ot_launch_info * 64)()
    cnt = ctypes.c_int32()
    ctx._raise(ctx.lib.ot_last_call_launches(ctx.h, buf, 64, ctypes.byref(cnt)), "ot_last_call_launches")
    return [{f: getattr(buf[i], f) for f, _ in ot_launch_info._fields_ if f != "reserved"}
            for i in range(min(cnt.value, 64))]


def ot_sinkhorn_solve(ctx: Context, C: torch.Tensor, eta: float, eps_rel: float = 1e-3, max_iter: int = 1000,
                      r=None, c=None, stream=None):
    """Log-domain Sinkhorn on a device cost matrix.  Returns (f, g) float32
    on C's device and (cost, residue, iterations)."""
    import numpy as np
    n, m, ldc = _check_cost(C)
    f = torch.empty(n, dtype=torch.float32, device=C.device)
    g = torch.empty(m, dtype=torch.float32, device=C.device)
    rr = None if r is None else np.ascontiguousarray(r, dtype=np.float64)
    cc = None if c is None else np.ascontiguousarray(c, dtype=np.float64)
    cost, res, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    rc = ctx.lib.ot_sinkhorn_solve(ctx.h, _ptr(C), ldc, n, m,
                                   None if rr is None else ctypes.c_void_p(rr.ctypes.data),
                                   None if cc is None else ctypes.c_void_p(cc.ctypes.data),
                                   float(eta), float(eps_rel), int(max_iter), _ptr(f), _ptr(g),
                                   ctypes.byref(cost), ctypes.byref(res), ctypes.byref(it), _stream_handle(stream))
    ctx._raise(rc, "ot_sinkhorn_solve")
    return f, g, (cost.value, res.value, it.value)


def ot_last_call_stats(ctx: Context) -> dict:
    """Counters of the most recent solve call, summed over its instances
    (synchronises); 'launches' is the number of kernels it launched."""
    st = ot_stats()
    ctx._raise(ctx.lib.ot_last_call_stats(ctx.h, ctypes.byref(st)), "ot_last_call_stats")
    d = {f: getattr(st, f) for f, _ in ot_stats._fields_ if f != "reserved"}
    d["launches"] = st.reserved[0]
    d["read_bytes"] = st.reserved[1]
    return d


def ot_assign_submit(ctx: Context, C: torch.Tensor, algo: int = OT_KM) -> int:
    n, m, ldc = _check_cost(C)
    t = ctypes.c_uint64()
    rc = ctx.lib.ot_assign_submit(ctx.h, _ptr(C), ldc, n, m, algo, ctypes.byref(t))
    ctx._raise(rc, "ot_assign_submit")
    return t.value


def ot_assign_poll(ctx: Context, ticket: int, out) -> int:
    """out = (row_to_col, cost[1], u, v) tensors (host or device).  Returns
    OT_PENDING or OT_OK; raises on a failed request."""
    r, c, u, v = out
    rc = ctx.lib.ot_assign_poll(ctx.h, ticket, _ptr(r), _ptr(c), _ptr(u), _ptr(v))
    if rc == OT_PENDING:
        return OT_PENDING
    ctx._raise(rc, "ot_assign_poll")
    return OT_OK


def ot_assign_completed(ctx: Context, max_count: int = 4096) -> list:
    """Tickets whose solve has ended since the last call (collect each with
    ot_assign_poll, which then returns OT_OK or raises)."""
    buf = getattr(ctx, "_done_buf", None)
    if buf is None or len(buf) < max_count:
        buf = (ctypes.c_uint64 * max_count)()
        ctx._done_buf = buf
    cnt = ctypes.c_int32()
    ctx._raise(ctx.lib.ot_assign_completed(ctx.h, buf, max_count, ctypes.byref(cnt)), "ot_assign_completed")
    return buf[: cnt.value]


def ot_assign_cancel(ctx: Context, ticket: int):
    """Cancel a submitted request (raises OtError OT_ERR_TICKET for an
    unknown, collected or already cancelled ticket)."""
    ctx._raise(ctx.lib.ot_assign_cancel(ctx.h, ticket), "ot_assign_cancel")


def ot_assign_drain(ctx: Context):
    ctx._raise(ctx.lib.ot_assign_drain(ctx.h), "ot_assign_drain")


def ot_serving_counters(ctx: Context) -> dict:
    out = (ctypes.c_int64 * 8)()
    ctx._raise(ctx.lib.ot_serving_counters(ctx.h, out), "ot_serving_counters")
    keys = ["submitted", "admitted", "completed", "waves", "max_concurrent_waves",
            "bytes_resident", "budget_bytes", "refused"]
    return dict(zip(keys, list(out)))


def ot_autotune(ctx: Context, Cs, algo: int = OT_KM, repeats: int = 2):
    a = BatchArgs(Cs)
    pp = ctypes.POINTER(ctypes.c_void_p)
    rc = ctx.lib.ot_autotune(ctx.h, a.k, ctypes.cast(a.cp, pp), a.ldc, a.n, a.m, algo, repeats)
    ctx._raise(rc, "ot_autotune")


def ot_tune_lookup(ctx: Context, algo: int, m: int):
    t, k = ctypes.c_int32(), ctypes.c_int32()
    ctx._raise(ctx.lib.ot_tune_lookup(ctx.h, algo, m, ctypes.byref(t), ctypes.byref(k)), "ot_tune_lookup")
    return t.value, k.value


OT_NOALLOC_MAX_INSTANCES = 1024


def ot_assign_solve_batched_noalloc(args: BatchArgs, algo: int = OT_KM, stream=None) -> int:
    """Batched solve through the entry point that allocates no device memory
    (no context; device tensors only; at most OT_NOALLOC_MAX_INSTANCES
    instances).  Returns the C return code; results land in ``args``."""
    lib = load()
    pp = ctypes.POINTER(ctypes.c_void_p)
    return lib.ot_assign_solve_batched_noalloc(args.k, ctypes.cast(args.cp, pp), args.ldc, args.n, args.m,
                                               algo, ctypes.cast(args.rp, pp), _ptr(args.cost),
                                               ctypes.cast(args.up, pp), ctypes.cast(args.vp, pp),
                                               _ptr(args.status), _stream_handle(stream))


def ot_tune_set(ctx: Context, algo: int, m: int, threads_per_instance: int, cols_per_thread: int):
    ctx._raise(ctx.lib.ot_tune_set(ctx.h, algo, m, threads_per_instance, cols_per_thread), "ot_tune_set")


def ot_version() -> str:
    return load().ot_version().decode()
