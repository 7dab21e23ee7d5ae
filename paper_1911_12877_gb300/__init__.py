"""Python binding of libgz (GraphZero pattern counting on GB300, sm_103a).

Argument marshalling only: every step of the counting path runs in libgz's CUDA
kernels and host C++ (planner, serving loop). PyTorch, when used, only provides
device buffers (``tensor.data_ptr()``) and streams. There is no CPU fallback:
if the library is missing this module raises at load time.

Build the library with ``paper_1911_12877_gb300.build.build()``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgz.so")

GZ_OK, GZ_EINVAL, GZ_ENOMEM, GZ_ECUDA, GZ_ETIMEOUT = 0, -1, -2, -3, -4
GZ_EUNSUPPORTED, GZ_EOVERFLOW, GZ_EBUSY = -5, -6, -7
GZ_VALIDATE, GZ_VALIDATE_SYMMETRIC = 1, 2
MAX_K = 8

#: every entry point declared in include/gz.h
EXPORTS = [
    "gz_load_csr", "gz_orient", "gz_graph_info", "gz_graph_export", "gz_graph_destroy",
    "gz_pattern_named", "gz_plan_create", "gz_plan_create_with_order", "gz_plan_info",
    "gz_plan_schedules", "gz_plan_describe", "gz_plan_destroy", "gz_count", "gz_count_ex", "gz_scratch_bytes",
    "gz_count_batch", "gz_count_batch_ranges", "gz_count_noalloc", "gz_prepare", "gz_autotune", "gz_server_create", "gz_server_submit", "gz_server_wait",
    "gz_server_replay", "gz_server_destroy", "gz_last_error", "gz_version", "gz_kernel_launches",
    "gz_allocations", "gz_count_merged",
    "gz_motif_patterns", "gz_count_motifs", "gz_plan_create_measured", "gz_schedule_times",
]


class GzError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libgz status {status}: {msg}")
        self.status = status


class GraphStats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("max_degree", ctypes.c_int64),
                ("max_out_degree_original", ctypes.c_int64),
                ("max_out_degree_oriented", ctypes.c_int64), ("oriented", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64)]


class CountOpts(ctypes.Structure):
    _fields_ = [("use_orientation", ctypes.c_int), ("root_lo", ctypes.c_int64),
                ("root_hi", ctypes.c_int64), ("block_warps", ctypes.c_int), ("chunk", ctypes.c_int),
                ("split_min", ctypes.c_int64), ("split_chunk", ctypes.c_int64)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("max_inflight_launches", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("scratch_budget", ctypes.c_uint64), ("heavy_ms", ctypes.c_double),
                ("slow_share", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def lib() -> ctypes.CDLL:
    """The loaded libgz; raises if the CUDA library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libgz.so not found at {LIB_PATH}: run paper_1911_12877_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    I, I64, S = ctypes.c_int, ctypes.c_int64, ctypes.c_int32
    L.gz_last_error.restype = ctypes.c_char_p
    L.gz_version.restype = ctypes.c_char_p
    L.gz_kernel_launches.restype = ctypes.c_uint64
    L.gz_kernel_launches.argtypes = []
    L.gz_allocations.restype = ctypes.c_uint64
    L.gz_allocations.argtypes = []
    sig = {
        "gz_load_csr": [_P, _P, I64, I64, I, ctypes.c_uint32, _P, ctypes.POINTER(_P)],
        "gz_orient": [_P, _P],
        "gz_graph_info": [_P, ctypes.POINTER(GraphStats)],
        "gz_graph_export": [_P, I, _i64p, _i32p, _i32p, _P],
        "gz_pattern_named": [ctypes.c_char_p, ctypes.POINTER(I), _u8p],
        "gz_plan_create": [I, _u8p, ctypes.c_uint32, ctypes.POINTER(_P)],
        "gz_plan_create_with_order": [I, _u8p, _i32p, ctypes.POINTER(_P)],
        "gz_plan_info": [_P, ctypes.POINTER(I), _i32p, _i32p, _u64p, ctypes.POINTER(ctypes.c_double)],
        "gz_plan_schedules": [I, _u8p, _i32p, I, ctypes.POINTER(I)],
        "gz_plan_describe": [_P, ctypes.c_char_p, I],
        "gz_count": [_P, _P, I, _P, _u64p],
        "gz_count_ex": [_P, _P, ctypes.POINTER(CountOpts), _P, _u64p],
        "gz_scratch_bytes": [_P, _P, I, _u64p],
        "gz_prepare": [_P, _P, I, _P],
        "gz_count_noalloc": [_P, _P, I, _P, _u64p],
        "gz_count_batch": [ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(I), I, _P, _u64p],
        "gz_count_batch_ranges": [ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(I), _i64p, _i64p, I, _P,
                                  _u64p],
        "gz_count_merged": [ctypes.POINTER(_P), I, _P, I, _P, _u64p],
        "gz_autotune": [_P, _P, I, _P, ctypes.POINTER(I), ctypes.POINTER(I), _i64p, _i64p],
        "gz_motif_patterns": [I, _u8p, I, ctypes.POINTER(I)],
        "gz_plan_create_measured": [I, _u8p, _P, I, _i64p, _i64p, I, _P, ctypes.POINTER(_P),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
        "gz_schedule_times": [I, _u8p, _P, I, _i64p, _i64p, I, _P, ctypes.c_double, _i32p,
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), I,
                              ctypes.POINTER(I)],
        "gz_count_motifs": [_P, I, I, _P, _u64p, I, ctypes.POINTER(I)],
        "gz_server_create": [ctypes.POINTER(ServerOpts), ctypes.POINTER(_P)],
        "gz_server_submit": [_P, _P, _P, I, _i64p],
        "gz_server_wait": [_P, I64, I64, _u64p, _i64p],
        "gz_server_replay": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(I), I64,
                             _i64p, _i32p, _i32p, I, _u64p, _i64p, ctypes.POINTER(ctypes.c_double)],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = S
    for name in ("gz_graph_destroy", "gz_plan_destroy", "gz_server_destroy"):
        getattr(L, name).argtypes = [_P]
        getattr(L, name).restype = None
    _lib = L
    return L


def _check(status: int, what: str = "") -> None:
    if status != GZ_OK:
        msg = lib().gz_last_error().decode(errors="replace")
        raise GzError(status, f"{what}: {msg}" if what else msg)


def _stream(stream) -> int | None:
    """cudaStream_t of a torch stream, an int handle, or the current torch stream."""
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def version() -> str:
    return lib().gz_version().decode()


def allocations() -> int:
    """Memory allocation calls libgz has made in this process (gz_allocations)."""
    return int(lib().gz_allocations())


def kernel_launches() -> int:
    """CUDA kernels libgz has launched in this process."""
    return int(lib().gz_kernel_launches())


# ------------------------------------------------------------------ patterns

def pattern_named(name: str) -> np.ndarray:
    k = ctypes.c_int()
    buf = (ctypes.c_uint8 * (MAX_K * MAX_K))()
    _check(lib().gz_pattern_named(name.encode(), ctypes.byref(k), buf), "gz_pattern_named")
    return np.frombuffer(bytes(buf), dtype=np.uint8)[: k.value * k.value].reshape(k.value, k.value).copy()


def _adj(adj):
    if isinstance(adj, str):
        adj = pattern_named(adj)
    a = np.ascontiguousarray(np.asarray(adj, dtype=np.uint8))
    return a, a.shape[0]


class Plan:
    """A compiled schedule (gz_plan)."""

    def __init__(self, adj, order=None):
        a, k = _adj(adj)
        self._a = a
        h = _P()
        if order is None:
            _check(lib().gz_plan_create(k, a.ctypes.data_as(_u8p), 0, ctypes.byref(h)), "gz_plan_create")
        else:
            o = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
            _check(lib().gz_plan_create_with_order(k, a.ctypes.data_as(_u8p), o.ctypes.data_as(_i32p),
                                                   ctypes.byref(h)), "gz_plan_create_with_order")
        self.handle = h

    def info(self) -> dict:
        k = ctypes.c_int()
        order = np.zeros(MAX_K, dtype=np.int32)
        bp = np.zeros(MAX_K, dtype=np.int32)
        aut = ctypes.c_uint64()
        cost = ctypes.c_double()
        _check(lib().gz_plan_info(self.handle, ctypes.byref(k), order.ctypes.data_as(_i32p),
                                  bp.ctypes.data_as(_i32p), ctypes.byref(aut), ctypes.byref(cost)))
        n = k.value
        return {"k": n, "order": order[:n].tolist(), "bound_parent": bp[:n].tolist(),
                "aut_size": aut.value, "est_cost": cost.value}

    def describe(self) -> str:
        buf = ctypes.create_string_buffer(16384)
        _check(lib().gz_plan_describe(self.handle, buf, len(buf)), "gz_plan_describe")
        return buf.value.decode()

    def close(self):
        if getattr(self, "handle", None):
            lib().gz_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ranges(samples):
    lo = np.ascontiguousarray([s[0] for s in samples], dtype=np.int64)
    hi = np.ascontiguousarray([s[1] for s in samples], dtype=np.int64)
    return lo, hi


def schedule_times(adj, graph: "Graph", samples, orientation: bool = True, cutoff: float = 0.0,
                   stream=None) -> list:
    """Every distinct schedule timed on the root ranges samples = [(lo, hi), ...]:
    a list of {"order", "est_cost", "ms"} in Algorithm 4's order (ms = -1: dropped
    past cutoff x the best)."""
    a, k = _adj(adj)
    lo, hi = _ranges(samples)
    cnt = ctypes.c_int()
    args = (k, a.ctypes.data_as(_u8p), graph.handle, int(orientation), lo.ctypes.data_as(_i64p),
            hi.ctypes.data_as(_i64p), len(samples), _stream(stream), float(cutoff))
    _check(lib().gz_schedule_times(*args, None, None, None, 0, ctypes.byref(cnt)), "gz_schedule_times")
    n = cnt.value
    orders = np.zeros((max(n, 1), k), dtype=np.int32)
    cost = np.zeros(max(n, 1))
    ms = np.zeros(max(n, 1))
    _dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().gz_schedule_times(*args, orders.ctypes.data_as(_i32p), cost.ctypes.data_as(_dp),
                                   ms.ctypes.data_as(_dp), n, ctypes.byref(cnt)), "gz_schedule_times")
    return [{"order": orders[i].tolist(), "est_cost": float(cost[i]), "ms": float(ms[i])}
            for i in range(n)]


def plan_measured(adj, graph: "Graph", samples, orientation: bool = True, stream=None):
    """The fastest distinct schedule of the pattern on graph, timed on the root
    ranges samples = [(lo, hi), ...]; returns (Plan, best_ms, model_ms)."""
    a, k = _adj(adj)
    lo, hi = _ranges(samples)
    h = _P()
    best, model = ctypes.c_double(), ctypes.c_double()
    _check(lib().gz_plan_create_measured(k, a.ctypes.data_as(_u8p), graph.handle, int(orientation),
                                         lo.ctypes.data_as(_i64p), hi.ctypes.data_as(_i64p), len(samples),
                                         _stream(stream), ctypes.byref(h), ctypes.byref(best),
                                         ctypes.byref(model)), "gz_plan_create_measured")
    p = Plan.__new__(Plan)
    p._a = a
    p.handle = h
    return p, best.value, model.value


def schedules(adj) -> np.ndarray:
    """Algorithm 4's distinct schedules (labels), in generation order."""
    a, k = _adj(adj)
    cnt = ctypes.c_int()
    _check(lib().gz_plan_schedules(k, a.ctypes.data_as(_u8p), None, 0, ctypes.byref(cnt)))
    out = np.zeros((max(cnt.value, 1), k), dtype=np.int32)
    _check(lib().gz_plan_schedules(k, a.ctypes.data_as(_u8p), out.ctypes.data_as(_i32p), cnt.value,
                                   ctypes.byref(cnt)))
    return out[: cnt.value]


# ------------------------------------------------------------------ graphs

class Graph:
    """A device-resident graph (gz_graph)."""

    def __init__(self, row_ptr, col, n: int | None = None, validate: int = GZ_VALIDATE, stream=None):
        """row_ptr/col: host numpy arrays (copied) or CUDA torch tensors (borrowed)."""
        dev = hasattr(row_ptr, "is_cuda") and row_ptr.is_cuda
        if dev:
            assert str(row_ptr.dtype) == "torch.int64" and str(col.dtype) == "torch.int32"
            self._keep = (row_ptr, col)
            rp_ptr, col_ptr = row_ptr.data_ptr(), col.data_ptr()
            n = row_ptr.numel() - 1
            nnz = col.numel()
        else:
            rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
            cl = np.ascontiguousarray(col, dtype=np.int32)
            if cl.size == 0:
                cl = np.zeros(1, dtype=np.int32)
            self._keep = (rp, cl)
            rp_ptr, col_ptr = rp.ctypes.data, cl.ctypes.data
            n = rp.shape[0] - 1
            nnz = int(np.asarray(col).shape[0])
        h = _P()
        _check(lib().gz_load_csr(rp_ptr, col_ptr, n, nnz, 1 if dev else 0, validate, _stream(stream),
                                 ctypes.byref(h)), "gz_load_csr")
        self.handle = h
        self.n, self.nnz = n, nnz
        if not dev:
            self._keep = None  # host arrays were copied

    @classmethod
    def from_csr(cls, csr, validate: int = GZ_VALIDATE, stream=None) -> "Graph":
        return cls(csr.row_ptr, csr.col, validate=validate, stream=stream)

    def orient(self, stream=None) -> "Graph":
        _check(lib().gz_orient(self.handle, _stream(stream)), "gz_orient")
        return self

    def info(self) -> dict:
        st = GraphStats()
        _check(lib().gz_graph_info(self.handle, ctypes.byref(st)), "gz_graph_info")
        return {f: getattr(st, f) for f, _ in GraphStats._fields_}

    def export(self, oriented: bool = False, stream=None):
        rp = np.zeros(self.n + 1, dtype=np.int64)
        col = np.zeros(max(self.nnz, 1), dtype=np.int32)
        nid = np.zeros(max(self.n, 1), dtype=np.int32)
        _check(lib().gz_graph_export(self.handle, int(oriented), rp.ctypes.data_as(_i64p),
                                     col.ctypes.data_as(_i32p),
                                     nid.ctypes.data_as(_i32p) if oriented else None,
                                     _stream(stream)), "gz_graph_export")
        return rp, col[: self.nnz], (nid[: self.n] if oriented else None)

    def close(self):
        if getattr(self, "handle", None):
            lib().gz_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ counting

def count(plan: Plan, graph: Graph, orientation: bool = False, root_lo: int = 0, root_hi: int = -1,
          block_warps: int = 0, chunk: int = 0, stream=None, split_min: int = 0, split_chunk: int = 0) -> int:
    """Exact number of vertex-induced instances of the plan's pattern."""
    o = CountOpts(int(orientation), root_lo, root_hi, block_warps, chunk, split_min, split_chunk)
    out = ctypes.c_uint64()
    _check(lib().gz_count_ex(plan.handle, graph.handle, ctypes.byref(o), _stream(stream),
                             ctypes.byref(out)), "gz_count")
    return out.value


def prepare(plan: Plan, graph: Graph, orientation: bool = False, stream=None) -> None:
    """gz_prepare: build the cached device state counts of this plan read (views,
    clique rows), so that a later count does only the counting."""
    _check(lib().gz_prepare(plan.handle, graph.handle, int(orientation), _stream(stream)), "gz_prepare")


def count_noalloc(plan: Plan, graph: Graph, orientation: bool = False, stream=None) -> int:
    """gz_count_noalloc: the same count without any device allocation (see include/gz.h)."""
    out = ctypes.c_uint64()
    _check(lib().gz_count_noalloc(plan.handle, graph.handle, int(orientation), _stream(stream),
                                  ctypes.byref(out)), "gz_count_noalloc")
    return out.value


def scratch_bytes(plan: Plan, graph: Graph, orientation: bool = False) -> int:
    out = ctypes.c_uint64()
    _check(lib().gz_scratch_bytes(plan.handle, graph.handle, int(orientation), ctypes.byref(out)))
    return out.value


def count_batch(plans, graphs, orientation, stream=None) -> list[int]:
    nq = len(plans)
    P = (_P * nq)(*[p.handle for p in plans])
    G = (_P * nq)(*[g.handle for g in graphs])
    O = (ctypes.c_int * nq)(*[int(o) for o in orientation])
    out = (ctypes.c_uint64 * nq)()
    _check(lib().gz_count_batch(P, G, O, nq, _stream(stream), out), "gz_count_batch")
    return list(out)


def count_batch_ranges(plans, graphs, orientation, ranges, stream=None) -> list[int]:
    """gz_count_batch_ranges: query i counts the roots in ranges[i] = (lo, hi)."""
    nq = len(plans)
    P = (_P * nq)(*[p.handle for p in plans])
    G = (_P * nq)(*[g.handle for g in graphs])
    O = (ctypes.c_int * nq)(*[int(o) for o in orientation])
    lo = (ctypes.c_int64 * nq)(*[int(r[0]) for r in ranges])
    hi = (ctypes.c_int64 * nq)(*[int(r[1]) for r in ranges])
    out = (ctypes.c_uint64 * nq)()
    _check(lib().gz_count_batch_ranges(P, G, O, lo, hi, nq, _stream(stream), out), "gz_count_batch_ranges")
    return list(out)


def count_merged(plans, graph: Graph, orientation: bool = False, stream=None) -> list[int]:
    """gz_count_merged: the counts of several patterns in one graph, counted by one
    merged program (shared loop-1 sets, one pass over the edges)."""
    n = len(plans)
    P = (_P * max(n, 1))(*[p.handle for p in plans])
    out = np.zeros(max(n, 1), dtype=np.uint64)
    _check(lib().gz_count_merged(P, n, graph.handle, int(orientation), _stream(stream),
                                 out.ctypes.data_as(_u64p)), "gz_count_merged")
    return [int(x) for x in out[:n]]


def autotune(plan: Plan, graph: Graph, orientation: bool = False, stream=None) -> dict:
    """gz_autotune: the launch settings chosen for (plan, graph, orientation)."""
    bw, ch = ctypes.c_int(), ctypes.c_int()
    sm, sc = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().gz_autotune(plan.handle, graph.handle, int(orientation), _stream(stream),
                             ctypes.byref(bw), ctypes.byref(ch), ctypes.byref(sm), ctypes.byref(sc)),
           "gz_autotune")
    return {"block_warps": bw.value, "chunk": ch.value, "split_min": sm.value, "split_chunk": sc.value}


def motif_patterns(k: int) -> list:
    """Every connected k-vertex pattern up to isomorphism (gz_motif_patterns)."""
    cnt = ctypes.c_int()
    _check(lib().gz_motif_patterns(k, None, 0, ctypes.byref(cnt)), "gz_motif_patterns")
    buf = np.zeros(max(cnt.value, 1) * k * k, dtype=np.uint8)
    _check(lib().gz_motif_patterns(k, buf.ctypes.data_as(_u8p), cnt.value, ctypes.byref(cnt)),
           "gz_motif_patterns")
    return [buf[i * k * k:(i + 1) * k * k].reshape(k, k).copy() for i in range(cnt.value)]


def count_motifs(graph: Graph, k: int, orientation: bool = False, stream=None) -> list[int]:
    """Exact counts of every connected k-vertex pattern, in motif_patterns(k) order."""
    cnt = ctypes.c_int()
    _check(lib().gz_count_motifs(graph.handle, k, int(orientation), _stream(stream), None, 0,
                                 ctypes.byref(cnt)), "gz_count_motifs")
    out = (ctypes.c_uint64 * max(cnt.value, 1))()
    _check(lib().gz_count_motifs(graph.handle, k, int(orientation), _stream(stream), out, cnt.value,
                                 ctypes.byref(cnt)), "gz_count_motifs")
    return list(out)[: cnt.value]


class Server:
    """Continuous-batching request loop (gz_server)."""

    def __init__(self, max_inflight: int = 4, max_batch: int = 64, scratch_budget: int = 0,
                 heavy_ms: float = 0.0, slow_share: float = 0.0):
        o = ServerOpts(max_inflight, max_batch, scratch_budget, heavy_ms, slow_share)
        h = _P()
        _check(lib().gz_server_create(ctypes.byref(o), ctypes.byref(h)), "gz_server_create")
        self.handle = h

    def submit(self, plan: Plan, graph: Graph, orientation: bool = False) -> int:
        t = ctypes.c_int64()
        _check(lib().gz_server_submit(self.handle, plan.handle, graph.handle, int(orientation),
                                      ctypes.byref(t)), "gz_server_submit")
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        c, lat = ctypes.c_uint64(), ctypes.c_int64()
        _check(lib().gz_server_wait(self.handle, ticket, timeout_ms, ctypes.byref(c),
                                    ctypes.byref(lat)), "gz_server_wait")
        return c.value, lat.value

    def replay(self, plans, graphs, orientation, arrival_ns, plan_idx, graph_idx, fifo=False):
        n = len(arrival_ns)
        P = (_P * len(plans))(*[p.handle for p in plans])
        G = (_P * len(graphs))(*[g.handle for g in graphs])
        O = (ctypes.c_int * max(n, 1))(*[int(o) for o in orientation])
        arr = np.ascontiguousarray(arrival_ns, dtype=np.int64)
        pi = np.ascontiguousarray(plan_idx, dtype=np.int32)
        gi = np.ascontiguousarray(graph_idx, dtype=np.int32)
        counts = np.zeros(max(n, 1), dtype=np.uint64)
        lat = np.zeros(max(n, 1), dtype=np.int64)
        stats = (ctypes.c_double * 4)()
        _check(lib().gz_server_replay(self.handle, P, G, O, n, arr.ctypes.data_as(_i64p),
                                      pi.ctypes.data_as(_i32p), gi.ctypes.data_as(_i32p), int(fifo),
                                      counts.ctypes.data_as(_u64p), lat.ctypes.data_as(_i64p), stats),
               "gz_server_replay")
        return counts[:n], lat[:n], {"achieved_rps": stats[0], "max_queue": stats[1],
                                     "launches": stats[2], "wall_s": stats[3]}

    def close(self):
        if getattr(self, "handle", None):
            lib().gz_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
