"""Python binding of libcoop.so: cooperative BFS / SSSP on GB300 (argument marshalling only).

Every function here has the name of the C entry point it wraps (``include/coop.h``)
and does nothing but check and convert arguments; all work runs in the CUDA kernels
of the shared library.  Device buffers are passed as torch CUDA tensors (only
``data_ptr()``, ``dtype``, ``numel()`` and ``is_cuda`` are used) or as raw integer
device addresses.  Streams are ``torch.cuda.Stream`` objects, raw ``cudaStream_t``
integers, or ``None`` for torch's current stream.

The library is loaded on first use; if it cannot be built or loaded the call raises
:class:`CoopUnavailable` -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import threading

from . import _build

__all__ = [
    "CoopError", "CoopUnavailable", "Stats", "CSR", "coop_init", "coop_destroy", "coop_bfs", "coop_sssp",
    "coop_sssp_topo", "coop_octree",
    "coop_request_resources", "coop_release", "coop_sync", "coop_get_stats", "coop_get_resize_log",
    "coop_get_request_log", "REQUEST_FIELDS",
    "coop_set_schedule", "coop_set_timeout", "coop_set_timing", "coop_set_kill_mode", "COOP_KILL_CHUNK",
    "COOP_KILL_QUERY", "COOP_KILL_SIMPLE", "coop_query", "coop_bfs_baseline", "coop_sssp_baseline",
    "coop_barrier_bench", "coop_saxpy", "coop_bfs_noalloc", "coop_status_string", "Job", "Batch", "make_job",
    "coop_batch_create", "coop_batch_set_ctas", "coop_batch_tune", "coop_batch_run", "coop_batch_get_stats",
    "coop_batch_destroy", "coop_last_cuda_error", "library_path", "load_library", "Server", "QueryResult",
    "coop_server_create", "coop_server_add_graph", "coop_server_submit", "coop_server_wait",
    "coop_server_request_resources", "coop_server_release", "coop_server_destroy",
]

COOP_OK, COOP_EINVAL, COOP_ENOMEM, COOP_ECUDA = 0, -1, -2, -3
COOP_ETIMEOUT, COOP_EBUSY, COOP_EOVERFLOW, COOP_EGRAPH = -4, -5, -6, -7


class CoopUnavailable(RuntimeError):
    """libcoop.so could not be built or loaded (no CPU fallback exists)."""


class CoopError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {coop_status_string(status)} ({status})"
        if status == COOP_ECUDA:
            msg += f" [{coop_last_cuda_error()}]"
        super().__init__(msg)


class CSR(ctypes.Structure):
    """coop_csr: V, E and device pointers row_off[V+1], col[E]."""
    _fields_ = [("num_vertices", ctypes.c_int32), ("num_edges", ctypes.c_int64),
                ("row_off", ctypes.c_void_p), ("col", ctypes.c_void_p)]


class Job(ctypes.Structure):
    """coop_job: one traversal of a batch (device pointers)."""
    _fields_ = [("graph", CSR), ("d_weights", ctypes.c_void_p), ("source", ctypes.c_int32),
                ("kind", ctypes.c_int32), ("d_out", ctypes.c_void_p)]


COOP_JOB_BFS, COOP_JOB_SSSP = 0, 1


class Stats(ctypes.Structure):
    """coop_stats (see include/coop.h)."""
    _fields_ = [("levels", ctypes.c_int32), ("barriers", ctypes.c_int32), ("kills", ctypes.c_int32),
                ("forks", ctypes.c_int32), ("min_active", ctypes.c_int32), ("max_active", ctypes.c_int32),
                ("initial_active", ctypes.c_int32), ("status", ctypes.c_int32),
                ("ctas_launched", ctypes.c_int32), ("joined", ctypes.c_int32),
                ("edges_scanned", ctypes.c_int64), ("frontier_total", ctypes.c_int64),
                ("vertices_reached", ctypes.c_int64), ("reached_edges", ctypes.c_int64),
                ("gather_us_max", ctypes.c_double), ("kernel_us", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class QueryResult(ctypes.Structure):
    """coop_query_result: one served query's outcome."""
    _fields_ = [("status", ctypes.c_int32), ("slot", ctypes.c_int32), ("ctas", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("queue_us", ctypes.c_double), ("latency_us", ctypes.c_double),
                ("stats", Stats)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load_library():
    """Build (if stale) and load libcoop.so; raises CoopUnavailable on failure."""
    global _lib
    with _lock:
        if _lib is None:
            try:
                path = _build.build_library()
                lib = ctypes.CDLL(path)
            except Exception as exc:  # no fallback: fail loudly
                raise CoopUnavailable(f"libcoop.so unavailable: {exc}") from exc
            vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
            ip = ctypes.POINTER(ctypes.c_int)
            sp = ctypes.POINTER(Stats)
            cp = ctypes.POINTER(CSR)
            sig = {
                "coop_init": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)],
                "coop_destroy": [vp],
                "coop_bfs": [vp, cp, i32, vp, vp, sp],
                "coop_sssp": [vp, cp, vp, i32, vp, vp, sp],
                "coop_sssp_topo": [vp, cp, vp, i32, vp, vp, sp],
                "coop_octree": [vp, vp, vp, vp, i32, i32, i32, vp, vp, vp, i32, vp, vp, vp, sp],
                "coop_bfs_baseline": [vp, cp, i32, vp, vp, sp],
                "coop_sssp_baseline": [vp, cp, vp, i32, vp, vp, sp],
                "coop_request_resources": [vp, ctypes.c_int, ctypes.c_int, ip],
                "coop_release": [vp, ctypes.c_int],
                "coop_sync": [vp],
                "coop_get_stats": [vp, sp],
                "coop_get_resize_log": [vp, ctypes.POINTER(i32), ctypes.c_int, ip],
                "coop_get_request_log": [vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ip, ctypes.c_int],
                "coop_set_schedule": [vp, u64, ctypes.c_double, ctypes.c_double],
                "coop_set_timeout": [vp, i64],
                "coop_set_timing": [vp, ctypes.c_int],
                "coop_set_kill_mode": [vp, ctypes.c_int],
                "coop_query": [vp, ip, ip, ip, ip],
                "coop_barrier_bench": [vp, i32, i32, vp, sp],
                "coop_saxpy": [ctypes.c_int, i64, ctypes.c_float, vp, vp, vp],
                "coop_bfs_noalloc": [cp, i32, vp, vp, vp],
                "coop_batch_create": [vp, ctypes.POINTER(Job), ctypes.c_int, ctypes.POINTER(vp)],
                "coop_batch_set_ctas": [vp, ctypes.POINTER(i32)],
                "coop_batch_tune": [vp, vp, ctypes.POINTER(i32)],
                "coop_batch_run": [vp, vp, ctypes.c_int],
                "coop_batch_get_stats": [vp, sp],
                "coop_batch_destroy": [vp],
                "coop_server_create": [ctypes.c_int, ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(vp)],
                "coop_server_add_graph": [vp, cp, vp, ip],
                "coop_server_submit": [vp, ctypes.c_int, ctypes.c_int, i32, vp, ctypes.POINTER(u64)],
                "coop_server_wait": [vp, u64, ctypes.c_int, ctypes.POINTER(QueryResult)],
                "coop_server_request_resources": [vp, ctypes.c_int, ctypes.c_int, ip],
                "coop_server_release": [vp, ctypes.c_int],
                "coop_server_destroy": [vp],
            }
            for name, args in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            lib.coop_last_cuda_error.argtypes = []
            lib.coop_last_cuda_error.restype = ctypes.c_char_p
            lib.coop_status_string.argtypes = [ctypes.c_int]
            lib.coop_status_string.restype = ctypes.c_char_p
            _lib = lib
    return _lib


def coop_last_cuda_error() -> str:
    try:
        return load_library().coop_last_cuda_error().decode()
    except CoopUnavailable:
        return ""


def coop_status_string(status: int) -> str:
    try:
        return load_library().coop_status_string(int(status)).decode()
    except CoopUnavailable:
        return f"status {status}"


def _check(status: int, where: str, ok=(COOP_OK,)) -> int:
    if status not in ok:
        raise CoopError(status, where)
    return status


def _ptr(x, dtype_name: str | None = None, numel: int | None = None, what: str = "buffer") -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if not getattr(x, "is_cuda", False):
        raise ValueError(f"{what} must be a CUDA tensor or a device address")
    if dtype_name is not None and str(x.dtype) != dtype_name:
        raise ValueError(f"{what} must have dtype {dtype_name}, got {x.dtype}")
    if numel is not None and x.numel() < numel:
        raise ValueError(f"{what} needs {numel} elements, has {x.numel()}")
    if hasattr(x, "is_contiguous") and not x.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return int(x.data_ptr())


def _stream(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def make_csr(row_off, col, num_vertices: int | None = None) -> CSR:
    """coop_csr from device tensors row_off (int32[V+1]) and col (int32[E])."""
    V = (row_off.numel() - 1) if num_vertices is None else num_vertices
    E = col.numel() if not isinstance(col, int) else 0
    return CSR(V, E, _ptr(row_off, "torch.int32", V + 1, "row_off"),
               _ptr(col, "torch.int32", None, "col") if E else 0)


class Context:
    """Owns a coop_ctx pointer; closes it on destroy / garbage collection."""

    def __init__(self, handle: int):
        self.handle = handle

    def __del__(self):
        try:
            coop_destroy(self)
        except Exception:
            pass


def _h(ctx) -> int:
    h = ctx.handle if isinstance(ctx, Context) else ctx
    if not h:
        raise ValueError("context is closed")
    return h


def coop_init(device: int = 0, max_ctas: int = 0, threads_per_cta: int = 0) -> Context:
    lib = load_library()
    out = ctypes.c_void_p()
    _check(lib.coop_init(device, max_ctas, threads_per_cta, ctypes.byref(out)), "coop_init")
    return Context(out.value)


def coop_destroy(ctx) -> None:
    if isinstance(ctx, Context):
        if ctx.handle:
            h, ctx.handle = ctx.handle, 0
            load_library().coop_destroy(h)
    elif ctx:
        load_library().coop_destroy(ctx)


def _stats_ptr(want):
    if not want:
        return None, None
    s = Stats()
    return s, ctypes.byref(s)


def coop_bfs(ctx, g: CSR, source: int, levels, stream=None, stats: bool = False, ok=(COOP_OK,)):
    """BFS levels into `levels` (int32[V] device).  Returns Stats when stats=True."""
    s, sp = _stats_ptr(stats)
    st = load_library().coop_bfs(_h(ctx), ctypes.byref(g), int(source),
                                 _ptr(levels, "torch.int32", g.num_vertices, "levels"), _stream(stream), sp)
    _check(st, "coop_bfs", ok)
    return s


def coop_sssp(ctx, g: CSR, weights, source: int, dist, stream=None, stats: bool = False, ok=(COOP_OK,)):
    """Shortest distances into `dist` (int32/uint32[V] device viewed as uint32)."""
    s, sp = _stats_ptr(stats)
    st = load_library().coop_sssp(_h(ctx), ctypes.byref(g), _ptr(weights, None, g.num_edges, "weights"),
                                  int(source), _ptr(dist, None, g.num_vertices, "dist"), _stream(stream), sp)
    _check(st, "coop_sssp", ok)
    return s


def coop_sssp_topo(ctx, g: CSR, weights, source: int, dist, stream=None, stats: bool = False, ok=(COOP_OK,)):
    """Topology-driven SSSP (p-sssp): same result as coop_sssp."""
    s, sp = _stats_ptr(stats)
    st = load_library().coop_sssp_topo(_h(ctx), ctypes.byref(g), _ptr(weights, None, g.num_edges, "weights"),
                                       int(source), _ptr(dist, None, g.num_vertices, "dist"), _stream(stream), sp)
    _check(st, "coop_sssp_topo", ok)
    return s


def coop_octree(ctx, x, y, z, leaf_cap: int, max_depth: int, leaf_code, leaf_begin, leaf_count, perm, n_leaves,
                stream=None, stats: bool = False, ok=(COOP_OK,)):
    """Octree partitioning of the points (x, y, z) (uint32 device tensors, coordinates
    below 2^21); leaves into leaf_code (int64/uint64), leaf_begin, leaf_count, perm
    (int32/uint32) and n_leaves (one int32).  See include/coop.h."""
    n = x.numel()
    s, sp = _stats_ptr(stats)
    st = load_library().coop_octree(
        _h(ctx), _ptr(x, None, n, "x"), _ptr(y, None, n, "y"), _ptr(z, None, n, "z"), int(n), int(leaf_cap),
        int(max_depth), _ptr(leaf_code, None, 0, "leaf_code"), _ptr(leaf_begin, None, 0, "leaf_begin"),
        _ptr(leaf_count, None, 0, "leaf_count"), int(leaf_code.numel()), _ptr(perm, None, n, "perm"),
        _ptr(n_leaves, None, 1, "n_leaves"), _stream(stream), sp)
    _check(st, "coop_octree", ok)
    return s


def coop_bfs_baseline(ctx, g: CSR, source: int, levels, stream=None, stats: bool = False, ok=(COOP_OK,)):
    s, sp = _stats_ptr(stats)
    st = load_library().coop_bfs_baseline(_h(ctx), ctypes.byref(g), int(source),
                                          _ptr(levels, "torch.int32", g.num_vertices, "levels"),
                                          _stream(stream), sp)
    _check(st, "coop_bfs_baseline", ok)
    return s


def coop_sssp_baseline(ctx, g: CSR, weights, source: int, dist, stream=None, stats: bool = False,
                       ok=(COOP_OK,)):
    s, sp = _stats_ptr(stats)
    st = load_library().coop_sssp_baseline(_h(ctx), ctypes.byref(g), _ptr(weights, None, g.num_edges, "weights"),
                                           int(source), _ptr(dist, None, g.num_vertices, "dist"),
                                           _stream(stream), sp)
    _check(st, "coop_sssp_baseline", ok)
    return s


def coop_barrier_bench(ctx, n_barriers: int, never_arrive: int = 0, stream=None, stats: bool = True,
                       ok=(COOP_OK,)):
    s, sp = _stats_ptr(stats)
    st = load_library().coop_barrier_bench(_h(ctx), int(n_barriers), int(never_arrive), _stream(stream), sp)
    _check(st, "coop_barrier_bench", ok)
    return s if stats else st


def coop_request_resources(ctx, n_ctas: int, timeout_us: int = 0, ok=(COOP_OK,)) -> int:
    n = ctypes.c_int(0)
    st = load_library().coop_request_resources(_h(ctx), int(n_ctas), int(timeout_us), ctypes.byref(n))
    _check(st, "coop_request_resources", ok)
    return n.value


def coop_release(ctx, n_ctas: int) -> None:
    _check(load_library().coop_release(_h(ctx), int(n_ctas)), "coop_release")


def coop_sync(ctx, ok=(COOP_OK,)) -> int:
    return _check(load_library().coop_sync(_h(ctx)), "coop_sync", ok)


def coop_get_stats(ctx, ok=(COOP_OK,)) -> Stats:
    s = Stats()
    _check(load_library().coop_get_stats(_h(ctx), ctypes.byref(s)), "coop_get_stats", ok)
    return s


LOG_FIELDS = ("barrier", "t_us", "m_before", "k_forked", "w_killed", "m_after", "spawned", "edges")


def coop_get_resize_log(ctx, cap: int = 4096):
    """Barrier records of the last traversal: tuples in the order of LOG_FIELDS."""
    buf = (ctypes.c_int32 * (8 * cap))()
    n = ctypes.c_int(0)
    _check(load_library().coop_get_resize_log(_h(ctx), buf, cap, ctypes.byref(n)), "coop_get_resize_log")
    return [tuple(buf[8 * i: 8 * i + 8]) for i in range(n.value)]


REQUEST_FIELDS = ("t_us", "n_ctas", "active_at_post", "active_at_grant", "gather_us", "granted", "lock_us",
                  "post_us")


def coop_get_request_log(ctx, cap: int = 4096, clear: bool = True):
    """The context's coop_request_resources records, oldest first, as dicts of REQUEST_FIELDS."""
    k = len(REQUEST_FIELDS)
    buf = (ctypes.c_double * (k * cap))()
    n = ctypes.c_int(0)
    _check(load_library().coop_get_request_log(_h(ctx), buf, cap, ctypes.byref(n), 1 if clear else 0),
           "coop_get_request_log")
    return [dict(zip(REQUEST_FIELDS, buf[k * i: k * i + k])) for i in range(n.value)]


def coop_set_schedule(ctx, seed: int, p_kill: float, p_fork: float) -> None:
    _check(load_library().coop_set_schedule(_h(ctx), seed & 0xFFFFFFFFFFFFFFFF, float(p_kill), float(p_fork)),
           "coop_set_schedule")


def coop_set_timeout(ctx, timeout_us: int) -> None:
    _check(load_library().coop_set_timeout(_h(ctx), int(timeout_us)), "coop_set_timeout")


COOP_KILL_CHUNK, COOP_KILL_QUERY, COOP_KILL_SIMPLE = 0, 1, 2


def coop_set_kill_mode(ctx, mode: int) -> None:
    _check(load_library().coop_set_kill_mode(_h(ctx), int(mode)), "coop_set_kill_mode")


def coop_set_timing(ctx, on: bool = True) -> None:
    _check(load_library().coop_set_timing(_h(ctx), 1 if on else 0), "coop_set_timing")


def coop_query(ctx) -> dict:
    a, b, c, d = (ctypes.c_int(0) for _ in range(4))
    _check(load_library().coop_query(_h(ctx), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)),
           "coop_query")
    return {"max_ctas": a.value, "threads_per_cta": b.value, "sm_count": c.value, "lent": d.value}


def coop_bfs_noalloc(g: CSR, source: int, levels, status=None, stream=None) -> None:
    """Allocation-free BFS (static scratch, at most 2^20 vertices); asynchronous."""
    st = load_library().coop_bfs_noalloc(ctypes.byref(g), int(source),
                                         _ptr(levels, "torch.int32", g.num_vertices, "levels"),
                                         _ptr(status, "torch.int32", 1, "status"), _stream(stream))
    _check(st, "coop_bfs_noalloc")


class Batch:
    """Owns a coop_batch pointer and keeps the jobs' tensors alive."""

    def __init__(self, handle: int, n: int, keep):
        self.handle, self.n, self._keep = handle, n, keep

    def __del__(self):
        try:
            coop_batch_destroy(self)
        except Exception:
            pass


def make_job(g: CSR, source: int, out, weights=None) -> Job:
    """coop_job for a BFS (weights None) or SSSP traversal writing into `out` ([V] int32 tensor)."""
    kind = COOP_JOB_BFS if weights is None else COOP_JOB_SSSP
    return Job(g, _ptr(weights, None, g.num_edges, "weights") if weights is not None else 0, int(source), kind,
               _ptr(out, None, g.num_vertices, "out"))


def coop_batch_create(ctx, jobs, keep=None) -> Batch:
    arr = (Job * len(jobs))(*jobs)
    out = ctypes.c_void_p()
    _check(load_library().coop_batch_create(_h(ctx), arr, len(jobs), ctypes.byref(out)), "coop_batch_create")
    return Batch(out.value, len(jobs), keep)


def coop_batch_set_ctas(batch: Batch, ctas) -> None:
    arr = (ctypes.c_int32 * batch.n)(*[int(c) for c in ctas])
    _check(load_library().coop_batch_set_ctas(batch.handle, arr), "coop_batch_set_ctas")


def coop_batch_tune(batch: Batch, stream=None):
    arr = (ctypes.c_int32 * batch.n)()
    _check(load_library().coop_batch_tune(batch.handle, _stream(stream), arr), "coop_batch_tune")
    return list(arr)


def coop_batch_run(batch: Batch, stream=None, use_graph: bool = True) -> None:
    _check(load_library().coop_batch_run(batch.handle, _stream(stream), 1 if use_graph else 0), "coop_batch_run")


def coop_batch_get_stats(batch: Batch, ok=(COOP_OK,)):
    arr = (Stats * batch.n)()
    _check(load_library().coop_batch_get_stats(batch.handle, arr), "coop_batch_get_stats", ok)
    return list(arr)


def coop_batch_destroy(batch) -> None:
    if isinstance(batch, Batch):
        if batch.handle:
            h, batch.handle = batch.handle, 0
            load_library().coop_batch_destroy(h)
    elif batch:
        load_library().coop_batch_destroy(batch)


class Server:
    """Owns a coop_server pointer and the registered graphs' tensors."""

    def __init__(self, handle: int):
        self.handle, self._keep = handle, []

    def __del__(self):
        try:
            coop_server_destroy(self)
        except Exception:
            pass


def coop_server_create(device: int = 0, slots: int = 4, hbm_budget_bytes: int = 0) -> Server:
    out = ctypes.c_void_p()
    _check(load_library().coop_server_create(int(device), int(slots), int(hbm_budget_bytes), ctypes.byref(out)),
           "coop_server_create")
    return Server(out.value)


def coop_server_add_graph(sv: Server, g: CSR, weights=None, keep=()) -> int:
    gid = ctypes.c_int(-1)
    _check(load_library().coop_server_add_graph(sv.handle, ctypes.byref(g),
                                                _ptr(weights, None, g.num_edges, "weights") if weights is not None
                                                else None, ctypes.byref(gid)), "coop_server_add_graph")
    sv._keep.append((g, weights, keep))
    return gid.value


def coop_server_submit(sv: Server, graph_id: int, kind: int, source: int, out) -> int:
    t = ctypes.c_uint64(0)
    _check(load_library().coop_server_submit(sv.handle, int(graph_id), int(kind), int(source),
                                             _ptr(out, None, None, "out"), ctypes.byref(t)), "coop_server_submit")
    return t.value


def coop_server_wait(sv: Server, ticket: int, timeout_us: int = 0, ok=(COOP_OK,)) -> QueryResult:
    r = QueryResult()
    _check(load_library().coop_server_wait(sv.handle, ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(r)),
           "coop_server_wait", ok)
    return r


def coop_server_request_resources(sv: Server, n_ctas: int, timeout_us: int = 0, ok=(COOP_OK,)) -> int:
    n = ctypes.c_int(0)
    _check(load_library().coop_server_request_resources(sv.handle, int(n_ctas), int(timeout_us), ctypes.byref(n)),
           "coop_server_request_resources", ok)
    return n.value


def coop_server_release(sv: Server, n_ctas: int) -> None:
    _check(load_library().coop_server_release(sv.handle, int(n_ctas)), "coop_server_release")


def coop_server_destroy(sv) -> None:
    if isinstance(sv, Server):
        if sv.handle:
            h, sv.handle = sv.handle, 0
            load_library().coop_server_destroy(h)
    elif sv:
        load_library().coop_server_destroy(sv)


def coop_saxpy(n_ctas: int, a: float, x, y, stream=None) -> None:
    n = x.numel() if not isinstance(x, int) else None
    if n is None:
        raise ValueError("pass tensors to coop_saxpy")
    _check(load_library().coop_saxpy(int(n_ctas), int(n), float(a), _ptr(x, "torch.float32", n, "x"),
                                     _ptr(y, "torch.float32", n, "y"), _stream(stream)), "coop_saxpy")
