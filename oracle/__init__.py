"""CPU oracle for cooperative BFS / SSSP.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / reference leg may import this package; the product path never
does.  It shares no code with the CUDA path (separate C file, separate build, no
common headers); the only shared module is :mod:`graphgen`, which generates inputs.

What it computes (Sorensen, Evrard and Donaldson, "Cooperative Kernels", FSE 2017):

* Sec. 2.2 Fig. 3 / Sec. 3.2 Fig. 4 - frontier graph traversal.  Under any schedule of
  kills and forks the cooperative kernel must produce what the plain kernel produces
  (Sec. 3.1: offer_kill may always be a no-op, request_fork may always return k = 0),
  and the plain level-synchronous traversal produces the textbook result.  So the
  oracle is that textbook result: FIFO-queue BFS levels (:func:`bfs`) and shortest
  distances by Dijkstra (:func:`dijkstra`), with Bellman-Ford (:func:`bellman_ford`)
  and Floyd-Warshall / simple-path enumeration as independent brute-force definitions.
* Table 1 names the Lonestar "l-sssp" application but not its algorithm; the result is
  the unique shortest-distance vector whatever the relaxation order.
* :mod:`oracle.semantics` models the programming model itself (Sec. 3.1 and the
  operational rules of Appendix A) for checking the runtime's kill / fork bookkeeping.

Conventions (readings of what the paper leaves unstated): unreached BFS level is -1
(int32); unreached distance is 0xFFFFFFFF (uint32); weights are uint32 and distances
are accumulated in uint64 and must stay below 2^32 - 1.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, brute force, scipy's Dijkstra, hand-checked special cases); none is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from itertools import permutations

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

UNREACHED_LEVEL = -1
UNREACHED_DIST = 0xFFFFFFFF


def build_library(force: bool = False, extra_flags=(), out: str | None = None) -> str:
    """Compile oracle.c with gcc (-O2).  ``extra_flags``/``out`` let tests build variants."""
    target = out or _LIB
    if force or out or not os.path.exists(target) or os.path.getmtime(target) < os.path.getmtime(_SRC):
        tmp = target + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", *extra_flags,
                               "-o", tmp, _SRC])
        os.replace(tmp, target)
    return target


def _declare(lib):
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
    u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
    lib.oracle_bfs.restype = ctypes.c_int64
    lib.oracle_bfs.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32, i32p]
    lib.oracle_dijkstra.restype = ctypes.c_int64
    lib.oracle_dijkstra.argtypes = [ctypes.c_int32, i32p, i32p, u32p, ctypes.c_int32, u32p]
    lib.oracle_bellman_ford.restype = ctypes.c_int64
    lib.oracle_bellman_ford.argtypes = [ctypes.c_int32, i32p, i32p, u32p, ctypes.c_int32, u32p]
    lib.oracle_floyd_warshall.restype = ctypes.c_int
    lib.oracle_floyd_warshall.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_void_p, u64p]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build_library()))
    return _lib


def load_variant(path: str):
    """Load a separately compiled oracle library (used to plant mistakes in tests)."""
    return _declare(ctypes.CDLL(path))


def _csr(g):
    return (np.ascontiguousarray(g.row_off, dtype=np.int32),
            np.ascontiguousarray(g.col if g.num_edges else np.zeros(1, np.int32), dtype=np.int32))


def _w(w, g):
    w = np.ascontiguousarray(w, dtype=np.uint32)
    return w if g.num_edges else np.zeros(1, np.uint32)


def bfs(g, src: int, lib=None) -> np.ndarray:
    """level[v] = fewest edges on a directed path src -> v; -1 if unreachable."""
    lib = lib or _load()
    ro, col = _csr(g)
    level = np.empty(g.num_vertices, dtype=np.int32)
    if lib.oracle_bfs(g.num_vertices, ro, col, src, level) < 0:
        raise ValueError("oracle_bfs: bad input")
    return level


def dijkstra(g, w, src: int, lib=None) -> np.ndarray:
    """dist[v] = least total weight of a path src -> v; 0xFFFFFFFF if unreachable."""
    lib = lib or _load()
    ro, col = _csr(g)
    dist = np.empty(g.num_vertices, dtype=np.uint32)
    rc = lib.oracle_dijkstra(g.num_vertices, ro, col, _w(w, g), src, dist)
    if rc == -2:
        raise OverflowError("a shortest distance does not fit below 2^32-1")
    if rc < 0:
        raise ValueError("oracle_dijkstra: bad input")
    return dist


def bellman_ford(g, w, src: int, lib=None) -> np.ndarray:
    """Independent second definition of the shortest distances (CLRS 24.1)."""
    lib = lib or _load()
    ro, col = _csr(g)
    dist = np.empty(g.num_vertices, dtype=np.uint32)
    rc = lib.oracle_bellman_ford(g.num_vertices, ro, col, _w(w, g), src, dist)
    if rc == -2:
        raise OverflowError("a shortest distance does not fit below 2^32-1")
    if rc < 0:
        raise ValueError("oracle_bellman_ford: bad input")
    return dist


def floyd_warshall(g, w=None, lib=None) -> np.ndarray:
    """All-pairs shortest path matrix (uint64, UINT64_MAX = unreachable); hop counts if w is None."""
    lib = lib or _load()
    V = g.num_vertices
    ro, col = _csr(g)
    D = np.empty(V * V, dtype=np.uint64)
    wk = None if w is None else _w(w, g)  # keep the array alive across the call
    wp = None if wk is None else wk.ctypes.data_as(ctypes.c_void_p)
    if lib.oracle_floyd_warshall(V, ro, col, wp, D) != 0:
        raise ValueError("oracle_floyd_warshall: bad input")
    return D.reshape(V, V)


def brute_force_paths(g, src: int, w=None):
    """Minimum over *every* simple path from src (explicit enumeration; V <= 8).

    Returns (hops, cost) lists with None for unreachable vertices.  Pure Python, used
    only to pin the fast definitions on tiny graphs.
    """
    V = g.num_vertices
    if V > 8:
        raise ValueError("brute force is for V <= 8")
    adj = {}
    for u in range(V):
        for e in range(g.row_off[u], g.row_off[u + 1]):
            adj[(u, int(g.col[e]))] = 1 if w is None else int(w[e])
    hops = [None] * V
    cost = [None] * V
    hops[src] = 0
    cost[src] = 0
    others = [v for v in range(V) if v != src]
    for length in range(1, V):
        for seq in permutations(others, length):
            path = (src,) + seq
            c = 0
            ok = True
            for a, b in zip(path, path[1:]):
                if (a, b) not in adj:
                    ok = False
                    break
                c += adj[(a, b)]
            if not ok:
                continue
            t = path[-1]
            if hops[t] is None or length < hops[t]:
                hops[t] = length
            if cost[t] is None or c < cost[t]:
                cost[t] = c
    return hops, cost


def traversal_work(g, reached_mask: np.ndarray):
    """(V_r, E_s): reached vertices and the out-edges they own (the TEPS numerator)."""
    deg = g.out_degree()
    return int(reached_mask.sum()), int(deg[reached_mask].sum())


def check_bfs_invariants(g, src: int, level: np.ndarray) -> None:
    """Properties any correct BFS level vector has on a directed graph (raises on failure).

    level[src] = 0; for every edge (u, v) with u reached, v is reached and
    level[v] <= level[u] + 1; every reached v != src has an in-edge from level[v] - 1;
    unreached vertices are exactly -1.
    """
    level = np.asarray(level, dtype=np.int64)
    V = g.num_vertices
    if level[src] != 0:
        raise AssertionError("level[src] != 0")
    if np.any((level < -1)):
        raise AssertionError("level below -1")
    u = np.repeat(np.arange(V), g.out_degree())
    v = g.col.astype(np.int64)
    lu, lv = level[u], level[v]
    reached_u = lu >= 0
    if np.any(reached_u & (lv < 0)):
        raise AssertionError("edge from a reached vertex to an unreached one")
    if np.any(reached_u & (lv > lu + 1)):
        raise AssertionError("edge (u,v) with level[v] > level[u] + 1")
    tight = reached_u & (lv == lu + 1)
    has_parent = np.zeros(V, dtype=bool)
    has_parent[v[tight]] = True
    has_parent[src] = True
    if np.any((level >= 0) & ~has_parent):
        raise AssertionError("reached vertex without a parent one level up")


def check_sssp_fixed_point(g, w, src: int, dist: np.ndarray) -> None:
    """Shortest distances are a fixed point of one more relaxation round (raises on failure).

    dist[src] = 0; for every edge (u, v) with u reached, dist[v] <= dist[u] + w(u, v);
    every reached v != src has a tight in-edge dist[v] = dist[u] + w(u, v).
    """
    d = np.asarray(dist, dtype=np.uint64)
    V = g.num_vertices
    inf = np.uint64(UNREACHED_DIST)
    if d[src] != 0:
        raise AssertionError("dist[src] != 0")
    u = np.repeat(np.arange(V), g.out_degree())
    v = g.col.astype(np.int64)
    wu = np.asarray(w, dtype=np.uint64)
    du, dv = d[u], d[v]
    reached_u = du != inf
    cand = du + wu
    if np.any(reached_u & (dv > cand)):
        raise AssertionError("a relaxation would still lower some distance")
    tight = reached_u & (dv == cand)
    has_parent = np.zeros(V, dtype=bool)
    has_parent[v[tight]] = True
    has_parent[src] = True
    if np.any((d != inf) & ~has_parent):
        raise AssertionError("reached vertex without a tight in-edge")
