"""Seeded synthetic graph inputs shared by the CPU oracle and the CUDA path.

This module only *generates inputs*: R-MAT and grid CSR graphs, small random or
hand-shaped graphs for edge cases, per-edge weights and the source-vertex rule.  It
contains none of the traversal arithmetic, so the oracle and the CUDA path can both
consume it without sharing any of the method's code.

The heavy lifting is in ``graphgen.c`` (compiled with gcc on first use, or by the
repository's ``build()``); every random draw is a SplitMix64 hash of
(seed, edge index, bit level), so a graph is a pure function of its parameters and
identical on x86 and Arm hosts.

Readings of unstated details (the paper publishes no generator):
  * R-MAT is directed as generated (not symmetrised), self-loops dropped, duplicates
    removed, rows sorted by column id; a/b/c/d = 0.57/0.19/0.19/0.05 by default.
  * The grid is 4-neighbour, undirected (both directions stored), without wraparound:
    a 256x256 grid has 4*256*255 = 261,120 directed edges.
  * Weights are uint32 in [1, 255], a hash of the edge (u, v) and the weight seed.
  * The source is the vertex of highest out-degree, ties broken by the smallest id.
"""
from __future__ import annotations

import ctypes
import functools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build_library(force: bool = False) -> str:
    """Compile graphgen.c into libgraphgen.so next to it (gcc, -O2, pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_library())
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
            lib.gg_splitmix64.restype = ctypes.c_uint64
            lib.gg_splitmix64.argtypes = [ctypes.c_uint64]
            lib.gg_rmat.restype = ctypes.c_int64
            lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.c_int, i32p, i32p]
            lib.gg_grid.restype = ctypes.c_int64
            lib.gg_grid.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p]
            lib.gg_edges_to_csr.restype = ctypes.c_int64
            lib.gg_edges_to_csr.argtypes = [ctypes.c_int32, ctypes.c_int64, u32p, u32p,
                                            ctypes.c_int, i32p, i32p]
            lib.gg_weights.restype = None
            lib.gg_weights.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_uint64,
                                       ctypes.c_uint32, ctypes.c_uint32, u32p]
            _lib = lib
    return _lib


def _threads(threads: int) -> int:
    return threads if threads > 0 else max(1, min(16, os.cpu_count() or 1))


class CSR:
    """A directed graph in int32 CSR form: row_off[V+1], col[E] (host, numpy)."""

    __slots__ = ("row_off", "col", "name")

    def __init__(self, row_off: np.ndarray, col: np.ndarray, name: str = ""):
        self.row_off = np.ascontiguousarray(row_off, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.name = name

    @property
    def num_vertices(self) -> int:
        return int(self.row_off.shape[0] - 1)

    @property
    def num_edges(self) -> int:
        return int(self.col.shape[0])

    def out_degree(self) -> np.ndarray:
        return np.diff(self.row_off.astype(np.int64))

    def __repr__(self) -> str:
        return f"CSR({self.name or '?'}, V={self.num_vertices}, E={self.num_edges})"


def splitmix64(x: int) -> int:
    return int(_load().gg_splitmix64(ctypes.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


@functools.lru_cache(maxsize=4)
def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 0, threads: int = 0) -> CSR:
    """Directed R-MAT graph with 2^scale vertices (deduplicated, no self-loops)."""
    V = 1 << scale
    m = edge_factor * V
    row_off = np.empty(V + 1, dtype=np.int32)
    col = np.empty(m, dtype=np.int32)
    E = _load().gg_rmat(scale, edge_factor, a, b, c, seed, _threads(threads), row_off, col)
    if E < 0:
        raise ValueError("gg_rmat failed")
    g = CSR(row_off, col[:E].copy(), f"rmat{scale}-ef{edge_factor}-s{seed}")
    for arr in (g.row_off, g.col):
        arr.setflags(write=False)
    return g


@functools.lru_cache(maxsize=4)
def grid(w: int, h: int) -> CSR:
    """w x h 4-neighbour grid, both directions stored, no wraparound; id = y*w + x."""
    V = w * h
    row_off = np.empty(V + 1, dtype=np.int32)
    col = np.empty(4 * V, dtype=np.int32)
    E = _load().gg_grid(w, h, row_off, col)
    g = CSR(row_off, col[:E].copy(), f"grid{w}x{h}")
    for arr in (g.row_off, g.col):
        arr.setflags(write=False)
    return g


def from_edges(num_vertices: int, src, dst, name: str = "") -> CSR:
    """CSR from an edge list: self-loops removed, duplicates removed, rows sorted."""
    src = np.ascontiguousarray(np.asarray(src, dtype=np.int64).astype(np.uint32))
    dst = np.ascontiguousarray(np.asarray(dst, dtype=np.int64).astype(np.uint32))
    if src.shape != dst.shape:
        raise ValueError("src and dst differ in length")
    if num_vertices < 1:
        raise ValueError("num_vertices must be >= 1")
    row_off = np.empty(num_vertices + 1, dtype=np.int32)
    col = np.empty(max(1, src.shape[0]), dtype=np.int32)
    E = _load().gg_edges_to_csr(num_vertices, src.shape[0], src, dst, 1, row_off, col)
    if E < 0:
        raise ValueError("edge endpoint out of range")
    return CSR(row_off, col[:E].copy(), name)


def random_graph(num_vertices: int, num_edges: int, seed: int, name: str = "") -> CSR:
    """Uniform random directed multigraph edges (then deduplicated) from numpy's PCG64."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, num_vertices, size=num_edges)
    dst = rng.integers(0, num_vertices, size=num_edges)
    return from_edges(num_vertices, src, dst, name or f"rand{num_vertices}-{num_edges}-s{seed}")


def path(n: int) -> CSR:
    return from_edges(n, np.arange(n - 1), np.arange(1, n), f"path{n}")


def star(n: int, undirected: bool = True) -> CSR:
    s = np.zeros(n - 1, dtype=np.int64)
    d = np.arange(1, n)
    if undirected:
        s, d = np.concatenate([s, d]), np.concatenate([d, s])
    return from_edges(n, s, d, f"star{n}")


def complete(n: int) -> CSR:
    s, d = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return from_edges(n, s.ravel(), d.ravel(), f"complete{n}")


def weights(g: CSR, seed: int, lo: int = 1, hi: int = 255) -> np.ndarray:
    """uint32 per-edge weights in [lo, hi], a hash of (seed, u, v)."""
    if not (0 <= lo <= hi <= 0xFFFFFFFF):
        raise ValueError("bad weight range")
    w = np.empty(max(1, g.num_edges), dtype=np.uint32)
    _load().gg_weights(g.num_vertices, g.row_off, g.col, seed, lo, hi, w)
    return w[: g.num_edges].copy()


def max_out_degree_vertex(g: CSR) -> int:
    """Source rule: the vertex of highest out-degree, ties to the smallest id."""
    return int(np.argmax(g.out_degree()))


def default_rmat_config(scale: int):
    """The R-MAT workloads: (graph seed, weight seed) per scale (20 -> 20/21, 22 -> 22/23)."""
    return scale, scale + 1


def points(n: int, seed: int, kind: str = "clustered"):
    """n points with integer coordinates in [0, 2^21)^3, the octree workload's input, as
    three uint32 arrays.  'uniform': independent uniform coordinates (a shallow, even
    tree); 'clustered': 16 Gaussian clusters with random centres and widths from 2^8 to
    2^18, clipped to the cube (deep, uneven trees, like the particle sets octrees are
    built for)."""
    rng = np.random.default_rng(seed)
    hi = 1 << 21
    if kind == "uniform":
        return tuple(rng.integers(0, hi, n, dtype=np.uint32) for _ in range(3))
    if kind != "clustered":
        raise ValueError(kind)
    k = 16
    centres = rng.integers(0, hi, (k, 3)).astype(np.float64)
    widths = 2.0 ** rng.uniform(8.0, 18.0, k)
    lab = rng.integers(0, k, n)
    pts = centres[lab] + rng.normal(0.0, 1.0, (n, 3)) * widths[lab, None]
    pts = np.clip(np.rint(pts), 0, hi - 1).astype(np.uint32)
    return np.ascontiguousarray(pts[:, 0]), np.ascontiguousarray(pts[:, 1]), np.ascontiguousarray(pts[:, 2])
