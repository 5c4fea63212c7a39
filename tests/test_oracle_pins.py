"""Pins for the CPU oracle against things other than itself.

Closed forms (grid levels), brute force on tiny graphs (every directed graph on 4
vertices, explicit simple-path enumeration), an independent library routine
(scipy.sparse.csgraph), hand-derived fixtures under tests/golden/, special cases and
invariants.  The last test plants plausible mistakes into a copy of oracle.c and
checks that these pins catch each one.
"""
import itertools
import os
import re
import shutil

import numpy as np
import pytest

import graphgen as gg
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF = oracle.UNREACHED_DIST


def _parse_tiny():
    edges, expect, V, src = [], {}, None, None
    for line in open(os.path.join(GOLDEN, "tiny_weighted.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        k, *rest = line.split()
        if k == "vertices":
            V = int(rest[0])
        elif k == "source":
            src = int(rest[0])
        elif k == "edge":
            edges.append(tuple(int(x) for x in rest))
        elif k == "expect":
            v, lv, d = rest
            expect[int(v)] = (int(lv), INF if d == "inf" else int(d))
    return V, src, edges, expect


def _weighted(V, edges):
    g = gg.from_edges(V, [e[0] for e in edges], [e[1] for e in edges])
    wmap = {(u, v): w for u, v, w in edges}
    w = np.array([wmap[(u, int(g.col[e]))] for u in range(V)
                  for e in range(g.row_off[u], g.row_off[u + 1])], dtype=np.uint32)
    return g, w


# ---- closed forms ------------------------------------------------------------------

def test_grid_closed_form_levels():
    W = H = 256
    g = gg.grid(W, H)
    lv = oracle.bfs(g, 0)
    y, x = np.divmod(np.arange(W * H), W)
    np.testing.assert_array_equal(lv, x + y)
    hist = np.bincount(lv)
    d = np.arange(511)
    np.testing.assert_array_equal(hist, np.minimum(d + 1, 511 - d))
    assert oracle.traversal_work(g, lv >= 0) == (65536, 261120)


def test_grid_unit_weight_sssp_equals_closed_form():
    g = gg.grid(64, 48)
    w = np.ones(g.num_edges, dtype=np.uint32)
    y, x = np.divmod(np.arange(64 * 48), 64)
    for src_xy in [(0, 0), (63, 47), (17, 30)]:
        s = src_xy[1] * 64 + src_xy[0]
        expect = np.abs(x - src_xy[0]) + np.abs(y - src_xy[1])
        np.testing.assert_array_equal(oracle.dijkstra(g, w, s), expect)
        np.testing.assert_array_equal(oracle.bellman_ford(g, w, s), expect)
        np.testing.assert_array_equal(oracle.bfs(g, s), expect)


def test_path_star_complete():
    n = 50
    np.testing.assert_array_equal(oracle.bfs(gg.path(n), 0), np.arange(n))
    lv = oracle.bfs(gg.path(n), 10)  # directed path: nothing before the source
    np.testing.assert_array_equal(lv, np.where(np.arange(n) >= 10, np.arange(n) - 10, -1))
    np.testing.assert_array_equal(oracle.bfs(gg.star(n), 0), np.r_[0, np.ones(n - 1)])
    np.testing.assert_array_equal(oracle.bfs(gg.star(n), 5), np.r_[1, 2 * np.ones(n - 1)] - np.eye(n)[5] * 2)
    np.testing.assert_array_equal(oracle.bfs(gg.complete(9), 3), 1 - np.eye(9)[3])
    g = gg.complete(9)
    assert g.num_edges == 72  # self-loops dropped


def test_isolated_and_single_vertex():
    g = gg.from_edges(5, [1, 2], [2, 3])
    np.testing.assert_array_equal(oracle.bfs(g, 0), [0, -1, -1, -1, -1])
    np.testing.assert_array_equal(oracle.dijkstra(g, np.ones(g.num_edges, np.uint32), 0),
                                  [0, INF, INF, INF, INF])
    g1 = gg.from_edges(1, [], [])
    assert oracle.bfs(g1, 0).tolist() == [0]
    assert oracle.dijkstra(g1, np.zeros(0, np.uint32), 0).tolist() == [0]


def test_disconnected_components():
    # two directed cycles; source in the second
    g = gg.from_edges(7, [0, 1, 2, 3, 4, 5, 6], [1, 2, 0, 4, 5, 6, 3])
    np.testing.assert_array_equal(oracle.bfs(g, 4), [-1, -1, -1, 3, 0, 1, 2])


def test_hand_derived_fixture():
    V, src, edges, expect = _parse_tiny()
    g, w = _weighted(V, edges)
    lv = oracle.bfs(g, src)
    for f in (oracle.dijkstra, oracle.bellman_ford):
        d = f(g, w, src)
        for v, (el, ed) in expect.items():
            assert d[v] == ed, (f.__name__, v)
    for v, (el, ed) in expect.items():
        assert lv[v] == el, v


# ---- brute force -------------------------------------------------------------------

def test_every_directed_graph_on_four_vertices():
    """All 2^12 edge subsets of K4 (no self-loops): BFS levels = explicit path minimum."""
    pairs = [(u, v) for u in range(4) for v in range(4) if u != v]
    for mask in range(1 << len(pairs)):
        es = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        g = gg.from_edges(4, [e[0] for e in es], [e[1] for e in es])
        hops, _ = oracle.brute_force_paths(g, 0)
        lv = oracle.bfs(g, 0)
        assert lv.tolist() == [-1 if h is None else h for h in hops], es


def test_random_tiny_weighted_vs_path_enumeration():
    rng = np.random.default_rng(1234)
    for trial in range(150):
        V = int(rng.integers(1, 8))
        m = int(rng.integers(0, 3 * V + 1))
        g = gg.random_graph(V, m, seed=trial)
        w = rng.integers(0, 20, size=g.num_edges).astype(np.uint32)
        src = int(rng.integers(0, V))
        hops, cost = oracle.brute_force_paths(g, src, w)
        assert oracle.bfs(g, src).tolist() == [-1 if h is None else h for h in hops]
        exp = [INF if c is None else c for c in cost]
        assert oracle.dijkstra(g, w, src).tolist() == exp
        assert oracle.bellman_ford(g, w, src).tolist() == exp
        fw = oracle.floyd_warshall(g, w)[src]
        assert [INF if x == np.iinfo(np.uint64).max else int(x) for x in fw] == exp


# ---- an independent library routine ------------------------------------------------

def _scipy_sp(g, w, src, unweighted=False):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    V = g.num_vertices
    data = np.ones(g.num_edges) if unweighted else np.asarray(w, dtype=np.float64)
    # scipy treats explicit zeros as missing edges; shift zero weights is avoided by w >= 1
    m = sp.csr_matrix((data, g.col, g.row_off), shape=(V, V))
    d = csgraph.shortest_path(m, method="D", directed=True, indices=src, unweighted=unweighted)
    return d


@pytest.mark.parametrize("V,m,seed", [(300, 900, 1), (2000, 5000, 2), (5000, 40000, 3)])
def test_random_graphs_vs_scipy(V, m, seed):
    g = gg.random_graph(V, m, seed)
    w = gg.weights(g, seed + 100, 1, 255)
    src = gg.max_out_degree_vertex(g)
    d_hops = _scipy_sp(g, None, src, unweighted=True)
    d_w = _scipy_sp(g, w, src)
    lv = oracle.bfs(g, src)
    np.testing.assert_array_equal(lv, np.where(np.isinf(d_hops), -1, d_hops).astype(np.int64))
    dist = oracle.dijkstra(g, w, src)
    np.testing.assert_array_equal(dist, np.where(np.isinf(d_w), INF, d_w).astype(np.uint64))


def test_rmat_vs_scipy_and_invariants():
    g = gg.rmat(13, 16, seed=7)
    w = gg.weights(g, 8)
    src = gg.max_out_degree_vertex(g)
    lv = oracle.bfs(g, src)
    oracle.check_bfs_invariants(g, src, lv)
    d_hops = _scipy_sp(g, None, src, unweighted=True)
    np.testing.assert_array_equal(lv, np.where(np.isinf(d_hops), -1, d_hops).astype(np.int64))
    dist = oracle.dijkstra(g, w, src)
    oracle.check_sssp_fixed_point(g, w, src, dist)
    np.testing.assert_array_equal(dist, oracle.bellman_ford(g, w, src))
    d_w = _scipy_sp(g, w, src)
    np.testing.assert_array_equal(dist, np.where(np.isinf(d_w), INF, d_w).astype(np.uint64))


def test_overflow_is_reported():
    g = gg.path(4)
    w = np.array([0x7FFFFFFF, 0x7FFFFFFF, 5], dtype=np.uint32)
    with pytest.raises(OverflowError):
        oracle.dijkstra(g, w, 0)
    with pytest.raises(OverflowError):
        oracle.bellman_ford(g, w, 0)


def test_invariant_checkers_reject_wrong_answers():
    g = gg.rmat(10, 8, seed=3)
    src = gg.max_out_degree_vertex(g)
    w = gg.weights(g, 4)
    lv = oracle.bfs(g, src)
    dist = oracle.dijkstra(g, w, src)
    reached = np.flatnonzero(lv > 0)
    bad = lv.copy(); bad[reached[0]] += 1
    with pytest.raises(AssertionError):
        oracle.check_bfs_invariants(g, src, bad)
    bad = lv.copy(); bad[reached[-1]] = -1
    with pytest.raises(AssertionError):
        oracle.check_bfs_invariants(g, src, bad)
    bad = dist.copy(); bad[reached[0]] += 1
    with pytest.raises(AssertionError):
        oracle.check_sssp_fixed_point(g, w, src, bad)
    bad = dist.copy(); bad[reached[1]] -= 1
    with pytest.raises(AssertionError):
        oracle.check_sssp_fixed_point(g, w, src, bad)


# ---- planted mistakes: the pins above must catch each one ---------------------------

MUTANTS = [
    ("level[v] = level[u] + 1;", "level[v] = level[u] + 2;"),          # wrong increment
    ("if (level[v] == -1) {", "if (level[v] <= 0) {"),                  # re-visits level 0
    ("e < row_off[u + 1]; ++e) {\n            int32_t v = col[e];\n            if (level",
     "e + 1 < row_off[u + 1]; ++e) {\n            int32_t v = col[e];\n            if (level"),  # drops last edge
    ("uint64_t nd = it.d + (uint64_t)w[e];", "uint64_t nd = it.d + (uint64_t)w[e] + 1;"),  # extra term
    ("uint64_t nd = it.d + (uint64_t)w[e];", "uint64_t nd = (uint64_t)w[e];"),            # dropped term
    ("if (h[p].d <= x.d) break;", "if (h[p].d >= x.d) break;"),          # heap order flipped
]


def _pins_pass(lib) -> bool:
    try:
        g = gg.grid(32, 32)
        y, x = np.divmod(np.arange(1024), 32)
        if not np.array_equal(oracle.bfs(g, 0, lib=lib), x + y):
            return False
        V, src, edges, expect = _parse_tiny()
        gt, wt = _weighted(V, edges)
        d = oracle.dijkstra(gt, wt, src, lib=lib)
        if [int(d[v]) for v in sorted(expect)] != [expect[v][1] for v in sorted(expect)]:
            return False
        rng = np.random.default_rng(5)
        for trial in range(40):
            Vr = int(rng.integers(2, 7))
            gr = gg.random_graph(Vr, 3 * Vr, seed=1000 + trial)
            wr = rng.integers(1, 9, size=gr.num_edges).astype(np.uint32)
            hops, cost = oracle.brute_force_paths(gr, 0, wr)
            if oracle.bfs(gr, 0, lib=lib).tolist() != [-1 if h is None else h for h in hops]:
                return False
            if oracle.dijkstra(gr, wr, 0, lib=lib).tolist() != [INF if c is None else c for c in cost]:
                return False
        return True
    except (AssertionError, ValueError, OverflowError):
        return False


def test_pins_catch_planted_mistakes(tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    clean = tmp_path / "clean.c"
    clean.write_text(src)
    lib_ok = oracle.load_variant(_compile(clean, tmp_path / "clean.so"))
    assert _pins_pass(lib_ok), "pins fail on the unmodified oracle"
    for i, (old, new) in enumerate(MUTANTS):
        assert src.count(old) >= 1, f"mutant {i} does not apply"
        mutated = tmp_path / f"m{i}.c"
        mutated.write_text(src.replace(old, new, 1))
        lib = oracle.load_variant(_compile(mutated, tmp_path / f"m{i}.so"))
        assert not _pins_pass(lib), f"planted mistake {i} ({new!r}) went unnoticed"


def _compile(c_path, so_path):
    import subprocess
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(so_path), str(c_path)])
    return str(so_path)
