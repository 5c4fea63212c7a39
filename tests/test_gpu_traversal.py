"""Parity of the CUDA traversals with the CPU oracle, element by element (bit-exact).

Small cases span many warps' edge ranges, several window slides and a ragged tail;
full-size cases are the R-MAT scale-20 SSSP and scale-22 BFS workloads, checked in
full against the oracle; edge cases cover V = 1, isolated / zero-out-degree sources,
deep paths, hubs, complete graphs, empty edge sets and malformed input.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1707_01989_gb300 as coop
from gpu_util import DevGraph, assert_same, hub_graph, run_bfs, run_sssp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_device):
    c = coop.coop_init(0)
    yield c
    coop.coop_destroy(c)


def test_context_facts(ctx):
    q = coop.coop_query(ctx)
    assert q["threads_per_cta"] == 992
    assert q["max_ctas"] == q["sm_count"]  # one traversal CTA per SM
    assert q["lent"] == 0


def test_bfs_grid_closed_form(ctx):
    g = gg.grid(256, 256)
    lv, st = run_bfs(ctx, DevGraph(g), 0)
    y, x = np.divmod(np.arange(65536), 256)
    assert_same(lv, x + y, "grid levels")
    assert st.levels == 511 and st.barriers == 511
    assert st.edges_scanned == 261120 and st.frontier_total == 65536
    assert st.kills == 0 and st.forks == 0


@pytest.mark.parametrize("scale,ef,seed", [(6, 4, 1), (10, 8, 2), (14, 16, 3), (17, 16, 4)])
def test_bfs_rmat_matches_oracle(ctx, scale, ef, seed):
    g = gg.rmat(scale, ef, seed=seed)
    src = gg.max_out_degree_vertex(g)
    lv, st = run_bfs(ctx, DevGraph(g), src)
    exp = oracle.bfs(g, src)
    assert_same(lv, exp, f"rmat{scale} levels")
    vr, es = oracle.traversal_work(g, exp >= 0)
    assert st.edges_scanned == es
    assert (st.vertices_reached, st.reached_edges) == (vr, es)
    # a level is expanded when some vertex on it has out-edges
    assert st.levels == exp[(exp >= 0) & (g.out_degree() > 0)].max() + 1


@pytest.mark.parametrize("scale,ef,seed", [(6, 4, 1), (10, 8, 2), (14, 16, 3), (17, 16, 5)])
def test_sssp_rmat_matches_oracle(ctx, scale, ef, seed):
    g = gg.rmat(scale, ef, seed=seed)
    w = gg.weights(g, seed + 1)
    src = gg.max_out_degree_vertex(g)
    d, st = run_sssp(ctx, DevGraph(g, w), src)
    exp = oracle.dijkstra(g, w, src)
    assert_same(d, exp, f"rmat{scale} dist")
    assert (st.vertices_reached, st.reached_edges) == oracle.traversal_work(g, exp != oracle.UNREACHED_DIST)


def test_random_graphs_many_sources(ctx):
    rng = np.random.default_rng(7)
    for trial in range(12):
        V = int(rng.integers(1, 3000))
        g = gg.random_graph(V, int(rng.integers(0, 6 * V + 1)), seed=trial)
        w = gg.weights(g, trial, 1, int(rng.integers(1, 1000)))
        dg = DevGraph(g, w)
        for src in rng.integers(0, V, size=3):
            lv, _ = run_bfs(ctx, dg, int(src))
            assert_same(lv, oracle.bfs(g, int(src)), f"random {trial} bfs")
            d, _ = run_sssp(ctx, dg, int(src))
            assert_same(d, oracle.dijkstra(g, w, int(src)), f"random {trial} sssp")


EDGE_CASES = {
    "single_vertex": lambda: (gg.from_edges(1, [], []), 0),
    "no_edges": lambda: (gg.from_edges(50, [], []), 7),
    "isolated_source": lambda: (gg.from_edges(6, [1, 2, 3], [2, 3, 4]), 0),
    "sink_source": lambda: (gg.from_edges(4, [0, 1], [1, 2]), 2),
    "deep_path": lambda: (gg.path(3000), 0),
    "path_from_middle": lambda: (gg.path(500), 250),
    "star_hub": lambda: (gg.star(40000), 0),
    "star_leaf": lambda: (gg.star(40000), 123),
    "complete": lambda: (gg.complete(180), 5),
    "two_cycles": lambda: (gg.from_edges(7, [0, 1, 2, 3, 4, 5, 6], [1, 2, 0, 4, 5, 6, 3]), 4),
    "long_row_ragged": lambda: (gg.from_edges(70001, np.zeros(70000, np.int64), np.arange(1, 70001)), 0),
}


@pytest.mark.parametrize("name", sorted(EDGE_CASES))
def test_edge_cases(ctx, name):
    g, src = EDGE_CASES[name]()
    w = gg.weights(g, 99, 1, 255)
    dg = DevGraph(g, w)
    lv, st = run_bfs(ctx, dg, src)
    assert_same(lv, oracle.bfs(g, src), f"{name} bfs")
    d, _ = run_sssp(ctx, dg, src)
    assert_same(d, oracle.dijkstra(g, w, src), f"{name} sssp")


def test_baselines_match(ctx):
    g = gg.rmat(15, 16, seed=8)
    w = gg.weights(g, 9)
    src = gg.max_out_degree_vertex(g)
    dg = DevGraph(g, w)
    lv, st = run_bfs(ctx, dg, src, baseline=True)
    assert_same(lv, oracle.bfs(g, src), "baseline bfs")
    assert st.max_active == coop.coop_query(ctx)["max_ctas"]
    d, _ = run_sssp(ctx, dg, src, baseline=True)
    assert_same(d, oracle.dijkstra(g, w, src), "baseline sssp")


def test_sssp_over_at_entry_writes_every_distance(ctx):
    """A source without out-edges ends the traversal at the master's entry.  Every CTA
    admitted there still copies its stripe of the distances out: the output is pre-filled
    with garbage, and the run is repeated, since a CTA that took the end of the run for a
    refusal of its admission would leave its stripe unwritten only now and then."""
    g = gg.rmat(16, 16, seed=5)
    src = int(np.flatnonzero(np.diff(np.array(g.row_off)) == 0)[0])
    w = gg.weights(g, 6)
    dg = DevGraph(g, w)
    exp = oracle.dijkstra(g, w, src)
    assert (exp != 0xFFFFFFFF).sum() == 1
    for i in range(50):
        out = dg.empty()
        out.fill_(0x5A5A5A5A)
        f = coop.coop_sssp_baseline if i % 5 == 4 else coop.coop_sssp
        f(ctx, dg.csr, dg.w, src, out, stats=True)
        assert_same(out.cpu().numpy().view(np.uint32), exp, f"source without out-edges, run {i}")


def test_repeated_runs_reuse_scratch(ctx):
    big = gg.rmat(16, 16, seed=21)
    small = gg.grid(40, 30)
    for g in (big, small, big):
        src = gg.max_out_degree_vertex(g)
        lv, _ = run_bfs(ctx, DevGraph(g), src)
        assert_same(lv, oracle.bfs(g, src), "repeat")


def test_sssp_overflow_reported(ctx):
    g = gg.path(4)
    w = np.array([0x7FFFFFFF, 0x7FFFFFFF, 5], dtype=np.uint32)
    d, st = run_sssp(ctx, DevGraph(g, w), 0, ok=(coop.COOP_EOVERFLOW,))
    assert st.status == coop.COOP_EOVERFLOW
    assert d[0] == 0 and d[1] == 0x7FFFFFFF


def test_malformed_graph_reported_not_faulted(ctx):
    """A column id >= V is caught by the kernel's bounds check and reported."""
    g = gg.rmat(10, 8, seed=4)
    col = g.col.copy()
    col[len(col) // 2] = g.num_vertices + 5
    bad = gg.CSR(g.row_off, col)
    src = gg.max_out_degree_vertex(g)
    _, st = run_bfs(ctx, DevGraph(bad), src, ok=(coop.COOP_EGRAPH, coop.COOP_OK))
    reached_bad = oracle.bfs(g, src)[np.searchsorted(g.row_off, len(col) // 2, side="right") - 1] >= 0
    if reached_bad:
        assert st.status == coop.COOP_EGRAPH
    # the context stays usable afterwards
    lv, _ = run_bfs(ctx, DevGraph(g), src)
    assert_same(lv, oracle.bfs(g, src), "after malformed input")


def test_invalid_arguments(ctx):
    g = gg.path(10)
    dg = DevGraph(g)
    out = dg.empty()
    with pytest.raises(coop.CoopError):
        coop.coop_bfs(ctx, dg.csr, 10, out)
    with pytest.raises(coop.CoopError):
        coop.coop_bfs(ctx, dg.csr, -1, out)
    with pytest.raises(coop.CoopError):
        coop.coop_release(ctx, 1)  # nothing lent


@pytest.mark.slow
def test_full_size_rmat20_sssp(ctx):
    g = gg.rmat(20, 16, seed=20)
    w = gg.weights(g, 21)
    src = gg.max_out_degree_vertex(g)
    d, st = run_sssp(ctx, DevGraph(g, w), src)
    exp = oracle.dijkstra(g, w, src)
    assert_same(d, exp, "rmat20 sssp")
    oracle.check_sssp_fixed_point(g, w, src, d)


@pytest.mark.slow
def test_full_size_rmat22_bfs(ctx):
    g = gg.rmat(22, 16, seed=22)
    src = gg.max_out_degree_vertex(g)
    lv, st = run_bfs(ctx, DevGraph(g), src)
    exp = oracle.bfs(g, src)
    assert_same(lv, exp, "rmat22 bfs")
    assert st.edges_scanned == oracle.traversal_work(g, exp >= 0)[1]


def _run_topo(ctx, dg, src, ok=(coop.COOP_OK,)):
    out = dg.empty()
    out.fill_(0x5A5A5A5A)
    st = coop.coop_sssp_topo(ctx, dg.csr, dg.w, src, out, stats=True, ok=ok)
    return out.cpu().numpy().view(np.uint32), st


@pytest.mark.parametrize("name", ["rmat13", "grid", "random", "path", "star", "no_out_edges"])
def test_topology_driven_sssp_matches_oracle(ctx, name):
    """p-sssp (Table 1): three barriers per iteration, same distances as Dijkstra."""
    if name == "rmat13":
        g = gg.rmat(13, 16, seed=31)
        src = gg.max_out_degree_vertex(g)
    elif name == "grid":
        g, src = gg.grid(50, 40), 0
    elif name == "random":
        g = gg.random_graph(3000, 24000, seed=32)
        src = 7
    elif name == "path":
        g, src = gg.path(300), 0
    elif name == "star":
        g, src = gg.star(500), 0
    else:
        g = gg.rmat(12, 8, seed=33)
        src = int(np.flatnonzero(np.diff(np.array(g.row_off)) == 0)[0])
    w = gg.weights(g, 34)
    dg = DevGraph(g, w)
    d, st = _run_topo(ctx, dg, src)
    exp = oracle.dijkstra(g, w, src)
    assert_same(d, exp, f"p-sssp {name}")
    assert st.barriers % 3 == 0  # whole iterations: relax, update, check
    assert st.vertices_reached == int((exp != 0xFFFFFFFF).sum())
    assert st.reached_edges == oracle.traversal_work(g, exp != 0xFFFFFFFF)[1]


@pytest.mark.parametrize("case", ["hubs", "star_center", "star_leaf", "dense_list_off"])
def test_topology_driven_sssp_heavy_rows(ctx, case):
    """p-sssp with rows of at least 512 edges, which the update interval lists as
    256-edge chunks for the next relax to deal out over the whole grid: hubs lowered in
    two different iterations, the source itself heavy (listed at entry), a heavy row
    reached through a leaf, and a dense graph where the list is off (it could outgrow
    its V-entry queue) and the stripe scan relaxes every row."""
    if case == "hubs":
        g, w, src = hub_graph(3)
    elif case.startswith("star"):
        g = gg.star(6000)
        w = gg.weights(g, 35)
        src = 0 if case == "star_center" else 17
    else:
        g = gg.complete(2100)
        w = gg.weights(g, 36)
        src = 5
    d, st = _run_topo(ctx, DevGraph(g, w), src)
    exp = oracle.dijkstra(g, w, src)
    assert_same(d, exp, f"p-sssp {case}")
    assert st.barriers % 3 == 0
    assert st.vertices_reached == int((exp != 0xFFFFFFFF).sum())
    assert st.reached_edges == oracle.traversal_work(g, exp != 0xFFFFFFFF)[1]


def test_topology_driven_sssp_overflow_reported(ctx):
    g = gg.path(4)
    w = np.array([0xFFFFFFF0, 0xFFFFFFF0, 1], dtype=np.uint32)
    d, st = _run_topo(ctx, DevGraph(g, w), 0, ok=(coop.COOP_EOVERFLOW,))
    assert st.status == coop.COOP_EOVERFLOW


@pytest.mark.slow
def test_full_size_rmat20_topology_driven_sssp(ctx):
    g = gg.rmat(20, 16, seed=20)
    w = gg.weights(g, 21)
    src = gg.max_out_degree_vertex(g)
    d, st = _run_topo(ctx, DevGraph(g, w), src)
    assert_same(d, oracle.dijkstra(g, w, src), "rmat20 p-sssp")
    assert st.barriers % 3 == 0
