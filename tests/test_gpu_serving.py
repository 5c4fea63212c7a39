"""Serving with continuous batching: queries overlap on the device, results do not change.

Queries arrive in bursts while others run, so they are admitted into free slots and
overlap (running traversals shrink through offer_kill and grow back through forks).
Every query's result must be bit-identical to the same query run alone on a context of
its own, and to the oracle.  A co-runner takes half the CTAs from the running queries in
the middle of the stream.
"""
import time

import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1707_01989_gb300 as coop
from gpu_util import DevGraph, assert_same

pytestmark = pytest.mark.gpu


def _graphs():
    gs = [gg.rmat(s, 16, seed=300 + s) for s in (10, 12, 14, 15, 16)] + [gg.grid(120, 80)]
    return [(g, gg.weights(g, 400 + i)) for i, g in enumerate(gs)]


def test_results_same_alone_and_in_the_mix(cuda_device):
    import torch
    graphs = _graphs()
    sv = coop.coop_server_create(0, slots=4)
    dgs = []
    for g, w in graphs:
        dg = DevGraph(g, w)
        dgs.append(dg)
        coop.coop_server_add_graph(sv, dg.csr, dg.w, keep=(dg,))
    rng = np.random.default_rng(9)
    queries = []
    for i in range(60):
        gi = int(rng.integers(0, len(graphs)))
        g = graphs[gi][0]
        src = gg.max_out_degree_vertex(g) if i % 3 else int(rng.integers(0, g.num_vertices))
        kind = coop.COOP_JOB_SSSP if i % 2 else coop.COOP_JOB_BFS
        queries.append((gi, kind, src, dgs[gi].empty()))
    N = coop.coop_query(coop.coop_init(0))["max_ctas"]
    x = torch.ones(1 << 22, device=cuda_device)
    y = torch.zeros_like(x)
    cs = torch.cuda.Stream(priority=-1)
    coop.coop_saxpy(N // 2, 1.0, x, y, stream=cs)  # load the co-runner's kernel
    torch.cuda.synchronize()
    tickets = []
    for k, (gi, kind, src, out) in enumerate(queries):
        tickets.append(coop.coop_server_submit(sv, gi, kind, src, out))
        if k == 30:  # a co-runner takes half the CTAs from the running queries
            got = coop.coop_server_request_resources(sv, N // 2, timeout_us=2_000_000)
            coop.coop_saxpy(N // 2, 1.0, x, y, stream=cs)
            cs.synchronize()
            coop.coop_server_release(sv, N // 2)
            assert got == N // 2
        if k % 10 == 9:
            time.sleep(0.001)
    results = [coop.coop_server_wait(sv, t, timeout_us=20_000_000) for t in tickets]
    assert all(r.status == coop.COOP_OK for r in results)
    assert any(r.ctas < N for r in results), "no query overlapped with another"
    assert sum(r.stats.kills + r.stats.forks for r in results) > 0, "no running query was resized"
    coop.coop_server_destroy(sv)
    # the same queries alone, each on a fresh context of its own
    ctx = coop.coop_init(0)
    for (gi, kind, src, out), r in zip(queries, results):
        g, w = graphs[gi]
        mixed = out.cpu().numpy()
        alone = dgs[gi].empty()
        if kind == coop.COOP_JOB_BFS:
            coop.coop_bfs(ctx, dgs[gi].csr, src, alone, stats=True)
            exp = oracle.bfs(g, src)
        else:
            coop.coop_sssp(ctx, dgs[gi].csr, dgs[gi].w, src, alone, stats=True)
            exp = oracle.dijkstra(g, w, src).view(np.int32)
        assert_same(mixed, alone.cpu().numpy(), f"query on graph {gi} from {src}: mix vs alone")
        assert_same(mixed, exp, f"query on graph {gi} from {src}: mix vs oracle")
        assert r.stats.reached_edges == oracle.traversal_work(g, exp != (-1 if kind == coop.COOP_JOB_BFS else -1))[1]
    coop.coop_destroy(ctx)


def test_server_budget_and_arguments(cuda_device):
    g = gg.rmat(14, 16, seed=1)
    dg = DevGraph(g)
    sv = coop.coop_server_create(0, slots=2, hbm_budget_bytes=1 << 20)  # far too small
    with pytest.raises(coop.CoopError) as ei:
        coop.coop_server_add_graph(sv, dg.csr, None, keep=(dg,))
    assert ei.value.status == coop.COOP_ENOMEM
    coop.coop_server_destroy(sv)
    sv = coop.coop_server_create(0, slots=2)
    gid = coop.coop_server_add_graph(sv, dg.csr, None, keep=(dg,))
    with pytest.raises(coop.CoopError):
        coop.coop_server_submit(sv, gid, coop.COOP_JOB_SSSP, 0, dg.empty())  # no weights registered
    with pytest.raises(coop.CoopError):
        coop.coop_server_submit(sv, gid, coop.COOP_JOB_BFS, g.num_vertices, dg.empty())
    out = dg.empty()
    t = coop.coop_server_submit(sv, gid, coop.COOP_JOB_BFS, 0, out)
    r = coop.coop_server_wait(sv, t, timeout_us=10_000_000)
    assert r.status == 0 and r.latency_us > 0
    assert_same(out.cpu().numpy(), oracle.bfs(g, 0), "single served query")
    coop.coop_server_destroy(sv)


@pytest.mark.slow
def test_serving_full_graph_set(cuda_device):
    """The serving workload's graph set at full size: 32 device-resident R-MAT graphs of
    scales 14..21 (seeded as in the benchmark), 4 slots under a 60 GB budget; 40 BFS /
    SSSP queries with random sources submitted in bursts so that they overlap and running
    queries are resized; every result against the oracle."""
    import torch
    rng_g, rng_s = np.random.default_rng(4), np.random.default_rng(16)
    scales = rng_g.integers(14, 22, size=32)
    sv = coop.coop_server_create(0, slots=4, hbm_budget_bytes=60 << 30)
    graphs = []
    for i, sc in enumerate(scales):
        g = gg.rmat(int(sc), 16, seed=3000 + i)
        w = gg.weights(g, 4000 + i)
        dg = DevGraph(g, w)
        coop.coop_server_add_graph(sv, dg.csr, dg.w, keep=(dg,))
        graphs.append((g, w, dg))
    queries = []
    for k in range(40):
        gi = int(rng_s.integers(0, 32))
        kind = coop.COOP_JOB_BFS if k % 2 else coop.COOP_JOB_SSSP
        src = int(rng_s.integers(0, graphs[gi][0].num_vertices))
        out = graphs[gi][2].empty()
        out.fill_(0x5A5A5A5A)
        queries.append((gi, kind, src, out))
    tickets = []
    for k, (gi, kind, src, out) in enumerate(queries):
        tickets.append(coop.coop_server_submit(sv, gi, kind, src, out))
        if k % 8 == 7:
            time.sleep(0.002)
    results = [coop.coop_server_wait(sv, t, timeout_us=30_000_000) for t in tickets]
    coop.coop_server_destroy(sv)
    assert all(r.status == coop.COOP_OK for r in results)
    assert any(r.ctas < coop.coop_query(coop.coop_init(0))["max_ctas"] for r in results)
    torch.cuda.synchronize()
    for (gi, kind, src, out), r in zip(queries, results):
        g, w, _ = graphs[gi]
        got = out.cpu().numpy()
        if kind == coop.COOP_JOB_BFS:
            assert_same(got, oracle.bfs(g, src), f"bfs on graph {gi} (scale {scales[gi]}) from {src}")
        else:
            assert_same(got.view(np.uint32), oracle.dijkstra(g, w, src), f"sssp on graph {gi} from {src}")
