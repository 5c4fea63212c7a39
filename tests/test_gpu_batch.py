"""Batched traversals: many independent BFS / SSSP jobs in one persistent launch.

Every job's output must equal the oracle's, whatever the blocks per job (uneven splits,
several waves of blocks, the autotuner's choice) and with or without CUDA-graph capture.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1707_01989_gb300 as coop
from gpu_util import DevGraph, assert_same

pytestmark = pytest.mark.gpu


def _batch_inputs(cuda_device, n_graphs=8, seed=3):
    import torch
    rng = np.random.default_rng(seed)
    items = []
    for i in range(n_graphs):
        scale = int(rng.integers(6, 16))
        g = gg.rmat(scale, 16, seed=100 + i)
        w = gg.weights(g, 200 + i)
        items.append((g, w, gg.max_out_degree_vertex(g)))
    items.append((gg.from_edges(1, [], []), np.zeros(0, np.uint32), 0))            # single vertex
    items.append((gg.from_edges(5, [1, 2], [2, 3]), np.ones(2, np.uint32), 0))     # isolated source
    items.append((gg.grid(40, 25), gg.weights(gg.grid(40, 25), 7), 0))
    jobs, keep, expect = [], [], []
    for g, w, src in items:
        dg = DevGraph(g, w)
        lv = dg.empty()
        dist = dg.empty()
        keep += [dg, lv, dist]
        jobs.append(coop.make_job(dg.csr, src, lv))
        jobs.append(coop.make_job(dg.csr, src, dist, dg.w))
        expect.append((lv, oracle.bfs(g, src), "bfs"))
        expect.append((dist, oracle.dijkstra(g, w, src), "sssp"))
    return jobs, keep, expect


def _check(expect):
    import torch
    torch.cuda.synchronize()
    for i, (out, exp, kind) in enumerate(expect):
        got = out.cpu().numpy()
        if kind == "sssp":
            got = got.view(np.uint32)
        assert_same(got, exp, f"job {i} ({kind})")


@pytest.fixture(scope="module")
def ctx(cuda_device):
    c = coop.coop_init(0)
    yield c
    coop.coop_destroy(c)


def test_batch_default_and_graph(ctx, cuda_device):
    import torch
    jobs, keep, expect = _batch_inputs(cuda_device)
    b = coop.coop_batch_create(ctx, jobs, keep)
    for use_graph in (False, True, True):
        for out, _, _ in expect:
            out.fill_(12345)
        coop.coop_batch_run(b, use_graph=use_graph)
        _check(expect)
    stats = coop.coop_batch_get_stats(b)
    assert all(s.status == coop.COOP_OK for s in stats)
    assert all(1 <= s.initial_active for s in stats)
    coop.coop_batch_destroy(b)


@pytest.mark.parametrize("rule", ["ones", "uneven", "waves"])
def test_batch_apportionments(ctx, cuda_device, rule):
    jobs, keep, expect = _batch_inputs(cuda_device, seed=11)
    b = coop.coop_batch_create(ctx, jobs, keep)
    N = coop.coop_query(ctx)["max_ctas"]
    n = len(jobs)
    rng = np.random.default_rng(5)
    if rule == "ones":
        ctas = [1] * n
    elif rule == "uneven":
        ctas = rng.integers(1, 9, size=n).tolist()
    else:  # far more blocks than fit at once: later jobs start as earlier ones finish
        ctas = rng.integers(N // 4, N, size=n).tolist()
    coop.coop_batch_set_ctas(b, ctas)
    coop.coop_batch_run(b, use_graph=True)
    _check(expect)
    stats = coop.coop_batch_get_stats(b)
    assert all(s.max_active <= c for s, c in zip(stats, ctas))
    coop.coop_batch_destroy(b)


def test_batch_tune(ctx, cuda_device):
    jobs, keep, expect = _batch_inputs(cuda_device, seed=21)
    b = coop.coop_batch_create(ctx, jobs, keep)
    ctas = coop.coop_batch_tune(b)
    assert len(ctas) == len(jobs) and min(ctas) >= 1
    for out, _, _ in expect:
        out.fill_(-7)
    coop.coop_batch_run(b, use_graph=True)
    _check(expect)
    coop.coop_batch_destroy(b)


@pytest.mark.slow
def test_batch_full_configuration(ctx, cuda_device):
    """The batched workload at its full size: 64 R-MAT instances, scales uniform in
    12..20 (seed 3, instance graphs seeded 1000 + i, weights 2000 + i), a BFS and an
    SSSP job each, blocks chosen by the autotuner, run from the captured CUDA graph;
    all 128 outputs against the oracle."""
    import torch
    rng = np.random.default_rng(3)
    scales = rng.integers(12, 21, size=64)
    jobs, keep, expect = [], [], []
    for i, sc in enumerate(scales):
        g = gg.rmat(int(sc), 16, seed=1000 + i)
        w = gg.weights(g, 2000 + i)
        src = gg.max_out_degree_vertex(g)
        dg = DevGraph(g, w)
        lv, dist = dg.empty(), dg.empty()
        keep += [dg, lv, dist]
        jobs += [coop.make_job(dg.csr, src, lv), coop.make_job(dg.csr, src, dist, dg.w)]
        expect += [(lv, (g, src), "bfs"), (dist, (g, w, src), "sssp")]
    b = coop.coop_batch_create(ctx, jobs, keep)
    try:
        coop.coop_batch_tune(b)
        for out, _, _ in expect:
            out.fill_(0x5A5A5A5A)
        coop.coop_batch_run(b, use_graph=True)
        coop.coop_batch_run(b, use_graph=True)
        torch.cuda.synchronize()
        for i, (out, args, kind) in enumerate(expect):
            got = out.cpu().numpy()
            if kind == "bfs":
                assert_same(got, oracle.bfs(*args), f"job {i} (bfs, scale {scales[i // 2]})")
            else:
                assert_same(got.view(np.uint32), oracle.dijkstra(*args), f"job {i} (sssp, scale {scales[i // 2]})")
    finally:
        coop.coop_batch_destroy(b)
