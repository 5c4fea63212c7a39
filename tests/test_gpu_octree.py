"""Octree partitioning on the GPU (the work-stealing application of Table 1) against the
oracle: every point's leaf code, the leaf count and each leaf's point set must match
exactly, alone and while the host takes and returns CTAs (Sec. 3.2: offer_kill and
request_fork at the head of the work-stealing loop)."""
import threading
import time

import numpy as np
import pytest

import graphgen as gg
import paper_1707_01989_gb300 as coop
from oracle import octree as ot

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_device):
    c = coop.coop_init(0)
    yield c
    coop.coop_destroy(c)


def _run(ctx, pts, cap, md, max_leaves=None, ok=(coop.COOP_OK,)):
    import torch
    x, y, z = (torch.from_numpy(a.view(np.int32)).cuda() for a in pts)
    n = len(pts[0])
    ml = max(1, n) if max_leaves is None else max_leaves
    code = torch.empty(ml, dtype=torch.int64, device="cuda")
    begin = torch.empty(ml, dtype=torch.int32, device="cuda")
    count = torch.empty(ml, dtype=torch.int32, device="cuda")
    perm = torch.empty(max(1, n), dtype=torch.int32, device="cuda")
    nl = torch.empty(1, dtype=torch.int32, device="cuda")
    st = coop.coop_octree(ctx, x, y, z, cap, md, code, begin, count, perm, nl, stats=True, ok=ok)
    k = int(nl.item())
    return (code[:k].cpu().numpy().view(np.uint64), begin[:k].cpu().numpy(), count[:k].cpu().numpy(),
            perm.cpu().numpy()[:n], st)


def _check(pts, cap, md, res):
    codes, begin, count, perm, st = res
    n = len(pts[0])
    exp = ot.octree_leaves(*pts, cap, md)
    assert len(codes) == len(exp), (len(codes), len(exp))
    got = np.zeros(n, dtype=np.uint64)
    covered = np.zeros(n, dtype=np.int64)
    for c, b, k in zip(codes, begin, count):
        idx = perm[b:b + k]
        got[idx] = c
        covered[idx] += 1
    assert np.all(covered == 1), "the leaves partition the points"
    assert np.array_equal(got, ot.leaf_code_of_points(*pts, cap, md))
    assert sorted(map(int, codes)) == sorted(int(c) for c, _, _ in exp)
    assert st.vertices_reached == len(exp) and st.status == coop.COOP_OK


@pytest.mark.parametrize("kind,n,cap,md", [("uniform", 50000, 32, 21), ("clustered", 120000, 16, 21),
                                           ("clustered", 30000, 1, 21), ("uniform", 20000, 8, 3),
                                           ("clustered", 5000, 64, 0), ("uniform", 1, 4, 21),
                                           ("clustered", 700, 1000, 21),
                                           # large inputs take the grid-wide partition of the top
                                           # levels: leaves above depth 3, and max_depth exactly 3
                                           ("clustered", 100000, 3000, 21), ("uniform", 70000, 8, 3),
                                           ("clustered", 300000, 32, 21)])
def test_octree_matches_oracle(ctx, kind, n, cap, md):
    pts = gg.points(n, 70 + n % 97, kind)
    _check(pts, cap, md, _run(ctx, pts, cap, md))


def test_octree_lattice_and_duplicates(ctx):
    m = 8
    i, j, k = (a.ravel().astype(np.uint32) << 18 for a in np.meshgrid(np.arange(m), np.arange(m), np.arange(m),
                                                                      indexing="ij"))
    _check((i, j, k), 1, 21, _run(ctx, (i, j, k), 1, 21))
    x, y, z = gg.points(3000, 5, "uniform")
    x[:1000], y[:1000], z[:1000] = 77, 88, 99  # a third identical: one leaf at max_depth
    _check((x, y, z), 10, 21, _run(ctx, (x, y, z), 10, 21))


def test_octree_under_host_requests(ctx):
    """A host arbiter takes and returns CTAs while octrees are built: offer_kill at the
    loop head lets CTAs leave (their queued tasks are stolen), forks join with queues of
    their own, and the leaves do not change."""
    pts = gg.points(400000, 81, "clustered")
    exp_codes = ot.leaf_code_of_points(*pts, 8, 21)
    stop = threading.Event()
    errors = []
    N = coop.coop_query(ctx)["max_ctas"]

    def arbiter():
        rng = np.random.default_rng(2)
        try:
            while not stop.is_set():
                got = coop.coop_request_resources(ctx, int(rng.integers(1, N // 2)), timeout_us=500_000,
                                                  ok=(coop.COOP_OK, coop.COOP_ETIMEOUT))
                time.sleep(0.0003)
                if got:
                    coop.coop_release(ctx, got)
        except Exception as exc:  # surfaced below
            errors.append(exc)

    t = threading.Thread(target=arbiter)
    t.start()
    kills = forks = 0
    try:
        for r in range(6):
            codes, begin, count, perm, st = _run(ctx, pts, 8, 21)
            got = np.zeros(len(pts[0]), dtype=np.uint64)
            for c, b, k in zip(codes, begin, count):
                got[perm[b:b + k]] = c
            assert np.array_equal(got, exp_codes), f"run {r}"
            kills += st.kills
            forks += st.forks
    finally:
        stop.set()
        t.join()
    assert not errors, errors
    assert kills > 0 and forks > 0, (kills, forks)
    coop.coop_sync(ctx)


def test_request_during_a_build_waits_for_its_ctas(ctx):
    """A request posted while an octree is being built is served by the build's CTAs
    leaving at the head of its loop, not granted at once: a build has a run id of its own,
    which the host sees published only when the build is over.  (A request granted at
    once is recorded with M = 0 and no wait; the traversal run first leaves a published
    M in the mailbox, which a request that waits records.)"""
    import torch
    from gpu_util import DevGraph, run_bfs
    run_bfs(ctx, DevGraph(gg.grid(64, 64)), 0)
    N = coop.coop_query(ctx)["max_ctas"]
    pts = gg.points(1 << 20, 91, "clustered")
    exp_codes = ot.leaf_code_of_points(*pts, 16, 21)
    x, y, z = (torch.from_numpy(a.view(np.int32)).cuda() for a in pts)
    n = len(pts[0])
    code = torch.empty(n, dtype=torch.int64, device="cuda")
    begin = torch.empty(n, dtype=torch.int32, device="cuda")
    count = torch.empty(n, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    nl = torch.empty(1, dtype=torch.int32, device="cuda")
    coop.coop_get_request_log(ctx, clear=True)
    coop.coop_octree(ctx, x, y, z, 16, 21, code, begin, count, perm, nl)  # returns once launched
    got = coop.coop_request_resources(ctx, N // 2, timeout_us=2_000_000)
    coop.coop_release(ctx, got)
    torch.cuda.synchronize()
    rec = coop.coop_get_request_log(ctx, clear=True)[-1]
    assert got == N // 2
    assert rec["active_at_post"] > 0, rec  # not granted at once
    assert rec["gather_us"] - rec["post_us"] > 1.0, rec
    k = int(nl.item())
    codes = code[:k].cpu().numpy().view(np.uint64)
    b, c, p = begin[:k].cpu().numpy(), count[:k].cpu().numpy(), perm.cpu().numpy()
    leaf_of = np.zeros(n, dtype=np.uint64)
    for cd, bb, cc in zip(codes, b, c):
        leaf_of[p[bb:bb + cc]] = cd
    assert np.array_equal(leaf_of, exp_codes)
    coop.coop_sync(ctx)


def test_octree_errors(ctx):
    pts = gg.points(2000, 3, "uniform")
    bad = (pts[0].copy(), pts[1], pts[2])
    bad[0][17] = 1 << 21
    assert _run(ctx, bad, 8, 21, ok=(coop.COOP_EGRAPH,))[4].status == coop.COOP_EGRAPH
    assert _run(ctx, pts, 8, 21, max_leaves=3, ok=(coop.COOP_EOVERFLOW,))[4].status == coop.COOP_EOVERFLOW
    with pytest.raises(coop.CoopError):
        _run(ctx, pts, 0, 21)
    with pytest.raises(coop.CoopError):
        _run(ctx, pts, 8, 22)
    codes, _, _, _, st = _run(ctx, (pts[0][:0], pts[1][:0], pts[2][:0]), 8, 21)
    assert len(codes) == 0
    # the context still works
    _check(pts, 8, 21, _run(ctx, pts, 8, 21))


@pytest.mark.slow
def test_octree_full_size(ctx):
    """4M clustered points, leaf_cap 32: the benchmark's octree, every point's leaf checked."""
    pts = gg.points(1 << 22, 90, "clustered")
    _check(pts, 32, 21, _run(ctx, pts, 32, 21))
