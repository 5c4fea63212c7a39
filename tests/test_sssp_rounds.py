"""Host models of the frontier SSSP's round structure (select, then expand).

Table 1's l-sssp is read as data-driven Bellman-Ford in rounds: a round expands the
pending vertices of lowest tentative distance (a select interval splits the pending queue
at a distance threshold when it is large) and every vertex whose distance drops becomes
pending for the next round.  These tests replay that structure on the host, with the
kernel's stamp rule (a vertex is queued at most once per round; a deferred vertex's stamp
is advanced), and check what the GPU's parity tests rely on:

* whatever thresholds the selects take -- the smallest, the largest, random ones, and
  the sampled-histogram rule of the kernel -- the distances equal Dijkstra's;
* the kernel's two-level threshold search (segment sums, then one segment) finds the
  same bucket as a direct cumulative search.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

INF = 0xFFFFFFFF
HIST, SHIFT = 1024, 2  # kHistBuckets, kHistShift


def bucket(d, base):
    return 0 if d <= base else min(HIST - 1, (d - base) >> SHIFT)


def rounds_sssp(g, w, src, choose, big=0):
    """Rounds over a pending list.  choose(pending, dist, base) returns the threshold
    bucket of a select; a round selects when the pending out-degree exceeds `big`."""
    ro = np.array(g.row_off, dtype=np.int64)
    col = np.array(g.col, dtype=np.int64)
    w = np.asarray(w, dtype=np.int64)
    V = g.num_vertices
    dist = np.full(V, INF, dtype=np.int64)
    stamp = np.zeros(V, dtype=np.int64)
    dist[src] = 0
    stamp[src] = 1
    pending, base, r, expanded = [src], 0, 0, 0
    while pending:
        tag = r + 2
        deg = ro[np.array(pending) + 1] - ro[np.array(pending)]
        if deg.sum() > big:
            b = choose(pending, dist, base)
            near = [v for v in pending if bucket(int(dist[v]), base) <= b]
            far = [v for v in pending if bucket(int(dist[v]), base) > b]
            for v in far:
                stamp[v] = tag
            nxt = list(far)
            dmin = min(int(dist[v]) for v in near) if near else None
        else:
            near, nxt, dmin = pending, [], None
        for u in near:  # relaxations in any order: here the queue order
            du = int(dist[u])
            for e in range(ro[u], ro[u + 1]):
                expanded += 1
                v, nd = int(col[e]), du + int(w[e])
                if nd < dist[v]:
                    dist[v] = nd
                    if stamp[v] != tag:
                        stamp[v] = tag
                        nxt.append(v)
        pending = [v for v in nxt if ro[v + 1] > ro[v]]  # rows without edges are not queued
        if dmin is not None:
            base = dmin
        r += 1
    return np.where(dist >= INF, INF, dist).astype(np.uint32), expanded


def sampled_rule(frac):
    """The kernel's rule on the whole pending list: first bucket whose cumulative count
    reaches `frac` of the total."""
    def choose(pending, dist, base):
        return 0 if not pending else _threshold(pending, dist, base, frac)
    return choose


def _threshold(pending, dist, base, frac):
    h = np.zeros(HIST, dtype=np.int64)
    for v in pending:
        h[bucket(int(dist[v]), base)] += 1
    tot = h.sum()
    cum = np.cumsum(h)
    hit = np.flatnonzero(cum >= frac * tot)
    return int(hit[0]) if hit.size else HIST - 1


@pytest.mark.parametrize("seed", range(6))
def test_any_selection_gives_dijkstras_distances(seed):
    rng = np.random.default_rng(seed)
    g = gg.rmat(9, 8, seed=seed) if seed % 2 else gg.from_edges(
        300, rng.integers(0, 300, 2000), rng.integers(0, 300, 2000), name="rand")
    w = gg.weights(g, seed + 50)
    src = gg.max_out_degree_vertex(g)
    exp = oracle.dijkstra(g, w, src)
    # a threshold is never below the lowest pending bucket (the kernel's is the first
    # bucket its sample reaches the target in, and a sample is never empty): every round
    # expands at least the closest pending vertex
    low = lambda p, d, b: min(bucket(int(d[v]), b) for v in p)
    rules = {
        "smallest": low,
        "largest": lambda p, d, b: HIST - 1,
        "random": lambda p, d, b: low(p, d, b) + int(rng.integers(0, 8)),
        "sampled 10%": sampled_rule(0.1),
        "sampled 50%": sampled_rule(0.5),
    }
    work = {}
    for name, rule in rules.items():
        got, expanded = rounds_sssp(g, w, src, rule)
        assert np.array_equal(got, exp), name
        work[name] = expanded
    # the small-queue shortcut (expand the pending queue whole) changes nothing either
    got, _ = rounds_sssp(g, w, src, sampled_rule(0.1), big=200)
    assert np.array_equal(got, exp)
    # expanding the closest vertices first does less work than expanding everything
    assert work["sampled 10%"] <= work["largest"]


def two_level_search(h, want_num, etot):
    """The kernel's search: lane l sums segment l, one scan over the 32 segment sums finds
    the first with cum * etot >= want_num, one scan within it finds the bucket."""
    seg = h.reshape(32, 32).sum(axis=1)
    sc = np.cumsum(seg)
    hits = np.flatnonzero(sc * etot >= want_num)
    if hits.size == 0:
        return HIST - 1
    sg = int(hits[0])
    before = int(sc[sg] - seg[sg])
    b = before + np.cumsum(h[sg * 32:(sg + 1) * 32])
    return sg * 32 + int(np.flatnonzero(b * etot >= want_num)[0])


@pytest.mark.parametrize("seed", range(30))
def test_two_level_threshold_search_matches_direct_search(seed):
    rng = np.random.default_rng(900 + seed)
    h = np.zeros(HIST, dtype=np.int64)
    k = int(rng.integers(1, 60))
    h[rng.integers(0, HIST if seed % 3 else 40, k)] = rng.integers(1, 5000, k)
    etot = int(rng.integers(1, 1 << 24))
    tot = int(h.sum())
    B = int(rng.integers(1, 1 << 22))
    want = B * tot
    direct = np.flatnonzero(np.cumsum(h) * etot >= want)
    exp = int(direct[0]) if direct.size else HIST - 1
    assert two_level_search(h, want, etot) == exp
