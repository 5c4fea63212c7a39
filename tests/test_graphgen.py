"""Checks on the seeded input generators (determinism, shape, the R-MAT distribution)."""
import numpy as np
import pytest

import graphgen as gg


def _edge_set(g):
    u = np.repeat(np.arange(g.num_vertices, dtype=np.int64), g.out_degree())
    return u, g.col.astype(np.int64)


def test_grid_shape():
    g = gg.grid(256, 256)
    assert g.num_vertices == 65536 and g.num_edges == 261120  # 4*256*255, no wraparound
    deg = g.out_degree()
    assert sorted(set(deg.tolist())) == [2, 3, 4]
    assert (deg == 2).sum() == 4 and (deg == 3).sum() == 4 * 254
    u, v = _edge_set(g)
    fwd = set(zip(u.tolist(), v.tolist()))
    assert all((b, a) in fwd for a, b in list(fwd)[:5000])  # undirected
    assert np.all(np.abs(u - v) != 0)


def test_csr_rows_sorted_dedup_no_self_loops():
    g = gg.rmat(14, 16, seed=9)
    u, v = _edge_set(g)
    assert np.all(u != v)
    same_row = u[1:] == u[:-1]
    assert np.all(v[1:][same_row] > v[:-1][same_row])  # strictly ascending => no duplicates
    assert g.row_off[0] == 0 and g.row_off[-1] == g.num_edges
    assert np.all(np.diff(g.row_off) >= 0)


def test_rmat_deterministic_across_thread_counts():
    a = gg.rmat.__wrapped__(12, 16, seed=5, threads=1)
    b = gg.rmat.__wrapped__(12, 16, seed=5, threads=7)
    np.testing.assert_array_equal(a.row_off, b.row_off)
    np.testing.assert_array_equal(a.col, b.col)
    c = gg.rmat.__wrapped__(12, 16, seed=6, threads=3)
    assert not np.array_equal(a.col[: min(a.num_edges, c.num_edges)], c.col[: min(a.num_edges, c.num_edges)])


def test_rmat_generated_edges_match_definition():
    """Recompute a few generated edges from the SplitMix64 / quadrant definition."""
    scale, ef, seed = 8, 4, 77
    g = gg.rmat(scale, ef, seed=seed)
    u_all, v_all = _edge_set(g)
    present = set(zip(u_all.tolist(), v_all.tolist()))
    s0 = gg.splitmix64(seed)
    M64 = (1 << 64) - 1
    checked = 0
    for i in range(200):
        u = v = 0
        for b in range(scale):
            h = gg.splitmix64(s0 ^ ((i << 6) | b))
            r = (h >> 11) * (1.0 / 9007199254740992.0)
            ub, vb = (0, 0) if r < 0.57 else (0, 1) if r < 0.76 else (1, 0) if r < 0.95 else (1, 1)
            u, v = (u << 1) | ub, (v << 1) | vb
        if u != v:
            assert (u, v) in present
            checked += 1
    assert checked > 150
    assert gg.splitmix64(0) == 0xE220A8397B1DCDAF  # SplitMix64 of 0 (published test value)
    del M64


def test_rmat_quadrant_frequencies():
    """Top-bit quadrant shares follow a, b, c, d (loose: dedup thins the dense quadrant)."""
    g = gg.rmat(16, 16, seed=1)
    u, v = _edge_set(g)
    half = g.num_vertices // 2
    qa = np.mean((u < half) & (v < half))
    qb = np.mean((u < half) & (v >= half))
    qc = np.mean((u >= half) & (v < half))
    qd = np.mean((u >= half) & (v >= half))
    assert abs(qb - qc) < 0.01
    assert qa > qb > qd and 0.45 < qa < 0.62 and 0.17 < qb < 0.24 and 0.03 < qd < 0.09
    assert g.num_edges > 0.8 * 16 * 65536


def test_weights():
    g = gg.rmat(10, 8, seed=2)
    w = gg.weights(g, 3)
    assert w.dtype == np.uint32 and w.min() >= 1 and w.max() <= 255
    np.testing.assert_array_equal(w, gg.weights(g, 3))
    assert not np.array_equal(w, gg.weights(g, 4))
    # a function of the edge: the same (u, v) in another graph gets the same weight
    u, v = _edge_set(g)
    sub = gg.from_edges(g.num_vertices, u[::3], v[::3])
    ws = gg.weights(sub, 3)
    lookup = dict(zip(zip(u.tolist(), v.tolist()), w.tolist()))
    su, sv = _edge_set(sub)
    assert all(lookup[(a, b)] == x for a, b, x in zip(su.tolist(), sv.tolist(), ws.tolist()))


def test_from_edges_cleanup_and_errors():
    g = gg.from_edges(4, [0, 0, 0, 1, 2, 2], [1, 1, 0, 2, 3, 2])
    assert g.row_off.tolist() == [0, 1, 2, 3, 3] and g.col.tolist() == [1, 2, 3]
    with pytest.raises(ValueError):
        gg.from_edges(3, [0], [3])


def test_source_rule():
    g = gg.from_edges(5, [1, 1, 3, 3, 4], [0, 2, 0, 1, 0])
    assert gg.max_out_degree_vertex(g) == 1  # tie between 1 and 3 goes to the smaller id
