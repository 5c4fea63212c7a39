"""Pins of the octree oracle (oracle/octree.py) against what the definition fixes.

The octree of the work-stealing application (Table 1 "octree"; Sec. 3.2 "Adapting Work
Stealing") under the reading stated in the oracle: cells split by coordinate bit
20 - depth while they hold more than leaf_cap points.  Pins: a lattice whose tree is known
in closed form, the non-recursive per-point characterisation (brute force), identical
points, the partition invariants, and planted mistakes that these pins must catch.
"""
import numpy as np
import pytest

import graphgen as gg
from oracle import octree as ot


def _morton3(i, j, k, levels):
    c = 1
    for b in range(levels - 1, -1, -1):
        c = (c << 3) | ((i >> b) & 1) | (((j >> b) & 1) << 1) | (((k >> b) & 1) << 2)
    return c


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_lattice_closed_form(levels):
    """8^L points on a lattice, one per cell at depth L: with leaf_cap 1 every point is a
    leaf at depth L named by its cell; with leaf_cap 8 the leaves are the depth-(L-1)
    cells, 8 points each."""
    m = 1 << levels
    i, j, k = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    sh = 21 - levels
    x, y, z = (a.astype(np.uint32) << sh for a in (i, j, k))
    leaves = ot.octree_leaves(x, y, z, 1)
    assert len(leaves) == m ** 3
    for code, d, idx in leaves:
        assert d == levels and len(idx) == 1
        p = int(idx[0])
        assert code == _morton3(int(i[p]), int(j[p]), int(k[p]), levels)
    leaves8 = ot.octree_leaves(x, y, z, 8)
    assert len(leaves8) == (m // 2) ** 3
    assert all(d == levels - 1 and len(idx) == 8 for _, d, idx in leaves8)


@pytest.mark.parametrize("case", range(12))
def test_recursive_equals_bruteforce(case):
    rng = np.random.default_rng(50 + case)
    n = int(rng.integers(1, 600))
    kind = ("uniform", "clustered")[case % 2]
    x, y, z = gg.points(n, 60 + case, kind)
    if case % 4 == 3:  # duplicates
        x[: n // 3], y[: n // 3], z[: n // 3] = x[0], y[0], z[0]
    cap = int(rng.integers(1, 20))
    md = int(rng.integers(0, 22))
    assert np.array_equal(ot.leaf_code_of_points(x, y, z, cap, md), ot.leaf_codes_bruteforce(x, y, z, cap, md))


def test_identical_points_stop_at_max_depth():
    x = np.full(50, 12345, np.uint32)
    y = np.full(50, 777, np.uint32)
    z = np.full(50, 2 ** 21 - 1, np.uint32)
    leaves = ot.octree_leaves(x, y, z, 4, 21)
    assert len(leaves) == 1
    code, d, idx = leaves[0]
    assert d == 21 and len(idx) == 50 and code == _morton3(12345, 777, 2 ** 21 - 1, 21)
    assert ot.octree_leaves(x, y, z, 4, 6)[0][1] == 6


def test_partition_invariants():
    x, y, z = gg.points(20000, 7, "clustered")
    cap = 16
    leaves = ot.octree_leaves(x, y, z, cap)
    allidx = np.concatenate([idx for _, _, idx in leaves])
    assert np.array_equal(np.sort(allidx), np.arange(20000))  # a partition of the points
    key = ot.octant_digits(x, y, z)
    for code, d, idx in leaves[::37]:
        assert len(idx) <= cap or d == 21
        assert ot.code_depth(code) == d
        # every point of the leaf has the leaf's prefix, and the parent cell held > cap
        assert np.all((key[idx] >> np.uint64(63 - 3 * d)) == np.uint64(code ^ (1 << 3 * d)))
        if d > 0:
            parent = (code >> 3) ^ (1 << 3 * (d - 1))
            assert np.sum((key >> np.uint64(63 - 3 * (d - 1))) == np.uint64(parent)) > cap


def test_planted_mistakes_are_caught(monkeypatch):
    x, y, z = gg.points(500, 3, "clustered")
    good = ot.leaf_codes_bruteforce(x, y, z, 6)
    # (1) octant bits in the wrong order
    real = ot.octant_digits

    def swapped(a, b, c):
        return real(c, b, a)

    monkeypatch.setattr(ot, "octant_digits", swapped)
    assert not np.array_equal(ot.leaf_code_of_points(x, y, z, 6), good)
    monkeypatch.setattr(ot, "octant_digits", real)
    # (2) splitting a cell that holds exactly leaf_cap points
    assert not np.array_equal(ot.leaf_code_of_points(x, y, z, 5), good)
    assert np.array_equal(ot.leaf_code_of_points(x, y, z, 6), good)


def test_points_generator_is_deterministic_and_in_range():
    a = gg.points(1000, 11, "clustered")
    b = gg.points(1000, 11, "clustered")
    for u, v in zip(a, b):
        assert u.dtype == np.uint32 and np.array_equal(u, v) and int(u.max()) < 2 ** 21
    assert not np.array_equal(a[0], gg.points(1000, 12, "clustered")[0])
