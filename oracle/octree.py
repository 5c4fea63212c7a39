"""CPU oracle for octree partitioning, the paper's work-stealing application.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` leg may import this module; the product path never does.  It shares
no code with the CUDA path; the inputs come from :mod:`graphgen` (``points``).

Table 1 lists "octree" among the work-stealing applications (no barriers, one kill and
one fork point at the head of the main loop, Sec. 3.2 "Adapting Work Stealing"); the
paper gives no construction rule.  Reading used here (and by the kernel):

* points have integer coordinates in [0, 2^21)^3; the root cell is the whole cube, at
  depth 0;
* a cell at depth d < max_depth holding more than ``leaf_cap`` points is split into its
  8 octants by coordinate bit (20 - d) of x, y and z, octant = bx | by << 1 | bz << 2;
  empty octants are dropped;
* every other cell holding points is a leaf.  A leaf is named by its path code: a 1
  followed by 3 bits (the octant) per level below the root, so the root is 1 and a
  depth-d code has its leading 1 at bit 3d.

The leaves and the set of points in each are then unique; only the order of points
inside a leaf, and of leaves in memory, depends on the schedule.

:func:`octree_leaves` builds the tree top-down over points sorted by their octant digits
(the recursive definition); :func:`leaf_codes_bruteforce` computes each point's leaf from
the non-recursive characterisation -- the shortest coordinate prefix shared by at most
``leaf_cap`` points, or max_depth -- and pins the first.
"""
from __future__ import annotations

import numpy as np

COORD_BITS = 21
MAX_DEPTH = COORD_BITS


def octant_digits(x, y, z) -> np.ndarray:
    """Key whose 3-bit digit d (most significant first) is the octant at depth d."""
    x = np.asarray(x, dtype=np.uint64)
    y = np.asarray(y, dtype=np.uint64)
    z = np.asarray(z, dtype=np.uint64)
    key = np.zeros(x.shape, dtype=np.uint64)
    for b in range(COORD_BITS - 1, -1, -1):
        o = ((x >> np.uint64(b)) & np.uint64(1)) | (((y >> np.uint64(b)) & np.uint64(1)) << np.uint64(1)) | \
            (((z >> np.uint64(b)) & np.uint64(1)) << np.uint64(2))
        key = (key << np.uint64(3)) | o
    return key


def _check_args(x, y, z, leaf_cap, max_depth):
    if not (len(x) == len(y) == len(z)):
        raise ValueError("coordinate arrays differ in length")
    if leaf_cap < 1 or not (0 <= max_depth <= MAX_DEPTH):
        raise ValueError("leaf_cap >= 1 and 0 <= max_depth <= 21")
    for a in (x, y, z):
        if len(a) and int(np.max(a)) >= (1 << COORD_BITS):
            raise ValueError("coordinates must be below 2^21")


def octree_leaves(x, y, z, leaf_cap: int, max_depth: int = MAX_DEPTH):
    """Leaves of the octree, top-down: a list of (code, depth, sorted point indices)."""
    _check_args(x, y, z, leaf_cap, max_depth)
    n = len(x)
    if n == 0:
        return []
    key = octant_digits(x, y, z)
    order = np.argsort(key, kind="stable")
    skey = key[order]
    leaves = []
    stack = [(0, n, 0, 1)]  # (lo, hi) in sorted order, depth, code
    while stack:
        lo, hi, d, code = stack.pop()
        if hi - lo <= leaf_cap or d == max_depth:
            leaves.append((code, d, np.sort(order[lo:hi])))
            continue
        shift = np.uint64(3 * (COORD_BITS - 1 - d))
        digit = (skey[lo:hi] >> shift) & np.uint64(7)  # sorted within the cell
        bounds = np.searchsorted(digit, np.arange(9, dtype=np.uint64))
        for o in range(8):
            a, b = lo + int(bounds[o]), lo + int(bounds[o + 1])
            if b > a:
                stack.append((a, b, d + 1, (code << 3) | o))
    return leaves


def leaf_code_of_points(x, y, z, leaf_cap: int, max_depth: int = MAX_DEPTH) -> np.ndarray:
    """Per point, the code of its leaf (from :func:`octree_leaves`)."""
    out = np.zeros(len(x), dtype=np.uint64)
    for code, _, idx in octree_leaves(x, y, z, leaf_cap, max_depth):
        out[idx] = np.uint64(code)
    return out


def leaf_codes_bruteforce(x, y, z, leaf_cap: int, max_depth: int = MAX_DEPTH) -> np.ndarray:
    """Per point, its leaf's code from the non-recursive characterisation: the leaf depth
    of a point is the smallest d with at most leaf_cap points sharing its d-bit coordinate
    prefixes (x >> (21 - d), y >> (21 - d), z >> (21 - d)), or max_depth; the code is
    assembled from those prefixes bit by bit."""
    _check_args(x, y, z, leaf_cap, max_depth)
    x = np.asarray(x, dtype=np.int64)
    y = np.asarray(y, dtype=np.int64)
    z = np.asarray(z, dtype=np.int64)
    n = len(x)
    depth = np.full(n, max_depth, dtype=np.int64)
    settled = np.zeros(n, dtype=bool)
    for d in range(0, max_depth + 1):
        s = COORD_BITS - d
        pre = np.stack([x >> s, y >> s, z >> s], axis=1)
        _, inv, cnt = np.unique(pre, axis=0, return_inverse=True, return_counts=True)
        small = (cnt[inv.reshape(-1)] <= leaf_cap) & ~settled
        depth[small] = d
        settled |= small
    codes = np.zeros(n, dtype=np.uint64)
    for i in range(n):
        c = 1
        for level in range(int(depth[i])):
            b = COORD_BITS - 1 - level
            c = (c << 3) | ((int(x[i]) >> b) & 1) | (((int(y[i]) >> b) & 1) << 1) | (((int(z[i]) >> b) & 1) << 2)
        codes[i] = c
    return codes


def code_depth(code: int) -> int:
    """Depth of a leaf code (position of its leading 1, in 3-bit steps)."""
    return (int(code).bit_length() - 1) // 3
