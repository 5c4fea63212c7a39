"""Host emulation of the expansion kernel's warp-level index arithmetic.

The persistent kernel cuts a frontier's edge space into CHUNK-edge chunks; the
enqueue records, for every chunk boundary, the queue slot of the entry holding it
(the chunk index).  A warp expanding a chunk starts a 32-entry window of frontier
entries at that slot and maps each lane to one edge with a ballot over ended entries,
a __reduce_or of start bits and a popc over lanemask_le.  This test replays exactly
that arithmetic in numpy (one vector = one warp) over random frontiers and checks that
every lane reads column start[u] + (e - off[u]) of the entry u that owns edge e, i.e.
that no column read can leave its row, and that every edge is expanded exactly once --
including the fast path that skips the per-group arithmetic when lane 0's entry covers a
whole 128-edge iteration.
It runs before any GPU code does.
"""
import numpy as np
import pytest

LANES = np.arange(32, dtype=np.int64)
FULL = 0xFFFFFFFF
MAXU = 0xFFFFFFFF


def ballot(pred):
    return int(np.sum((pred.astype(np.int64)) << LANES))


def popc(x):
    return bin(x & FULL).count("1")


def find_entry(qo, F, x):
    lo, hi = 0, F
    while hi - lo > 32:
        step = (hi - lo + 31) // 32
        idx = lo + LANES * step
        pred = np.array([i < hi and qo[i] <= x for i in idx])
        b = ballot(pred)
        L = b.bit_length() - 1
        nlo = lo + L * step
        hi = min(nlo + step, hi)
        lo = nlo
    idx = lo + LANES
    pred = np.array([i < hi and qo[i] <= x for i in idx])
    return lo + ballot(pred).bit_length() - 1


def load(qo, qs, F, Etot, i):
    if i < F:
        return qo[i], (qo[i + 1] if i + 1 < F else Etot), qs[i]
    return MAXU, MAXU, 0


CHUNK = 128  # the index granularity (kIndexEdges); chunks are 1..8 units


def index_chunks(qo, degs, nchunks):
    """The enqueue's chunk index: slot of the entry holding edge j*CHUNK, for every j."""
    qx = np.full(nchunks, -1, dtype=np.int64)
    for slot, (o, d) in enumerate(zip(qo, degs)):
        j = (o + CHUNK - 1) // CHUNK
        while j * CHUNK < o + d:
            qx[j] = slot
            j += 1
    return qx


def emulate_warp(qo, qs, F, Etot, E0, E1, wb=None):
    """Returns a list of (edge, column position) exactly as the kernel computes them."""
    out = []
    if wb is None:
        wb = find_entry(qo, F, E0)
    win = [load(qo, qs, F, Etot, wb + l) for l in range(32)]
    while True:  # catch-up slides until lane 0 holds the entry containing E0
        ended = ballot(np.array([w[1] <= E0 for w in win]))
        if not ended:
            break
        n = popc(ended)
        wb += n
        win = [win[(l + n) & 31] if l + n < 32 else load(qo, qs, F, Etot, wb + l) for l in range(32)]
    for it in range(E0, E1, 128):  # one kernel iteration: 4 groups of 32 edges
        if win[0][1] >= it + 128:  # fast path: lane 0's entry covers the whole iteration
            s0, o0 = win[0][2], win[0][0]
            for e in range(it, min(it + 128, E1)):
                out.append((e, (s0 + ((e - o0) & FULL)) & FULL))
            continue
        for c in range(it, min(it + 128, E1), 32):
            ended = ballot(np.array([w[1] <= c for w in win]))
            if ended:
                n = popc(ended)
                wb += n
                new = []
                for l in range(32):
                    new.append(win[(l + n) & 31] if l + n < 32 else load(qo, qs, F, Etot, wb + l))
                win = new
            bits = 0
            for l in range(32):
                rel = (win[l][0] - c) & FULL
                if l != 0 and rel < 32:
                    bits |= 1 << rel
            for l in range(32):
                idx = popc(bits & ((2 << l) - 1))
                s0, o0 = win[idx][2], win[idx][0]
                e = c + l
                if e < E1:
                    out.append((e, (s0 + ((e - o0) & FULL)) & FULL))
    return out


def check_frontier_chunks(degs, rng):
    """The chunked scheme: every chunk starts at its indexed entry, no search."""
    F = len(degs)
    qo = np.concatenate([[0], np.cumsum(degs)[:-1]]).astype(np.int64)
    Etot = int(np.sum(degs))
    gaps = rng.integers(0, 5, size=F)
    qs = np.concatenate([[0], np.cumsum(degs + gaps)[:-1]]).astype(np.int64)
    owner = np.repeat(np.arange(F), degs)
    nchunks = (Etot + CHUNK - 1) // CHUNK
    qx = index_chunks(qo, degs, nchunks)
    assert np.all(qx >= 0)
    assert np.array_equal(qx, owner[np.arange(nchunks) * CHUNK])
    for mult in (1, 3, 8, 16):  # chunks of 32*mult edges, started from the 128-edge index
        units = (Etot + 31) // 32
        seen = np.zeros(Etot, dtype=np.int64)
        for j in rng.permutation((units + mult - 1) // mult):
            c0, c1 = j * 32 * mult, min((j + 1) * 32 * mult, Etot)
            for e, pos in emulate_warp(qo, qs, F, Etot, c0, c1, wb=int(qx[c0 // CHUNK])):
                u = owner[e]
                assert pos == qs[u] + (e - qo[u])
                seen[e] += 1
        assert np.all(seen == 1)


@pytest.mark.parametrize("seed", range(12))
def test_chunk_index_random_frontiers(seed):
    rng = np.random.default_rng(100 + seed)
    F = int(rng.integers(1, 300))
    if seed % 3 == 0:
        degs = rng.integers(1, 40, size=F)
    elif seed % 3 == 1:
        degs = np.minimum(rng.zipf(1.5, size=F), 9000)
    else:
        degs = rng.integers(1, 20, size=F)
        degs[rng.integers(0, F)] = 3 * CHUNK + 17   # a hub spanning several chunks
    check_frontier_chunks(degs.astype(np.int64), rng)


def check_frontier(degs, n_warps, rng):
    F = len(degs)
    qo = np.concatenate([[0], np.cumsum(degs)[:-1]]).astype(np.int64)
    Etot = int(np.sum(degs))
    # rows placed at arbitrary, non-overlapping column positions
    gaps = rng.integers(0, 5, size=F)
    qs = np.concatenate([[0], np.cumsum(degs + gaps)[:-1]]).astype(np.int64) + int(rng.integers(0, 9))
    owner = np.repeat(np.arange(F), degs)
    seen = np.zeros(Etot, dtype=np.int64)
    for gw in range(n_warps):
        E0 = Etot * gw // n_warps
        E1 = Etot * (gw + 1) // n_warps
        if E0 >= E1:
            continue
        for e, pos in emulate_warp(qo, qs, F, Etot, E0, E1):
            u = owner[e]
            assert pos == qs[u] + (e - qo[u]), (e, pos)
            assert qs[u] <= pos < qs[u] + degs[u]
            seen[e] += 1
    assert np.all(seen == 1), "every edge of the frontier exactly once"


@pytest.mark.parametrize("seed", range(40))
def test_window_arithmetic_random_frontiers(seed):
    rng = np.random.default_rng(seed)
    F = int(rng.integers(1, 400))
    kind = seed % 4
    if kind == 0:
        degs = rng.integers(1, 5, size=F)             # grid-like
    elif kind == 1:
        degs = np.minimum(rng.zipf(1.6, size=F), 3000)  # skewed, R-MAT-like
    elif kind == 2:
        degs = np.ones(F, dtype=np.int64)              # 32 entries end per chunk
    else:
        degs = rng.integers(1, 70, size=F)
        degs[rng.integers(0, F)] = 5000                # one hub spanning many warps
    check_frontier(degs.astype(np.int64), int(rng.integers(1, 80)), rng)


def test_window_arithmetic_single_entry_and_exact_multiples():
    rng = np.random.default_rng(0)
    check_frontier(np.array([1]), 5, rng)
    check_frontier(np.array([32]), 1, rng)
    check_frontier(np.array([32] * 10), 3, rng)
    check_frontier(np.array([31, 1, 33, 64, 1, 1]), 7, rng)
