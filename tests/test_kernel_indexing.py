"""Host emulation of the expansion kernel's warp-level index arithmetic.

The persistent kernel maps each lane of a warp to one edge of the frontier's edge
space with a 32-ary search, a 32-entry window of frontier entries held in registers,
a ballot over ended entries, a __reduce_or of start bits and a popc over
lanemask_le.  This test replays exactly that arithmetic in numpy (one vector = one
warp) over random frontiers and checks that every lane reads column
start[u] + (e - off[u]) of the entry u that owns edge e, i.e. that no column read can
leave its row.  It runs before any GPU code does.
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


def emulate_warp(qo, qs, F, Etot, E0, E1):
    """Returns a list of (edge, column position) exactly as the kernel computes them."""
    out = []
    wb = find_entry(qo, F, E0)
    win = [load(qo, qs, F, Etot, wb + l) for l in range(32)]
    c = E0
    while c < E1:
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
        c += 32
    return out


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
