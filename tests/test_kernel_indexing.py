"""Host emulation of the expansion kernel's warp-level index arithmetic.

The persistent kernel cuts a frontier's edge space into chunks (ChunkSched: one 32-edge
chunk per warp on small frontiers, else rounds of chunks of 1..cap 128-edge units, each
round about half of what is left); the enqueue records, for every 128-edge boundary,
the queue slot of the entry holding it (the chunk index).  A warp expanding a chunk starts a 32-entry window of frontier
entries at that slot and maps each lane to one edge with a ballot over ended entries,
a __reduce_or of start bits and a popc over lanemask_le.  This test replays exactly
that arithmetic in numpy (one vector = one warp) over random frontiers and checks that
every lane reads column start[u] + (e - off[u]) of the entry u that owns edge e, i.e.
that no column read can leave its row, and that every edge is expanded exactly once --
including the fast path that skips the per-group arithmetic when lane 0's entry covers a
whole 128-edge iteration, and the path that maps all four groups of an iteration from
one window position when its 32 entries reach the iteration's end.
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


CHUNK = 128  # the index granularity (kIndexEdges)
CAP_BFS, CAP_SSSP = 16, 4  # kChunkUnitsMax, kChunkUnitsMaxSssp: units per chunk at most


def round_units(rem, gw, cap):
    return min(cap, max(1, (rem + 2 * gw - 1) // (2 * gw)))


class Sched:
    """ChunkSched of one warp: sched_init, then sched_chunk for growing chunk ids."""

    def __init__(self, E, gw, cap):
        small = E <= gw * 32
        self.E, self.gw, self.cap = E, gw, cap
        self.shift = 5 if small else 7
        self.U = (E + (1 << self.shift) - 1) >> self.shift
        self.k0, self.base = 0, 0
        self.s = 1 if small else round_units(self.U, gw, cap)

    def more(self):
        return self.U > self.gw * self.s

    def chunk(self, k):
        k0, base, s = self.k0, self.base, self.s
        ok = True
        while k - k0 >= self.gw:
            base += self.gw * s
            assert base < 1 << 32
            if base >= self.U:
                ok = False
                break
            k0 += self.gw
            s = round_units(self.U - base, self.gw, self.cap)
        self.k0, self.base, self.s = k0, base, s
        u0 = base + (k - k0) * s
        if not ok or u0 >= self.U:
            return None
        return u0 << self.shift, min((u0 + s) << self.shift, self.E)


def schedule_chunks(E, gw, cap, rng):
    """Every chunk the warps of one interval expand, in a random interleaving of their
    cursor claims: round 0's chunk w is warp w's, later ids come from one counter."""
    warps = [Sched(E, gw, cap) for _ in range(gw)]
    more = warps[0].more()
    out, live, cursor = [], [], 0
    for w in range(gw):
        r = warps[w].chunk(w)
        if r is not None:
            out.append(r)
            live.append(w)
    while more and live:
        i = int(rng.integers(0, len(live)))
        w = live[i]
        r = warps[w].chunk(gw + cursor)
        cursor += 1
        if r is None:
            live.pop(i)
        else:
            out.append(r)
    return out, more


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
        # one slide to the iteration's first edge; if the window then reaches the
        # iteration's end, the groups map their lanes without sliding again
        ended = ballot(np.array([w[1] <= it for w in win]))
        if ended:
            n = popc(ended)
            wb += n
            win = [win[(l + n) & 31] if l + n < 32 else load(qo, qs, F, Etot, wb + l) for l in range(32)]
        if win[31][1] >= min(it + 128, E1):
            for c in range(it, min(it + 128, E1), 32):
                km = ballot(np.array([w[0] <= c for w in win]))
                k = km.bit_length() - 1
                assert k >= 0
                bits = 0
                for l in range(32):
                    rel = (win[l][0] - c) & FULL
                    if ((rel - 1) & FULL) < 31:
                        bits |= 1 << rel
                for l in range(32):
                    idx = k + popc(bits & ((2 << l) - 1))
                    e = c + l
                    if e < E1:
                        assert idx < 32
                        s0, o0 = win[idx][2], win[idx][0]
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
    for gw in (1, 3, 8, 31, 64, 4712):  # warps of the interval (M * NW)
        for cap in (CAP_BFS, CAP_SSSP):
            seen = np.zeros(Etot, dtype=np.int64)
            chunks, _ = schedule_chunks(Etot, gw, cap, rng)
            for c0, c1 in chunks:
                if Etot > gw * 32:  # wide frontier: indexed starts, at most cap units
                    assert c0 % CHUNK == 0 and c1 - c0 <= cap * CHUNK
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


@pytest.mark.parametrize("E", [1, 31, 32, 33, 127, 128, 129, 4095, 150784, 150785, 300000, 36508052, 27740094,
                               (1 << 31) - 1])
@pytest.mark.parametrize("gw", [1, 2, 31, 4712, 63488])
def test_chunk_schedule_covers_the_edge_space_once(E, gw):
    """The chunk ranges of ChunkSched tile [0, E) exactly, whatever order the cursor's ids
    reach the warps in; each round takes about half of what is left; the counts stay in
    32 bits.  (R-MAT 22's two wide BFS levels are among the sizes.)"""
    rng = np.random.default_rng(E % 1000 + gw)
    for cap in (CAP_BFS, CAP_SSSP):
        if E > 50_000_000 and (gw < 31 or cap == CAP_SSSP):
            continue  # the emulation walks every chunk: keep the host time small
        chunks, more = schedule_chunks(E, gw, cap, rng)
        chunks.sort()
        assert chunks[0][0] == 0 and chunks[-1][1] == E
        for (a0, a1), (b0, b1) in zip(chunks, chunks[1:]):
            assert a1 == b0 and a0 < a1
        if E <= gw * 32:
            assert not more and len(chunks) == (E + 31) // 32 and all(c1 - c0 <= 32 for c0, c1 in chunks)
        else:
            assert all(c0 % CHUNK == 0 and c1 - c0 <= cap * CHUNK for c0, c1 in chunks)


def test_chunk_schedule_shrinks_towards_the_end():
    """R-MAT 22's first wide level with 152 CTAs of 31 warps: most edges go in chunks of
    the cap, the last chunks are single 128-edge units, and there are far fewer chunk
    starts than with fixed 512-edge chunks."""
    E, gw = 36508052, 152 * 31
    chunks, _ = schedule_chunks(E, gw, CAP_BFS, np.random.default_rng(1))
    sizes = np.array(sorted(chunks))[:, 1] - np.array(sorted(chunks))[:, 0]
    assert sizes[0] == CAP_BFS * CHUNK and sizes[-2] == CHUNK
    big = sizes[sizes == CAP_BFS * CHUNK].sum()
    assert big > 0.5 * E
    assert len(chunks) < (E + 511) // 512 / 2


def test_claim_ring_never_overwrites_a_pending_candidate():
    """The BFS claim ring (kCand = 64 slots): after every 32-edge group at most 32 new
    candidates arrive, and 32 are claimed whenever 32 or more are pending, so no slot is
    rewritten while it still holds a pending candidate."""
    rng = np.random.default_rng(9)
    ring = [None] * 64
    ch = ct = 0
    for _ in range(20000):
        n = int(rng.integers(0, 33)) if rng.random() < 0.3 else int(rng.integers(0, 4))
        for i in range(n):
            slot = (ct + i) & 63
            assert ring[slot] is None, "a pending candidate would be overwritten"
            ring[slot] = ct + i
        ct += n
        if ct - ch >= 32:
            for i in range(32):
                assert ring[(ch + i) & 63] == ch + i
                ring[(ch + i) & 63] = None
            ch += 32
        assert ct - ch <= 63


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


# ---- p-sssp relax interval: heavy rows as a chunk list dealt out over the grid --------
TOPO_HEAVY, TOPO_CHUNK = 512, 256  # kTopoHeavy, kTopoChunk


def topo_heavy_enabled(V, E):
    """The host's condition for listing heavy rows (the list lives in a V-entry queue)."""
    return E // TOPO_CHUNK + E // TOPO_HEAVY + 1 <= V


def relax_edges_cover(cnt, e0, e1):
    """relax_edges: 32 lanes, two edges per lane in flight, steps of 64 edges."""
    if e1 <= e0:
        return
    e = (np.arange(e0, e1, 64)[:, None, None] + 32 * np.arange(2)[None, :, None]
         + np.arange(32)[None, None, :]).ravel()
    np.add.at(cnt, e[e < e1], 1)


def emulate_topo_relax(row_off, flagged, M, NW, rng):
    """The update interval lists the flagged heavy rows (in any order: lanes race on the
    counter); the relax interval deals chunk j to warp j mod G and every warp scans its
    32-vertex stripes, skipping listed rows.  Returns relaxations per edge and the list
    length."""
    V, E = len(row_off) - 1, int(row_off[-1])
    on = topo_heavy_enabled(V, E)
    lst = []
    for v in rng.permutation(np.asarray(flagged, dtype=np.int64)):
        a, b = int(row_off[v]), int(row_off[v + 1])
        if on and b - a >= TOPO_HEAVY:
            n = (b - a + TOPO_CHUNK - 1) // TOPO_CHUNK
            assert len(lst) + n <= V, "the list would outgrow its queue"
            lst.extend((int(v), a + k * TOPO_CHUNK) for k in range(n))
    fl = np.zeros(V, dtype=bool)
    fl[np.asarray(flagged, dtype=np.int64)] = True
    cnt = np.zeros(E, dtype=np.int64)
    G = M * NW
    nch = min(len(lst), V)
    for gw in range(G):
        for j in range(gw, nch, G):
            u, e0 = lst[j]
            b = int(row_off[u + 1])
            assert 0 <= u < V and e0 < b
            relax_edges_cover(cnt, e0, min(b, e0 + TOPO_CHUNK))
        for base in range(gw * 32, V, G * 32):
            for u in np.flatnonzero(fl[base:base + 32]) + base:
                a, b = int(row_off[u]), int(row_off[u + 1])
                if on and b - a >= TOPO_HEAVY:
                    continue
                relax_edges_cover(cnt, a, b)
    return cnt, len(lst)


def rows_with_degrees(degs):
    return np.concatenate([[0], np.cumsum(degs)]).astype(np.int64)


@pytest.mark.parametrize("seed", range(8))
def test_topo_heavy_rows_relaxed_exactly_once(seed):
    """Every edge of a flagged row is relaxed once (heavy rows through the chunk list,
    the others by the stripe scan), no other edge is, for grids of any size."""
    rng = np.random.default_rng(700 + seed)
    V = int(rng.integers(3000, 9000))
    degs = rng.integers(0, 12, size=V)
    hubs = rng.choice(V, size=int(rng.integers(1, 6)), replace=False)
    degs[hubs] = rng.integers(TOPO_HEAVY - 1, 4 * TOPO_HEAVY + 300, size=len(hubs))
    degs[hubs[0]] = TOPO_HEAVY  # exactly at the threshold
    row_off = rows_with_degrees(degs)
    assert topo_heavy_enabled(V, int(row_off[-1]))
    flagged = np.union1d(rng.choice(V, size=V // 5, replace=False), hubs[: max(1, len(hubs) - 1)])
    M, NW = int(rng.integers(1, 5)), int(rng.choice([1, 3, 31]))
    cnt, n_list = emulate_topo_relax(row_off, flagged, M, NW, rng)
    want = np.zeros_like(cnt)
    for v in flagged:
        want[row_off[v]:row_off[v + 1]] = 1
    assert np.array_equal(cnt, want)
    assert n_list > 0


def test_topo_heavy_list_bound_is_tight_but_safe():
    """Adversarial degree sequences at the host's condition: every row heavy and flagged
    (at the threshold, one edge over it, one edge short of a further chunk, and three
    times over) still fits the V-entry queue."""
    rng = np.random.default_rng(5)
    for d in (TOPO_HEAVY, TOPO_HEAVY + 1, TOPO_HEAVY + TOPO_CHUNK - 1, 3 * TOPO_HEAVY + 1):
        H = 7
        E = H * d
        V = E // TOPO_CHUNK + E // TOPO_HEAVY + 1  # the smallest V the host accepts
        degs = np.zeros(V, dtype=np.int64)
        degs[:H] = d
        row_off = rows_with_degrees(degs)
        cnt, n_list = emulate_topo_relax(row_off, np.arange(H), 1, 2, rng)
        assert n_list <= V
        assert np.all(cnt == 1)
    # one vertex fewer and the host turns the list off: the stripe scan relaxes everything
    degs = np.zeros(V - 1, dtype=np.int64)
    degs[:H] = d
    row_off = rows_with_degrees(degs)
    assert not topo_heavy_enabled(V - 1, int(row_off[-1]))
    cnt, n_list = emulate_topo_relax(row_off, np.arange(H), 1, 2, rng)
    assert n_list == 0 and np.all(cnt == 1)
