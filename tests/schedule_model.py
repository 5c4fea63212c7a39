"""Host model of the forced kill/fork schedule the releaser draws (coop_set_schedule).

At barrier b (1-based) the releaser draws r = mix64(seed ^ mix64(b)) and r2 = mix64(r)
(SplitMix64's finaliser); with probability p_fork (the high half of r against
p_fork * 2^32) it wants kcap = r2 mod (N - M + 1) CTAs in flight and launches the ones
not yet pending; it admits every registered joiner, up to N - M; with probability
p_kill (the low half of r) it accepts W = (r2 >> 32) mod M offer_kills, never CTA 0.
The model assumes that CTAs launched at one barrier have registered by the next, which
holds when intervals last longer than a device-side launch (the wide R-MAT levels).
"""
M64 = (1 << 64) - 1


def mix64(z):
    z = (z + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def simulate(seed, p_kill, p_fork, N, n_barriers):
    """(kills, forks admitted, CTAs spawned, final M) over n_barriers resizing barriers."""
    pk = min(0xFFFFFFFF, int(p_kill * 4294967296.0))
    pf = min(0xFFFFFFFF, int(p_fork * 4294967296.0))
    M, admitted, launched, registered = N, N - 1, N, N - 1
    kills = forks = spawned = 0
    for b in range(1, n_barriers + 1):
        r = mix64((seed ^ mix64(b)) & M64)
        r2 = mix64(r)
        k = min(N - M, registered - admitted)
        kcap = r2 % (N - M + 1) if (r >> 32) < pf else 0
        spawn = kcap - (launched - 1 - admitted)
        if spawn > 0:
            launched += spawn
            spawned += spawn
        ws = (r2 >> 32) % M if (r & 0xFFFFFFFF) < pk else 0
        w = min(ws, M + k - 1)
        M = M + k - w
        admitted += k
        kills += w
        forks += k
        registered = launched - 1
    return kills, forks, spawned, M


# R-MAT scale 22 BFS from its highest out-degree vertex: six levels, so five resizing
# barriers open a further interval (the sixth ends the traversal); the bench's schedules
RMAT22_RESIZING_BARRIERS = 5
RMAT22_SCHEDULE = (0.5, 1.0)  # (p_kill, p_fork)
RMAT22_SEEDS = (0, 1, 2, 3)
