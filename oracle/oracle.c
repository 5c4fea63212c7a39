/*
 * oracle.c - plain, slow, obviously correct CPU reference for the traversal results.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this file;
 * only the tests, the smoke check and the benchmark's CPU-baseline leg do.  It shares
 * no code with the CUDA path.
 *
 * Cooperative graph traversal (Sec. 2.2 Fig. 3 and Sec. 3.2 Fig. 4 of Sorensen, Evrard
 * and Donaldson, "Cooperative Kernels", FSE 2017) reaches, under any schedule of kills
 * and forks (Sec. 3.1: an offer_kill may always be a no-op and k = 0 forks is always
 * legal, so every schedule must compute the same thing), the textbook result.  So the
 * oracle is that textbook result written out:
 *
 *   BFS   level[v] = fewest edges on a directed path src -> v, -1 if none
 *         (first-in first-out queue, Moore 1959 / CLRS 22.2)
 *   SSSP  dist[v]  = least total weight of a directed path src -> v, UINT32_MAX if none
 *         (Dijkstra 1959 with a binary heap, CLRS 24.3; and Bellman-Ford, CLRS 24.1,
 *          as an independent second definition; uint64 accumulators)
 *
 * Brute-force definitions for tiny graphs (Floyd-Warshall, CLRS 25.2) are here too so
 * that the tests can pin the fast definitions against them.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_INF64 UINT64_MAX

/* Breadth-first search from src.  Returns the number of reached vertices, or -1. */
int64_t oracle_bfs(int32_t V, const int32_t *row_off, const int32_t *col, int32_t src,
                   int32_t *level) {
    if (V < 1 || src < 0 || src >= V) return -1;
    int32_t *queue = (int32_t *)malloc((size_t)V * sizeof(int32_t));
    if (!queue) return -1;
    for (int32_t v = 0; v < V; ++v) level[v] = -1;
    int64_t head = 0, tail = 0;
    level[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int32_t e = row_off[u]; e < row_off[u + 1]; ++e) {
            int32_t v = col[e];
            if (level[v] == -1) {
                level[v] = level[u] + 1;
                queue[tail++] = v;
            }
        }
    }
    free(queue);
    return tail;
}

/* ---- Dijkstra with a binary min-heap keyed by tentative distance (lazy deletion) ---- */
typedef struct { uint64_t d; int32_t v; } heap_item;

static void heap_push(heap_item *h, int64_t *n, heap_item x) {
    int64_t i = (*n)++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p].d <= x.d) break;
        h[i] = h[p];
        i = p;
    }
    h[i] = x;
}

static heap_item heap_pop(heap_item *h, int64_t *n) {
    heap_item top = h[0];
    heap_item x = h[--(*n)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        uint64_t md = x.d;
        if (l < *n && h[l].d < md) { m = l; md = h[l].d; }
        if (r < *n && h[r].d < md) { m = r; }
        if (m == i) break;
        h[i] = h[m];
        i = m;
    }
    if (*n > 0) h[i] = x;
    return top;
}

/*
 * Dijkstra from src over non-negative uint32 weights.  dist[v] = UINT32_MAX when v is
 * unreachable.  Returns the number of reached vertices, -1 on bad input, -2 if some
 * shortest distance does not fit below UINT32_MAX.
 */
int64_t oracle_dijkstra(int32_t V, const int32_t *row_off, const int32_t *col, const uint32_t *w,
                        int32_t src, uint32_t *dist) {
    if (V < 1 || src < 0 || src >= V) return -1;
    int64_t E = row_off[V];
    uint64_t *d = (uint64_t *)malloc((size_t)V * sizeof(uint64_t));
    uint8_t *done = (uint8_t *)calloc((size_t)V, 1);
    heap_item *h = (heap_item *)malloc(((size_t)E + 1) * sizeof(heap_item));
    if (!d || !done || !h) { free(d); free(done); free(h); return -1; }
    for (int32_t v = 0; v < V; ++v) d[v] = OR_INF64;
    int64_t n = 0, reached = 0;
    d[src] = 0;
    heap_push(h, &n, (heap_item){0, src});
    while (n > 0) {
        heap_item it = heap_pop(h, &n);
        if (done[it.v] || it.d != d[it.v]) continue;
        done[it.v] = 1;
        ++reached;
        for (int32_t e = row_off[it.v]; e < row_off[it.v + 1]; ++e) {
            int32_t v = col[e];
            uint64_t nd = it.d + (uint64_t)w[e];
            if (nd < d[v]) {
                d[v] = nd;
                heap_push(h, &n, (heap_item){nd, v});
            }
        }
    }
    int64_t rc = reached;
    for (int32_t v = 0; v < V; ++v) {
        if (d[v] == OR_INF64) dist[v] = UINT32_MAX;
        else if (d[v] >= UINT32_MAX) { dist[v] = UINT32_MAX; rc = -2; }
        else dist[v] = (uint32_t)d[v];
    }
    free(d);
    free(done);
    free(h);
    return rc;
}

/*
 * Bellman-Ford from src: relax every edge, round after round, until a round changes
 * nothing (at most V-1 rounds for non-negative weights).  Same output convention as
 * oracle_dijkstra; returns the number of rounds that changed something, or -1/-2.
 */
int64_t oracle_bellman_ford(int32_t V, const int32_t *row_off, const int32_t *col,
                            const uint32_t *w, int32_t src, uint32_t *dist) {
    if (V < 1 || src < 0 || src >= V) return -1;
    uint64_t *d = (uint64_t *)malloc((size_t)V * sizeof(uint64_t));
    if (!d) return -1;
    for (int32_t v = 0; v < V; ++v) d[v] = OR_INF64;
    d[src] = 0;
    int64_t rounds = 0;
    for (int32_t r = 0; r < V; ++r) {
        int changed = 0;
        for (int32_t u = 0; u < V; ++u) {
            if (d[u] == OR_INF64) continue;
            for (int32_t e = row_off[u]; e < row_off[u + 1]; ++e) {
                uint64_t nd = d[u] + (uint64_t)w[e];
                if (nd < d[col[e]]) { d[col[e]] = nd; changed = 1; }
            }
        }
        if (!changed) break;
        ++rounds;
    }
    int64_t rc = rounds;
    for (int32_t v = 0; v < V; ++v) {
        if (d[v] == OR_INF64) dist[v] = UINT32_MAX;
        else if (d[v] >= UINT32_MAX) { dist[v] = UINT32_MAX; rc = -2; }
        else dist[v] = (uint32_t)d[v];
    }
    free(d);
    return rc;
}

/*
 * All-pairs shortest paths by Floyd-Warshall on a dense V x V matrix (V <= 4096).
 * w == NULL means every edge weighs 1 (then D holds hop counts).  D[i*V+j] =
 * UINT64_MAX when j is unreachable from i.  Returns 0, or -1 on bad input.
 */
int oracle_floyd_warshall(int32_t V, const int32_t *row_off, const int32_t *col,
                          const uint32_t *w, uint64_t *D) {
    if (V < 1 || V > 4096) return -1;
    for (int64_t i = 0; i < (int64_t)V * V; ++i) D[i] = OR_INF64;
    for (int32_t i = 0; i < V; ++i) D[(int64_t)i * V + i] = 0;
    for (int32_t u = 0; u < V; ++u)
        for (int32_t e = row_off[u]; e < row_off[u + 1]; ++e) {
            uint64_t c = w ? (uint64_t)w[e] : 1;
            uint64_t *cell = &D[(int64_t)u * V + col[e]];
            if (c < *cell) *cell = c;
        }
    for (int32_t k = 0; k < V; ++k)
        for (int32_t i = 0; i < V; ++i) {
            uint64_t dik = D[(int64_t)i * V + k];
            if (dik == OR_INF64) continue;
            for (int32_t j = 0; j < V; ++j) {
                uint64_t dkj = D[(int64_t)k * V + j];
                if (dkj == OR_INF64) continue;
                if (dik + dkj < D[(int64_t)i * V + j]) D[(int64_t)i * V + j] = dik + dkj;
            }
        }
    return 0;
}
