/*
 * graphgen.c - seeded synthetic CSR graphs (input generation only).
 *
 * This file builds the inputs that both the CPU oracle and the CUDA path consume:
 * R-MAT edge lists, 2-D grids, deduplicated CSR assembly and per-edge weights.
 * It holds none of the traversal arithmetic (no BFS, no relaxation).
 *
 * Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used as a counter-based generator:
 * every draw is a pure function of (seed, edge index, bit level), so the output does
 * not depend on the thread count or on the host architecture.
 *
 * R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): each of the ef * 2^scale edges
 * descends `scale` levels of the adjacency matrix; at each level one uniform double in
 * [0,1) picks the quadrant with probabilities a, b, c, d = 1-a-b-c (a = row 0 / col 0,
 * b = row 0 / col 1, c = row 1 / col 0, d = row 1 / col 1), most significant bit first.
 * No noise and no vertex permutation.  Self-loops are dropped, duplicates removed,
 * rows stored with ascending column ids.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

uint64_t gg_splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* uniform double in [0,1) from the top 53 bits of one SplitMix64 output */
static inline double u01(uint64_t s0, uint64_t edge, unsigned bit) {
    uint64_t h = gg_splitmix64(s0 ^ ((edge << 6) | (uint64_t)bit));
    return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

typedef struct {
    int scale;
    double ta, tb, tc; /* cumulative thresholds a, a+b, a+b+c */
    uint64_t s0;
    uint64_t lo, hi;   /* edge index range of this worker */
    uint32_t *src, *dst;
} rmat_job;

static void *rmat_worker(void *arg) {
    rmat_job *j = (rmat_job *)arg;
    for (uint64_t i = j->lo; i < j->hi; ++i) {
        uint32_t u = 0, v = 0;
        for (int b = 0; b < j->scale; ++b) {
            double r = u01(j->s0, i, (unsigned)b);
            uint32_t ub, vb;
            if (r < j->ta) { ub = 0; vb = 0; }
            else if (r < j->tb) { ub = 0; vb = 1; }
            else if (r < j->tc) { ub = 1; vb = 0; }
            else { ub = 1; vb = 1; }
            u = (u << 1) | ub;
            v = (v << 1) | vb;
        }
        j->src[i] = u;
        j->dst[i] = v;
    }
    return NULL;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static void sort_small(int32_t *a, int64_t n) {
    if (n > 24) { qsort(a, (size_t)n, sizeof(int32_t), cmp_i32); return; }
    for (int64_t i = 1; i < n; ++i) {
        int32_t x = a[i];
        int64_t k = i - 1;
        while (k >= 0 && a[k] > x) { a[k + 1] = a[k]; --k; }
        a[k + 1] = x;
    }
}

typedef struct {
    int64_t row_lo, row_hi;
    const int64_t *start; /* pre-dedup row starts (V+1) */
    int32_t *buf;
    int64_t *uniq;        /* out: unique count per row */
} sort_job;

static void *sort_worker(void *arg) {
    sort_job *j = (sort_job *)arg;
    for (int64_t r = j->row_lo; r < j->row_hi; ++r) {
        int32_t *a = j->buf + j->start[r];
        int64_t n = j->start[r + 1] - j->start[r];
        sort_small(a, n);
        int64_t k = 0;
        for (int64_t i = 0; i < n; ++i)
            if (k == 0 || a[i] != a[k - 1]) a[k++] = a[i];
        j->uniq[r] = k;
    }
    return NULL;
}

/*
 * Assemble a deduplicated CSR from an edge list (self-loops removed, rows sorted).
 * row_off: V+1 entries, col: capacity >= m.  Returns the edge count, or -1 on
 * allocation failure / a vertex id out of range.
 */
int64_t gg_edges_to_csr(int32_t V, int64_t m, const uint32_t *src, const uint32_t *dst,
                        int threads, int32_t *row_off, int32_t *col) {
    if (threads < 1) threads = 1;
    int64_t *start = (int64_t *)calloc((size_t)V + 1, sizeof(int64_t));
    int64_t *uniq = (int64_t *)malloc(((size_t)V + 1) * sizeof(int64_t));
    if (!start || !uniq) { free(start); free(uniq); return -1; }
    for (int64_t i = 0; i < m; ++i) {
        if (src[i] >= (uint32_t)V || dst[i] >= (uint32_t)V) { free(start); free(uniq); return -1; }
        if (src[i] != dst[i]) start[src[i] + 1]++;
    }
    for (int64_t r = 0; r < V; ++r) start[r + 1] += start[r];
    int64_t *fill = (int64_t *)malloc((size_t)V * sizeof(int64_t));
    if (!fill) { free(start); free(uniq); return -1; }
    memcpy(fill, start, (size_t)V * sizeof(int64_t));
    for (int64_t i = 0; i < m; ++i)
        if (src[i] != dst[i]) col[fill[src[i]]++] = (int32_t)dst[i];
    free(fill);

    pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    sort_job *jobs = (sort_job *)malloc(sizeof(sort_job) * (size_t)threads);
    for (int t = 0; t < threads; ++t) {
        jobs[t].row_lo = (int64_t)V * t / threads;
        jobs[t].row_hi = (int64_t)V * (t + 1) / threads;
        jobs[t].start = start;
        jobs[t].buf = col;
        jobs[t].uniq = uniq;
        pthread_create(&tid[t], NULL, sort_worker, &jobs[t]);
    }
    for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
    free(tid);
    free(jobs);

    /* compact rows to the left: every row moves to an offset <= its old one */
    int64_t out = 0;
    for (int64_t r = 0; r < V; ++r) {
        row_off[r] = (int32_t)out;
        if (out != start[r]) memmove(col + out, col + start[r], (size_t)uniq[r] * sizeof(int32_t));
        out += uniq[r];
    }
    row_off[V] = (int32_t)out;
    free(start);
    free(uniq);
    return out;
}

/*
 * R-MAT graph with V = 2^scale and ef * V generated edges.  col must hold ef * V
 * entries.  Returns the edge count after dedup, or -1 on failure.
 */
int64_t gg_rmat(int scale, int ef, double a, double b, double c, uint64_t seed, int threads,
                int32_t *row_off, int32_t *col) {
    if (scale < 1 || scale > 30 || ef < 1) return -1;
    int32_t V = (int32_t)1 << scale;
    int64_t m = (int64_t)ef << scale;
    if (m >= ((int64_t)1 << 31)) return -1;
    if (threads < 1) threads = 1;
    uint32_t *src = (uint32_t *)malloc((size_t)m * sizeof(uint32_t));
    uint32_t *dst = (uint32_t *)malloc((size_t)m * sizeof(uint32_t));
    if (!src || !dst) { free(src); free(dst); return -1; }
    pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    rmat_job *jobs = (rmat_job *)malloc(sizeof(rmat_job) * (size_t)threads);
    uint64_t s0 = gg_splitmix64(seed);
    for (int t = 0; t < threads; ++t) {
        jobs[t].scale = scale;
        jobs[t].ta = a;
        jobs[t].tb = a + b;
        jobs[t].tc = a + b + c;
        jobs[t].s0 = s0;
        jobs[t].lo = (uint64_t)m * (uint64_t)t / (uint64_t)threads;
        jobs[t].hi = (uint64_t)m * (uint64_t)(t + 1) / (uint64_t)threads;
        jobs[t].src = src;
        jobs[t].dst = dst;
        pthread_create(&tid[t], NULL, rmat_worker, &jobs[t]);
    }
    for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
    free(tid);
    free(jobs);
    int64_t E = gg_edges_to_csr(V, m, src, dst, threads, row_off, col);
    free(src);
    free(dst);
    return E;
}

/*
 * w x h grid, 4-neighbour, no wraparound, both directions stored.  Vertex id
 * y*w + x.  col must hold 4*w*h entries.  Returns the edge count.
 */
int64_t gg_grid(int32_t w, int32_t h, int32_t *row_off, int32_t *col) {
    int64_t e = 0;
    for (int32_t y = 0; y < h; ++y)
        for (int32_t x = 0; x < w; ++x) {
            int32_t id = y * w + x;
            row_off[id] = (int32_t)e;
            if (y > 0) col[e++] = id - w;
            if (x > 0) col[e++] = id - 1;
            if (x + 1 < w) col[e++] = id + 1;
            if (y + 1 < h) col[e++] = id + w;
        }
    row_off[(int64_t)w * h] = (int32_t)e;
    return e;
}

/*
 * Per-edge weight w(u,v) = lo + SplitMix64(s ^ (u<<32 | v)) mod (hi-lo+1), with
 * s = SplitMix64(seed).  A function of the edge itself, so independent of the order
 * in which duplicates were removed.
 */
void gg_weights(int32_t V, const int32_t *row_off, const int32_t *col, uint64_t seed, uint32_t lo,
                uint32_t hi, uint32_t *w) {
    uint64_t s = gg_splitmix64(seed);
    uint64_t span = (uint64_t)hi - (uint64_t)lo + 1;
    for (int32_t u = 0; u < V; ++u)
        for (int32_t e = row_off[u]; e < row_off[u + 1]; ++e) {
            uint64_t key = ((uint64_t)(uint32_t)u << 32) | (uint32_t)col[e];
            w[e] = lo + (uint32_t)(gg_splitmix64(s ^ key) % span);
        }
}
