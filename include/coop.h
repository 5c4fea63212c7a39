/*
 * coop.h - C ABI of libcoop.so: cooperative BFS / SSSP on one GB300 (sm_103a).
 *
 * Implements the cooperative-kernels programming model of Sorensen, Evrard and
 * Donaldson, "Cooperative Kernels: GPU Multitasking for Blocking Algorithms"
 * (FSE 2017), for its frontier graph-traversal application (Sec. 3.2, Fig. 4;
 * Table 1's bfs and l-sssp).  A traversal runs as one persistent kernel whose CTAs
 * (the paper's workgroups) synchronise through a resizing global barrier
 * (Sec. 3.1; the query barrier of Sec. 4.2) and cooperate with a host-side
 * scheduler: CTAs leave through offer_kill when the host asks for SMs
 * (coop_request_resources) and new CTAs join through request_fork when the host
 * returns them (coop_release).  Results do not depend on the schedule.
 *
 * Entry points: frontier traversals (coop_bfs, coop_sssp; their non-cooperative
 * baselines), the topology-driven SSSP of Table 1's p-sssp (coop_sssp_topo), the
 * work-stealing octree of Table 1 (coop_octree), many traversals in one persistent
 * launch (coop_batch_*), a request loop with continuous batching (coop_server_*), the
 * co-running task (coop_saxpy), and the place where host requests are served
 * (coop_set_kill_mode: regular barrier, query barrier, or query barrier plus kill points
 * between chunks).
 *
 * Conventions
 *  - Every pointer argument named d_* or inside coop_csr is DEVICE memory owned by the
 *    caller (e.g. a torch tensor); it must stay valid until the traversal's stream
 *    has synchronised.  Scratch (frontier queues, visited bitmap, control block) and
 *    the host mailbox are owned by the context.  A traversal's stream completes only
 *    after every CTA it forked has left.
 *  - Calls return coop_status; negative values are errors.  No call aborts or throws.
 *  - A coop_stream is a cudaStream_t (same type, declared here without CUDA headers);
 *    NULL is the legacy default stream.
 *  - Graphs are int32 CSR: row_off[V+1] with row_off[0] = 0, non-decreasing,
 *    row_off[V] = E < 2^31; col[E] with 0 <= col[e] < V.  The kernels bounds-check
 *    every vertex id and row offset they read and report COOP_EGRAPH instead of
 *    touching memory out of range.
 *  - One context drives one traversal at a time.  coop_request_resources and
 *    coop_release may be called from another host thread while a traversal runs.
 *    Device-synchronising CUDA calls (cudaMalloc, cudaFree, work on the legacy default
 *    stream) made while a traversal runs wait for it to finish, and so does the first
 *    launch of a kernel whose module is loaded lazily; a co-running task must allocate
 *    its buffers and launch its kernels once beforehand, and use its own non-blocking
 *    stream.  coop_init loads all of this library's kernels eagerly.
 */
#ifndef COOP_H
#define COOP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *coop_stream; /* == cudaStream_t */
typedef struct coop_ctx coop_ctx;        /* opaque, library-owned */

typedef enum {
    COOP_OK = 0,
    COOP_EINVAL = -1,    /* bad argument (null pointer, source out of range, V < 1 ...) */
    COOP_ENOMEM = -2,    /* device or pinned host allocation failed */
    COOP_ECUDA = -3,     /* a CUDA runtime call failed */
    COOP_ETIMEOUT = -4,  /* a device wait or a host gather exceeded its time limit */
    COOP_EBUSY = -5,     /* the context is busy (e.g. destroy with a traversal in flight) */
    COOP_EOVERFLOW = -6, /* an SSSP distance did not fit below 2^32 - 1; octree: out of leaf or queue room */
    COOP_EGRAPH = -7     /* malformed CSR detected on the device (id or offset out of range); octree: a
                            coordinate at or above 2^21 */
} coop_status;

/* A directed graph in int32 CSR form; row_off and col are device pointers. */
typedef struct {
    int32_t num_vertices; /* V >= 1 */
    int64_t num_edges;    /* E, 0 <= E < 2^31, must equal row_off[V] */
    const int32_t *row_off;
    const int32_t *col;
} coop_csr;

/* What one traversal did (all counters cover the whole run). */
typedef struct {
    int32_t levels;         /* frontier rounds expanded (BFS levels; SSSP rounds, each a select
                               and an expand interval, so barriers = 2 x levels) */
    int32_t barriers;       /* resizing barriers passed, excluding the entry one */
    int32_t kills;          /* CTAs that left through offer_kill */
    int32_t forks;          /* CTAs that joined through request_fork after entry */
    int32_t min_active;     /* smallest active CTA count M seen */
    int32_t max_active;     /* largest active CTA count M seen */
    int32_t initial_active; /* M after the entry barrier */
    int32_t status;         /* coop_status of the run */
    int32_t ctas_launched;  /* CTAs launched for the run: main grid + every forked CTA */
    int32_t joined;         /* of forks, the CTAs that joined a BFS level while it ran (they
                               take chunks from the level's shared cursor) rather than
                               waiting for the next barrier */
    int64_t edges_scanned;  /* sum of out-degrees over every expanded frontier (BFS: E_s;
                               SSSP: over the near queues, E_s x work inflation) */
    int64_t frontier_total; /* sum of expanded frontier sizes */
    int64_t vertices_reached; /* V_r: vertices reached from the source (incl. it) */
    int64_t reached_edges;  /* E_s: out-edges of the reached vertices (the TEPS numerator) */
    double gather_us_max;   /* longest coop_request_resources wait during the run */
    double kernel_us;       /* persistent-kernel time on the launch stream (0 unless timing is on) */
} coop_stats;

/*
 * Create a context on `device`.  max_ctas is N, the launch limit of Sec. 3.1
 * ("a maximum of N workgroups"); 0 picks every CTA that can be co-resident (one per
 * SM).  threads_per_cta is the number of worker threads per CTA: 0 (default, 992),
 * 992, 736 or 480 (31, 23 or 15 worker warps; each CTA adds one scheduler warp).
 * Allocates the control block and a mapped pinned mailbox.  *out = NULL on error.
 */
coop_status coop_init(int device, int max_ctas, int threads_per_cta, coop_ctx **out);

/* Free everything the context owns.  Waits for its last traversal; NULL is a no-op. */
coop_status coop_destroy(coop_ctx *ctx);

/*
 * Level-synchronous BFS from `source` (Sec. 2.2 Fig. 3 made cooperative as in Sec. 3.2
 * Fig. 4; Table 1 "bfs").  Writes d_levels[v] = fewest edges on a path source -> v,
 * -1 if unreachable (int32[V], device).  Asynchronous on `stream` unless stats is
 * non-NULL, in which case it waits for the traversal and fills *stats.
 */
coop_status coop_bfs(coop_ctx *ctx, const coop_csr *g, int32_t source, int32_t *d_levels,
                     coop_stream stream, coop_stats *stats);

/*
 * Frontier single-source shortest paths (Table 1 "l-sssp": two resizing barriers per
 * iteration, read as data-driven Bellman-Ford in rounds): each round's first interval
 * selects the pending vertices of lowest tentative distance (enough out-edges to keep
 * the GPU busy, all of them if fewer) and defers the rest; its second relaxes the
 * selected vertices' out-edges, and every vertex whose distance drops is pending for the
 * next round.  d_dist[v] = least total weight of a path source -> v, 0xFFFFFFFF if
 * unreachable (uint32[V], device); d_weights is uint32[E] (device).  Every shortest
 * distance must fit below 2^32 - 1, else the run reports COOP_EOVERFLOW.
 * Asynchronous unless stats is non-NULL (as coop_bfs).
 */
coop_status coop_sssp(coop_ctx *ctx, const coop_csr *g, const uint32_t *d_weights,
                      int32_t source, uint32_t *d_dist, coop_stream stream, coop_stats *stats);

/*
 * Topology-driven single-source shortest paths (Table 1 "p-sssp", read as Pannotia's
 * formulation): every iteration scans all vertices in three resizing-barrier intervals --
 * relax (each vertex lowered by the previous update relaxes its out-edges into a cost
 * array), update (dist = min(dist, cost); the lowered vertices are the next relax's), and
 * check (the run ends after an iteration that lowered nothing).  Same arguments, result
 * and errors as coop_sssp; host requests are served at its barriers.
 */
coop_status coop_sssp_topo(coop_ctx *ctx, const coop_csr *g, const uint32_t *d_weights, int32_t source,
                           uint32_t *d_dist, coop_stream stream, coop_stats *stats);

/*
 * The scheduler asks the running cooperative kernel for n_ctas CTAs (Sec. 4.2,
 * "Launching Kernels and Managing Workgroups": command K_c to provide N - N_a
 * workgroups via offer_kill).  Blocks until the CTAs have left (or, with no traversal
 * in flight, grants them at once), at most timeout_us microseconds (<= 0: no limit).
 * *n_freed (nullable) receives how many left.  On COOP_ETIMEOUT the request stays
 * pending; CTAs it frees later are also lent to the caller.  CTA 0 is never
 * surrendered, so at most N-1 CTAs can be lent at a time (else COOP_EINVAL).
 */
coop_status coop_request_resources(coop_ctx *ctx, int n_ctas, int timeout_us, int *n_freed);

/*
 * Return n_ctas lent CTAs (Sec. 4.2: the scheduler signals that extra workgroups
 * should join at the next request_fork).  If a traversal is running, the running
 * kernel launches n_ctas new CTAs of itself from the device (a follow-up launch into a
 * fire-and-forget stream); they join at a resizing barrier with the transmitted state
 * of the running interval.  Otherwise the next traversal simply starts with them.
 * COOP_EINVAL if more than are lent.  Never blocks.
 */
coop_status coop_release(coop_ctx *ctx, int n_ctas);

/* Wait for the last traversal (both streams) and return its status (sticky device error). */
coop_status coop_sync(coop_ctx *ctx);

/* Statistics of the last completed traversal (call after it has finished). */
coop_status coop_get_stats(coop_ctx *ctx, coop_stats *stats);

/*
 * Barrier trace of the last completed traversal: one record per resizing barrier (after
 * the first 2048, only barriers that admitted, removed or launched CTAs), in order,
 * eight int32 each: {barrier index, microseconds since the run started, M_before,
 * k_forked, W_killed, M_after, CTAs launched there by a forced schedule, out-edges of the
 * frontier the next interval expands}.  Writes min(cap, available) records to out (host
 * memory, 8*cap int32) and the number written to *n.  At most 4096 records per run.
 */
coop_status coop_get_resize_log(coop_ctx *ctx, int32_t *out, int cap, int *n);

/*
 * Record of the scheduler's requests (Sec. 4.2: the gather time of a request for
 * workgroups): one record per coop_request_resources call, eight doubles each:
 * {microseconds from coop_init to the request, CTAs asked for, active CTAs M when the
 * request was posted, M when it was granted, gather microseconds (request to grant),
 * CTAs granted, microseconds spent waiting for the context's lock, microseconds from
 * the call to the request's posting (the lock wait included)}.  M is the count the
 * device published at its latest resizing barrier (0 for a request granted at once,
 * with no traversal in flight).  Writes the latest min(cap, available) records, oldest
 * first, to out (host memory, 8*cap doubles) and
 * the number written to *n; with clear != 0 the context's record is emptied after the
 * copy.  A context keeps its latest 4096 records.  Host-side only: it never waits for
 * the GPU.
 */
coop_status coop_get_request_log(coop_ctx *ctx, double *out, int cap, int *n, int clear);

/*
 * Forced random schedule (tests and the multitasking benchmark).  At every resizing
 * barrier, with probability p_kill the scheduler accepts W in [0, M-1] offer_kills, and
 * with probability p_fork it grants k in [0, N-M] new CTAs, which the kernel launches
 * from the device at once and admits when they arrive.  p_kill = p_fork = 0 disables
 * the schedule (the default).  Draws are SplitMix64 hashes of (seed, barrier index).
 */
coop_status coop_set_schedule(coop_ctx *ctx, uint64_t seed, double p_kill, double p_fork);

/* Time limit for every device-side wait (default 2 s).  Exceeding it ends the run with COOP_ETIMEOUT. */
coop_status coop_set_timeout(coop_ctx *ctx, int64_t timeout_us);

/*
 * Where the context's traversals serve coop_request_resources (Sec. 4.2, "An Efficient
 * Resizing Barrier"); takes effect at the next launch.
 *   COOP_KILL_CHUNK   (default) the query barrier -- the releaser fixes W, the CTAs with
 *                     the W largest ids leave, and a CTA that sees the request while
 *                     waiting leaves at once -- plus a kill point between two chunks of
 *                     an interval, so a request is served within one chunk of work.
 *   COOP_KILL_QUERY   the query barrier alone: requests are served at resizing barriers.
 *   COOP_KILL_SIMPLE  the regular barrier: every CTA offers to leave once, on arriving at
 *                     a barrier, and only the CTA with the largest live id may, so the
 *                     order of arrival decides how many leave per barrier.
 * The results do not depend on the mode; COOP_EINVAL for an unknown mode.
 */
enum { COOP_KILL_CHUNK = 0, COOP_KILL_QUERY = 1, COOP_KILL_SIMPLE = 2 };
coop_status coop_set_kill_mode(coop_ctx *ctx, int mode);

/*
 * Kernel timing: when on, every traversal records CUDA events around its persistent
 * kernel on the launch stream and coop_stats.kernel_us reports the elapsed time.
 */
coop_status coop_set_timing(coop_ctx *ctx, int on);

/* Context facts: N, worker threads per CTA, SM count, CTAs currently lent to the host. */
coop_status coop_query(coop_ctx *ctx, int *max_ctas, int *threads_per_cta, int *sm_count,
                       int *lent);

/*
 * Non-cooperative baselines (Sec. 2.2 Fig. 3): the same traversal with a plain global
 * barrier, a fixed set of N CTAs and no scheduler interaction.  Used to measure the
 * overhead of the cooperative primitives when nothing is resized (Sec. 5.3, Table 2).
 */
coop_status coop_bfs_baseline(coop_ctx *ctx, const coop_csr *g, int32_t source, int32_t *d_levels,
                              coop_stream stream, coop_stats *stats);
coop_status coop_sssp_baseline(coop_ctx *ctx, const coop_csr *g, const uint32_t *d_weights,
                               int32_t source, uint32_t *d_dist, coop_stream stream,
                               coop_stats *stats);

/*
 * Barrier benchmark / self-test: the persistent kernel with empty intervals passes
 * n_barriers resizing barriers (schedule and host requests apply as usual).  With
 * never_arrive > 0 the barrier waits for that many extra arrivals that never come, so
 * the run must end with COOP_ETIMEOUT after the context's time limit (the way the
 * failure path is tested without faulting or hanging the GPU).  Synchronous when
 * stats is non-NULL.
 */
coop_status coop_barrier_bench(coop_ctx *ctx, int32_t n_barriers, int32_t never_arrive,
                               coop_stream stream, coop_stats *stats);

/* ---- batched traversals (many independent jobs in one persistent launch) ---- */

enum { COOP_JOB_BFS = 0, COOP_JOB_SSSP = 1 };

/* One traversal of a batch.  All pointers are caller-owned device memory. */
typedef struct {
    coop_csr graph;            /* the job's graph */
    const uint32_t *d_weights; /* uint32[E] for COOP_JOB_SSSP, ignored for BFS */
    int32_t source;
    int32_t kind;              /* COOP_JOB_BFS or COOP_JOB_SSSP */
    void *d_out;               /* int32 levels[V] (BFS) or uint32 dist[V] (SSSP) */
} coop_job;

typedef struct coop_batch coop_batch; /* opaque, library-owned */

/*
 * Prepare a batch of n_jobs independent traversals (the batched form of Sec. 3.2's
 * traversal: every job is a cooperative kernel of its own -- own barrier, queues and
 * control block -- and all of them share one persistent launch).  Allocates the jobs'
 * scratch.  Blocks (CTAs) per job default to one wave of N blocks split in proportion
 * to the jobs' edges; coop_batch_set_ctas or coop_batch_tune change that.  Batched jobs
 * have no host scheduler (coop_request_resources / coop_release do not apply).
 */
coop_status coop_batch_create(coop_ctx *ctx, const coop_job *jobs, int n_jobs, coop_batch **out);

/* Set the blocks of every job (ctas[i] >= 1; the sum may exceed the resident capacity:
 * jobs whose blocks are not resident yet start when earlier jobs free their SMs).  Waits
 * for the batch's last run, on whatever stream, before it rewrites the job table. */
coop_status coop_batch_set_ctas(coop_batch *b, const int32_t *ctas);

/*
 * Autotuner: times the batch under candidate apportionments (blocks proportional to
 * edges^alpha for alpha in {0.5, 0.75, 1}, totals of 1, 2 and 4 waves of N blocks) and
 * keeps the fastest; ctas_out (nullable, n_jobs entries) receives the choice.
 * Synchronous; runs the batch 27 times.
 */
coop_status coop_batch_tune(coop_batch *b, coop_stream stream, int32_t *ctas_out);

/*
 * Run every job once: one initialisation kernel and one persistent launch on `stream`.
 * With use_graph != 0 both are captured once into a CUDA graph (re-captured after the
 * apportionment changes) and the graph is launched.  Asynchronous.
 */
coop_status coop_batch_run(coop_batch *b, coop_stream stream, int use_graph);

/* Per-job statistics of the last run (waits for the device); per_job has n_jobs entries.
 * Returns the first failing job's status, if any. */
coop_status coop_batch_get_stats(coop_batch *b, coop_stats *per_job);

/* Free the batch (waits for the device).  NULL is a no-op. */
coop_status coop_batch_destroy(coop_batch *b);

/* ---- serving: a request loop with continuous batching ---- */

typedef struct coop_server coop_server; /* opaque, library-owned */

/* The outcome of one query. */
typedef struct {
    int32_t status;    /* coop_status of the traversal */
    int32_t slot;      /* slot that ran it */
    int32_t ctas;      /* CTAs it was admitted with */
    int32_t reserved;
    double queue_us;   /* submit -> launch */
    double latency_us; /* submit -> completion seen by the server */
    coop_stats stats;  /* the traversal's statistics */
} coop_query_result;

/*
 * Create a server on `device` with `slots` concurrent query slots (each a context of its
 * own).  hbm_budget_bytes (0 = no limit) bounds the device memory of the registered
 * graphs (CSR and weights) plus the scratch every slot holds for the largest of them;
 * coop_server_add_graph fails with COOP_ENOMEM beyond it.  Since every slot is sized for
 * every graph before the first query, admission while serving is by free slot: a query
 * that finds a slot free runs within the budget.  Query outputs are the caller's memory
 * and are not counted.
 */
coop_status coop_server_create(int device, int slots, size_t hbm_budget_bytes, coop_server **out);

/*
 * Register a device-resident graph (caller-owned CSR and optional weights, which must
 * stay valid until the server is destroyed) before the first query.  Sizes every
 * slot's scratch for it.  *graph_id receives its index.
 */
coop_status coop_server_add_graph(coop_server *sv, const coop_csr *g, const uint32_t *d_weights, int *graph_id);

/*
 * Queue a query: kind COOP_JOB_BFS (d_out int32[V]) or COOP_JOB_SSSP (d_out uint32[V],
 * the graph must have weights) from `source` on graph `graph_id`.  Queries are admitted
 * in arrival order as slots free up; a query that arrives while others run overlaps with
 * them: running traversals are shrunk (offer_kill) so that every running query holds an
 * equal share of the CTAs, and grown back (request_fork) when queries finish.  Never
 * blocks.  *ticket identifies the query.
 */
coop_status coop_server_submit(coop_server *sv, int graph_id, int kind, int32_t source, void *d_out,
                               uint64_t *ticket);

/* Wait for a query (timeout_us <= 0: no limit) and fetch its result; returns its status. */
coop_status coop_server_wait(coop_server *sv, uint64_t ticket, int timeout_us, coop_query_result *res);

/*
 * Take n_ctas CTAs for a co-running task: CTAs no running query holds count first, the
 * rest is requested from the running queries in proportion to what each can lend (each
 * keeps at least one), all requests posted before any is waited for.  Blocks like
 * coop_request_resources, at most timeout_us in all (timeout_us <= 0: no limit); returns
 * COOP_ETIMEOUT with *n_freed < n_ctas if fewer could be freed in time (the requests stay
 * pending).  The n_ctas are held for the co-runner either way until coop_server_release.
 */
coop_status coop_server_request_resources(coop_server *sv, int n_ctas, int timeout_us, int *n_freed);
/* Give n_ctas co-runner CTAs back; running queries grow into them (request_fork). */
coop_status coop_server_release(coop_server *sv, int n_ctas);

/* Drain the queue, wait for running queries and free everything.  NULL is a no-op. */
coop_status coop_server_destroy(coop_server *sv);

/* ---- octree partitioning (work stealing) ---- */

/*
 * Octree partitioning of n points, the work-stealing application of Table 1 (Sec. 2.2
 * Fig. 2; Sec. 3.2 "Adapting Work Stealing"), run as a cooperative kernel on this
 * context: per-CTA task queues guarded by compare-and-swap mutexes, stealing from other
 * queues, offer_kill at the head of the main loop and forked CTAs taking queues of
 * their own -- coop_request_resources / coop_release apply while it runs.
 *
 * d_x, d_y, d_z: uint32[n] device coordinates, each below 2^21 (else COOP_EGRAPH).  The
 * root cell is the cube [0, 2^21)^3 at depth 0; a cell at depth d < max_depth (0..21)
 * holding more than leaf_cap (>= 1) points splits into its octants by coordinate bit
 * 20 - d (octant = bx | by << 1 | bz << 2); every other non-empty cell is a leaf.  Output
 * (caller-owned device memory): *d_n_leaves leaves, leaf i with path code d_leaf_code[i]
 * (a 1 followed by 3 bits per level below the root) holding the d_leaf_count[i] point
 * indices d_perm[d_leaf_begin[i] .. + count); d_perm is uint32[n], the leaf arrays hold
 * max_leaves entries (n always suffices).  The leaves and each leaf's point set are
 * unique; their order in memory is not.  Asynchronous unless stats is non-NULL; with
 * stats: kills, forks, initial_active, ctas_launched as for traversals, frontier_total =
 * tasks processed, edges_scanned = steals, vertices_reached = leaves, reached_edges =
 * points moved by partitioning.  COOP_EOVERFLOW if more than max_leaves leaves or a task
 * queue overflowed; COOP_ETIMEOUT on a device wait beyond coop_set_timeout.
 */
coop_status coop_octree(coop_ctx *ctx, const uint32_t *d_x, const uint32_t *d_y, const uint32_t *d_z, int32_t n,
                        int32_t leaf_cap, int32_t max_depth, uint64_t *d_leaf_code, uint32_t *d_leaf_begin,
                        uint32_t *d_leaf_count, int32_t max_leaves, uint32_t *d_perm, int32_t *d_n_leaves,
                        coop_stream stream, coop_stats *stats);

/*
 * The co-running latency-critical task: y[i] = a * x[i] + y[i] for i < n (fp32,
 * device pointers), on n_ctas CTAs whose shared-memory reservation keeps them off any
 * SM that holds a traversal CTA, so they run only on SMs the traversal gave up (the
 * compute stand-in for the paper's graphics / matrix-multiplication tasks, Sec. 5.4).
 */
coop_status coop_saxpy(int n_ctas, int64_t n, float a, const float *d_x, float *d_y,
                       coop_stream stream);

/*
 * Allocation-free BFS.  The paper has no counterpart: this is a deployment variant of
 * coop_bfs for callers that must not allocate device memory -- processes that reserve
 * their whole device-memory budget up front through their own pool, code running inside
 * an allocator's or memory pool's callbacks (which must not re-enter the allocator), and
 * latency-critical loops that cannot take cudaMalloc's implicit device synchronisation
 * (which would also wait for any running traversal).  It needs no context and calls no
 * allocating routine: its scratch (control block, mailbox, visited bitmap, frontier
 * queues) is one static device array compiled into libcoop.so, about 25 MB, which every
 * GPU that loads the library holds until the process exits.
 *
 *  - Limit: graphs of at most 2^20 (1,048,576) vertices and 2^25 (33,554,432) edges;
 *    larger ones are rejected with COOP_EINVAL (coop_last_cuda_error() names the limit)
 *    before any GPU work.
 *  - Inputs and outputs as coop_bfs: g (device CSR), source, d_levels (int32[V], device);
 *    d_status (nullable, device int32) receives the run's coop_status when it finishes.
 *  - Asynchronous on `stream`.  It runs with every CTA that fits (no host scheduler:
 *    coop_request_resources / coop_release do not apply).
 *  - The first call on a device (the current device) looks up the array's device address
 *    and sets kernel attributes; make that first call before any stream capture.
 *  - Every call shares the one array, which keeps the last call's contents; each call
 *    clears what must start at zero.  Calls whose work overlaps on the GPU race with each
 *    other and corrupt each other's results: order them (one stream, or events).
 */
coop_status coop_bfs_noalloc(const coop_csr *g, int32_t source, int32_t *d_levels, int32_t *d_status,
                             coop_stream stream);

/*
 * Text of the last failing CUDA runtime call made by this library on the calling
 * thread ("" if none): which step failed, the CUDA error name and its description.
 * Useful after COOP_ECUDA; the string stays valid until the thread's next failure.
 */
const char *coop_last_cuda_error(void);

/* Human-readable name of a status code (static string). */
const char *coop_status_string(coop_status s);

#ifdef __cplusplus
}
#endif

#endif /* COOP_H */
