// coop_runtime.cuh - device runtime of the cooperative kernels (sm_103a).
//
// Implements the primitives of Sec. 3.1 of "Cooperative Kernels" (Sorensen, Evrard and
// Donaldson, FSE 2017) for persistent CUDA kernels:
//
//  * active CTAs and logical ids: a CTA is *active* once admitted; active CTAs hold the
//    contiguous logical ids [0, M-1]; logical id 0 (block 0 of the main launch, the
//    master) is never killed.  Logical ids are decoupled from blockIdx so that CTAs of
//    a later launch (forks) can take ids M..M+k-1.
//  * resizing_global_barrier as the query barrier of Sec. 4.2: all active CTAs arrive
//    on one L2-resident counter (acq_rel, gpu scope); the last arrival releases the
//    barrier by bumping an epoch word (sense reversal by epoch parity).  Inside the
//    release it (2) forks: admits up to N-M CTAs that are waiting to join, (3) queries
//    the scheduler for W, (4) broadcasts the next interval (the transmitted state) and
//    the new M; (5) the CTAs with logical ids >= M' leave.  Fork happens before kill,
//    so ids [0, min(M, M')-1] are untouched (Sec. 3.1).
//  * request_fork via join-on-arrival: new CTAs come from device-side (fire-and-forget)
//    launches of the same kernel made by the running kernel itself -- by the scheduler
//    warp when the host returns SMs, by the releaser under a forced schedule.  Every CTA
//    other than the master first registers (takes a ticket) and waits for the release
//    that admits it; a CTA counts towards M only after admission, so a launched but not
//    yet resident CTA never holds a barrier up.
//  * transmit: the interval record (level, input queue, frontier size) is written by
//    the releaser before the release and read by every CTA after it; joiners read the
//    same record, which is "thread 0 of workgroup 0's" transmitted state since those
//    values are uniform across the kernel (the observation of Appendix B).
//  * the scheduler side of query(): a scheduler warp in the master CTA turns the host's
//    request counter (mapped pinned memory, system scope) into an epoch-stamped kill
//    target in L2 -- CTAs with logical ids at or above it leave at their next offer_kill
//    point, and the releaser closes it for the interval -- so the release path reads only
//    L2; it also launches the CTAs the host gives back.  Where requests are served is a
//    per-context mode (KillMode): the regular barrier of Sec. 4.2, the query barrier, or
//    the query barrier plus a kill point between chunks of an interval.
//
// Every spin-wait reads %globaltimer and gives up after the context's limit, setting a
// sticky error that all other waits observe; nothing here can wait forever.
#pragma once
#include <stdint.h>

namespace coopdev {

// Worker warps per CTA is a template parameter NW of the kernels (31, 23 or 15); every
// CTA has NW worker warps plus one scheduler (poller) warp, (NW + 1) * 32 <= 1024 threads.
constexpr int kDefaultWorkerWarps = 31;
constexpr int kMaxCtas = 2048;              // admission slot table; N <= kMaxCtas
constexpr int kLogCap = 4096;               // resize-log records per run
// SM exclusivity by shared memory: a traversal CTA takes at least kTraverseSmemMin of an
// SM's 228 KB and a co-runner CTA kCorunnerSmem, more than the SM holds together, so a
// co-runner only ever starts on an SM that no traversal CTA occupies.  A traversal CTA
// asks for no more than its staging needs, so that the rest of the SM's 256 KB of
// L1/shared storage serves as L1 (the BFS visited bitmap is read through L1).
constexpr int kTraverseSmemMin = 56 * 1024;
constexpr int kCorunnerSmem = 176 * 1024;
static_assert(kTraverseSmemMin + kCorunnerSmem + 2 * 1024 > 228 * 1024, "co-runner must not fit beside a traversal CTA");
constexpr uint64_t kEntryGatherNs = 20000;  // master waits this long for its launch to register
constexpr uint32_t kIndexShift = 7;
constexpr uint32_t kIndexEdges = 1u << kIndexShift;  // granularity of the chunk index (edges per unit)
constexpr uint32_t kChunkUnitsMax = 16;     // a chunk of a wide BFS level spans 1..16 units of kIndexEdges edges
constexpr uint32_t kChunkUnitsMaxSssp = 4;  // SSSP: 1..4 units
// A claim reads the target's state (visited bit, distance) before its atomic on frontiers
// of at least kPrecheckEdges edges, where the read saves most atomics (claim atomics in
// bulk are far slower than loads).  On smaller frontiers the read is one more dependent
// round trip on the level's critical path, and the claim goes straight to the atomic.
constexpr uint32_t kPrecheckEdges = 65536;
// BFS: a CTA that the host's kill target dooms in the middle of a chunk hands the rest of
// the chunk back (the warp stops after its current iteration) into a list of returned
// edge ranges in the control block; the release turns them into a continuation interval
// of the same level.  kRetCap ranges per level at most (beyond that a doomed warp
// finishes its chunk).
constexpr uint32_t kRetCap = 32768;
// p-sssp: a flagged row of at least kTopoHeavy edges is not relaxed by the one warp whose
// vertex stripe holds it but listed, as chunks of kTopoChunk edges, by the update interval
// that flagged it; the relax interval deals the chunks out over every warp of the grid.
// (An R-MAT hub's 10^4-10^5 edges on one warp would leave the rest of the grid waiting.)
constexpr uint32_t kTopoHeavy = 512;
constexpr uint32_t kTopoChunk = 256;
// Frontier SSSP in rounds (Table 1 l-sssp: two barriers per iteration).  A round whose
// pending queue has more than kNearUnits * kIndexEdges out-edges per worker warp has two
// intervals: a select interval moves the pending vertices of lowest tentative distance,
// about that many out-edges, into the near queue (queue kNearQueue) and defers the rest
// to the next round's pending queue; the expand interval relaxes the near queue's
// out-edges into that pending queue.  A smaller pending queue is expanded whole, in one
// interval.  Each CTA splits its own stripes of the pending queue at a distance threshold
// found from a sample of its stripes: a histogram of their out-degrees over current
// distance in kHistBuckets buckets of 2^kHistShift distance units above the round's
// base (no pending distance is below it; the last bucket takes every larger distance).
// Relaxing the closest vertices first keeps most vertices from being expanded again at a
// distance that later drops (work inflation).
constexpr uint32_t kNearQueue = 2;
constexpr uint32_t kNearUnits = 4;
constexpr uint32_t kHistBuckets = 1024;
constexpr uint32_t kHistShift = 2;

// MODE_PSSSP: topology-driven SSSP (Table 1's p-sssp, read as Pannotia's formulation):
// every iteration scans all vertices in three intervals -- relax, update, check.
enum Mode : int { MODE_BFS = 0, MODE_SSSP = 1, MODE_BARRIER = 2, MODE_PSSSP = 3 };

// Where the host's requests for CTAs are served (Sec. 4.2, "An Efficient Resizing Barrier"):
//  KILL_CHUNK   the query barrier, plus a kill point between two chunks of an interval
//  KILL_QUERY   the query barrier alone: the scheduler's W is fixed at a release, and the
//               CTAs with the W largest ids leave at the barrier
//  KILL_SIMPLE  the regular barrier: each CTA offers to leave once, on arrival, and only
//               the CTA with the largest live id can, so arrival order decides how many
//               leave per barrier
enum KillMode : uint32_t { KILL_CHUNK = 0, KILL_QUERY = 1, KILL_SIMPLE = 2 };

enum Err : int {
  ERR_TIMEOUT = -4,   // COOP_ETIMEOUT
  ERR_OVERFLOW = -6,  // COOP_EOVERFLOW
  ERR_GRAPH = -7      // COOP_EGRAPH
};

// The transmitted state of one resizing-barrier interval (Fig. 4: level, in_nodes,
// out_nodes) plus the active count M that holds during the interval.
struct Interval {
  int32_t M;       // active CTAs in this interval
  int32_t level;   // BFS level whose frontier is expanded / SSSP interval (round = level / 2)
  uint32_t sel;    // input queue index; the output queue is sel ^ 1
  uint32_t count;  // frontier vertices in the input queue
  uint32_t edges;  // frontier out-edges (size of this interval's edge space)
  uint32_t done;   // 1: the traversal is over, every CTA leaves
  uint32_t epoch;  // epoch number that opened this interval
  uint32_t doom;   // CTAs of the previous interval with logical id >= doom leave (host kills)
  uint32_t precheck;  // 1: read a target's state before its claim atomic (kPrecheckEdges)
  uint32_t base;      // SSSP: the round's histogram base (no pending distance is below it)
  // SSSP: round r << 3 | select << 2 | xq.  Round r's pending queue is queue sel, the
  // next round's sel ^ 1; select is 1 in a round's select interval, 0 in an expand
  // interval, which expands queue xq (kNearQueue, or the pending queue whole)
  uint32_t sssp;
  // BFS continuation interval (nonzero): the returned ranges [lo, lo + n) of the level's
  // edge space to expand, as lo << 16 | n
  uint32_t cont;
};

__host__ __device__ constexpr uint32_t sssp_word(uint32_t round, uint32_t select, uint32_t xq) {
  return round << 3 | select << 2 | xq;
}
__host__ __device__ constexpr uint32_t sssp_round(const Interval &iv) { return iv.sssp >> 3; }
__host__ __device__ constexpr bool sssp_select(const Interval &iv) { return ((iv.sssp >> 2) & 1u) != 0u; }
__host__ __device__ constexpr uint32_t sssp_xq(const Interval &iv) { return iv.sssp & 3u; }

// One barrier record (the run's trace): barrier index, microseconds since the run
// started, the active count before, CTAs admitted (fork), CTAs leaving (kill), the active
// count after, CTAs launched at this barrier by a forced schedule, and the out-edges of
// the frontier the next interval expands.
struct LogRec {
  int32_t barrier, t_us, m_before, k, w, m_after, spawned, edges;
};

struct alignas(128) Word {
  uint32_t v;
  uint32_t pad[31];
};
struct alignas(128) Word64 {
  unsigned long long v;
  uint32_t pad[30];
};

// The barrier's arrival word: epoch << 32 | joined << 16 | arrived.  `arrived` counts the
// interval's CTAs that have reached the barrier; `joined` the CTAs that joined the interval
// after it opened (a forked CTA takes part in the running BFS level instead of waiting for
// the next barrier).  The barrier releases when arrived reaches M + joined, so a join and
// the last arrival are ordered by the one atomic word: a CTA can join only while someone
// is still working, and the release then waits for it.
__host__ __device__ constexpr unsigned long long arrive_word(uint32_t epoch, uint32_t joined, uint32_t arrived) {
  return ((unsigned long long)epoch << 32) | ((unsigned long long)(joined & 0xFFFFu) << 16) |
         (unsigned long long)(arrived & 0xFFFFu);
}

// Control block in device memory (L2-resident), zeroed before every run.
struct Ctl {
  Word64 arrive;      // arrivals at the current barrier (arrive_word)
  Word epoch;         // release word: bumped by the releaser
  Word join_ticket;   // registrations of CTAs waiting to be admitted
  Word cursor;        // chunks claimed beyond the first M * NW in the current interval
  alignas(128) unsigned long long qctr[3];  // per queue: (vertices << 32) | edges
  uint64_t pad_q[13];
  alignas(128) Interval iv;  // the current interval (written only by releasers)
  uint32_t pad_iv[24];
  // host kill target of the running interval: (epoch << 32) | closed << 31 | T, where
  // CTAs with logical id >= T leave; lowered by the scheduler warp, closed by the releaser
  alignas(128) unsigned long long kill_target;
  uint32_t surrendered;   // CTAs that left on a host request
  uint32_t host_decided;  // host kills fixed at releases (releaser)
  uint32_t host_req;      // KILL_SIMPLE: the host's requests of this run (scheduler warp)
  uint32_t pad_k0;
  // KILL_SIMPLE: (live CTAs << 32) | CTAs that left at this barrier's offer_kill
  unsigned long long live;
  uint32_t pad_k[24];
  // header line: written once per run by the init kernel, then by error/done paths
  alignas(128) uint32_t run;
  uint32_t unused_h;
  uint32_t err;              // sticky error (negative coop_status as uint32)
  uint32_t done;             // set by the final release
  uint32_t ovf;              // SSSP distance overflow seen
  uint32_t pad_h[27];
  alignas(128) uint32_t launched_total;  // CTAs launched for this run (main grid + forks)
  uint32_t pad_l[31];
  alignas(128) unsigned long long reached_edges;  // out-edges of reached vertices (E_s)
  unsigned long long reached;                     // reached vertices (V_r)
  uint64_t pad_r[14];
  // releaser-private bookkeeping (serialised by the barrier)
  alignas(128) uint32_t admitted;  // forked CTAs admitted at barriers (join tickets)
  uint32_t joined;                 // forked CTAs that joined a running interval
  int32_t barriers, kills, forks, min_active, max_active, initial_active;
  unsigned long long edges_scanned, frontier_total;
  unsigned long long t_start;  // %globaltimer at the master's entry
  uint32_t log_n;
  uint32_t pad_b[13];
  // SSSP: least distance selected in the current round (atomicMin by the select's CTAs),
  // the next round's histogram base
  alignas(128) uint32_t dmin;
  uint32_t pad_s[31];
  alignas(128) uint32_t ret_n;  // BFS: edge ranges handed back in the current level
  uint32_t pad_r2[31];
  alignas(128) unsigned long long slot[kMaxCtas];  // admission records, by ticket % kMaxCtas
  LogRec log[kLogCap];
  unsigned long long ret[kRetCap];  // BFS: returned ranges, first edge << 32 | end (not cleared)
};

// Host <-> device mailbox in mapped pinned host memory.
struct alignas(128) Mailbox {
  // kill_req and fork_req share one 8-byte word, read by the device in one load
  uint32_t kill_req;  // host -> device: cumulative CTAs requested by the scheduler
  uint32_t fork_req;  // host -> device: cumulative CTAs the scheduler gave back
  uint32_t pad0[30];
  uint32_t freed;     // device -> host: cumulative requested CTAs that have left
  int32_t err;        // device -> host: sticky error of the current run
  uint32_t run_done;  // device -> host: id of the last run that finished
  int32_t active;     // device -> host: active CTAs (M) after the latest resizing barrier
  uint32_t pad1[28];
  int32_t levels, barriers, kills, forks, min_active, max_active, initial_active, status;
  int32_t ctas_launched, joined;
  unsigned long long edges_scanned, frontier_total;
  unsigned long long reached, reached_edges;
};

// Kernel parameters: immutable for the whole run and identical for forked CTAs
// (Sec. 3.1, "the parameters to a cooperative kernel are immutable").
struct Params {
  const int32_t *row_off;
  const int32_t *col;
  const uint32_t *w;
  int32_t *level;
  uint32_t *dist;
  uint32_t *visited;  // BFS: 1 bit per vertex
  // SSSP: per vertex (tentative distance << 32) | stamp, the stamp being the frontier
  // round the vertex was last queued for; the distances are copied out to `dist` when
  // the traversal ends
  unsigned long long *ds;
  // frontier queues 0 and 1 (BFS levels, SSSP pending vertices) and 2 (SSSP near queue)
  uint32_t *qv[3];    // vertex id (SSSP)
  uint32_t *qs[3];    // first column index (row_off[v])
  uint32_t *qo[3];    // exclusive prefix of out-degrees (edge space)
  uint32_t *qx[3];    // chunk index: entry holding edge j * kIndexEdges, per expanded queue
  Ctl *ctl;
  Mailbox *mbox;
  int32_t V;
  uint32_t E;
  int32_t src;
  int32_t N;
  uint32_t launched;   // CTAs in the main launch (the master waits for them at entry)
  uint32_t kill_base;  // scheduler requests already served when the run started
  uint32_t fork_base;  // host fork grants already consumed when the run started
  uint64_t timeout_ns;
  uint64_t sched_seed;
  uint32_t p_kill;     // schedule: kill probability * 2^32 (0 = never)
  uint32_t p_fork;     // schedule: fork probability * 2^32 (0 = never)
  uint32_t sched_on;
  uint32_t run;
  int32_t n_barriers;  // MODE_BARRIER: intervals to run
  uint32_t extra_wait; // barrier self-test: arrivals that never come
  uint32_t coop;       // 0: non-cooperative baseline (fixed ids, no scheduler)
  uint32_t kill_mode;  // where host requests are served: KILL_CHUNK, KILL_QUERY or KILL_SIMPLE
  int32_t mode;        // MODE_BFS / MODE_SSSP (read by the batch kernel)
  // MODE_PSSSP: heavy rows are listed as chunks in queue 0 (qv: vertex, qs: first edge),
  // their count in ctl->cursor.  Set only when the list cannot outgrow the queue:
  // E / kTopoChunk + E / kTopoHeavy + 1 <= V.
  uint32_t topo_heavy;
};

struct CtaShared {
  Interval iv;
  uint32_t split[2];  // SSSP select interval: threshold bucket, least distance selected
  // SSSP select interval, by batch parity: per queue (near, pending) the CTA's
  // (entries << 32 | edges) of a batch, then the CTA's base in the queue
  unsigned long long take[2][2];
  int32_t id;
  int32_t ok;
  int32_t exit;
  int32_t workers_left;  // set when this CTA's worker warps have left (bounds the poller)
  int32_t leave;         // this CTA leaves at the current barrier (host kill)
  uint32_t doom;         // BFS: epoch of the interval in which the host's kill target dooms
                         // this CTA (set by the CTA's doom watcher warp)
};

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_acquire64(const unsigned long long *p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_relaxed64(const unsigned long long *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed64(unsigned long long *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t *p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ uint64_t atom_add_acq_rel64(unsigned long long *p, uint64_t v) {
  uint64_t old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}
// mapped pinned host memory: generic addressing, system scope
__device__ __forceinline__ uint32_t ld_sys(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.sys.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_sys64(const void *p) {
  uint64_t v;
  asm volatile("ld.relaxed.sys.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_sys(uint32_t *p, uint32_t v) {
  asm volatile("st.relaxed.sys.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_sys64(unsigned long long *p, uint64_t v) {
  asm volatile("st.relaxed.sys.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
template <int NW>
__device__ __forceinline__ void workers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(NW * 32) : "memory");
}
__device__ __forceinline__ unsigned lanemask_le() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
  return m;
}
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {  // SplitMix64 finaliser
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Read the interval record with strong (relaxed, gpu-scope) loads after an acquire.
__device__ __forceinline__ Interval read_iv(const Ctl *c) {
  Interval r;
  const uint32_t *s = reinterpret_cast<const uint32_t *>(&c->iv);
  uint32_t *d = reinterpret_cast<uint32_t *>(&r);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(Interval) / 4); ++i) d[i] = ld_relaxed(s + i);
  return r;
}

// ---------------------------------------------------------------- host kill target
constexpr unsigned long long kTargetClosed = 1ull << 31;

// Does the kill target word `kt` make logical id `id` of interval `epoch` (M CTAs at its
// opening) leave?  A CTA that joined the interval after it opened (id >= M) is never
// taken by that interval's target: the target counts the opening CTAs only.
__device__ __forceinline__ bool doomed(uint64_t kt, uint32_t epoch, int32_t id, int32_t M) {
  return id < M && (uint32_t)(kt >> 32) == epoch && (uint32_t)id >= (uint32_t)(kt & 0x7FFFFFFFull);
}

// ---------------------------------------------------------------- errors / stats
__device__ __forceinline__ void raise_err(const Params &p, int code) {
  if (atomicCAS(&p.ctl->err, 0u, (uint32_t)code) == 0u) {
    st_sys((uint32_t *)&p.mbox->err, (uint32_t)code);
    __threadfence_system();
  }
}

__device__ __forceinline__ void publish_stats(const Params &p, int status) {
  Ctl *c = p.ctl;
  Mailbox *m = p.mbox;
  // SSSP: rounds (an expand interval each, some also a select interval)
  st_sys((uint32_t *)&m->levels, p.mode == MODE_SSSP ? sssp_round(c->iv) : (uint32_t)c->iv.level);
  st_sys((uint32_t *)&m->barriers, (uint32_t)c->barriers);
  st_sys((uint32_t *)&m->kills, (uint32_t)c->kills);
  st_sys((uint32_t *)&m->forks, (uint32_t)c->forks);
  st_sys((uint32_t *)&m->min_active, (uint32_t)c->min_active);
  st_sys((uint32_t *)&m->max_active, (uint32_t)c->max_active);
  st_sys((uint32_t *)&m->initial_active, (uint32_t)c->initial_active);
  st_sys((uint32_t *)&m->status, (uint32_t)status);
  st_sys((uint32_t *)&m->ctas_launched, ld_relaxed(&c->launched_total));
  st_sys((uint32_t *)&m->joined, c->joined);
  st_sys64(&m->edges_scanned, c->edges_scanned);
  st_sys64(&m->reached, ld_relaxed64(&c->reached));
  st_sys64(&m->reached_edges, ld_relaxed64(&c->reached_edges));
  st_sys64(&m->frontier_total, c->frontier_total);
  __threadfence_system();
  st_sys(&m->run_done, p.run);
  __threadfence_system();
}

// ---------------------------------------------------------------- admission slots
// slot = epoch << 32 | killed << 31 | logical id << 19 | (ticket & 0x7FFFF)
__device__ __forceinline__ uint64_t slot_pack(uint32_t epoch, uint32_t killed, uint32_t id, uint32_t t) {
  return ((uint64_t)epoch << 32) | ((uint64_t)(killed & 1u) << 31) | ((uint64_t)(id & 0xFFFu) << 19) |
         (uint64_t)(t & 0x7FFFFu);
}

// Wait until the epoch word differs from `e` (a release happened): returns 1.  A CTA
// with logical id `id` (>= 0) of an interval that opened with M CTAs, which the host's
// kill target dooms while it waits, returns 2
// at once (it has arrived already, and the closed target will include it).  0 on error
// or timeout.
__device__ __forceinline__ int wait_release(const Params &p, uint32_t e, int32_t id = -1, int32_t M = 0) {
  Ctl *c = p.ctl;
  const uint64_t t0 = gtime();
  for (uint32_t spin = 0;; ++spin) {
    if (ld_acquire(&c->epoch.v) != e) return 1;
    if (id > 0 && doomed(ld_relaxed64(&c->kill_target), e, id, M)) return 2;
    if (ld_relaxed(&c->err) != 0u) return 0;
    if ((spin & 31u) == 31u) {
      if (gtime() - t0 > p.timeout_ns) {
        raise_err(p, ERR_TIMEOUT);
        return 0;
      }
      __nanosleep(spin < 4096 ? 20 : 200);
    }
  }
}

// Wait until the epoch word reaches `e` (a joiner waiting for its admission release).
__device__ __forceinline__ bool wait_epoch_at_least(const Params &p, uint32_t e) {
  Ctl *c = p.ctl;
  const uint64_t t0 = gtime();
  for (uint32_t spin = 0;; ++spin) {
    if ((int32_t)(ld_acquire(&c->epoch.v) - e) >= 0) return true;
    if (ld_relaxed(&c->err) != 0u) return false;
    if ((spin & 31u) == 31u) {
      if (gtime() - t0 > p.timeout_ns) {
        raise_err(p, ERR_TIMEOUT);
        return false;
      }
      __nanosleep(50);
    }
  }
}

// ---------------------------------------------------------------- release (query barrier)
// Runs in thread 0 of the last CTA to arrive, while every other active CTA waits.
// Computes the next interval from the output queue, admits joiners (fork), asks the
// scheduler for W (query), kills from the top, logs the resize and publishes.
template <int MODE, int NW>
__device__ void spawn_forks(const Params &p, uint32_t n);

__device__ __forceinline__ uint32_t precheck_hint(uint32_t edges) { return edges >= kPrecheckEdges ? 1u : 0u; }

// Releaser-private books of one release, stored after the epoch word is released: no
// waiter reads them, and this thread's next arrival (a release) orders them before the
// next releaser's loads.
struct Books {
  int32_t m_after;  // the new interval's M, for the host mailbox
  uint32_t admitted, joined;
  int32_t barriers, kills, forks, min_active, max_active;
  unsigned long long edges_scanned, frontier_total;
  uint32_t log_n;
  bool has_kill, has_rec;  // trace records to append: the host kills, the resize
  LogRec kill_rec, rec;
  int32_t status;  // final status when the traversal is over, else 1
};

// J CTAs joined the interval after it opened (logical ids M .. M + J - 1): they stay,
// renumbered right after the opening CTAs that stay, and count as admitted here.
template <int MODE, int NW>
__device__ __forceinline__ Interval release_step(const Params &p, const Interval cur, uint32_t J, Books &bk) {
  Ctl *c = p.ctl;
  const int32_t M = cur.M;
  // (5) of the query barrier for the host's requests: close this interval's kill target.
  // CTAs with ids >= Mmid leave (those that saw it while waiting already left; the
  // others leave right after this release).  The word is stamped closed for this epoch
  // even when no target was set, so that a scheduler update computed before this
  // release can no longer land on this epoch; a lower open target is then put back.
  // Issued first so that its round trip overlaps the loads below.
  unsigned long long closed = 0ull, kt = 0ull;
  const bool simple = p.kill_mode == KILL_SIMPLE;
  if (p.coop && !simple) {
    closed = ((unsigned long long)cur.epoch << 32) | kTargetClosed;
    kt = atomicExch(&c->kill_target, closed | (unsigned long long)(uint32_t)M);
  }
  // regular barrier: the CTAs that left at their offer_kill on arrival (largest ids first)
  const unsigned long long live = simple ? ld_relaxed64(&c->live) : 0ull;
  // Everything else the release needs, in one batch of independent loads: the output
  // queue's counters and the releaser-private books.
  const uint32_t out = cur.sel ^ 1u;
  // the output queue's (vertices << 32 | edges); topology-driven SSSP: the vertices its
  // update interval lowered, and the edges its relax interval scanned
  // SSSP: after a select the near queue is expanded next, after an expand the pending queue
  const bool was_select = MODE == MODE_SSSP && sssp_select(cur);
  const unsigned long long packed = (MODE == MODE_BARRIER) ? 0ull
                                    : (MODE == MODE_PSSSP) ? c->qctr[0]
                                    : was_select           ? c->qctr[kNearQueue]
                                                           : c->qctr[out];
  const uint32_t dmin = (MODE == MODE_SSSP && !was_select) ? ld_relaxed(&c->dmin) : 0xFFFFFFFFu;
  const unsigned long long relaxed = (MODE == MODE_PSSSP) ? c->qctr[1] : 0ull;
  const uint32_t A = c->admitted, Jt = c->joined;
  const uint32_t decided = c->host_decided;
  const int32_t barriers = c->barriers + 1, kills0 = c->kills, forks0 = c->forks;
  const int32_t mina = c->min_active, maxa = c->max_active;
  const unsigned long long es0 = c->edges_scanned, ft0 = c->frontier_total, t_start = c->t_start;
  uint32_t log_n = c->log_n;
  const uint32_t err = ld_relaxed(&c->err);
  const uint32_t ret_raw = MODE == MODE_BFS ? ld_relaxed(&c->ret_n) : 0u;
  const uint32_t R = p.coop ? ld_relaxed(&c->join_ticket.v) : 0u;
  const uint64_t now = gtime();
  int32_t Mmid = M;
  if (simple) {
    Mmid = (int32_t)(live >> 32);
  } else {
    if (p.coop && (uint32_t)(kt >> 32) == cur.epoch) Mmid = min(M, max(1, (int32_t)(kt & 0x7FFFFFFFull)));
    if (Mmid < M) st_relaxed64(&c->kill_target, closed | (unsigned long long)(uint32_t)Mmid);
  }

  Interval nxt = cur;
  nxt.epoch = cur.epoch + 1u;
  nxt.level = cur.level + 1;
  // BFS: ranges handed back by doomed CTAs and not yet expanded open a continuation
  // interval of the same level
  const uint32_t ret_n = min(ret_raw, kRetCap);
  const uint32_t ret_done = (cur.cont >> 16) + (cur.cont & 0xFFFFu);
  const bool cont = MODE == MODE_BFS && err == 0u && ret_n > ret_done;
  uint32_t count, edges;
  if (cont) {
    nxt.level = cur.level;
    nxt.cont = ret_done << 16 | (ret_n - ret_done);
    count = cur.count;
    edges = cur.edges;
    c->cursor.v = 0u;
  } else if (MODE == MODE_BARRIER) {
    count = (cur.level + 1 < p.n_barriers) ? 1u : 0u;
    edges = 0u;
  } else if (MODE == MODE_PSSSP) {
    // intervals relax, update, check: after the check, stop if the update lowered nothing
    count = 1u;
    edges = 0u;
    if ((uint32_t)cur.level % 3u == 2u) {
      count = (uint32_t)packed;
      edges = (uint32_t)relaxed;
      c->qctr[0] = 0ull;
      c->qctr[1] = 0ull;
    }
    // the relax interval has used the heavy-row list: the next update builds it anew
    if ((uint32_t)cur.level % 3u == 0u) c->cursor.v = 0u;
  } else if (MODE == MODE_SSSP) {
    count = (uint32_t)(packed >> 32);
    edges = (uint32_t)packed;
    c->cursor.v = 0u;
    c->qctr[cur.sel] = 0ull;  // this round's pending queue is used up: it holds round r + 2's
    if (was_select) {
      nxt.sssp = sssp_word(sssp_round(cur), 0u, kNearQueue);
    } else {
      c->qctr[kNearQueue] = 0ull;
      nxt.sel = out;
      // every distance of round r + 1 is above the least one expanded in round r (recorded
      // by a select interval; without one the old base still bounds it)
      if (dmin != 0xFFFFFFFFu) nxt.base = dmin;
      st_relaxed(&c->dmin, 0xFFFFFFFFu);
      const uint64_t B = (uint64_t)M * NW * kNearUnits * kIndexEdges;
      nxt.sssp = sssp_word(sssp_round(cur) + 1u, (uint64_t)edges > B ? 1u : 0u, out);
    }
  } else {
    count = (uint32_t)(packed >> 32);
    edges = (uint32_t)packed;
    c->qctr[cur.sel] = 0ull;  // the finished input queue becomes the next output queue
    c->cursor.v = 0u;
    nxt.sel = out;
    if (MODE == MODE_BFS) {
      nxt.cont = 0u;
      if (ret_n) st_relaxed(&c->ret_n, 0u);
    }
  }
  nxt.count = count;
  nxt.edges = edges;
  // an SSSP round's expand interval runs even on an empty near queue: the traversal ends
  // when a round leaves nothing pending
  nxt.done = ((count == 0u && !was_select) || err != 0u) ? 1u : 0u;

  const int32_t Wmid = M - Mmid;
  const int32_t Mj = Mmid + (int32_t)J;  // the opening CTAs that stay, then the joiners
  int32_t k = 0, W = 0, spawned = 0;
  if (!nxt.done && p.coop) {
    // (2) fork: admit CTAs that registered and wait, up to N - Mmid - J
    k = (int32_t)min((uint32_t)(p.N - Mj), R - A);
    int32_t Ws = 0;
    if (p.sched_on) {
      // forced schedule: the scheduler grants up to kcap in [0, N-M] new CTAs (spawned
      // now, admitted when they arrive) and accepts W in [0, M-1] offer_kills
      const uint64_t r = mix64(p.sched_seed ^ mix64((uint64_t)barriers));
      const uint64_t r2 = mix64(r);
      const int32_t kcap = ((uint32_t)(r >> 32) < p.p_fork) ? (int32_t)(r2 % (uint64_t)(p.N - Mj + 1)) : 0;
      // launched, and neither admitted at an earlier barrier nor joined
      const int32_t pending = (int32_t)(ld_relaxed(&c->launched_total) - 1u - A - Jt - J);
      const int32_t spawn = kcap - pending;
      if (spawn > 0) {
        atomicAdd(&c->launched_total, (uint32_t)spawn);
        spawn_forks<MODE, NW>(p, (uint32_t)spawn);
        spawned = spawn;
      }
      if ((uint32_t)r < p.p_kill) Ws = (int32_t)((r2 >> 32) % (uint64_t)Mmid);
    }
    // (3) query for the forced schedule's kills (never CTA 0)
    W = min(Ws, Mj + k - 1);
  }
  const int32_t Mn = Mj + k - W;
  for (int32_t i = 0; i < k; ++i) {
    const uint32_t t = A + (uint32_t)i;
    const uint32_t idv = (uint32_t)(Mj + i);
    st_relaxed64(&c->slot[t % kMaxCtas], slot_pack(nxt.epoch, idv >= (uint32_t)Mn, idv, t));
  }
  // read by the scheduler warp together with the interval: published with it
  c->host_decided = decided + (uint32_t)Wmid;
  nxt.M = Mn;
  nxt.doom = (uint32_t)Mmid;
  if (simple) st_relaxed64(&c->live, (unsigned long long)(uint32_t)Mn << 32);
  if (!cont) nxt.precheck = precheck_hint(edges);
  c->iv = nxt;
  if (nxt.done) st_release(&c->done, 1u);  // after the admission slots (join_enter relies on it)

  bk.m_after = Mn;
  bk.admitted = A + (uint32_t)k;
  bk.joined = Jt + J;
  bk.barriers = barriers;
  bk.kills = kills0 + Wmid + W;
  bk.forks = forks0 + k + (int32_t)J;
  bk.min_active = min(mina, min(Mmid, Mn));
  bk.max_active = max(maxa, max(M + (int32_t)J, Mn));
  // edges and vertices of the frontiers the traversal expands (SSSP: not the pending
  // queues that a select interval splits)
  const bool expands = !nxt.done && !cont && (MODE != MODE_SSSP || !sssp_select(nxt));
  bk.edges_scanned = expands ? es0 + edges : es0;
  bk.frontier_total = expands ? ft0 + count : ft0;
  // every barrier while the first half of the trace has room, resize events always
  const int32_t t_us = (int32_t)((now - t_start) / 1000ull);
  bk.has_kill = Wmid > 0 && log_n < (uint32_t)kLogCap;  // the host kills of the interval
  bk.kill_rec = LogRec{barriers, t_us, M, 0, Wmid, Mmid, 0, (int32_t)edges};
  const uint32_t ln = log_n + (bk.has_kill ? 1u : 0u);
  // the joiners are logged as admitted at this barrier (the trace's fork count)
  const int32_t kj = k + (int32_t)J;
  bk.has_rec = ln < (uint32_t)kLogCap && (ln < (uint32_t)kLogCap / 2u || (kj | W | spawned) != 0);
  bk.rec = LogRec{barriers, t_us, Mmid, kj, W, Mn, spawned, (int32_t)edges};
  bk.log_n = log_n;
  bk.status = nxt.done ? (err ? (int)err : (ld_relaxed(&c->ovf) ? (int)ERR_OVERFLOW : 0)) : 1;
  return nxt;
}

// The second half of a release, after the epoch word has been released.
__device__ __forceinline__ void release_books(const Params &p, const Books &bk) {
  Ctl *c = p.ctl;
  c->admitted = bk.admitted;
  c->joined = bk.joined;
  c->barriers = bk.barriers;
  c->kills = bk.kills;
  c->forks = bk.forks;
  c->min_active = bk.min_active;
  c->max_active = bk.max_active;
  c->edges_scanned = bk.edges_scanned;
  c->frontier_total = bk.frontier_total;
  uint32_t ln = bk.log_n;
  if (bk.has_kill) c->log[ln++] = bk.kill_rec;
  if (bk.has_rec) c->log[ln++] = bk.rec;
  c->log_n = ln;
  if (p.coop) st_sys((uint32_t *)&p.mbox->active, (uint32_t)bk.m_after);
  if (bk.status != 1) publish_stats(p, bk.status);
}

// The resizing global barrier, called by all worker threads of an active CTA.
// Returns false when the run is aborting (error or timeout).
template <int MODE, int NW>
__device__ __forceinline__ bool resizing_barrier(const Params &p, CtaShared &cs) {
  workers_sync<NW>();  // the CTA's work for the interval is done
  if (threadIdx.x == 0) {
    Ctl *c = p.ctl;
    const Interval cur = cs.iv;
    // offer_kill: a CTA inside the host's kill target leaves as soon as it sees the target
    // while waiting (it has arrived, and the target is only ever lowered until the
    // releaser stamps it closed, so the closed target includes it)
    bool leave = false;
    if (p.coop && p.kill_mode == KILL_SIMPLE && cs.id > 0) {
      // the regular barrier's offer_kill, once, on arrival: leave if the host still
      // wants CTAs and this CTA has the largest live id
      const uint32_t want = ld_relaxed(&c->host_req) - ld_relaxed(&c->host_decided);
      unsigned long long lv = ld_relaxed64(&c->live);
      for (;;) {
        const uint32_t ml = (uint32_t)(lv >> 32), kd = (uint32_t)lv;
        if (kd >= want || (uint32_t)cs.id + 1u != ml) break;
        const unsigned long long prev =
            atomicCAS(&c->live, lv, ((unsigned long long)(ml - 1u) << 32) | (unsigned long long)(kd + 1u));
        if (prev == lv) {
          leave = true;
          break;
        }
        lv = prev;
      }
    }
    const uint64_t old = atom_add_acq_rel64(&c->arrive.v, 1ull);
    const uint32_t J = (uint32_t)(old >> 16) & 0xFFFFu;  // final: no CTA joins once all have arrived
    bool ok = true, next = false;
    Interval nxt;
    if (((uint32_t)old & 0xFFFFu) == (uint32_t)(cur.M - 1) + J + p.extra_wait) {
      Books bk;
      nxt = release_step<MODE, NW>(p, cur, J, bk);
      st_relaxed64(&c->arrive.v, arrive_word(cur.epoch + 1u, 0u, 0u));
      st_release(&c->epoch.v, cur.epoch + 1u);
      release_books(p, bk);
      next = true;
    } else if (!leave) {
      const int w = wait_release(p, cur.epoch, (p.coop && p.kill_mode != KILL_SIMPLE) ? cs.id : -1, cur.M);
      ok = w != 0;
      if (w == 1) {
        nxt = read_iv(c);
        next = true;
      }
      if (w == 2) leave = true;
    }
    if (next) {
      int32_t id = cs.id;
      if (id >= cur.M) {
        id = (int32_t)nxt.doom + (id - cur.M);  // joined during cur: after the opening CTAs that stay
      } else if (p.coop && id >= (int32_t)nxt.doom) {
        leave = true;  // a CTA that waited may still be inside the target as the release closed it
      }
      // the id before the interval: the doom watcher reads the interval's epoch first
      *(volatile int32_t *)&cs.id = id;
      __threadfence_block();
      cs.iv = nxt;
    }
    if (leave) {
      // the host sees the CTA go at once; the scheduler warp republishes the count in order
      // (two leavers' stores may reach the host out of order)
      const uint32_t v = atomicAdd(&c->surrendered, 1u) + 1u;
      if (p.coop) st_sys(&p.mbox->freed, p.kill_base + v);
    }
    cs.ok = ok ? 1 : 0;
    cs.leave = leave ? 1 : 0;
  }
  workers_sync<NW>();
  return cs.ok != 0 && cs.leave == 0;
}

// ---------------------------------------------------------------- entry
// Units per chunk in a round of the guided chunk schedule that has `rem` units left to
// deal over GW warps: half the remainder spread evenly, 1 .. cap.
__host__ __device__ __forceinline__ uint32_t round_units(uint32_t rem, uint32_t GW, uint32_t cap) {
  return min(cap, max(1u, (rem + 2u * GW - 1u) / (2u * GW)));
}

// Can a CTA join interval iv while it runs?  A BFS level (not a continuation of one)
// whose chunk schedule deals chunks beyond its first round -- claimed from the shared
// cursor by whichever warp is free, so a CTA that arrives late can take some.
template <int MODE, int NW>
__device__ __forceinline__ bool joinable(const Params &p, const Interval &iv) {
  if (MODE != MODE_BFS || !p.coop || p.kill_mode == KILL_SIMPLE || p.extra_wait != 0u) return false;
  if (iv.done || iv.cont != 0u || iv.M < 1) return false;
  const uint32_t GW = (uint32_t)iv.M * NW;
  if (iv.edges <= GW * 32u) return false;  // one 32-edge chunk per warp, nothing left over
  const uint32_t U = (iv.edges + kIndexEdges - 1u) >> kIndexShift;
  return U > GW * round_units(U, GW, kChunkUnitsMax);
}

// A forked CTA joins the running interval if it can (joinable; fewer than N CTAs in it;
// not all of its CTAs at the barrier yet): one CAS on the arrival word adds it to the
// barrier's count, and its logical id for the interval is M + (joiners before it).
// False if it cannot; it then registers for admission at the next barrier.
template <int MODE, int NW>
__device__ __forceinline__ bool join_running(const Params &p, CtaShared &cs) {
  Ctl *c = p.ctl;
  const uint32_t e = ld_acquire(&c->epoch.v);
  if (e == 0u) return false;  // the master has not opened the first interval
  const Interval iv = read_iv(c);
  if (iv.epoch != e || !joinable<MODE, NW>(p, iv)) return false;
  unsigned long long w = ld_relaxed64(&c->arrive.v);
  for (int tries = 0; tries < 64; ++tries) {
    const uint32_t J = (uint32_t)(w >> 16) & 0xFFFFu, a = (uint32_t)w & 0xFFFFu;
    // another epoch (released since), everyone arrived (releasing), or full
    if ((uint32_t)(w >> 32) != e || a >= (uint32_t)iv.M + J || (int32_t)((uint32_t)iv.M + J) >= p.N) return false;
    const unsigned long long prev = atomicCAS(&c->arrive.v, w, w + (1ull << 16));
    if (prev == w) {
      cs.iv = iv;
      cs.id = iv.M + (int32_t)J;
      return true;
    }
    w = prev;
  }
  return false;
}

// A CTA that is not the master joins the running interval (join_running), or registers
// and waits for a release that admits it (request_fork seen from the forked side).
// Returns false if it should leave.
template <int MODE, int NW>
__device__ __forceinline__ bool join_enter(const Params &p, CtaShared &cs) {
  Ctl *c = p.ctl;
  if (ld_relaxed(&c->run) != p.run || ld_relaxed(&c->done) != 0u || ld_relaxed(&c->err) != 0u) return false;
  if (join_running<MODE, NW>(p, cs)) return true;
  const uint32_t t = atomicAdd(&c->join_ticket.v, 1u);
  const uint64_t t0 = gtime();
  uint64_t s = 0;
  auto admitted = [&](uint64_t v) { return v != 0ull && (uint32_t)(v & 0x7FFFFull) == (t & 0x7FFFFu); };
  for (uint32_t spin = 0;; ++spin) {
    s = ld_acquire64(&c->slot[t % kMaxCtas]);
    if (admitted(s)) break;
    if (ld_acquire(&c->done) != 0u) {
      // The run is over -- possibly already at the master's entry, with this CTA among
      // the admitted.  The slots are written before `done` is released, so a second look
      // at the slot is conclusive: an admitted CTA goes on (it copies its share of the
      // result), any other leaves.
      s = ld_acquire64(&c->slot[t % kMaxCtas]);
      if (admitted(s)) break;
      return false;
    }
    if (ld_relaxed(&c->err) != 0u || ld_relaxed(&c->run) != p.run) return false;
    // a CTA that is never admitted simply leaves after the limit; it holds nobody up
    if ((spin & 15u) == 15u && gtime() - t0 > 4ull * p.timeout_ns) return false;
    __nanosleep(100);
  }
  if ((s >> 31) & 1ull) return false;  // admitted and killed in the same barrier
  const uint32_t ea = (uint32_t)(s >> 32);
  if (!wait_epoch_at_least(p, ea)) return false;
  cs.iv = read_iv(c);
  cs.id = (int32_t)((s >> 19) & 0xFFFull);
  return true;
}

// Non-cooperative baseline entry: fixed id = blockIdx.x, wait for the master's start.
__device__ __forceinline__ bool plain_enter(const Params &p, CtaShared &cs) {
  Ctl *c = p.ctl;
  if (!wait_epoch_at_least(p, 1u)) return false;
  cs.iv = read_iv(c);
  cs.id = (int32_t)blockIdx.x;
  return true;
}

// The master (block 0 of the main launch, logical id 0) seeds the frontier, waits
// briefly for its launch to register, admits them and opens interval 1 (level 0).
template <int MODE>
__device__ __forceinline__ void master_enter(const Params &p, CtaShared &cs) {
  Ctl *c = p.ctl;
  uint32_t count = 0u, edges = 0u;
  if (MODE == MODE_BARRIER) {
    count = p.n_barriers > 0 ? 1u : 0u;
  } else {
    const int32_t s = p.src;
    const int32_t rs = __ldg(p.row_off + s), re = __ldg(p.row_off + s + 1);
    if (rs < 0 || re < rs || (uint32_t)re > p.E) {
      raise_err(p, ERR_GRAPH);
    } else {
      if (MODE == MODE_BFS) {
        p.level[s] = 0;
        atomicOr(p.visited + (s >> 5), 1u << (s & 31));
      } else if (MODE == MODE_SSSP) {
        p.ds[s] = 1ull;  // distance 0, queued for round 1
      } else {
        p.dist[s] = 0u;  // topology-driven: distance 0, cost 0, changed
        reinterpret_cast<uint32_t *>(p.ds)[s] = 0u;
        atomicOr(p.visited + (s >> 5), 1u << (s & 31));
      }
      c->reached = 1ull;
      c->reached_edges = (unsigned long long)(re - rs);
      if (MODE == MODE_PSSSP) {
        count = 1u;  // the iterations run until one lowers nothing
        if (p.topo_heavy && (uint32_t)(re - rs) >= kTopoHeavy) {
          uint32_t n = 0u;
          for (uint64_t e = (uint64_t)rs; e < (uint64_t)re; e += kTopoChunk, ++n) {
            p.qv[0][n] = (uint32_t)s;
            p.qs[0][n] = (uint32_t)e;
          }
          c->cursor.v = n;
        }
      } else if (re > rs) {
        p.qo[0][0] = 0u;
        p.qs[0][0] = (uint32_t)rs;
        p.qv[0][0] = (uint32_t)s;
        count = 1u;
        edges = (uint32_t)(re - rs);
        for (uint32_t j = 0; j * kIndexEdges < edges; ++j) p.qx[0][j] = 0u;
      }
    }
  }
  int32_t k = 0;
  if (p.coop) {
    const uint64_t t0 = gtime();
    while (ld_relaxed(&c->join_ticket.v) + 1u < p.launched && gtime() - t0 < kEntryGatherNs) __nanosleep(200);
    const uint32_t R = ld_relaxed(&c->join_ticket.v);
    k = (int32_t)min(R, (uint32_t)(p.N - 1));
    for (int32_t i = 0; i < k; ++i)
      st_relaxed64(&c->slot[(uint32_t)i % kMaxCtas], slot_pack(1u, 0u, (uint32_t)(1 + i), (uint32_t)i));
  } else {
    k = (int32_t)gridDim.x - 1;
  }
  Interval iv;
  iv.M = 1 + k;
  iv.level = 0;
  iv.sel = 0u;
  iv.count = count;
  iv.edges = edges;
  iv.done = (count == 0u || ld_relaxed(&c->err) != 0u) ? 1u : 0u;
  iv.epoch = 1u;
  iv.doom = (uint32_t)(1 + k);
  iv.precheck = 0u;  // only the source is reached yet: every target is a candidate
  iv.base = 0u;
  iv.sssp = sssp_word(0u, 0u, 0u);  // SSSP round 0 expands the source's pending queue whole
  iv.cont = 0u;
  c->dmin = 0xFFFFFFFFu;
  c->admitted = (uint32_t)k;
  c->live = (unsigned long long)(uint32_t)iv.M << 32;
  c->t_start = gtime();
  st_relaxed(&c->launched_total, p.coop ? p.launched : gridDim.x);
  c->initial_active = iv.M;
  c->min_active = iv.M;
  c->max_active = iv.M;
  c->edges_scanned = edges;
  c->frontier_total = count;
  c->iv = iv;
  if (iv.done) {
    st_release(&c->done, 1u);  // after the admission slots (join_enter relies on it)
    const uint32_t e = ld_relaxed(&c->err);
    publish_stats(p, (int)e);
  }
  c->arrive.v = arrive_word(1u, 0u, 0u);
  st_release(&c->epoch.v, 1u);
  if (p.coop) st_sys((uint32_t *)&p.mbox->active, (uint32_t)iv.M);
  cs.iv = iv;
  cs.id = 0;
}

}  // namespace coopdev
