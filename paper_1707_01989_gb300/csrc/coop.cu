// coop.cu - cooperative kernels for GB300 (sm_103a) and the C ABI of libcoop.so.
//
// One traversal = one init kernel + one persistent kernel (+ CTAs the kernel itself
// launches from the device when it grows).  Inside the persistent kernel each interval
// between two resizing barriers expands one frontier (Fig. 4 of "Cooperative Kernels",
// Sec. 3.2):
//
//  * the frontier lives in a queue of (first column, edge-space offset[, vertex]) entries;
//    the offsets are the exclusive prefix sums of the frontier's out-degrees, built on
//    the fly by the warp-aggregated enqueue (one 64-bit atomic per warp adds both the
//    vertex count and the edge count), which also writes a chunk index (the entry holding
//    every 128th edge);
//  * the interval's edge space [0, edges) is cut into chunks of 32-edge units; a warp's
//    first chunk follows from its logical id -- the paper's tid / stride re-partition,
//    recomputed after every resizing barrier, applied to edges instead of vertices so that
//    skewed degrees (R-MAT hubs) are balanced -- and further chunks come from a shared
//    cursor; the claim of the next chunk is also the expansion's offer_kill point;
//  * a warp walks a chunk 128 edges (4 groups of 32) per iteration: a window of 32
//    frontier entries sits in registers, a ballot finds the entries that ended, one
//    __reduce_or marks the entries that start inside a group, and a popc over lanemask_le
//    gives each lane its source entry; the columns (and weights) of the next iteration
//    are copied into a shared-memory landing slot with cp.async while the current one is
//    claimed;
//  * BFS claims a vertex with an atomicOr on a 1-bit-per-vertex visited bitmap (checked
//    first with a plain load; stale reads only cost an extra atomic), writes its level
//    and enqueues it if its out-degree is non-zero; SSSP keeps (distance, round stamp)
//    of a vertex in one 64-bit word, so a single 64-bit atomicMin both lowers the
//    distance and tells whether the vertex is already queued for the next round.
//
// Also here: the topology-driven SSSP (Table 1 p-sssp), the work-stealing octree (Table 1
// octree), the batched launch, the serving loop, the co-runner and the allocation-free BFS.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <unordered_map>
#include <numeric>
#include <vector>
#include <chrono>
#include <cmath>
#include <mutex>
#include <thread>

#include "../../include/coop.h"
#include "coop_runtime.cuh"

using namespace coopdev;

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

struct Window {
  uint32_t off, end, start, u, du;
};

// entry i of the input queue (or an empty marker past its end)
template <int MODE>
__device__ __forceinline__ void load_entry(const Params &p, const uint32_t *qo, const uint32_t *qs,
                                           const uint32_t *qv, uint32_t F, uint32_t Etot, uint32_t i,
                                           Window &w) {
  if (i < F) {
    w.off = qo[i];
    w.start = qs[i];
    w.end = (i + 1u < F) ? qo[i + 1u] : Etot;
    if (MODE == MODE_SSSP) {
      w.u = qv[i];
      // a weak (L1-cacheable) read: after the barrier's acquire it returns the distance
      // at the barrier or a later, lower one, and a lowering after the barrier queues
      // the vertex again for the next round
      w.du = (uint32_t)(p.ds[w.u] >> 32);
    }
  } else {
    w.off = 0xFFFFFFFFu;
    w.end = 0xFFFFFFFFu;
    w.start = 0u;
    w.u = 0u;
    w.du = 0u;
  }
}

// Per-warp staging of enqueued vertices in shared memory: lanes append (v, first column,
// degree) without atomics; once 32 or more are staged the warp publishes them with ONE
// 64-bit atomicAdd on the output queue's (vertices << 32 | edges) counter, a two-pass
// warp scan of the degrees for their edge-space offsets, and coalesced stores.
constexpr int kStage = 64;

// BFS claim candidates: targets whose visited bit read as clear are compacted into a
// per-warp ring and claimed one per lane, so that the claim (atomic, level write, row
// bounds, enqueue) runs once per 32 candidates with every lane busy, instead of once per
// 32-edge group with a few lanes busy.  A ring holds at most 63 entries: whenever 32 are
// pending after a group they are claimed at once; the rest when the warp's part of the
// interval is done.  (Claiming what is pending at the end of every iteration instead
// measured 8 % slower on R-MAT 22.)
constexpr uint32_t kCand = 64;
constexpr uint32_t kNoChunk = 0xFFFFFFFFu;  // no further chunk for this warp

// Queue q (0, 1 or 2) of a per-queue pointer array of the kernel parameters, chosen by
// selects: an index into the parameter array itself would make the compiler copy it to
// local memory.
template <typename T>
__device__ __forceinline__ T *queue(T *const (&a)[3], uint32_t q) {
  return q == 0u ? a[0] : q == 1u ? a[1] : a[2];
}

// The chunk schedule of one interval.  A frontier of at most GW * 32 edges (GW = M * NW
// worker warps) gets one 32-edge chunk per warp.  A larger one is cut into units of
// kIndexEdges edges, handed out in rounds of GW chunks: round r's chunks span
// s_r = clamp(ceil(rem_r / (2 GW)), 1, cap) units each, rem_r being the units no earlier
// round covered, so that each round takes about half of what is left.  Most of a wide
// level then goes in large chunks (few chunk starts, each a chain of dependent loads) and
// its end in single units (a short tail).  The cap is larger for BFS than for SSSP, whose
// relaxations read distances at the start of a chunk: long chunks there expand more edges
// (kChunkUnitsMax, kChunkUnitsMaxSssp).  Round 0's chunk j is warp j's -- Fig. 4's
// tid/stride split, recomputed from the current M -- and later chunk ids come from the
// shared cursor.  On wide levels every chunk starts at a unit boundary, an indexed edge.
struct ChunkSched {  // per warp, in shared memory: touched only between chunks
  uint32_t U;      // units of the interval
  uint32_t shift;  // log2 of the edges per unit: 5 on small frontiers, else log2(kIndexEdges)
  uint32_t k0, base, s;  // the current round: first chunk id, first unit, units per chunk
  uint32_t cap;          // units per chunk at most
};

// Chunk index: for every unit boundary j*kIndexEdges inside an entry's edge range
// [o, o + d), record the entry's queue slot.  Called by a whole warp, one entry per lane
// (`valid`); a lane whose entry spans more than 8 boundaries (an R-MAT hub spans
// hundreds) is helped by the others, so no lane loops alone over a long row.
__device__ __forceinline__ void index_chunks(uint32_t *qx, uint32_t o, uint32_t d, uint32_t slot, bool valid,
                                             unsigned lane) {
  const uint32_t j0 = (o + kIndexEdges - 1u) / kIndexEdges;
  const uint32_t j1 = valid ? (o + d + kIndexEdges - 1u) / kIndexEdges : j0;
  const bool big = j1 - j0 > 8u;
  if (!big)
    for (uint32_t j = j0; j < j1; ++j) qx[j] = slot;
  for (unsigned m = __ballot_sync(0xFFFFFFFFu, big); m != 0u; m &= m - 1u) {
    const int l = __ffs(m) - 1;
    const uint32_t b0 = __shfl_sync(0xFFFFFFFFu, j0, l), b1 = __shfl_sync(0xFFFFFFFFu, j1, l);
    const uint32_t bs = __shfl_sync(0xFFFFFFFFu, slot, l);
    for (uint32_t j = b0 + lane; j < b1; j += 32u) qx[j] = bs;
  }
}

struct WarpStage {
  uint32_t v[kStage];
  uint32_t rs[kStage];
  uint32_t deg[kStage];
};

template <int MODE>
__device__ __forceinline__ void stage_flush(const Params &p, uint32_t out, WarpStage &b, uint32_t n, unsigned lane,
                                            bool index = true) {
  __syncwarp();
  const uint32_t d0 = lane < n ? b.deg[lane] : 0u;
  const uint32_t d1 = lane + 32u < n ? b.deg[lane + 32u] : 0u;
  uint32_t s0 = d0, s1 = d1;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y0 = __shfl_up_sync(kFull, s0, o);
    const uint32_t y1 = __shfl_up_sync(kFull, s1, o);
    if ((int)lane >= o) {
      s0 += y0;
      s1 += y1;
    }
  }
  const uint32_t t0 = __shfl_sync(kFull, s0, 31);
  const uint32_t total = t0 + __shfl_sync(kFull, s1, 31);
  unsigned long long base = 0ull;
  if (lane == 0) base = atomicAdd(&p.ctl->qctr[out], ((unsigned long long)n << 32) | (unsigned long long)total);
  base = __shfl_sync(kFull, base, 0);
  const uint32_t bc = (uint32_t)(base >> 32), be = (uint32_t)base;
  uint32_t *qo = out ? p.qo[1] : p.qo[0];  // the output of an expansion: queue 0 or 1
  uint32_t *qs = out ? p.qs[1] : p.qs[0];
  uint32_t *qv = out ? p.qv[1] : p.qv[0];
  uint32_t *qx = out ? p.qx[1] : p.qx[0];
  const uint32_t o0 = be + s0 - d0, o1 = be + t0 + s1 - d1;
  if (lane < n) {
    qo[bc + lane] = o0;
    qs[bc + lane] = b.rs[lane];
    if (MODE == MODE_SSSP) qv[bc + lane] = b.v[lane];
  }
  if (lane + 32u < n) {
    qo[bc + 32u + lane] = o1;
    qs[bc + 32u + lane] = b.rs[lane + 32u];
    if (MODE == MODE_SSSP) qv[bc + 32u + lane] = b.v[lane + 32u];
  }
  if (index) {
    index_chunks(qx, o0, d0, bc + lane, lane < n, lane);
    if (n > 32u) index_chunks(qx, o1, d1, bc + 32u + lane, lane + 32u < n, lane);
  }
  __syncwarp();
}

template <int MODE>
__device__ __forceinline__ void stage_push(const Params &p, uint32_t out, WarpStage &b, uint32_t &n, bool push,
                                           uint32_t v, uint32_t rs, uint32_t deg, unsigned lane, bool index = true) {
  const unsigned pm = __ballot_sync(kFull, push);
  if (pm == 0u) return;
  if (push) {
    const uint32_t at = n + (uint32_t)__popc(pm & lanemask_lt());
    b.v[at] = v;
    b.rs[at] = rs;
    b.deg[at] = deg;
  }
  n += (uint32_t)__popc(pm);
  if (n >= 32u) {
    stage_flush<MODE>(p, out, b, n, lane, index);
    n = 0u;
  }
}

// Claim the n (<= 32) candidates at ring positions head.. of a BFS warp, one per lane:
// the row bounds are read before the atomicOr so the two round trips overlap; a lane
// whose atomicOr set the bit writes the level and enqueues the vertex if it has
// out-edges.  A candidate that another warp claimed meanwhile costs one failed atomic.
__device__ __forceinline__ void claim_batch(const Params &p, uint32_t out, WarpStage &stage, uint32_t &staged,
                                            const uint32_t *cand, uint32_t head, uint32_t n, uint32_t next_level,
                                            bool &bad, uint32_t &nreach, uint64_t &ereach, unsigned lane) {
  __syncwarp();  // the ring's entries written by other lanes
  const bool has = lane < n;
  const uint32_t v = has ? cand[(head + lane) & (kCand - 1u)] : 0u;
  int32_t ra = 0, rb = 0;
  if (has) {
    ra = __ldg(p.row_off + v);
    rb = __ldg(p.row_off + v + 1);
  }
  const uint32_t m = 1u << (v & 31u);
  const bool claim = has && (atomicOr(p.visited + (v >> 5), m) & m) == 0u;
  uint32_t rs = 0u, deg = 0u;
  bool push = false;
  if (claim) {
    p.level[v] = (int32_t)next_level;
    if (ra < 0 || rb < ra || (uint32_t)rb > p.E) bad = true;
    else {
      rs = (uint32_t)ra;
      deg = (uint32_t)(rb - ra);
      push = deg > 0u;
    }
    nreach += 1u;
    ereach += deg;
  }
  stage_push<MODE_BFS>(p, out, stage, staged, push, v, rs, deg, lane);
  __syncwarp();  // the ring's slots just read may be written again by the next group
}

// Read row_off[v], row_off[v+1] of a vertex about to be enqueued; false if malformed.
__device__ __forceinline__ bool row_of(const Params &p, uint32_t v, uint32_t &rs, uint32_t &deg) {
  const int32_t a = __ldg(p.row_off + v), b = __ldg(p.row_off + v + 1);
  if (a < 0 || b < a || (uint32_t)b > p.E) return false;
  rs = (uint32_t)a;
  deg = (uint32_t)(b - a);
  return true;
}

constexpr int kUnroll = 4;  // 32-edge groups a warp handles per iteration

// Per-warp landing buffer of the column stream: two slots of kUnroll x 32 edges, each
// edge's column (and, for SSSP, its weight and its source's distance).  While a warp
// claims the targets of one slot, the asynchronous copies of the next 128 edges fill the
// other, so the DRAM latency of the column stream overlaps the L2 round trips of the
// claim.  Every lane copies and later reads only its own words of a slot.
constexpr int kStages = 2;  // landing slots: copies run kStages - 1 iterations ahead
template <int MODE>
struct Landing {  // BFS (and the barrier self-test): columns, the claim ring, the schedule
  uint32_t col[kStages][kUnroll][32];
  uint32_t cand[kCand];
  ChunkSched sched;
};
template <>
struct Landing<MODE_SSSP> {
  uint32_t col[kStages][kUnroll][32];
  uint32_t w[kStages][kUnroll][32];
  uint32_t du[kStages][kUnroll][32];
  ChunkSched sched;
};

// Dynamic shared memory of a traversal CTA: NW enqueue stages, then NW landing buffers,
// and at least kTraverseSmemMin (SM exclusivity).  The batch kernel runs both kinds of
// job and takes the SSSP size.
__host__ __device__ constexpr int traverse_smem(int mode, int nw) {
  const size_t need =
      (size_t)nw * (sizeof(WarpStage) + (mode == MODE_SSSP ? sizeof(Landing<MODE_SSSP>) : sizeof(Landing<MODE_BFS>)));
  const int rounded = (int)((need + 1023) / 1024 * 1024);
  return rounded > kTraverseSmemMin ? rounded : kTraverseSmemMin;
}
static_assert(traverse_smem(MODE_SSSP, kDefaultWorkerWarps) <= 227 * 1024, "traversal CTA shared memory");
static_assert(15 * sizeof(Landing<MODE_SSSP>) >= kHistBuckets * sizeof(uint32_t),
              "an SSSP CTA's landing buffers hold its histogram in a select interval");

__device__ __forceinline__ void cp_async4(void *sdst, const void *gsrc) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Drop the window's entries that end at or before edge x (32 at most per call); true if
// any did.  Once it returns false, lane 0 holds the entry containing x.
template <int MODE>
__device__ __forceinline__ bool slide(const Params &p, const uint32_t *qo, const uint32_t *qs, const uint32_t *qv,
                                      uint32_t F, uint32_t Etot, uint32_t x, Window &w, uint32_t &wb,
                                      unsigned lane) {
  const unsigned ended = __ballot_sync(kFull, w.end <= x);
  if (!ended) return false;
  const unsigned n = (unsigned)__popc(ended);
  wb += n;
  const unsigned srcl = (lane + n) & 31u;
  Window t;
  t.off = __shfl_sync(kFull, w.off, srcl);
  t.end = __shfl_sync(kFull, w.end, srcl);
  t.start = __shfl_sync(kFull, w.start, srcl);
  if (MODE == MODE_SSSP) {
    t.u = __shfl_sync(kFull, w.u, srcl);
    t.du = __shfl_sync(kFull, w.du, srcl);
  }
  if (lane + n < 32u) w = t;
  else load_entry<MODE>(p, qo, qs, qv, F, Etot, wb + lane, w);
  return true;
}

// The index arithmetic of the kUnroll groups starting at edge c (window slide, source
// entry of each lane's edge) and the start of their column (and weight) copies into
// slot sb of the landing buffer.
template <int MODE>
__device__ __forceinline__ void issue_groups(const Params &p, const uint32_t *qo, const uint32_t *qs,
                                             const uint32_t *qv, uint32_t F, uint32_t Etot, uint32_t c,
                                             uint32_t E1, Window &w, uint32_t &wb, Landing<MODE> &pf, int sb,
                                             unsigned lane, unsigned lm_le) {
  // Fast path: lane 0 holds the entry containing edge c - 32 (or c itself); if that entry
  // also covers all of [c, c + 32 kUnroll) -- most iterations on wide R-MAT levels, whose
  // rows run to hundreds of edges -- the positions are contiguous and the window stays.
  const uint32_t end0 = __shfl_sync(kFull, w.end, 0);
  if (end0 >= c + 32u * kUnroll) {
    const uint32_t s0 = __shfl_sync(kFull, w.start, 0);
    const uint32_t o0 = __shfl_sync(kFull, w.off, 0);
    uint32_t du = 0u;
    if (MODE == MODE_SSSP) du = __shfl_sync(kFull, w.du, 0);
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint32_t e = c + 32u * (uint32_t)u + lane;
      if (e < E1) {
        const uint32_t pos = s0 + (e - o0);
        cp_async4(&pf.col[sb][u][lane], p.col + pos);
        if constexpr (MODE == MODE_SSSP) {
          cp_async4(&pf.w[sb][u][lane], p.w + pos);
          pf.du[sb][u][lane] = du;
        }
      }
    }
    cp_async_commit();
    return;
  }
  // One slide to c: lane 0 then holds the entry containing c.  When the window's 32
  // entries reach the end of the iteration (rows of 4 or more edges on average: nearly
  // every iteration of a wide R-MAT level that spans several rows), every group's source
  // entries are found in the window as it is -- the entry containing the group's first
  // edge is the last lane whose entry starts at or before it -- and the next iteration's
  // slide drops at most 32 entries.  Otherwise the window slides group by group.
  slide<MODE>(p, qo, qs, qv, F, Etot, c, w, wb, lane);
  if (__shfl_sync(kFull, w.end, 31) >= min(c + 32u * kUnroll, E1)) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint32_t cu = c + 32u * (uint32_t)u;
      if (cu >= E1) break;  // warp-uniform
      const unsigned k = 31u - (unsigned)__clz(__ballot_sync(kFull, w.off <= cu));  // lane 0's entry qualifies
      // entries starting strictly inside (cu, cu + 32) -> source entry of each lane's edge
      const uint32_t rel = w.off - cu;
      const unsigned bit = (rel - 1u < 31u) ? (1u << rel) : 0u;
      const unsigned bits = __reduce_or_sync(kFull, bit);
      const unsigned idx = k + (unsigned)__popc(bits & lm_le);
      const uint32_t s0 = __shfl_sync(kFull, w.start, idx);
      const uint32_t o0 = __shfl_sync(kFull, w.off, idx);
      uint32_t du = 0u;
      if (MODE == MODE_SSSP) du = __shfl_sync(kFull, w.du, idx);
      const uint32_t e = cu + lane;
      if (e < E1) {
        const uint32_t pos = s0 + (e - o0);
        cp_async4(&pf.col[sb][u][lane], p.col + pos);
        if constexpr (MODE == MODE_SSSP) {
          cp_async4(&pf.w[sb][u][lane], p.w + pos);
          pf.du[sb][u][lane] = du;
        }
      }
    }
    cp_async_commit();
    return;
  }
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const uint32_t cu = c + 32u * (uint32_t)u;
    if (cu >= E1) break;  // warp-uniform
    // every entry holds at least one edge, so one slide covers a 32-edge step
    if (u > 0) slide<MODE>(p, qo, qs, qv, F, Etot, cu, w, wb, lane);
    // entries starting strictly inside [cu, cu+32) -> source entry of each lane's edge
    const uint32_t rel = w.off - cu;
    const unsigned bit = (lane != 0u && rel < 32u) ? (1u << rel) : 0u;
    const unsigned bits = __reduce_or_sync(kFull, bit);
    const unsigned idx = (unsigned)__popc(bits & lm_le);
    const uint32_t s0 = __shfl_sync(kFull, w.start, idx);
    const uint32_t o0 = __shfl_sync(kFull, w.off, idx);
    uint32_t du = 0u;
    if (MODE == MODE_SSSP) du = __shfl_sync(kFull, w.du, idx);
    const uint32_t e = cu + lane;
    if (e < E1) {
      const uint32_t pos = s0 + (e - o0);
      cp_async4(&pf.col[sb][u][lane], p.col + pos);
      if constexpr (MODE == MODE_SSSP) {
        cp_async4(&pf.w[sb][u][lane], p.w + pos);
        pf.du[sb][u][lane] = du;
      }
    }
  }
  cp_async_commit();
}

// ---- frontier SSSP rounds: select, then expand (Table 1 l-sssp: two barriers per iteration)

// Histogram bucket of tentative distance d in a pending queue whose bucket 0 starts at base.
__device__ __forceinline__ uint32_t dist_bucket(uint32_t d, uint32_t base) {
  return d <= base ? 0u : min(kHistBuckets - 1u, (d - base) >> kHistShift);
}

// Stamp of "queued in the pending queue of round r + 1" during round r (the source is
// queued for round 0 with stamp 1; a never-queued vertex has stamp 0).
__device__ __forceinline__ uint32_t sssp_tag(const Interval &iv) { return sssp_round(iv) + 2u; }

// The select interval of round r: split the pending queue (queue iv.sel).  The CTA with
// logical id `id` owns the queue's 32-entry stripes id * NW + w, id * NW + w + GW, ...
// (Fig. 4's tid / stride over the current M), spread over the whole queue.  Its first
// stripe per warp is a sample: a histogram of their out-degrees over their current
// distances (hs, kHistBuckets words of shared memory) gives the threshold b*, the first
// bucket at which the sample's cumulative out-degree reaches the fraction of the queue's
// edges that the round's target B = GW * kNearUnits * kIndexEdges is.  Then the entries
// in buckets up to b* go to the near queue, any other stays pending for round r + 1 --
// its stamp advanced so that a lowering in this round's expand interval does not queue it
// twice -- kSelectBatch stripes per warp at a time, the CTA's warps taking their places
// in each queue from one atomic of the CTA's (all warps at once on one counter would
// queue behind each other at the L2).  The least distance
// selected goes to the control block: the next round's base.  No distance changes in a
// select interval.  Every selection gives the same result: a vertex whose distance
// dropped is pending until it has been expanded at that distance, and the traversal ends
// only when nothing is pending.
constexpr int kSelectBatch = 4;

template <int NW>
__device__ __forceinline__ void select_interval(const Params &p, const Interval &iv, int32_t id, uint32_t *hs,
                                                CtaShared &cs) {
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt();
  const uint32_t in = iv.sel, out = in ^ 1u;
  const uint32_t GW = (uint32_t)iv.M * NW;
  const uint32_t F = iv.count, Etot = iv.edges;
  const uint32_t *qo = queue(p.qo, in), *qs = queue(p.qs, in), *qv = queue(p.qv, in);
  const uint32_t first = ((uint32_t)id * NW + warp) * 32u;
  for (uint32_t b = threadIdx.x; b < kHistBuckets; b += NW * 32) hs[b] = 0u;
  if (threadIdx.x == 0) {
    cs.split[1] = 0xFFFFFFFFu;
    cs.take[0][0] = cs.take[0][1] = cs.take[1][0] = cs.take[1][1] = 0ull;
  }
  workers_sync<NW>();
  if (first + lane < F) {
    const uint32_t i = first + lane;
    const uint32_t deg = (i + 1u < F ? qo[i + 1u] : Etot) - qo[i];
    atomicAdd(&hs[dist_bucket((uint32_t)(__ldcg(p.ds + qv[i]) >> 32), iv.base)], deg);
  }
  workers_sync<NW>();
  if (warp == 0) {
    // the first bucket with cum * Etot >= B * total: lane l sums segment l (32 buckets),
    // one scan over the segments finds the segment, one more the bucket in it
    static_assert(kHistBuckets == 32u * 32u, "the threshold search takes 32 segments of 32 buckets");
    uint32_t seg = 0u;
#pragma unroll 8
    for (uint32_t k = 0; k < 32u; ++k) seg += hs[lane * 32u + ((k + lane) & 31u)];  // rotated: no bank conflicts
    uint32_t sc = seg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, sc, o);
      if ((int)lane >= o) sc += y;
    }
    const uint64_t want = (uint64_t)GW * kNearUnits * kIndexEdges * __shfl_sync(kFull, sc, 31);
    const unsigned hs_hit = __ballot_sync(kFull, (uint64_t)sc * Etot >= want);
    uint32_t bstar = kHistBuckets - 1u;
    if (hs_hit != 0u) {
      const uint32_t sg = (uint32_t)(__ffs(hs_hit) - 1);
      const uint64_t before = __shfl_sync(kFull, sc - seg, (int)sg);  // buckets below segment sg
      uint32_t b = hs[sg * 32u + lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, b, o);
        if ((int)lane >= o) b += y;
      }
      const unsigned hit = __ballot_sync(kFull, (before + b) * (uint64_t)Etot >= want);
      bstar = sg * 32u + (uint32_t)(__ffs(hit) - 1);  // the segment's total reaches want: hit != 0
    }
    if (lane == 0) cs.split[0] = bstar;
  }
  workers_sync<NW>();
  const uint32_t bstar = cs.split[0];
  const uint32_t tag = sssp_tag(iv);
  uint32_t dmin = 0xFFFFFFFFu;
  const uint32_t step = GW * 32u;
  // batches: the same count for every warp of the CTA (they meet at two CTA syncs each)
  const uint32_t nb = (F + kSelectBatch * step - 1u) / (kSelectBatch * step);
  for (uint32_t bi = 0, i0 = first; bi < nb; ++bi, i0 += kSelectBatch * step) {
    unsigned long long *take = cs.take[bi & 1u];
    uint32_t v[kSelectBatch], rs[kSelectBatch], deg[kSelectBatch];
    bool near[kSelectBatch], far[kSelectBatch];
#pragma unroll
    for (int k = 0; k < kSelectBatch; ++k) {
      const uint32_t i = i0 + (uint32_t)k * step + lane;
      v[k] = 0u;
      rs[k] = 0u;
      deg[k] = 0u;
      if (i < F) {
        v[k] = qv[i];
        rs[k] = qs[i];
        deg[k] = (i + 1u < F ? qo[i + 1u] : Etot) - qo[i];
      }
    }
    uint32_t nN = 0u, nF = 0u, eN = 0u, eF = 0u;
#pragma unroll
    for (int k = 0; k < kSelectBatch; ++k) {
      const bool valid = i0 + (uint32_t)k * step + lane < F;
      const uint32_t d = valid ? (uint32_t)(__ldcg(p.ds + v[k]) >> 32) : 0u;
      near[k] = valid && dist_bucket(d, iv.base) <= bstar;
      far[k] = valid && !near[k];
      if (near[k]) dmin = min(dmin, d);
      nN += (uint32_t)__popc(__ballot_sync(kFull, near[k]));
      nF += (uint32_t)__popc(__ballot_sync(kFull, far[k]));
      eN += near[k] ? deg[k] : 0u;
      eF += far[k] ? deg[k] : 0u;
    }
    eN = __reduce_add_sync(kFull, eN);
    eF = __reduce_add_sync(kFull, eF);
    // the warp's places within the CTA's part, then the CTA's part of each queue
    unsigned long long lN = 0ull, lF = 0ull;
    if (lane == 0) {
      lN = atomicAdd(&take[0], ((unsigned long long)nN << 32) | eN);
      lF = atomicAdd(&take[1], ((unsigned long long)nF << 32) | eF);
    }
    workers_sync<NW>();
    if (threadIdx.x == 0) {
      const unsigned long long tN = take[0], tF = take[1];
      take[0] = tN ? atomicAdd(&p.ctl->qctr[kNearQueue], tN) : 0ull;
      take[1] = tF ? atomicAdd(&p.ctl->qctr[out], tF) : 0ull;
      // every warp read the other parity's bases before the first sync of this batch
      cs.take[(bi & 1u) ^ 1u][0] = cs.take[(bi & 1u) ^ 1u][1] = 0ull;
    }
    workers_sync<NW>();
    const unsigned long long bN = __shfl_sync(kFull, lN, 0) + take[0];
    const unsigned long long bF = __shfl_sync(kFull, lF, 0) + take[1];
    uint32_t atN = (uint32_t)(bN >> 32), oN = (uint32_t)bN, atF = (uint32_t)(bF >> 32), oF = (uint32_t)bF;
#pragma unroll
    for (int k = 0; k < kSelectBatch; ++k) {
      // exclusive scans of this stripe's near and far degrees
      uint32_t sN = near[k] ? deg[k] : 0u, sF = far[k] ? deg[k] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t yN = __shfl_up_sync(kFull, sN, o), yF = __shfl_up_sync(kFull, sF, o);
        if ((int)lane >= o) {
          sN += yN;
          sF += yF;
        }
      }
      const unsigned mN = __ballot_sync(kFull, near[k]), mF = __ballot_sync(kFull, far[k]);
      const uint32_t atn = atN + (uint32_t)__popc(mN & lt), on = oN + sN - deg[k];
      const uint32_t atf = atF + (uint32_t)__popc(mF & lt), of = oF + sF - deg[k];
      if (near[k]) {
        p.qo[kNearQueue][atn] = on;
        p.qs[kNearQueue][atn] = rs[k];
        p.qv[kNearQueue][atn] = v[k];
      }
      if (far[k]) {
        reinterpret_cast<uint32_t *>(p.ds + v[k])[0] = tag;  // the stamp half of the packed word
        queue(p.qo, out)[atf] = of;
        queue(p.qs, out)[atf] = rs[k];
        queue(p.qv, out)[atf] = v[k];
      }
      if (mN) index_chunks(p.qx[kNearQueue], on, deg[k], atn, near[k], lane);
      if (mF) index_chunks(queue(p.qx, out), of, deg[k], atf, far[k], lane);
      atN += (uint32_t)__popc(mN);
      atF += (uint32_t)__popc(mF);
      oN += __shfl_sync(kFull, sN, 31);
      oF += __shfl_sync(kFull, sF, 31);
    }
  }
  dmin = __reduce_min_sync(kFull, dmin);
  if (lane == 0 && dmin != 0xFFFFFFFFu) atomicMin(&cs.split[1], dmin);
  workers_sync<NW>();
  if (threadIdx.x == 0 && cs.split[1] != 0xFFFFFFFFu) atomicMin(&p.ctl->dmin, cs.split[1]);
}

// BFS expansion of edges [c0, c1) (the contract is expand_range's).  Software-pipelined
// like it; per iteration the visited word of every target is read (on small frontiers no
// pre-check: every target is a candidate) and the targets it shows unvisited are
// compacted into the warp's claim ring, 32 pending candidates claimed at once.  (Loading
// the visited words one iteration ahead, with a third landing slot, measured no faster.)
template <int MODE>
__device__ __forceinline__ uint32_t expand_range_bfs(const Params &p, const Interval &iv, uint32_t c0, uint32_t c1,
                                                     uint32_t wb, WarpStage &stage, Landing<MODE> &pf,
                                                     uint32_t &staged, bool &bad, uint32_t &nreach, uint64_t &ereach,
                                                     bool more, int32_t id, uint32_t GW, uint32_t &ch,
                                                     uint32_t &ct, const volatile uint32_t *doom) {
  const unsigned lane = threadIdx.x & 31u;
  const uint32_t Etot = iv.edges;
  const uint32_t F = iv.count;
  const uint32_t in = iv.sel, out = in ^ 1u;
  const uint32_t *qo = in ? p.qo[1] : p.qo[0];
  const uint32_t *qs = in ? p.qs[1] : p.qs[0];
  const uint32_t *qv = in ? p.qv[1] : p.qv[0];
  const unsigned lm_le = lanemask_le();
  const unsigned lt = lm_le & ~(1u << lane);
  const uint32_t next_level = (uint32_t)iv.level + 1u;
  const uint32_t V = (uint32_t)p.V;
  const uint32_t E1 = c1;
  const bool pre = iv.precheck != 0u;
  constexpr uint32_t kIt = 32u * kUnroll;

  Window w;
  load_entry<MODE>(p, qo, qs, qv, F, Etot, wb + lane, w);
  while (slide<MODE>(p, qo, qs, qv, F, Etot, c0, w, wb, lane)) {
  }
  uint32_t ci = c0;
#pragma unroll
  for (int k = 0; k < kStages - 1; ++k, ci += kIt) {
    if (ci < E1) issue_groups<MODE>(p, qo, qs, qv, F, Etot, ci, E1, w, wb, pf, k, lane, lm_le);
    else cp_async_commit();
  }
  int sb = 0, sn = kStages - 1;
  uint32_t jn = kNoChunk;
  // Kill point inside the chunk (KILL_CHUNK): once the CTA's doom watcher has seen the
  // host's kill target take this CTA, a warp hands the rest of its chunk back (from a
  // unit boundary, an indexed edge) and stops, so that the CTA leaves within about one
  // iteration.
  const bool handback = p.coop && p.kill_mode == KILL_CHUNK && MODE == MODE_BFS && id > 0;
  uint32_t dm = handback ? *doom : 0u;  // read one iteration before it is tested
  for (uint32_t c = c0; c < E1; c += kIt, ci += kIt) {
    if (handback && dm == iv.epoch && (c & (kIndexEdges - 1u)) == 0u) {
      uint32_t pushed = 0u;
      if (lane == 0) {
        const uint32_t slot = atomicAdd(&p.ctl->ret_n, 1u);
        if (slot < kRetCap) {
          p.ctl->ret[slot] = ((unsigned long long)c << 32) | E1;
          pushed = 1u;
        }
      }
      if (__shfl_sync(kFull, pushed, 0) != 0u) {
        cp_async_wait<0>();  // the copies in flight land before the buffers are left
        return kNoChunk;
      }
      // the list is full: this iteration goes on (the next one tries again)
    }
    if (more && lane == 0 && c + kIt >= E1 &&
        !(p.coop && p.kill_mode == KILL_CHUNK && doomed(ld_relaxed64(&p.ctl->kill_target), iv.epoch, id, iv.M)))
      jn = GW + atomicAdd(&p.ctl->cursor.v, 1u);
    if (ci < E1) issue_groups<MODE>(p, qo, qs, qv, F, Etot, ci, E1, w, wb, pf, sn, lane, lm_le);
    else cp_async_commit();
    cp_async_wait<kStages - 1>();  // this iteration's slot has landed; later ones stay in flight
    uint32_t vv[kUnroll], word[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      vv[u] = pf.col[sb][u][lane];
      word[u] = 0xFFFFFFFFu;  // past the range or out of [0, V): reads as visited
      if (c + 32u * (uint32_t)u + lane < E1) {
        if (vv[u] >= V) bad = true;
        else word[u] = pre ? *(p.visited + (vv[u] >> 5)) : 0u;
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const bool cnd = word[u] != 0xFFFFFFFFu && ((word[u] >> (vv[u] & 31u)) & 1u) == 0u;
      const unsigned m = __ballot_sync(kFull, cnd);
      if (cnd) pf.cand[(ct + (uint32_t)__popc(m & lt)) & (kCand - 1u)] = vv[u];
      ct += (uint32_t)__popc(m);
      if (ct - ch >= 32u) {
        claim_batch(p, out, stage, staged, pf.cand, ch, 32u, next_level, bad, nreach, ereach, lane);
        ch += 32u;
      }
    }
    sb = sb + 1 == kStages ? 0 : sb + 1;
    sn = sn + 1 == kStages ? 0 : sn + 1;
    if (handback) dm = *doom;
  }
  return __shfl_sync(kFull, jn, 0);
}

// Expand edges [c0, c1) of the interval's edge space (SSSP); entry wb of the input queue
// holds edge c0.  Software-pipelined over iterations of kUnroll 32-edge groups: the copies
// of iteration i+1 are started, then iteration i's targets are relaxed, so every lane keeps
// the next kUnroll column loads in flight while it works on the current ones.
//
// Returns the warp's next chunk id (kNoChunk: none).  With `more`, lane 0 claims it from the
// cursor at the start of the range's last iteration, so the atomic's latency overlaps
// that iteration's work.  This is also the offer_kill point of the expansion: a CTA inside
// the host's kill target claims nothing more (the other CTAs take the rest of the level)
// and leaves at the barrier, at most one iteration after the check.
template <int MODE>
__device__ __forceinline__ uint32_t expand_range(const Params &p, const Interval &iv, uint32_t c0, uint32_t c1,
                                                 uint32_t wb, WarpStage &stage, Landing<MODE> &pf,
                                                 uint32_t &staged, bool &bad, bool &ovf, uint32_t &nreach,
                                                 uint64_t &ereach, bool more, int32_t id, uint32_t GW) {
  const unsigned lane = threadIdx.x & 31u;
  const uint32_t Etot = iv.edges;
  const uint32_t F = iv.count;
  const uint32_t out = iv.sel ^ 1u;  // the next round's pending queue
  const uint32_t *qo = queue(p.qo, sssp_xq(iv));  // the near queue, or the whole pending queue
  const uint32_t *qs = queue(p.qs, sssp_xq(iv));
  const uint32_t *qv = queue(p.qv, sssp_xq(iv));
  const unsigned lm_le = lanemask_le();
  const uint32_t V = (uint32_t)p.V;
  const uint32_t E1 = c1;
  const bool pre = iv.precheck != 0u;

  Window w;
  load_entry<MODE>(p, qo, qs, qv, F, Etot, wb + lane, w);
  // the index names the entry holding the 128-edge unit boundary at or before c0, up to
  // 127 entries back: catch up until lane 0 holds the entry containing c0
  while (slide<MODE>(p, qo, qs, qv, F, Etot, c0, w, wb, lane)) {
  }
  // prologue: the first kStages - 1 iterations' copies (an empty group past the end, so
  // that every iteration below commits exactly one group)
  uint32_t ci = c0;
#pragma unroll
  for (int k = 0; k < kStages - 1; ++k, ci += 32u * kUnroll) {
    if (ci < E1) issue_groups<MODE>(p, qo, qs, qv, F, Etot, ci, E1, w, wb, pf, k, lane, lm_le);
    else cp_async_commit();
  }
  int sb = 0, sn = kStages - 1;
  uint32_t jn = kNoChunk;
  for (uint32_t c = c0; c < E1; c += 32u * kUnroll, ci += 32u * kUnroll) {
    if (more && lane == 0 && c + 32u * kUnroll >= E1 &&
        !(p.coop && p.kill_mode == KILL_CHUNK && doomed(ld_relaxed64(&p.ctl->kill_target), iv.epoch, id, iv.M)))
      jn = GW + atomicAdd(&p.ctl->cursor.v, 1u);
    if (ci < E1) issue_groups<MODE>(p, qo, qs, qv, F, Etot, ci, E1, w, wb, pf, sn, lane, lm_le);
    else cp_async_commit();
    cp_async_wait<kStages - 1>();  // this iteration's slot has landed; later ones stay in flight
    bool val[kUnroll];
    uint32_t vv[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      val[u] = c + 32u * (uint32_t)u + lane < E1;
      vv[u] = val[u] ? pf.col[sb][u][lane] : 0xFFFFFFFFu;
    }

    {
      // Relaxation on the packed word ds[v] = (dist << 32) | stamp.  One 64-bit atomicMin
      // with (nd << 32) | tag lowers the distance exactly when nd < dist (stamps only grow,
      // so an equal distance never rewrites the word), and the old word it returns says
      // whether this relaxation lowered it (nd < old dist) and whether the vertex was
      // already queued for the next round (old stamp == tag): the first lowering of a
      // round enqueues, later ones find the vertex queued and its expansion reads the
      // distance then current.  The phases run across the kUnroll groups -- all
      // pre-check loads, then all atomics, then all row reads -- so their chains overlap.
      bool push[kUnroll];
      uint32_t rs[kUnroll], deg[kUnroll];
      uint32_t wt[kUnroll], du[kUnroll], dv[kUnroll];
      unsigned long long old[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        wt[u] = val[u] ? pf.w[sb][u][lane] : 0u;
        du[u] = val[u] ? pf.du[sb][u][lane] : 0u;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        if (val[u] && vv[u] >= V) {
          bad = true;
          val[u] = false;
        }
        dv[u] = !val[u] ? 0u : pre ? (uint32_t)(p.ds[vv[u]] >> 32) : 0xFFFFFFFFu;
      }
      const uint32_t tag = sssp_tag(iv);  // stamp of "queued for the next round"
      bool imp[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        imp[u] = false;
        old[u] = 0ull;
        if (val[u]) {
          const uint64_t nd64 = (uint64_t)du[u] + (uint64_t)wt[u];
          if (nd64 >= 0xFFFFFFFFull) ovf = true;
          else if ((uint32_t)nd64 < dv[u]) {
            old[u] = atomicMin(p.ds + vv[u], (nd64 << 32) | (unsigned long long)tag);
            imp[u] = (uint32_t)nd64 < (uint32_t)(old[u] >> 32);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        rs[u] = 0u;
        deg[u] = 0u;
        push[u] = imp[u] && (uint32_t)old[u] != tag;
        const bool first = imp[u] && (uint32_t)(old[u] >> 32) == 0xFFFFFFFFu;  // first time reached
        if (push[u] || first) {
          if (!row_of(p, vv[u], rs[u], deg[u])) bad = true;
        }
        if (first) {
          nreach += 1u;
          ereach += deg[u];
        }
        push[u] = push[u] && deg[u] > 0u;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) stage_push<MODE>(p, out, stage, staged, push[u], vv[u], rs[u], deg[u], lane);
    }
    sb = sb + 1 == kStages ? 0 : sb + 1;
    sn = sn + 1 == kStages ? 0 : sn + 1;
  }
  return __shfl_sync(kFull, jn, 0);
}

__device__ __forceinline__ void sched_init(ChunkSched &s, uint32_t E, uint32_t GW, uint32_t cap) {
  const bool small = E <= GW * 32u;
  const uint32_t shift = small ? 5u : kIndexShift;
  const uint32_t U = (E + (1u << shift) - 1u) >> shift;
  __syncwarp();
  if ((threadIdx.x & 31u) == 0u) {
    s.U = U;
    s.shift = shift;
    s.k0 = 0u;
    s.base = 0u;
    s.s = small ? 1u : round_units(U, GW, cap);
    s.cap = cap;
  }
  __syncwarp();
}

// The edge range [c0, c1) of chunk k (warp-uniform); false past the end of the schedule.
// The chunk ids one warp is given only grow, so the round is advanced in place.
__device__ __forceinline__ bool sched_chunk(ChunkSched &sc, uint32_t k, uint32_t E, uint32_t GW, uint32_t &c0,
                                            uint32_t &c1) {
  const uint32_t U = sc.U, shift = sc.shift;
  uint32_t k0 = sc.k0, base = sc.base, s = sc.s;
  bool ok = true;
  if (k - k0 >= GW) {
    while (k - k0 >= GW) {
      base += GW * s;
      if (base >= U) {
        ok = false;
        break;
      }
      k0 += GW;
      s = round_units(U - base, GW, sc.cap);
    }
    __syncwarp();
    if ((threadIdx.x & 31u) == 0u) {
      sc.k0 = k0;
      sc.base = base;
      sc.s = s;
    }
    __syncwarp();
  }
  const uint32_t u0 = base + (k - k0) * s;
  if (!ok || u0 >= U) return false;
  c0 = u0 << shift;
  c1 = min((u0 + s) << shift, E);
  return true;
}

// Expand this warp's part of the interval, chunk by chunk (ChunkSched).  The enqueue
// built a chunk index (the entry holding every kIndexEdges-th edge), so a chunk starts
// without any search.  BFS expands queue iv.sel into the other one; SSSP queue xq (the
// near queue, or a small pending queue whole) into the next pending queue.
template <int MODE, int NW>
__device__ void expand(const Params &p, const Interval &iv, int32_t id, WarpStage &stage, Landing<MODE> &pf,
                       const volatile uint32_t *doom) {
  const unsigned lane = threadIdx.x & 31u;
  const uint32_t Etot = iv.edges;
  const uint32_t GW = (uint32_t)iv.M * NW;
  ChunkSched &sc = pf.sched;
  sched_init(sc, Etot, GW, MODE == MODE_SSSP ? kChunkUnitsMaxSssp : kChunkUnitsMax);
  uint32_t c0 = 0u, c1 = 0u;
  const uint32_t *qx = MODE == MODE_SSSP ? queue(p.qx, sssp_xq(iv)) : iv.sel ? p.qx[1] : p.qx[0];
  const uint32_t out = iv.sel ^ 1u;
  uint32_t staged = 0u, nreach = 0u;
  uint32_t ch = 0u, ct = 0u;  // BFS claim ring: head and tail (warp-uniform)
  uint64_t ereach = 0ull;
  bool bad = false, ovf = false;
  const uint32_t gw = (uint32_t)id * NW + (threadIdx.x >> 5);
  // BFS continuation interval: the returned ranges [lo, lo + n) of the level, range j for
  // warp j mod GW; otherwise the chunks of the schedule (a CTA that joined the interval
  // after it opened, id >= M, takes its chunks from the cursor only)
  const uint32_t cont = MODE == MODE_BFS ? iv.cont : 0u;
  const uint32_t lo = cont >> 16, n = cont & 0xFFFFu;
  uint32_t j = gw;
  auto next_range = [&]() -> bool {
    while (j < n) {
      const unsigned long long r = __ldcg(p.ctl->ret + lo + j);
      j += GW;
      c0 = (uint32_t)(r >> 32);
      c1 = (uint32_t)r;
      if (c0 < c1 && c1 <= Etot && (c0 & (kIndexEdges - 1u)) == 0u) return true;
      bad = true;
    }
    return false;
  };
  const bool more = !cont && sc.U > GW * sc.s;  // chunks beyond round 0 are claimed from the cursor
  bool have;
  if (cont) {
    have = next_range();
  } else if (id >= iv.M) {
    uint32_t k = kNoChunk;
    if (more && lane == 0) k = GW + atomicAdd(&p.ctl->cursor.v, 1u);
    k = __shfl_sync(kFull, k, 0);
    have = k != kNoChunk && sched_chunk(sc, k, Etot, GW, c0, c1);
  } else {
    have = sched_chunk(sc, gw, Etot, GW, c0, c1);
  }
  while (have) {
    uint32_t k;
    if constexpr (MODE == MODE_SSSP)
      k = expand_range<MODE>(p, iv, c0, c1, qx[c0 / kIndexEdges], stage, pf, staged, bad, ovf, nreach, ereach, more,
                             id, GW);
    else
      k = expand_range_bfs<MODE>(p, iv, c0, c1, qx[c0 / kIndexEdges], stage, pf, staged, bad, nreach, ereach, more,
                                 id, GW, ch, ct, doom);
    if (cont) have = next_range();
    else have = k != kNoChunk && sched_chunk(sc, k, Etot, GW, c0, c1);
  }
  if constexpr (MODE != MODE_SSSP) {
    if (ct != ch) claim_batch(p, out, stage, staged, pf.cand, ch, ct - ch, (uint32_t)iv.level + 1u, bad, nreach,
                              ereach, lane);
  }
  if (staged) stage_flush<MODE>(p, out, stage, staged, lane);
  // this warp's newly reached vertices and their out-edges (the TEPS numerator)
  for (int o = 16; o > 0; o >>= 1) {
    nreach += __shfl_xor_sync(kFull, nreach, o);
    ereach += __shfl_xor_sync(kFull, ereach, o);
  }
  if (lane == 0 && nreach) {
    atomicAdd(&p.ctl->reached, (unsigned long long)nreach);
    atomicAdd(&p.ctl->reached_edges, (unsigned long long)ereach);
  }
  if (bad) raise_err(p, ERR_GRAPH);
  if (ovf) p.ctl->ovf = 1u;
}

template <int MODE, int NW>
__global__ void __launch_bounds__((NW + 1) * 32, 1) coop_traverse(const __grid_constant__ Params p, int join);

}  // namespace

namespace coopdev {
// request_fork seen from the scheduler: n new CTAs of this very kernel, launched from
// the device into a fire-and-forget stream.  They register on arrival and are admitted
// at the next resizing barrier; the parent grid completes only after they have left.
template <int MODE, int NW>
__device__ void spawn_forks(const Params &p, uint32_t n) {
  coop_traverse<MODE, NW><<<n, (NW + 1) * 32, traverse_smem(MODE, NW), cudaStreamFireAndForget>>>(p, 1);
}
}  // namespace coopdev

namespace {

// The scheduler warp of the master CTA (the scheduler side of query(), kill and fork).
// It turns the host's outstanding CTA requests into the running interval's kill target
// (ids >= M - pending leave at their next offer_kill point), publishes how many CTAs
// have left, and launches the CTAs the host gives back.  Runs until the traversal is
// over or the master's own workers have left.
template <int MODE, int NW>
__device__ __forceinline__ void scheduler_warp(const Params &p, const volatile int32_t *workers_left) {
  Ctl *c = p.ctl;
  uint32_t forks_seen = p.fork_base, freed_seen = 0u, host_req_seen = 0u;
  for (;;) {
    // both host counters in one system-scope load: (fork_req << 32) | kill_req; and the
    // count of freed CTAs the host sees (issued together: two independent round trips)
    const uint64_t req = ld_sys64(&p.mbox->kill_req);
    const uint32_t host_freed = ld_sys(&p.mbox->freed);
    const uint32_t r = (uint32_t)req, f = (uint32_t)(req >> 32);
    if (p.kill_mode == KILL_SIMPLE) {
      // the regular barrier: arriving CTAs compare this with the kills already decided
      if (r - p.kill_base != host_req_seen) {
        host_req_seen = r - p.kill_base;
        st_relaxed(&c->host_req, host_req_seen);
      }
    } else if ((int32_t)(r - p.kill_base - ld_relaxed(&c->host_decided)) > 0) {
      // a consistent (epoch, interval, decided) snapshot: epoch read before and after
      const uint32_t e = ld_acquire(&c->epoch.v);
      const uint32_t decided = ld_relaxed(&c->host_decided);
      const Interval iv = read_iv(c);
      const int32_t pend = (int32_t)(r - p.kill_base - decided);
      if (pend > 0 && iv.epoch == e && !iv.done && ld_acquire(&c->epoch.v) == e) {
        const int32_t T = max(1, iv.M - pend);
        unsigned long long kt = ld_relaxed64(&c->kill_target);
        for (;;) {
          const uint32_t ke = (uint32_t)(kt >> 32);
          if ((int32_t)(ke - e) > 0) break;  // the word already belongs to a later interval
          const bool same = ke == e;
          if (same && ((kt & kTargetClosed) || (int32_t)(kt & 0x7FFFFFFFull) <= T)) break;
          const unsigned long long nv = ((unsigned long long)e << 32) | (unsigned long long)(uint32_t)T;
          const unsigned long long prev = atomicCAS(&c->kill_target, kt, nv);
          if (prev == kt) break;
          kt = prev;
        }
      }
    }
    // A CTA that leaves on a host request publishes the count itself (the host sees it at
    // once), but two such stores from different SMs can reach host memory in either
    // order, the lower count last; the host would then wait for the traversal's end.  So
    // the count is rewritten here whenever it changed or the host's copy differs from it
    // (until the traversal is over: the host then grants what is left itself).
    const uint32_t sur = ld_relaxed(&c->surrendered);
    if ((sur != freed_seen || host_freed != p.kill_base + sur) && ld_relaxed(&c->done) == 0u) {
      st_sys(&p.mbox->freed, p.kill_base + sur);
      freed_seen = sur;
    }
    if ((int32_t)(f - forks_seen) > 0) {
      const uint32_t n = f - forks_seen;
      forks_seen = f;
      atomicAdd(&c->launched_total, n);
      spawn_forks<MODE, NW>(p, n);
    }
    if (ld_relaxed(&c->done) != 0u || ld_relaxed(&c->err) != 0u || *workers_left != 0) return;
    __nanosleep(200);
  }
}

// The doom watcher of a BFS CTA other than the master (its otherwise idle 32nd warp, in
// KILL_CHUNK mode): polls the host's kill target and records in shared memory the epoch
// of the interval in which the target takes this CTA, so that the worker warps see it
// with a shared-memory read per iteration and hand their chunks back.  Runs until the
// CTA's workers have left or the traversal is over.
__device__ __forceinline__ void doom_watcher(const Params &p, CtaShared &cs) {
  const volatile Interval *iv = &cs.iv;
  const volatile int32_t *left = &cs.workers_left;
  const volatile int32_t *idp = &cs.id;
  volatile uint32_t *doom = &cs.doom;
  for (;;) {
    // the epoch first: a barrier writes the CTA's new id before the new interval
    const uint32_t e = iv->epoch;
    __threadfence_block();
    const int32_t M = iv->M, id = *idp;
    if (doomed(ld_relaxed64(&p.ctl->kill_target), e, id, M)) *doom = e;
    if (*left != 0 || ld_relaxed(&p.ctl->done) != 0u || ld_relaxed(&p.ctl->err) != 0u) return;
    __nanosleep(256);
  }
}

// p-sssp relax of edges [e0, e1) of one row whose source distance is du, by the 32 lanes
// of a warp, two edges per lane in flight.
__device__ __forceinline__ void relax_edges(const Params &p, uint32_t *cost, uint32_t du, uint32_t e0, uint32_t e1,
                                            unsigned lane, bool &bad, bool &ovf) {
  const uint32_t V = (uint32_t)p.V;
  for (uint32_t e00 = e0; e00 < e1; e00 += 64u) {
    uint32_t v[2], wt[2];
    bool ok[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const uint32_t e = e00 + 32u * (uint32_t)k + lane;
      ok[k] = e < e1;
      v[k] = ok[k] ? (uint32_t)__ldg(p.col + e) : 0u;
      wt[k] = ok[k] ? __ldg(p.w + e) : 0u;
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (!ok[k]) continue;
      if (v[k] >= V) {
        bad = true;
        continue;
      }
      const uint64_t nd = (uint64_t)du + (uint64_t)wt[k];
      if (nd >= 0xFFFFFFFFull) ovf = true;
      else if ((uint32_t)nd < cost[v[k]]) atomicMin(cost + v[k], (uint32_t)nd);
    }
  }
}

// Topology-driven SSSP, one interval of an iteration (Table 1, p-sssp: three resizing
// barriers per iteration).  cost[] lives in the packed-word scratch, the "changed" flags
// in the bitmap.  Work is partitioned by logical id as in Fig. 4, recomputed from the
// current M: warp id * NW + w of stride M * NW, 32 vertices at a time.
//   relax  (level % 3 == 0): every vertex lowered by the last update relaxes its
//          out-edges into cost[] (atomicMin); rows of at least kTopoHeavy edges come
//          from the update's chunk list, dealt out over every warp of the grid;
//   update (level % 3 == 1): dist = min(dist, cost); the flags of the next relax are the
//          vertices lowered now, and the heavy rows among them are listed as chunks; the
//          number lowered is counted;
//   check  (level % 3 == 2): no work -- the releaser ends the run when the update
//          lowered nothing.
template <int NW>
__device__ __forceinline__ void topo_interval(const Params &p, const Interval &iv, int32_t id) {
  const unsigned lane = threadIdx.x & 31u;
  const uint32_t V = (uint32_t)p.V;
  uint32_t *cost = reinterpret_cast<uint32_t *>(p.ds);
  const uint32_t phase = (uint32_t)iv.level % 3u;
  if (phase == 0u) {
    unsigned long long nrel = 0ull;
    bool bad = false, ovf = false;
    // heavy rows first: chunk j of the list (built by the update interval that flagged
    // the rows) goes to warp j mod G of the grid
    const uint32_t G = (uint32_t)iv.M * NW;
    const uint32_t nch = p.topo_heavy ? min(ld_relaxed(&p.ctl->cursor.v), V) : 0u;
    for (uint32_t j = (uint32_t)id * NW + (threadIdx.x >> 5); j < nch; j += G) {
      const uint32_t u = p.qv[0][j], e0 = p.qs[0][j];
      if (u >= V) {
        bad = true;
        continue;
      }
      const int32_t b = __ldg(p.row_off + u + 1);
      if (b < 0 || (uint32_t)b > p.E || e0 >= (uint32_t)b) {
        bad = true;
        continue;
      }
      const uint32_t e1 = min((uint32_t)b, e0 + kTopoChunk);  // b < 2^31: no wrap
      nrel += (unsigned long long)(e1 - e0);
      relax_edges(p, cost, p.dist[u], e0, e1, lane, bad, ovf);
    }
    // the other flagged rows, warp-cooperatively: warp id * NW + w takes 32 vertices at a
    // time; for each flagged one, the 32 lanes stride over its out-edges
    for (uint32_t base = ((uint32_t)id * NW + (threadIdx.x >> 5)) * 32u; base < V;
         base += (uint32_t)iv.M * NW * 32u) {
      unsigned m = p.visited[base >> 5];
      if (base + 32u > V) m &= (1u << (V - base)) - 1u;
      while (m) {
        const uint32_t u = base + (uint32_t)(__ffs(m) - 1);
        m &= m - 1u;
        const int32_t a = __ldg(p.row_off + u), b = __ldg(p.row_off + u + 1);
        if (a < 0 || b < a || (uint32_t)b > p.E) {
          bad = true;
          continue;
        }
        if (p.topo_heavy && (uint32_t)(b - a) >= kTopoHeavy) continue;  // listed: relaxed above
        nrel += (unsigned long long)(b - a);
        relax_edges(p, cost, p.dist[u], (uint32_t)a, (uint32_t)b, lane, bad, ovf);
      }
    }
    if (lane == 0 && nrel) atomicAdd(&p.ctl->qctr[1], nrel);
    if (__any_sync(kFull, bad) && lane == 0) raise_err(p, ERR_GRAPH);
    if (__any_sync(kFull, ovf) && lane == 0) p.ctl->ovf = 1u;
  } else if (phase == 1u) {
    uint32_t lowered = 0u, nreach = 0u;
    unsigned long long ereach = 0ull;
    for (uint32_t base = ((uint32_t)id * NW + (threadIdx.x >> 5)) * 32u; base < V;
         base += (uint32_t)iv.M * NW * 32u) {
      const uint32_t v = base + lane;
      bool low = false;
      if (v < V) {
        const uint32_t cv = cost[v], dv = p.dist[v];
        if (cv < dv) {
          p.dist[v] = cv;
          low = true;
          const int32_t a = __ldg(p.row_off + v), b = __ldg(p.row_off + v + 1);
          if (dv == 0xFFFFFFFFu) {  // first time reached
            nreach += 1u;
            ereach += (unsigned long long)(b - a);
          }
          // a heavy row flagged for the next relax is listed there as chunks
          if (p.topo_heavy && a >= 0 && b >= a && (uint32_t)b <= p.E && (uint32_t)(b - a) >= kTopoHeavy) {
            const uint32_t n = ((uint32_t)(b - a) + kTopoChunk - 1u) / kTopoChunk;
            const uint32_t at = atomicAdd(&p.ctl->cursor.v, n);
            if (at > V || n > V - at) {
              raise_err(p, ERR_GRAPH);  // only rows that overlap can outgrow the list
            } else {
              for (uint32_t k = 0; k < n; ++k) {
                p.qv[0][at + k] = v;
                p.qs[0][at + k] = (uint32_t)a + k * kTopoChunk;
              }
            }
          }
        }
      }
      const unsigned m = __ballot_sync(kFull, low);
      if (lane == 0) p.visited[base >> 5] = m;  // the whole word: flags of the next relax
      lowered += (uint32_t)__popc(m);
    }
    for (int o = 16; o > 0; o >>= 1) {
      nreach += __shfl_xor_sync(kFull, nreach, o);
      ereach += __shfl_xor_sync(kFull, ereach, o);
    }
    if (lane == 0) {
      if (lowered) atomicAdd(&p.ctl->qctr[0], (unsigned long long)lowered);
      if (nreach) {
        atomicAdd(&p.ctl->reached, (unsigned long long)nreach);
        atomicAdd(&p.ctl->reached_edges, ereach);
      }
    }
  }
}

template <int NW>
__device__ __forceinline__ void copy_dist(const Params &p, int32_t id, int32_t M) {
  const size_t V = (size_t)p.V;
  const size_t lo = V * (size_t)id / (size_t)M, hi = V * (size_t)(id + 1) / (size_t)M;
  for (size_t i = lo + threadIdx.x; i < hi; i += NW * 32) p.dist[i] = (uint32_t)(__ldcg(p.ds + i) >> 32);
}

template <int MODE, int NW>
__device__ __forceinline__ void worker_loop(const Params &p, CtaShared &cs, WarpStage *stages, Landing<MODE> *pfs) {
  WarpStage &stage = stages[threadIdx.x >> 5];
  Landing<MODE> &pf = pfs[threadIdx.x >> 5];
  for (bool first = true;; first = false) {
    const Interval iv = cs.iv;
    const int32_t id = cs.id;
    if (iv.done) {
      // SSSP's result: the active CTAs copy the distances out of the packed words, CTA
      // `id` of M taking the id-th stripe
      if (MODE == MODE_SSSP && id < iv.M) copy_dist<NW>(p, id, iv.M);
      return;
    }
    // left through offer_kill at the barrier (a CTA that has just joined the running
    // interval has an id >= M there)
    if (id >= iv.M && !first) return;
    if constexpr (MODE == MODE_PSSSP) {
      topo_interval<NW>(p, iv, id);
    } else if constexpr (MODE == MODE_SSSP) {
      // the landing buffers are idle in a select interval: their first kHistBuckets words
      // hold the CTA's histogram
      if (sssp_select(iv)) select_interval<NW>(p, iv, id, reinterpret_cast<uint32_t *>(pfs), cs);
      else expand<MODE, NW>(p, iv, id, stage, pf, &cs.doom);
    } else if constexpr (MODE != MODE_BARRIER) {
      expand<MODE, NW>(p, iv, id, stage, pf, &cs.doom);
    }
    if (!resizing_barrier<MODE, NW>(p, cs)) return;
  }
}

// One CTA's life in a cooperative traversal: enter (as the master, or by registering
// and waiting to be admitted), then either run the scheduler warp (master only) or the
// worker loop until the traversal ends or the CTA is killed.
template <int MODE, int NW>
__device__ __forceinline__ void traverse_body(const Params &p, bool master, CtaShared &cs, unsigned char *dyn) {
  if (threadIdx.x == 0) {
    bool active;
    if (master) {
      master_enter<MODE>(p, cs);
      active = true;
    } else if (p.coop) {
      active = join_enter<MODE, NW>(p, cs);
    } else {
      active = plain_enter(p, cs);
    }
    cs.exit = active ? 0 : 1;
    cs.workers_left = 0;
    cs.doom = 0u;
  }
  __syncthreads();
  if (cs.exit) return;
  if (threadIdx.x >= NW * 32) {
    if (p.coop && threadIdx.x == NW * 32) {
      if (cs.id == 0) scheduler_warp<MODE, NW>(p, &cs.workers_left);
      else if (MODE == MODE_BFS && p.kill_mode == KILL_CHUNK) doom_watcher(p, cs);
    }
    return;
  }
  // dynamic shared memory: NW enqueue stages, then NW landing buffers
  worker_loop<MODE, NW>(p, cs, reinterpret_cast<WarpStage *>(dyn),
                        reinterpret_cast<Landing<MODE> *>(dyn + NW * sizeof(WarpStage)));
  if (threadIdx.x == 0) *(volatile int32_t *)&cs.workers_left = 1;
}

template <int MODE, int NW>
__global__ void __launch_bounds__((NW + 1) * 32, 1) coop_traverse(const __grid_constant__ Params p, int join) {
  __shared__ CtaShared cs;
  extern __shared__ __align__(16) unsigned char dyn_smem[];  // per-warp enqueue staging (+ SM reservation)
  traverse_body<MODE, NW>(p, !join && blockIdx.x == 0, cs, dyn_smem);
}

// Many traversals in one persistent launch.  Job g owns blocks [first[g], first[g+1]) and
// is a cooperative kernel of its own (own control block, queues and barrier); its first
// block is its master.  A job whose blocks are not resident yet simply starts later:
// admission is join-on-arrival, so no barrier ever waits for a block that has not run.
template <int NW>
__global__ void __launch_bounds__((NW + 1) * 32, 1)
    coop_traverse_batch(const Params *__restrict__ jobs, const uint32_t *__restrict__ first, int njobs) {
  __shared__ Params P;
  __shared__ int32_t s_master;
  __shared__ CtaShared cs;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  if (threadIdx.x == 0) {
    int lo = 0, hi = njobs - 1;  // the last job whose first block is <= blockIdx.x
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (first[mid] <= blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    s_master = first[lo] == blockIdx.x ? 1 : 0;
    P = jobs[lo];
  }
  __syncthreads();
  if (P.mode == MODE_SSSP) traverse_body<MODE_SSSP, NW>(P, s_master != 0, cs, dyn_smem);
  else traverse_body<MODE_BFS, NW>(P, s_master != 0, cs, dyn_smem);
}

// Per-run initialisation: outputs, scratch and the control block (up to its resize log,
// which is only ever read up to its record count).
template <int MODE>
__device__ __forceinline__ void init_body(const Params &p, size_t tid, size_t nth) {
  const size_t V = (size_t)(p.V > 0 ? p.V : 0);
  if (MODE == MODE_BFS) {
    for (size_t i = tid; i < V; i += nth) p.level[i] = -1;
    for (size_t i = tid; i < (V + 31) / 32; i += nth) p.visited[i] = 0u;
  } else if (MODE == MODE_SSSP) {
    for (size_t i = tid; i < V; i += nth) p.ds[i] = 0xFFFFFFFF00000000ull;  // unreached, never queued
  } else if (MODE == MODE_PSSSP) {
    uint32_t *cost = reinterpret_cast<uint32_t *>(p.ds);
    for (size_t i = tid; i < V; i += nth) {
      p.dist[i] = 0xFFFFFFFFu;
      cost[i] = 0xFFFFFFFFu;
    }
    for (size_t i = tid; i < (V + 31) / 32; i += nth) p.visited[i] = 0u;
  }
  // zero the control block except its header line, which thread 0 writes
  uint32_t *cw = reinterpret_cast<uint32_t *>(p.ctl);
  const size_t hdr = offsetof(Ctl, run) / 4, hdr_end = hdr + 32;
  for (size_t i = tid; i < offsetof(Ctl, log) / 4; i += nth)
    if (i < hdr || i >= hdr_end) cw[i] = 0u;
  if (tid == 0) {
    p.ctl->run = p.run;
    p.ctl->err = 0u;
    p.ctl->done = 0u;
    p.ctl->ovf = 0u;
  }
}

template <int MODE>
__global__ void __launch_bounds__(512) coop_init_kernel(const __grid_constant__ Params p) {
  init_body<MODE>(p, (size_t)blockIdx.x * blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
}

// Batch initialisation: blockIdx.y selects the job; its device-resident mailbox is
// cleared too (batched jobs have no host scheduler).
__global__ void __launch_bounds__(512) coop_init_batch_kernel(const Params *__restrict__ jobs) {
  const Params &p = jobs[blockIdx.y];
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (size_t)gridDim.x * blockDim.x;
  if (p.mode == MODE_SSSP) init_body<MODE_SSSP>(p, tid, nth);
  else init_body<MODE_BFS>(p, tid, nth);
  uint32_t *mw = reinterpret_cast<uint32_t *>(p.mbox);
  for (size_t i = tid; i < sizeof(Mailbox) / 4; i += nth) mw[i] = 0u;
}

// Device-side launch warm-up: the first launch from the device in a process sets up the
// device runtime's launch path, which must not happen inside the scheduler warp of a
// running traversal (it would hold up the host's next request).
__global__ void coop_warm_child() {}
__global__ void coop_warm_parent() { coop_warm_child<<<1, 32, 0, cudaStreamFireAndForget>>>(); }

// The co-running task: y = a*x + y, grid-stride, vectorised where aligned.
__global__ void __launch_bounds__(1024) coop_saxpy_kernel(int64_t n, float a, const float *__restrict__ x,
                                                        float *__restrict__ y) {
  extern __shared__ uint4 reserve[];  // SM-exclusivity reservation only
  (void)reserve;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15u) == 0u;
  int64_t done = 0;
  if (vec) {
    const int64_t n4 = n / 4;
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    float4 *y4 = reinterpret_cast<float4 *>(y);
    for (int64_t i = tid; i < n4; i += nth) {
      const float4 xv = __ldg(x4 + i);
      float4 yv = y4[i];
      yv.x = fmaf(a, xv.x, yv.x);
      yv.y = fmaf(a, xv.y, yv.y);
      yv.z = fmaf(a, xv.z, yv.z);
      yv.w = fmaf(a, xv.w, yv.w);
      y4[i] = yv;
    }
    done = n4 * 4;
  }
  for (int64_t i = done + tid; i < n; i += nth) y[i] = fmaf(a, x[i], y[i]);
}

}  // namespace

// ===================================================================== octree (work stealing)
// Octree partitioning, the work-stealing application of Table 1 (Sec. 2.2 Fig. 2 and
// Sec. 3.2 "Adapting Work Stealing").  A task is a cell: a range of points and the cell's
// path code (a 1 followed by 3 bits per level).  A CTA pops a task from its own queue
// (newest first, so the queue stays short) or steals one from another queue (oldest
// first); a cell holding more than leaf_cap points (and above max_depth) is partitioned
// into its octants by coordinate bit 20 - depth, into the other of two buffers, and its
// non-empty octants are pushed as new tasks; any other cell is a leaf.  Every queue is
// guarded by a mutex (compare-and-swap).  There are no barriers: offer_kill sits at the
// head of the main loop (a leaving CTA's queued tasks are stolen by the others) and the
// master's scheduler warp launches forked CTAs, which take a queue slot of their own.
namespace {

struct OctTask {
  uint32_t begin, count;
  unsigned long long code;  // leading 1 at bit 3 * depth, then the octants from the root
};
constexpr uint32_t kOctQueues = 256;      // queue slots; CTAs take them in arrival order
constexpr uint32_t kOctQueueCap = 1024;   // tasks per queue (depth-first pops: ~7 per level)

struct alignas(128) OctQueue {
  uint32_t lock;  // 0 free, 1 held
  uint32_t head;  // thieves take from here
  uint32_t tail;  // the owner pushes and pops here
  uint32_t pad[29];
};

struct OctCtl {  // zeroed by the init kernel
  Word outstanding;  // tasks pushed and not yet completed
  Word slots;        // queue slots handed out
  Word leaves;       // leaf records written
  Word done;
  Word err;
  Word killed;       // CTAs that left at offer_kill
  Word host_req;     // the host's requests of this run (scheduler warp)
  Word launched;     // CTAs launched (main grid + forks)
  alignas(128) unsigned long long tasks, steals, moved;
};

struct OctParams {
  const uint32_t *x, *y, *z;  // caller's coordinates
  uint32_t *bx[2], *by[2], *bz[2], *bi[2];  // ping-pong: coordinates and point index
  uint32_t *perm;             // out: point indices, each leaf's points in its range
  unsigned long long *leaf_code;
  uint32_t *leaf_begin, *leaf_count;
  int32_t *n_leaves;
  uint32_t max_leaves;
  OctQueue *queues;
  OctTask *tasks;
  OctCtl *ctl;
  Mailbox *mbox;
  uint32_t n, leaf_cap, max_depth;
  uint32_t launched, kill_base, fork_base, coop;
  uint64_t timeout_ns;
  uint32_t pre;  // 1: the top kPreDepth levels are partitioned grid-wide before the work stealing
  uint32_t *cell_count, *cell_begin, *cell_cursor, *cell_leaf;  // kPreCells each
  uint32_t run;  // the context's run id, published to the host when the build is over
};

// Grid-wide partition of the top levels: the first kPreDepth levels of a large tree would
// otherwise be partitioned by one CTA at a time (the root's n points by a single CTA).
constexpr uint32_t kPreDepth = 3;
constexpr uint32_t kPreCells = 1u << (3 * kPreDepth);  // 512 cells at depth 3
constexpr uint32_t kPreMinPoints = 65536;

__device__ __forceinline__ void oct_error(const OctParams &p, int code) {
  atomicCAS(&p.ctl->err.v, 0u, (uint32_t)code);
}

__device__ __forceinline__ bool oct_lock(const OctParams &p, uint32_t q) {
  uint32_t *l = &p.queues[q].lock;
  const uint64_t t0 = gtime();
  for (uint32_t spin = 0;; ++spin) {
    if (ld_relaxed(l) == 0u && atomicCAS(l, 0u, 1u) == 0u) {
      __threadfence();  // acquire: the queue's tasks and what they describe
      return true;
    }
    if ((spin & 63u) == 63u && (gtime() - t0 > p.timeout_ns || ld_relaxed(&p.ctl->err.v) != 0u)) {
      oct_error(p, ERR_TIMEOUT);
      return false;
    }
    __nanosleep(32);
  }
}

__device__ __forceinline__ void oct_unlock(const OctParams &p, uint32_t q) {
  __threadfence();
  st_release(&p.queues[q].lock, 0u);
}

// Take a task from queue q: its newest (own queue) or its oldest (a steal).
__device__ __forceinline__ bool oct_pop(const OctParams &p, uint32_t q, bool own, OctTask &t) {
  OctQueue &Q = p.queues[q];
  if (ld_relaxed(&Q.tail) == ld_relaxed(&Q.head)) return false;  // hint, without the lock
  if (!oct_lock(p, q)) return false;
  const uint32_t h = ld_relaxed(&Q.head), tl = ld_relaxed(&Q.tail);
  bool ok = false;
  if (tl != h) {
    const uint32_t at = own ? tl - 1u : h;
    t = p.tasks[(size_t)q * kOctQueueCap + at % kOctQueueCap];
    if (own) st_relaxed(&Q.tail, tl - 1u);
    else st_relaxed(&Q.head, h + 1u);
    ok = true;
  }
  oct_unlock(p, q);
  return ok;
}

__device__ __forceinline__ bool oct_push(const OctParams &p, uint32_t q, const OctTask *c, uint32_t n) {
  OctQueue &Q = p.queues[q];
  if (!oct_lock(p, q)) return false;
  const uint32_t h = ld_relaxed(&Q.head), tl = ld_relaxed(&Q.tail);
  const bool ok = tl - h + n <= kOctQueueCap;
  if (ok) {
    for (uint32_t i = 0; i < n; ++i) p.tasks[(size_t)q * kOctQueueCap + (tl + i) % kOctQueueCap] = c[i];
    st_relaxed(&Q.tail, tl + n);
  }
  oct_unlock(p, q);
  if (!ok) oct_error(p, ERR_OVERFLOW);
  return ok;
}

__device__ __forceinline__ uint32_t octant(uint32_t x, uint32_t y, uint32_t z, uint32_t b) {
  return ((x >> b) & 1u) | (((y >> b) & 1u) << 1) | (((z >> b) & 1u) << 2);
}

template <int NW>
__global__ void __launch_bounds__((NW + 1) * 32, 1) coop_octree_kernel(const __grid_constant__ OctParams p, int join);

// The scheduler side for the octree (master CTA only): mirrors the host's requests for
// the CTAs' offer_kill, reports CTAs that left, launches the CTAs the host gives back.
template <int NW>
__device__ void oct_scheduler(const OctParams &p, const volatile int32_t *workers_left) {
  OctCtl *c = p.ctl;
  uint32_t forks_seen = p.fork_base, freed_seen = 0u, req_seen = 0u;
  for (;;) {
    const uint64_t req = ld_sys64(&p.mbox->kill_req);
    const uint32_t r = (uint32_t)req - p.kill_base, f = (uint32_t)(req >> 32);
    if (r != req_seen) {
      req_seen = r;
      st_relaxed(&c->host_req.v, r);
    }
    const uint32_t k = ld_relaxed(&c->killed.v);
    if (k != freed_seen) {
      st_sys(&p.mbox->freed, p.kill_base + k);
      freed_seen = k;
    }
    if ((int32_t)(f - forks_seen) > 0) {
      const uint32_t n = f - forks_seen;
      forks_seen = f;
      atomicAdd(&c->launched.v, n);
      coop_octree_kernel<NW><<<n, (NW + 1) * 32, kTraverseSmemMin, cudaStreamFireAndForget>>>(p, 1);
    }
    if (ld_relaxed(&c->done.v) != 0u || ld_relaxed(&c->err.v) != 0u || *workers_left != 0) return;
    __nanosleep(200);
  }
}

// A cell's partition state in shared memory: octant counts, first places, scatter cursors,
// and which octants become leaves.
struct OctCell {
  uint32_t hist[8], off[8], cur[8], leafmask;
};
// Cells below this many points are processed several at a time, one per warp group of a
// CTA; larger ones by the whole CTA (they lie on the tree's critical path).
constexpr uint32_t kOctSmall = 2048;
__host__ __device__ constexpr int oct_groups(int nw) { return nw >= 24 ? 4 : nw >= 12 ? 2 : 1; }

// One cell's work by T threads (gt = 0 .. T-1: a warp group, or the CTA's workers), whose
// meeting point is sync(): a leaf's points copied to perm and its record written, or the
// partition into octants (histogram, offsets, scatter; ballots aggregate each warp's
// points per octant, shared-memory atomics per warp).  Children that will be leaves are
// emitted here, not queued: their points go straight to perm during the scatter and their
// records are written by thread 0, which also queues the other children on queue `slot`.
template <typename Sync>
__device__ __forceinline__ void oct_cell(const OctParams &p, const OctTask t, uint32_t gt, uint32_t T, OctCell &cs,
                                         uint32_t slot, Sync sync) {
  OctCtl *c = p.ctl;
  const unsigned lane = threadIdx.x & 31u;
  const uint32_t d = (uint32_t)(63 - __clzll((long long)t.code)) / 3u;
  const uint32_t src = d & 1u, dst = src ^ 1u;
  const bool leaf = t.count <= p.leaf_cap || d >= p.max_depth;
  if (leaf) {
    for (uint32_t i = gt; i < t.count; i += T) p.perm[t.begin + i] = __ldcg(p.bi[src] + t.begin + i);
    if (gt == 0) {
      const uint32_t li = atomicAdd(&c->leaves.v, 1u);
      if (li < p.max_leaves) {
        p.leaf_code[li] = t.code;
        p.leaf_begin[li] = t.begin;
        p.leaf_count[li] = t.count;
      } else {
        oct_error(p, ERR_OVERFLOW);
      }
    }
  } else {
    const uint32_t b = 20u - d;
    if (gt < 8) cs.hist[gt] = 0u;
    sync();
    bool bad = false;
    for (uint32_t i0 = 0; i0 < t.count; i0 += T) {
      const uint32_t i = i0 + gt;
      uint32_t o = 8u;
      if (i < t.count) {
        const uint32_t x = __ldcg(p.bx[src] + t.begin + i), y = __ldcg(p.by[src] + t.begin + i),
                       z = __ldcg(p.bz[src] + t.begin + i);
        if ((x | y | z) >> 21) bad = true;
        o = octant(x, y, z, b);
      }
#pragma unroll
      for (uint32_t k = 0; k < 8u; ++k) {
        const unsigned m = __ballot_sync(kFull, o == k);
        if (lane == 0 && m) atomicAdd(&cs.hist[k], (uint32_t)__popc(m));
      }
    }
    if (bad) oct_error(p, ERR_GRAPH);
    sync();
    if (gt == 0) {
      uint32_t acc = 0u, lm = 0u;
      for (int k = 0; k < 8; ++k) {
        cs.off[k] = acc;
        cs.cur[k] = acc;
        acc += cs.hist[k];
        if (cs.hist[k] && (cs.hist[k] <= p.leaf_cap || d + 1u >= p.max_depth)) lm |= 1u << k;
      }
      cs.leafmask = lm;
    }
    sync();
    const uint32_t leafmask = cs.leafmask;
    const unsigned lt = lanemask_lt();
    for (uint32_t i0 = 0; i0 < t.count; i0 += T) {
      const uint32_t i = i0 + gt;
      uint32_t o = 8u, x = 0u, y = 0u, z = 0u, id = 0u;
      if (i < t.count) {
        x = __ldcg(p.bx[src] + t.begin + i);
        y = __ldcg(p.by[src] + t.begin + i);
        z = __ldcg(p.bz[src] + t.begin + i);
        id = __ldcg(p.bi[src] + t.begin + i);
        o = octant(x, y, z, b) & 7u;
      }
      uint32_t pos = 0u;
#pragma unroll
      for (uint32_t k = 0; k < 8u; ++k) {
        const unsigned m = __ballot_sync(kFull, o == k && i < t.count);
        if (m) {
          const unsigned first = (unsigned)__ffs(m) - 1u;
          uint32_t base = 0u;
          if (lane == first) base = atomicAdd(&cs.cur[k], (uint32_t)__popc(m));
          base = __shfl_sync(kFull, base, first);
          if (o == k && i < t.count) pos = base + (uint32_t)__popc(m & lt);
        }
      }
      if (i < t.count) {
        const uint32_t at = t.begin + pos;
        if ((leafmask >> o) & 1u) {
          p.perm[at] = id;
        } else {
          p.bx[dst][at] = x;
          p.by[dst][at] = y;
          p.bz[dst][at] = z;
          p.bi[dst][at] = id;
        }
      }
    }
  }
  __threadfence();  // these threads' writes before the tasks that will read them
  sync();
  if (gt == 0) {
    OctTask ch[8];
    uint32_t nc = 0u;
    if (!leaf) {
      const uint32_t lm = cs.leafmask;
      const uint32_t nleaf = (uint32_t)__popc(lm);
      if (nleaf) {
        const uint32_t li = atomicAdd(&c->leaves.v, nleaf);
        uint32_t j = 0u;
        for (uint32_t k = 0; k < 8u; ++k) {
          if (!((lm >> k) & 1u)) continue;
          if (li + j < p.max_leaves) {
            p.leaf_code[li + j] = (t.code << 3) | k;
            p.leaf_begin[li + j] = t.begin + cs.off[k];
            p.leaf_count[li + j] = cs.hist[k];
          } else {
            oct_error(p, ERR_OVERFLOW);
          }
          ++j;
        }
      }
      for (uint32_t k = 0; k < 8u; ++k)
        if (cs.hist[k] && !((lm >> k) & 1u)) ch[nc++] = OctTask{t.begin + cs.off[k], cs.hist[k], (t.code << 3) | k};
      atomicAdd(&c->moved, (unsigned long long)t.count);
    }
    bool ok = true;
    if (nc) ok = oct_push(p, slot, ch, nc);
    atomicAdd(&c->tasks, 1ull);
    if (ok) {
      // this task is done and nc are new: the run ends when none is outstanding
      const uint32_t prev = atomicAdd(&c->outstanding.v, nc - 1u);
      if (prev + nc - 1u == 0u) st_release(&c->done.v, 1u);
    }
  }
}

template <int NW>
__global__ void __launch_bounds__((NW + 1) * 32, 1) coop_octree_kernel(const __grid_constant__ OctParams p, int join) {
  extern __shared__ __align__(16) unsigned char oct_reserve[];  // SM-exclusivity reservation only
  (void)oct_reserve;
  constexpr int G = oct_groups(NW);
  __shared__ OctTask s_task[G];
  __shared__ OctCell s_cell[G];
  __shared__ int32_t s_state, s_workers_left;
  __shared__ uint32_t s_slot, s_ntask;
  OctCtl *c = p.ctl;
  const bool master = !join && blockIdx.x == 0;
  const unsigned tid = threadIdx.x;
  constexpr uint32_t T = NW * 32;
  if (tid == 0) {
    s_slot = atomicAdd(&c->slots.v, 1u) % kOctQueues;
    s_workers_left = 0;
  }
  __syncthreads();
  if (tid >= T) {
    if (master && p.coop && tid == T) oct_scheduler<NW>(p, &s_workers_left);
    return;
  }
  // warp group g: warps [g * NW / G, (g + 1) * NW / G), named barrier 2 + g
  const uint32_t warp = tid >> 5;
  uint32_t g = 0;
  while (g + 1 < (uint32_t)G && warp >= (g + 1) * NW / G) ++g;
  const uint32_t w0 = g * NW / G, Tg = ((g + 1) * NW / G - w0) * 32u;
  const auto cta_sync = [] { workers_sync<NW>(); };
  const auto group_sync = [g, Tg] { asm volatile("bar.sync %0, %1;" ::"r"(2u + g), "r"(Tg) : "memory"); };
  uint64_t idle0 = 0;
  for (;;) {
    if (tid == 0) {
      int st = 0;
      // offer_kill at the head of the main loop; the master never leaves
      if (p.coop && !master) {
        uint32_t k = ld_relaxed(&c->killed.v);
        while (k < ld_relaxed(&c->host_req.v)) {
          const uint32_t prev = atomicCAS(&c->killed.v, k, k + 1u);
          if (prev == k) {
            st = 2;
            break;
          }
          k = prev;
        }
      }
      if (st == 0) {
        OctTask t;
        if (oct_pop(p, s_slot, true, t)) {
          st = 1;
        } else {
          // steal: every other queue in use, starting after this CTA's own
          const uint32_t nq = min(ld_relaxed(&c->slots.v), kOctQueues);
          for (uint32_t i = 1; i < nq && st == 0; ++i) {
            if (oct_pop(p, (s_slot + i) % nq, false, t)) {
              st = 1;
              atomicAdd(&c->steals, 1ull);
            }
          }
        }
        if (st == 1) {
          s_task[0] = t;
          uint32_t n = 1u;
          // a small cell: take more small ones from this CTA's own queue, one per group
          // (a large one popped meanwhile goes back, to be taken whole next time)
          while (G > 1 && t.count < kOctSmall && n < (uint32_t)G) {
            OctTask u;
            if (!oct_pop(p, s_slot, true, u)) break;
            if (u.count >= kOctSmall) {
              oct_push(p, s_slot, &u, 1u);
              break;
            }
            s_task[n++] = u;
          }
          s_ntask = n;
          idle0 = 0;
        } else if (ld_acquire(&c->outstanding.v) == 0u || ld_relaxed(&c->done.v) != 0u ||
                   ld_relaxed(&c->err.v) != 0u) {
          st = 3;
        } else {
          const uint64_t now = gtime();
          if (idle0 == 0) idle0 = now;
          if (now - idle0 > p.timeout_ns) {
            oct_error(p, ERR_TIMEOUT);
            st = 3;
          } else {
            // nothing to steal yet: back off (up to ~4 us) so idle CTAs leave the queue
            // headers to the working ones
            const uint64_t back = 200ull + (now - idle0) / 8ull;
            __nanosleep(back < 4000ull ? (unsigned)back : 4000u);
          }
        }
      }
      s_state = st;
    }
    workers_sync<NW>();
    const int st = s_state;
    if (st >= 2) {
      if (tid == 0 && st == 2) __threadfence();
      break;
    }
    if (st == 1) {
      const uint32_t nt = s_ntask;
      if (nt == 1u) oct_cell(p, s_task[0], tid, T, s_cell[0], s_slot, cta_sync);
      else if (g < nt) oct_cell(p, s_task[g], tid - w0 * 32u, Tg, s_cell[g], s_slot, group_sync);
    }
    workers_sync<NW>();  // s_state and s_task are rewritten only after every worker read them
  }
  if (tid == 0) *(volatile int32_t *)&s_workers_left = 1;
}

__global__ void __launch_bounds__(512) coop_octree_init(const __grid_constant__ OctParams p) {
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (size_t)gridDim.x * blockDim.x;
  if (p.pre) {
    for (size_t i = tid; i < kPreCells; i += nth) p.cell_count[i] = 0u;
  } else {
    for (size_t i = tid; i < p.n; i += nth) {
      p.bx[0][i] = p.x[i];
      p.by[0][i] = p.y[i];
      p.bz[0][i] = p.z[i];
      p.bi[0][i] = (uint32_t)i;
    }
  }
  if (tid == 0) {
    uint32_t *cw = reinterpret_cast<uint32_t *>(p.ctl);
    for (size_t i = 0; i < sizeof(OctCtl) / 4; ++i) cw[i] = 0u;
    for (uint32_t q = 0; q < kOctQueues; ++q) {
      p.queues[q].lock = 0u;
      p.queues[q].head = 0u;
      p.queues[q].tail = 0u;
    }
    if (!p.pre) {
      p.tasks[0] = OctTask{0u, p.n, 1ull};  // the root cell, in queue 0
      p.queues[0].tail = 1u;
      p.ctl->outstanding.v = 1u;
    }
    p.ctl->launched.v = p.launched;
    *p.n_leaves = 0;
  }
}

__device__ __forceinline__ uint32_t pre_cell(uint32_t x, uint32_t y, uint32_t z) {
  uint32_t c = 0u;
#pragma unroll
  for (uint32_t d = 0; d < kPreDepth; ++d) c = (c << 3) | octant(x, y, z, 20u - d);
  return c;
}

// Top levels, step 1: points per depth-3 cell (a shared-memory histogram per block).
__global__ void __launch_bounds__(512) coop_octree_pre_hist(const __grid_constant__ OctParams p) {
  __shared__ uint32_t h[kPreCells];
  for (uint32_t i = threadIdx.x; i < kPreCells; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  bool bad = false;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t x = p.x[i], y = p.y[i], z = p.z[i];
    if ((x | y | z) >> 21) bad = true;
    atomicAdd(&h[pre_cell(x, y, z)], 1u);
  }
  if (bad) oct_error(p, ERR_GRAPH);
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < kPreCells; i += blockDim.x)
    if (h[i]) atomicAdd(&p.cell_count[i], h[i]);
}

// Top levels, step 2 (one block): the cells' ranges in octant order (so every cell above
// depth 3 is contiguous), the leaves above depth 3 -- recorded here, their points go to
// perm in step 3 -- and one task per non-empty depth-3 cell below no leaf, spread over the
// queues.  The tree is the one a root task would have produced.
__global__ void __launch_bounds__(kPreCells) coop_octree_pre_plan(const __grid_constant__ OctParams p) {
  __shared__ uint32_t cnt[kPreCells], beg[kPreCells], n2[64], n1[8];
  __shared__ uint32_t s_tasks;
  const uint32_t t = threadIdx.x;
  cnt[t] = p.cell_count[t];
  if (t == 0) s_tasks = 0u;
  __syncthreads();
  if (t < 64) {
    uint32_t a = 0u;
    for (int k = 0; k < 8; ++k) a += cnt[t * 8 + k];
    n2[t] = a;
  }
  if (t == 0) {  // exclusive prefix over the 512 cells, in octant order
    uint32_t acc = 0u;
    for (uint32_t i = 0; i < kPreCells; ++i) {
      beg[i] = acc;
      acc += cnt[i];
    }
  }
  __syncthreads();
  if (t < 8) {
    uint32_t a = 0u;
    for (int k = 0; k < 8; ++k) a += n2[t * 8 + k];
    n1[t] = a;
  }
  __syncthreads();
  // which level, if any, ends this cell's branch above depth 3 (the root always splits:
  // this path runs only for n > leaf_cap and max_depth >= 3)
  const uint32_t d0 = t >> 6, d01 = t >> 3;
  uint32_t leaf_depth = 0u;  // 0: none, the depth-3 cell is a task
  if (n1[d0] <= p.leaf_cap || p.max_depth <= 1u) leaf_depth = 1u;
  else if (n2[d01] <= p.leaf_cap || p.max_depth <= 2u) leaf_depth = 2u;
  p.cell_leaf[t] = leaf_depth;
  p.cell_begin[t] = beg[t];
  p.cell_cursor[t] = beg[t];
  // one record per leaf, written by the leaf's first cell
  const bool first1 = (t & 63u) == 0u, first2 = (t & 7u) == 0u;
  if ((leaf_depth == 1u && first1 && n1[d0]) || (leaf_depth == 2u && first2 && n2[d01])) {
    const uint32_t li = atomicAdd(&p.ctl->leaves.v, 1u);
    const unsigned long long code = leaf_depth == 1u ? (8ull | d0) : (64ull | d01);
    if (li < p.max_leaves) {
      p.leaf_code[li] = code;
      p.leaf_begin[li] = beg[t];
      p.leaf_count[li] = leaf_depth == 1u ? n1[d0] : n2[d01];
    } else {
      oct_error(p, ERR_OVERFLOW);
    }
  }
  if (leaf_depth == 0u && cnt[t]) {
    // over the queues of the launched CTAs only: a CTA looks at the queue slots taken so
    // far, and the main grid's CTAs take the first min(launched, kOctQueues)
    const uint32_t k = atomicAdd(&s_tasks, 1u);
    const uint32_t nq = min(p.launched, kOctQueues);
    const uint32_t q = k % nq, at = k / nq;  // at <= 511 < kOctQueueCap
    p.tasks[(size_t)q * kOctQueueCap + at] = OctTask{beg[t], cnt[t], 512ull | t};
    atomicAdd(&p.queues[q].tail, 1u);
  }
  __syncthreads();
  if (t == 0) p.ctl->outstanding.v = s_tasks;
}

// Top levels, step 3: every point to its depth-3 cell (buffer 1, as the depth-3 tasks read
// it) or, below a leaf, straight to perm.  Each block reserves its points' places per cell
// with one atomic, then ranks them in shared memory.
__global__ void __launch_bounds__(512) coop_octree_pre_scatter(const __grid_constant__ OctParams p) {
  __shared__ uint32_t h[kPreCells], base[kPreCells];
  const size_t per = (p.n + gridDim.x - 1) / gridDim.x;
  const size_t lo = (size_t)blockIdx.x * per, hi = min((size_t)p.n, lo + per);
  for (uint32_t i = threadIdx.x; i < kPreCells; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) atomicAdd(&h[pre_cell(p.x[i], p.y[i], p.z[i])], 1u);
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < kPreCells; i += blockDim.x) {
    base[i] = h[i] ? atomicAdd(&p.cell_cursor[i], h[i]) : 0u;
    h[i] = 0u;
  }
  __syncthreads();
  for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const uint32_t x = p.x[i], y = p.y[i], z = p.z[i];
    const uint32_t c = pre_cell(x, y, z);
    const uint32_t at = base[c] + atomicAdd(&h[c], 1u);
    if (p.cell_leaf[c]) {
      p.perm[at] = (uint32_t)i;
    } else {
      p.bx[1][at] = x;
      p.by[1][at] = y;
      p.bz[1][at] = z;
      p.bi[1][at] = (uint32_t)i;
    }
  }
}

__global__ void coop_octree_finish(const __grid_constant__ OctParams p) {
  *p.n_leaves = (int32_t)min(p.ctl->leaves.v, p.max_leaves);
  // the build is over: a host request still waiting is granted from the remaining CTAs
  __threadfence_system();
  st_sys(&p.mbox->run_done, p.run);
  __threadfence_system();
}

const void *octree_fn(int nw) {
  switch (nw) {
    case 31: return (const void *)coop_octree_kernel<31>;
    case 23: return (const void *)coop_octree_kernel<23>;
    default: return (const void *)coop_octree_kernel<15>;
  }
}


}  // namespace

// ===================================================================== host side

constexpr int kReqFields = 8;  // doubles per coop_request_resources record

struct coop_ctx {
  int device = 0;
  int nw = kDefaultWorkerWarps;  // worker warps per traversal CTA
  int N = 0;
  int sm_count = 0;
  cudaEvent_t ev_done = nullptr;
  cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;  // kernel timing (optional)
  bool timing = false;
  uint32_t kill_mode = 0;  // KILL_CHUNK
  void *oct_scratch = nullptr;  // octree: buffers, queues, tasks, control block
  int64_t oct_cap = 0;
  Mailbox *mbox = nullptr;    // host view
  Mailbox *mbox_d = nullptr;  // device view of the same pinned page
  Ctl *ctl = nullptr;
  void *scratch = nullptr;
  int64_t cap_V = 0, cap_chunks = 0;
  uint32_t *visited = nullptr;
  unsigned long long *ds = nullptr;
  uint32_t *qx[3] = {nullptr, nullptr, nullptr};
  uint32_t *qv[3] = {nullptr, nullptr, nullptr}, *qs[3] = {nullptr, nullptr, nullptr};
  uint32_t *qo[3] = {nullptr, nullptr, nullptr};
  std::mutex mu;         // host bookkeeping (kill/fork counters, run state)
  std::mutex launch_mu;  // serialises traversal launches
  uint32_t run = 0;
  bool launched = false;
  bool launching = false;  // a traversal's parameters are fixed and its launch is under way
  Params cur{};
  int cur_mode = MODE_BFS;
  uint32_t kill_req = 0, served = 0, returned = 0, fork_req = 0;
  int64_t timeout_us = 2000000;
  uint64_t sched_seed = 0;
  double p_kill = 0.0, p_fork = 0.0;
  double gather_us_max = 0.0;
  // coop_request_resources records: {posted (us since coop_init), CTAs asked for, M when
  // posted, M when granted, gather us, CTAs granted, us waiting for the context lock, us
  // posting}; the latest kReqLog
  std::chrono::steady_clock::time_point t_init = std::chrono::steady_clock::now();
  std::deque<std::array<double, kReqFields>> req_log;
};

namespace {

thread_local char g_last_error[256] = "";
constexpr size_t kReqLog = 4096;  // coop_request_resources records kept per context

// Record a failing CUDA call (what + the runtime's error name and string) for
// coop_last_cuda_error(); returns true when `e` is an error.
bool cuda_failed(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return false;
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  (void)cudaGetLastError();
  return true;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int now = -1;
    if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
  }
};

inline uint32_t load_acquire(const uint32_t *p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }
inline void store_release(uint32_t *p, uint32_t v) { __atomic_store_n(p, v, __ATOMIC_RELEASE); }

// A traversal kernel's dynamic shared memory, and the carveout hint that leaves the rest
// of the SM's L1/shared storage to L1 (the driver takes the smallest carveout that holds
// the CTA's shared memory).
bool set_traverse_attrs(const void *k, int smem) {
  return !cuda_failed(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                      "set traversal smem") &&
         !cuda_failed(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                           (int)cudaSharedmemCarveoutMaxL1),
                      "set traversal carveout");
}

bool running(coop_ctx *c) {
  return c->launching || (c->launched && cudaEventQuery(c->ev_done) == cudaErrorNotReady);
}

// The latest traversal has made its final release (the device wrote its run id after
// the stats): its CTAs are leaving, so a request need not wait for its completion event.
bool finished_locked(coop_ctx *c) {
  return c->launched && !c->launching && load_acquire(&c->mbox->run_done) == c->cur.run;
}

// A traversal holds CTAs that a request must wait for.
bool busy_locked(coop_ctx *c) { return !finished_locked(c) && running(c); }

// The same from host memory alone (no CUDA call, which can wait behind another thread's
// driver calls): a launched run that has not published its end counts as running.  A
// run that ended without publishing it (an error) is found by the request wait's
// periodic busy_locked.
bool busy_nowait_locked(coop_ctx *c) { return !finished_locked(c) && (c->launching || c->launched); }

// Fold the CTAs the device has surrendered into the host's books (always), and once no
// traversal holds CTAs grant every still-outstanding request at once.
void finalize_locked(coop_ctx *c, bool nowait = false) {
  const uint32_t f = load_acquire(&c->mbox->freed);
  if ((int32_t)(f - c->served) > 0) c->served = f;
  if (nowait ? busy_nowait_locked(c) : busy_locked(c)) return;
  (void)cudaGetLastError();
  if ((int32_t)(c->kill_req - c->served) > 0) c->served = c->kill_req;  // idle grant
  store_release(&c->mbox->freed, c->served);
}

// The two halves of coop_request_resources.  post_kill raises the cumulative request by
// n (offer_kill asked of the running kernel) and returns the count the device's `freed`
// must reach and the id of the run asked (*run); with no traversal holding CTAs the
// request is granted at once (*granted).
coop_status post_kill(coop_ctx *c, int n, uint32_t *target, bool *granted, double *lock_us, uint32_t *run) {
  const auto t0 = std::chrono::steady_clock::now();
  std::lock_guard<std::mutex> lk(c->mu);
  *lock_us = std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
  finalize_locked(c, true);
  const int outstanding = (int)(c->kill_req - c->returned);
  if (outstanding + n > c->N - 1) return COOP_EINVAL;
  c->kill_req += (uint32_t)n;
  *target = c->kill_req;
  store_release(&c->mbox->kill_req, c->kill_req);
  *run = c->cur.run;
  *granted = !busy_nowait_locked(c);
  if (*granted) finalize_locked(c, true);
  return COOP_OK;
}

// Waits until the device has freed the CTAs of a posted request (or the traversal ended,
// which grants the rest: seen first as the run's id in the mailbox, then as its
// completion), or until `deadline`; *got = the request's CTAs freed so far.  While the
// traversal runs the loop reads host memory only: the completion event is queried (a
// CUDA call, which can wait behind another process's driver queries) only once the run
// has published its end, and otherwise once a millisecond, in case it never does.
coop_status wait_kill(coop_ctx *c, uint32_t target, int n, uint32_t run, bool bounded,
                      std::chrono::steady_clock::time_point deadline, int *got) {
  const auto t0 = std::chrono::steady_clock::now();
  auto fallback = t0 + std::chrono::milliseconds(1);
  for (uint32_t spin = 0;; ++spin) {
    const uint32_t f = load_acquire(&c->mbox->freed);
    *got = std::max(0, std::min(n, (int)(f - (target - (uint32_t)n))));
    if ((int32_t)(f - target) >= 0) break;
    const bool ended = load_acquire(&c->mbox->run_done) == run;
    if (ended || (spin & 63u) == 0u) {
      const auto now = std::chrono::steady_clock::now();
      if (ended || now >= fallback) {
        fallback = now + std::chrono::milliseconds(1);
        std::lock_guard<std::mutex> lk(c->mu);
        if (!busy_locked(c)) {
          finalize_locked(c);
          break;
        }
      }
    }
    if (bounded && std::chrono::steady_clock::now() > deadline) return COOP_ETIMEOUT;
    if (spin > 2048) std::this_thread::yield();
  }
  *got = n;
  const double us = std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
  std::lock_guard<std::mutex> lk(c->mu);
  c->gather_us_max = std::max(c->gather_us_max, us);
  return COOP_OK;
}

coop_status ensure_scratch(coop_ctx *c, int64_t V, int64_t E) {
  const int64_t chunks = E / kIndexEdges + 2;
  if (V <= c->cap_V && chunks <= c->cap_chunks) return COOP_OK;
  if (c->scratch) {
    if (c->launched) cudaEventSynchronize(c->ev_done);
    cudaFree(c->scratch);
    c->scratch = nullptr;
    c->cap_V = 0;
    c->cap_chunks = 0;
  }
  const int64_t cap = std::max<int64_t>(std::max(V, c->cap_V), 1024);
  const int64_t capx = std::max<int64_t>(chunks, 1024);
  const size_t words = (size_t)(cap + 31) / 32;
  const size_t qbytes = (size_t)cap * 4;
  const size_t xbytes = (size_t)capx * 4;
  const size_t total = words * 4 + qbytes * 11 + xbytes * 3 + 14 * 256;
  char *base = nullptr;
  if (cudaMalloc(&base, total) != cudaSuccess) {
    (void)cudaGetLastError();
    return COOP_ENOMEM;
  }
  size_t at = 0;
  auto take = [&](size_t b) {
    char *p = base + at;
    at += (b + 255) & ~(size_t)255;
    return reinterpret_cast<uint32_t *>(p);
  };
  c->visited = take(words * 4);
  for (int i = 0; i < 3; ++i) {
    c->qv[i] = take(qbytes);
    c->qs[i] = take(qbytes);
    c->qo[i] = take(qbytes);
    c->qx[i] = take(xbytes);
  }
  c->ds = reinterpret_cast<unsigned long long *>(take(qbytes * 2));
  c->scratch = base;
  c->cap_V = cap;
  c->cap_chunks = capx;
  return COOP_OK;
}

coop_status check_graph(const coop_csr *g, int32_t source) {
  if (!g || !g->row_off || g->num_vertices < 1) return COOP_EINVAL;
  if (g->num_edges < 0 || g->num_edges >= ((int64_t)1 << 31)) return COOP_EINVAL;
  if (g->num_edges > 0 && !g->col) return COOP_EINVAL;
  if (source < 0 || source >= g->num_vertices) return COOP_EINVAL;
  return COOP_OK;
}

// The traversal kernel instantiations: worker warps NW in {31, 23, 15} (+ 1 poller warp).
template <int MODE>
const void *traverse_fn(int nw) {
  switch (nw) {
    case 31: return (const void *)coop_traverse<MODE, 31>;
    case 23: return (const void *)coop_traverse<MODE, 23>;
    default: return (const void *)coop_traverse<MODE, 15>;
  }
}

template <int MODE>
void launch_traverse(int nw, int grid, const Params &p, int join, cudaStream_t s) {
  switch (nw) {
    case 31: coop_traverse<MODE, 31><<<grid, 32 * 32, traverse_smem(MODE, 31), s>>>(p, join); break;
    case 23: coop_traverse<MODE, 23><<<grid, 24 * 32, traverse_smem(MODE, 23), s>>>(p, join); break;
    default: coop_traverse<MODE, 15><<<grid, 16 * 32, traverse_smem(MODE, 15), s>>>(p, join); break;
  }
}

template <int MODE>
coop_status launch_run(coop_ctx *c, const coop_csr *g, const uint32_t *w, int32_t source, int32_t *level,
                       uint32_t *dist, cudaStream_t stream, coop_stats *stats, bool coop, int32_t n_barriers,
                       int32_t extra_wait) {
  DeviceGuard guard(c->device);
  // One traversal at a time.  The wait for the previous one happens without holding the
  // state lock, so the scheduler's calls from other threads never queue behind a GPU wait.
  std::lock_guard<std::mutex> launch_lk(c->launch_mu);
  if (c->launched) cudaEventSynchronize(c->ev_done);
  Params p{};
  int launched = 0;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    finalize_locked(c);
    const int64_t V = g ? g->num_vertices : 0;
    coop_status st = ensure_scratch(c, std::max<int64_t>(V, 1), g ? g->num_edges : 0);
    if (st != COOP_OK) return st;
    const int held = (int)(c->served - c->returned);
    launched = coop ? std::max(1, c->N - held) : c->N;
    if (g) {
      p.row_off = g->row_off;
      p.col = g->col;
      p.V = g->num_vertices;
      p.E = (uint32_t)g->num_edges;
      // p-sssp's heavy-row chunk list lives in queue 0 (at least V entries)
      const uint64_t E = (uint64_t)g->num_edges;
      p.topo_heavy = (MODE == MODE_PSSSP && E / kTopoChunk + E / kTopoHeavy + 1 <= (uint64_t)g->num_vertices) ? 1u : 0u;
    }
    p.w = w;
    p.level = level;
    p.dist = dist;
    p.visited = c->visited;
    p.ds = c->ds;
    for (int i = 0; i < 3; ++i) {
      p.qv[i] = c->qv[i];
      p.qs[i] = c->qs[i];
      p.qo[i] = c->qo[i];
      p.qx[i] = c->qx[i];
    }
    p.ctl = c->ctl;
    p.mbox = c->mbox_d;
    p.src = source;
    p.N = c->N;
    p.launched = (uint32_t)launched;
    p.kill_base = c->served;
    p.fork_base = c->fork_req;
    p.timeout_ns = (uint64_t)std::max<int64_t>(c->timeout_us, 1) * 1000ull;
    p.sched_seed = c->sched_seed;
    p.p_kill = (uint32_t)std::min(4294967295.0, std::max(0.0, c->p_kill) * 4294967296.0);
    p.p_fork = (uint32_t)std::min(4294967295.0, std::max(0.0, c->p_fork) * 4294967296.0);
    p.sched_on = (coop && (c->p_kill > 0.0 || c->p_fork > 0.0)) ? 1u : 0u;
    p.run = ++c->run;
    p.n_barriers = n_barriers;
    p.extra_wait = (uint32_t)std::max(0, extra_wait);
    p.coop = coop ? 1u : 0u;
    p.kill_mode = c->kill_mode;
    p.mode = MODE;

    c->mbox->err = 0;
    c->mbox->status = 0;
    store_release(&c->mbox->freed, c->served);
    store_release(&c->mbox->kill_req, c->kill_req);
    store_release(&c->mbox->fork_req, c->fork_req);
    // From here on a request or a release is the new traversal's (kill_base and fork_base
    // are fixed above); the launch calls run without the state lock, so that a request
    // never waits behind them.
    c->launching = true;
    c->cur = p;
    c->cur_mode = MODE;
    c->gather_us_max = 0.0;
  }
  coop_init_kernel<MODE><<<c->sm_count * 4, 512, 0, stream>>>(p);
  if (c->timing) cudaEventRecord(c->ev_t0, stream);
  launch_traverse<MODE>(c->nw, launched, p, 0, stream);
  if (c->timing) cudaEventRecord(c->ev_t1, stream);
  cudaEventRecord(c->ev_done, stream);
  const bool failed = cuda_failed(cudaGetLastError(), "traversal launch");
  {
    std::lock_guard<std::mutex> lk(c->mu);
    c->launching = false;
    c->launched = !failed;
  }
  if (failed) return COOP_ECUDA;
  if (stats) {
    if (cudaEventSynchronize(c->ev_done) != cudaSuccess) return COOP_ECUDA;
    return coop_get_stats(c, stats);
  }
  return COOP_OK;
}

}  // namespace

extern "C" {

const char *coop_last_cuda_error(void) { return g_last_error; }

const char *coop_status_string(coop_status s) {
  switch (s) {
    case COOP_OK: return "COOP_OK";
    case COOP_EINVAL: return "COOP_EINVAL";
    case COOP_ENOMEM: return "COOP_ENOMEM";
    case COOP_ECUDA: return "COOP_ECUDA";
    case COOP_ETIMEOUT: return "COOP_ETIMEOUT";
    case COOP_EBUSY: return "COOP_EBUSY";
    case COOP_EOVERFLOW: return "COOP_EOVERFLOW";
    case COOP_EGRAPH: return "COOP_EGRAPH";
  }
  return "COOP_UNKNOWN";
}

coop_status coop_init(int device, int max_ctas, int threads_per_cta, coop_ctx **out) {
  if (!out) return COOP_EINVAL;
  *out = nullptr;
  if (max_ctas < 0) return COOP_EINVAL;
  int nw = 0;
  if (threads_per_cta == 0) nw = kDefaultWorkerWarps;
  else if (threads_per_cta == 31 * 32 || threads_per_cta == 23 * 32 || threads_per_cta == 15 * 32)
    nw = threads_per_cta / 32;
  else
    return COOP_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    (void)cudaGetLastError();
    return COOP_EINVAL;
  }
  DeviceGuard guard(device);
  coop_ctx *c = new coop_ctx();
  c->device = device;
  auto fail = [&](coop_status s) {
    coop_destroy(c);
    (void)cudaGetLastError();
    return s;
  };
  if (cuda_failed(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device), "sm count"))
    return fail(COOP_ECUDA);
  c->nw = nw;
  const void *kernels[] = {traverse_fn<MODE_BFS>(nw), traverse_fn<MODE_SSSP>(nw), traverse_fn<MODE_BARRIER>(nw),
                           traverse_fn<MODE_PSSSP>(nw)};
  const int modes[] = {MODE_BFS, MODE_SSSP, MODE_BARRIER, MODE_PSSSP};
  int per_sm = 1 << 30;
  for (int i = 0; i < 4; ++i) {
    const int smem = traverse_smem(modes[i], nw);
    if (!set_traverse_attrs(kernels[i], smem)) return fail(COOP_ECUDA);
    int nb = 0;
    if (cuda_failed(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernels[i], (nw + 1) * 32, smem), "occupancy"))
      return fail(COOP_ECUDA);
    per_sm = std::min(per_sm, nb);
  }
  if (cuda_failed(cudaFuncSetAttribute((const void *)coop_saxpy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kCorunnerSmem),
                  "set co-runner smem"))
    return fail(COOP_ECUDA);
  if (!set_traverse_attrs(octree_fn(nw), kTraverseSmemMin)) return fail(COOP_ECUDA);
  if (per_sm < 1) {
    snprintf(g_last_error, sizeof(g_last_error), "traversal kernel cannot be resident (%d per SM)", per_sm);
    return fail(COOP_ECUDA);
  }
  // Load every kernel now.  With lazy module loading the first launch of a kernel
  // waits for kernels already running, so a co-runner launched for the first time
  // while a traversal runs would not start until the traversal ended.
  {
    const void *all[] = {traverse_fn<MODE_BFS>(nw), traverse_fn<MODE_SSSP>(nw), traverse_fn<MODE_BARRIER>(nw),
                         traverse_fn<MODE_PSSSP>(nw), (const void *)coop_init_kernel<MODE_PSSSP>, octree_fn(nw),
                         (const void *)coop_octree_init, (const void *)coop_octree_finish,
                         (const void *)coop_octree_pre_hist, (const void *)coop_octree_pre_plan,
                         (const void *)coop_octree_pre_scatter,
                         (const void *)coop_init_kernel<MODE_BFS>, (const void *)coop_init_kernel<MODE_SSSP>,
                         (const void *)coop_init_kernel<MODE_BARRIER>, (const void *)coop_saxpy_kernel};
    for (const void *k : all) {
      cudaFuncAttributes fa;
      if (cuda_failed(cudaFuncGetAttributes(&fa, k), "kernel attributes")) return fail(COOP_ECUDA);
    }
    coop_saxpy_kernel<<<1, 1024, kCorunnerSmem>>>(0, 0.f, nullptr, nullptr);  // n = 0: no work
    if (cuda_failed(cudaGetLastError(), "co-runner warm-up")) return fail(COOP_ECUDA);
    cudaStream_t ws = nullptr;
    if (cuda_failed(cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking), "warm-up stream")) return fail(COOP_ECUDA);
    coop_warm_parent<<<1, 1, 0, ws>>>();
    const bool warm_ok = !cuda_failed(cudaGetLastError(), "device launch warm-up") &&
                         !cuda_failed(cudaStreamSynchronize(ws), "device launch warm-up");
    cudaStreamDestroy(ws);
    if (!warm_ok) return fail(COOP_ECUDA);
  }
  const int cap = std::min(per_sm * c->sm_count, kMaxCtas);
  c->N = max_ctas == 0 ? cap : std::min(max_ctas, cap);
  if (cuda_failed(cudaEventCreateWithFlags(&c->ev_done, cudaEventDisableTiming), "event")) return fail(COOP_ECUDA);
  if (cuda_failed(cudaHostAlloc((void **)&c->mbox, sizeof(Mailbox), cudaHostAllocMapped | cudaHostAllocPortable),
                  "mailbox"))
    return fail(COOP_ENOMEM);
  memset(c->mbox, 0, sizeof(Mailbox));
  if (cuda_failed(cudaHostGetDevicePointer((void **)&c->mbox_d, c->mbox, 0), "mailbox device pointer"))
    return fail(COOP_ECUDA);
  if (cuda_failed(cudaMalloc((void **)&c->ctl, sizeof(Ctl)), "control block")) return fail(COOP_ENOMEM);
  if (cuda_failed(cudaMemset(c->ctl, 0, sizeof(Ctl)), "control block memset")) return fail(COOP_ECUDA);
  if (cuda_failed(cudaDeviceSynchronize(), "init sync")) return fail(COOP_ECUDA);
  *out = c;
  return COOP_OK;
}

coop_status coop_destroy(coop_ctx *c) {
  if (!c) return COOP_OK;
  DeviceGuard guard(c->device);
  if (c->ev_done && c->launched) cudaEventSynchronize(c->ev_done);
  if (c->scratch) cudaFree(c->scratch);
  if (c->oct_scratch) cudaFree(c->oct_scratch);
  if (c->ctl) cudaFree(c->ctl);
  if (c->mbox) cudaFreeHost(c->mbox);
  if (c->ev_done) cudaEventDestroy(c->ev_done);
  if (c->ev_t0) cudaEventDestroy(c->ev_t0);
  if (c->ev_t1) cudaEventDestroy(c->ev_t1);
  (void)cudaGetLastError();
  delete c;
  return COOP_OK;
}

coop_status coop_bfs(coop_ctx *c, const coop_csr *g, int32_t source, int32_t *d_levels, coop_stream stream,
                     coop_stats *stats) {
  if (!c || !d_levels) return COOP_EINVAL;
  const coop_status st = check_graph(g, source);
  if (st != COOP_OK) return st;
  return launch_run<MODE_BFS>(c, g, nullptr, source, d_levels, nullptr, (cudaStream_t)stream, stats, true, 0, 0);
}

coop_status coop_sssp(coop_ctx *c, const coop_csr *g, const uint32_t *d_weights, int32_t source, uint32_t *d_dist,
                      coop_stream stream, coop_stats *stats) {
  if (!c || !d_dist) return COOP_EINVAL;
  const coop_status st = check_graph(g, source);
  if (st != COOP_OK) return st;
  if (g->num_edges > 0 && !d_weights) return COOP_EINVAL;
  return launch_run<MODE_SSSP>(c, g, d_weights, source, nullptr, d_dist, (cudaStream_t)stream, stats, true, 0, 0);
}

coop_status coop_sssp_topo(coop_ctx *c, const coop_csr *g, const uint32_t *d_weights, int32_t source,
                           uint32_t *d_dist, coop_stream stream, coop_stats *stats) {
  if (!c || !d_dist) return COOP_EINVAL;
  const coop_status st = check_graph(g, source);
  if (st != COOP_OK) return st;
  if (g->num_edges > 0 && !d_weights) return COOP_EINVAL;
  return launch_run<MODE_PSSSP>(c, g, d_weights, source, nullptr, d_dist, (cudaStream_t)stream, stats, true, 0, 0);
}

coop_status coop_bfs_baseline(coop_ctx *c, const coop_csr *g, int32_t source, int32_t *d_levels,
                              coop_stream stream, coop_stats *stats) {
  if (!c || !d_levels) return COOP_EINVAL;
  const coop_status st = check_graph(g, source);
  if (st != COOP_OK) return st;
  return launch_run<MODE_BFS>(c, g, nullptr, source, d_levels, nullptr, (cudaStream_t)stream, stats, false, 0, 0);
}

coop_status coop_sssp_baseline(coop_ctx *c, const coop_csr *g, const uint32_t *d_weights, int32_t source,
                               uint32_t *d_dist, coop_stream stream, coop_stats *stats) {
  if (!c || !d_dist) return COOP_EINVAL;
  const coop_status st = check_graph(g, source);
  if (st != COOP_OK) return st;
  if (g->num_edges > 0 && !d_weights) return COOP_EINVAL;
  return launch_run<MODE_SSSP>(c, g, d_weights, source, nullptr, d_dist, (cudaStream_t)stream, stats, false, 0,
                               0);
}

coop_status coop_barrier_bench(coop_ctx *c, int32_t n_barriers, int32_t never_arrive, coop_stream stream,
                               coop_stats *stats) {
  if (!c || n_barriers < 0 || never_arrive < 0) return COOP_EINVAL;
  return launch_run<MODE_BARRIER>(c, nullptr, nullptr, 0, nullptr, nullptr, (cudaStream_t)stream, stats, true,
                                  n_barriers, never_arrive);
}

coop_status coop_request_resources(coop_ctx *c, int n, int timeout_us, int *n_freed) {
  if (n_freed) *n_freed = 0;
  if (!c || n < 1) return COOP_EINVAL;
  uint32_t target = 0;
  bool granted = false;
  const auto t0 = std::chrono::steady_clock::now();
  const int m_post = __atomic_load_n(&c->mbox->active, __ATOMIC_ACQUIRE);
  double lock_us = 0.0;
  uint32_t run = 0;
  const coop_status st = post_kill(c, n, &target, &granted, &lock_us, &run);
  if (st != COOP_OK) return st;
  const double post_us = std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
  int got = n;
  coop_status w = COOP_OK;
  if (!granted) {
    const auto deadline = t0 + std::chrono::microseconds(std::max(0, timeout_us));
    w = wait_kill(c, target, n, run, timeout_us > 0, deadline, &got);
  }
  if (n_freed) *n_freed = got;
  const auto t1 = std::chrono::steady_clock::now();
  const int m_grant = __atomic_load_n(&c->mbox->active, __ATOMIC_ACQUIRE);
  std::lock_guard<std::mutex> lk(c->mu);
  c->req_log.push_back({std::chrono::duration<double, std::micro>(t0 - c->t_init).count(), (double)n,
                        granted ? 0.0 : (double)m_post, granted ? 0.0 : (double)m_grant,
                        std::chrono::duration<double, std::micro>(t1 - t0).count(), (double)got, lock_us, post_us});
  if (c->req_log.size() > kReqLog) c->req_log.pop_front();
  return w;
}

coop_status coop_get_request_log(coop_ctx *c, double *out, int cap, int *n, int clear) {
  if (!c || !n || cap < 0 || (cap > 0 && !out)) return COOP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  const int take = std::min<int>(cap, (int)c->req_log.size());
  const size_t first = c->req_log.size() - (size_t)take;  // the latest `take` records
  for (int i = 0; i < take; ++i)
    for (int j = 0; j < kReqFields; ++j) out[kReqFields * (size_t)i + j] = c->req_log[first + (size_t)i][j];
  *n = take;
  if (clear) c->req_log.clear();
  return COOP_OK;
}

coop_status coop_release(coop_ctx *c, int n) {
  if (!c || n < 1) return COOP_EINVAL;
  DeviceGuard guard(c->device);
  std::lock_guard<std::mutex> lk(c->mu);
  finalize_locked(c);
  const int held = (int)(c->served - c->returned);
  if (n > held) return COOP_EINVAL;
  c->returned += (uint32_t)n;
  if (running(c)) {
    // the running kernel's scheduler warp launches the n CTAs; they join at a barrier
    c->fork_req += (uint32_t)n;
    store_release(&c->mbox->fork_req, c->fork_req);
  }
  return COOP_OK;
}

coop_status coop_sync(coop_ctx *c) {
  if (!c) return COOP_EINVAL;
  DeviceGuard guard(c->device);
  if (c->launched && cudaEventSynchronize(c->ev_done) != cudaSuccess) return COOP_ECUDA;
  std::lock_guard<std::mutex> lk(c->mu);
  finalize_locked(c);
  const int32_t e = __atomic_load_n(&c->mbox->err, __ATOMIC_ACQUIRE);
  if (e != 0) return (coop_status)e;
  return (coop_status)__atomic_load_n(&c->mbox->status, __ATOMIC_ACQUIRE);
}

coop_status coop_get_stats(coop_ctx *c, coop_stats *s) {
  if (!c || !s) return COOP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  if (running(c)) return COOP_EBUSY;
  finalize_locked(c);
  const Mailbox *m = c->mbox;
  memset(s, 0, sizeof(*s));
  s->levels = m->levels;
  s->barriers = m->barriers;
  s->kills = m->kills;
  s->forks = m->forks;
  s->min_active = m->min_active;
  s->max_active = m->max_active;
  s->initial_active = m->initial_active;
  s->ctas_launched = m->ctas_launched;
  s->joined = m->joined;
  s->edges_scanned = (int64_t)m->edges_scanned;
  s->frontier_total = (int64_t)m->frontier_total;
  s->vertices_reached = (int64_t)m->reached;
  s->reached_edges = (int64_t)m->reached_edges;
  s->gather_us_max = c->gather_us_max;
  if (c->timing && c->launched) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev_t0, c->ev_t1) == cudaSuccess) s->kernel_us = 1000.0 * ms;
    (void)cudaGetLastError();
  }
  int32_t status = m->err != 0 ? m->err : m->status;
  if (c->launched && m->run_done != c->run && status == 0) status = COOP_ETIMEOUT;  // never finished cleanly
  s->status = status;
  return (coop_status)status;
}

coop_status coop_get_resize_log(coop_ctx *c, int32_t *out, int cap, int *n) {
  if (!c || !n || cap < 0 || (cap > 0 && !out)) return COOP_EINVAL;
  DeviceGuard guard(c->device);
  *n = 0;
  if (c->launched && cudaEventSynchronize(c->ev_done) != cudaSuccess) return COOP_ECUDA;
  uint32_t ln = 0;
  if (cudaMemcpy(&ln, &c->ctl->log_n, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return COOP_ECUDA;
  const int take = std::min<int>((int)std::min<uint32_t>(ln, (uint32_t)kLogCap), cap);
  if (take > 0) {
    LogRec *tmp = new LogRec[take];
    const cudaError_t e = cudaMemcpy(tmp, c->ctl->log, sizeof(LogRec) * (size_t)take, cudaMemcpyDeviceToHost);
    for (int i = 0; e == cudaSuccess && i < take; ++i) {
      int32_t *r = out + 8 * (size_t)i;
      r[0] = tmp[i].barrier;
      r[1] = tmp[i].t_us;
      r[2] = tmp[i].m_before;
      r[3] = tmp[i].k;
      r[4] = tmp[i].w;
      r[5] = tmp[i].m_after;
      r[6] = tmp[i].spawned;
      r[7] = tmp[i].edges;
    }
    delete[] tmp;
    if (cuda_failed(e, "resize log copy")) return COOP_ECUDA;
  }
  *n = take;
  return COOP_OK;
}

coop_status coop_set_schedule(coop_ctx *c, uint64_t seed, double p_kill, double p_fork) {
  if (!c || p_kill < 0.0 || p_kill > 1.0 || p_fork < 0.0 || p_fork > 1.0) return COOP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  c->sched_seed = seed;
  c->p_kill = p_kill;
  c->p_fork = p_fork;
  return COOP_OK;
}

coop_status coop_set_timeout(coop_ctx *c, int64_t timeout_us) {
  if (!c || timeout_us < 1) return COOP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  c->timeout_us = timeout_us;
  return COOP_OK;
}

coop_status coop_set_kill_mode(coop_ctx *c, int mode) {
  if (!c || mode < COOP_KILL_CHUNK || mode > COOP_KILL_SIMPLE) return COOP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  c->kill_mode = (uint32_t)mode;
  return COOP_OK;
}

coop_status coop_set_timing(coop_ctx *c, int on) {
  if (!c) return COOP_EINVAL;
  DeviceGuard guard(c->device);
  std::lock_guard<std::mutex> lk(c->mu);
  if (on && !c->ev_t0) {
    if (cudaEventCreate(&c->ev_t0) != cudaSuccess || cudaEventCreate(&c->ev_t1) != cudaSuccess) {
      (void)cudaGetLastError();
      return COOP_ECUDA;
    }
  }
  c->timing = on != 0;
  return COOP_OK;
}

coop_status coop_query(coop_ctx *c, int *max_ctas, int *threads_per_cta, int *sm_count, int *lent) {
  if (!c) return COOP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  finalize_locked(c);
  if (max_ctas) *max_ctas = c->N;
  if (threads_per_cta) *threads_per_cta = c->nw * 32;
  if (sm_count) *sm_count = c->sm_count;
  if (lent) *lent = (int)(c->served - c->returned);
  return COOP_OK;
}

coop_status coop_saxpy(int n_ctas, int64_t n, float a, const float *d_x, float *d_y, coop_stream stream) {
  if (n_ctas < 1 || n < 0 || (n > 0 && (!d_x || !d_y))) return COOP_EINVAL;
  if (n == 0) return COOP_OK;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute((const void *)coop_saxpy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kCorunnerSmem);
  });
  coop_saxpy_kernel<<<n_ctas, 1024, kCorunnerSmem, (cudaStream_t)stream>>>(n, a, d_x, d_y);
  return cuda_failed(cudaGetLastError(), "co-runner launch") ? COOP_ECUDA : COOP_OK;
}

}  // extern "C"

// ===================================================================== batched traversals
//
// A batch is a set of independent traversals (jobs) run by one persistent launch of
// coop_traverse_batch: each job is a cooperative kernel of its own over a contiguous
// range of blocks.  Jobs are laid out largest first, so that when the grid is larger than
// what fits on the GPU at once, small jobs fill SMs as big ones finish.  The blocks per
// job come from coop_batch_set_ctas, the autotuner (coop_batch_tune), or the default
// rule (proportional to the job's edges, one wave of blocks in total).

struct coop_batch {
  coop_ctx *ctx = nullptr;
  int n = 0;
  std::vector<coop_job> jobs;
  std::vector<Params> params;   // host copy, in launch order
  std::vector<int> order;       // launch position -> job index
  std::vector<int32_t> ctas;    // per job (job order)
  Params *d_params = nullptr;
  uint32_t *d_first = nullptr;
  void *scratch = nullptr;
  uint32_t total = 0;
  uint32_t run = 0;
  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false;
  cudaStream_t capture = nullptr;  // private stream the graph is recorded on
  cudaEvent_t ran = nullptr;       // recorded after every run: the job table is in use until then
  bool any_run = false;
  int64_t max_V = 0;
};

namespace {

int64_t job_edges(const coop_job &j) { return std::max<int64_t>(j.graph.num_edges, 1); }

// blocks per job proportional to edges^alpha, `total` blocks in all, at least 1 and at
// most `cap` each (largest-remainder rounding)
std::vector<int32_t> apportion(const std::vector<coop_job> &jobs, double alpha, int total, int cap) {
  const int n = (int)jobs.size();
  std::vector<double> w(n);
  double sw = 0.0;
  for (int i = 0; i < n; ++i) sw += (w[i] = std::pow((double)job_edges(jobs[i]), alpha));
  total = std::max(total, n);
  std::vector<int32_t> c(n, 1);
  int left = total - n;
  std::vector<std::pair<double, int>> rem;
  for (int i = 0; i < n; ++i) {
    const double ideal = (double)left * w[i] / sw;
    const int add = std::min(cap - 1, (int)ideal);
    c[i] += add;
    rem.push_back({ideal - add, i});
  }
  int used = 0;
  for (int v : c) used += v;
  std::sort(rem.begin(), rem.end(), [](auto &a, auto &b) { return a.first > b.first; });
  for (size_t k = 0; used < total && k < rem.size(); ++k)
    if (c[rem[k].second] < cap) {
      ++c[rem[k].second];
      ++used;
    }
  return c;
}

// (Re)build the device job table for the current block counts.
coop_status batch_layout(coop_batch *b) {
  const int n = b->n;
  b->order.resize(n);
  std::iota(b->order.begin(), b->order.end(), 0);
  std::stable_sort(b->order.begin(), b->order.end(),
                   [&](int x, int y) { return job_edges(b->jobs[x]) > job_edges(b->jobs[y]); });
  std::vector<uint32_t> first(n);
  std::vector<Params> ps(n);
  uint32_t at = 0;
  for (int k = 0; k < n; ++k) {
    const int j = b->order[k];
    first[k] = at;
    ps[k] = b->params[j];
    ps[k].launched = (uint32_t)b->ctas[j];
    ps[k].N = b->ctas[j];
    at += (uint32_t)b->ctas[j];
  }
  b->total = at;
  // a run still in flight (on any stream) reads the table: let it finish first
  if (b->any_run && cuda_failed(cudaEventSynchronize(b->ran), "batch run")) return COOP_ECUDA;
  if (cuda_failed(cudaMemcpy(b->d_params, ps.data(), sizeof(Params) * n, cudaMemcpyHostToDevice), "batch table") ||
      cuda_failed(cudaMemcpy(b->d_first, first.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice), "batch table"))
    return COOP_ECUDA;
  b->graph_valid = false;
  return COOP_OK;
}

void batch_enqueue(coop_batch *b, cudaStream_t s) {
  coop_ctx *c = b->ctx;
  const dim3 ig((unsigned)std::max<int64_t>(1, std::min<int64_t>((b->max_V + 511) / 512, 64)), (unsigned)b->n);
  coop_init_batch_kernel<<<ig, 512, 0, s>>>(b->d_params);
  switch (c->nw) {
    case 31:
      coop_traverse_batch<31><<<b->total, 32 * 32, traverse_smem(MODE_SSSP, 31), s>>>(b->d_params, b->d_first, b->n);
      break;
    case 23:
      coop_traverse_batch<23><<<b->total, 24 * 32, traverse_smem(MODE_SSSP, 23), s>>>(b->d_params, b->d_first, b->n);
      break;
    default:
      coop_traverse_batch<15><<<b->total, 16 * 32, traverse_smem(MODE_SSSP, 15), s>>>(b->d_params, b->d_first, b->n);
      break;
  }
}

const void *batch_fn(int nw) {
  switch (nw) {
    case 31: return (const void *)coop_traverse_batch<31>;
    case 23: return (const void *)coop_traverse_batch<23>;
    default: return (const void *)coop_traverse_batch<15>;
  }
}

}  // namespace

extern "C" {

coop_status coop_batch_create(coop_ctx *c, const coop_job *jobs, int n, coop_batch **out) {
  if (!out) return COOP_EINVAL;
  *out = nullptr;
  if (!c || !jobs || n < 1 || n > 65535) return COOP_EINVAL;
  for (int i = 0; i < n; ++i) {
    const coop_job &j = jobs[i];
    if (check_graph(&j.graph, j.source) != COOP_OK || !j.d_out) return COOP_EINVAL;
    if (j.kind != COOP_JOB_BFS && j.kind != COOP_JOB_SSSP) return COOP_EINVAL;
    if (j.kind == COOP_JOB_SSSP && j.graph.num_edges > 0 && !j.d_weights) return COOP_EINVAL;
  }
  DeviceGuard guard(c->device);
  coop_batch *b = new coop_batch();
  b->ctx = c;
  b->n = n;
  b->jobs.assign(jobs, jobs + n);
  // scratch per job: control block, mailbox, bitmap or stamps, 3 x 3 queues, 3 chunk indexes
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  std::vector<size_t> off(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    const size_t V = (size_t)jobs[i].graph.num_vertices, X = (size_t)(jobs[i].graph.num_edges / kIndexEdges + 2);
    const size_t need = al(sizeof(Ctl)) + al(sizeof(Mailbox)) +
                        (jobs[i].kind == COOP_JOB_SSSP ? al(V * 8) : al((V + 31) / 32 * 4)) + 9 * al(V * 4) +
                        3 * al(X * 4);
    off[i + 1] = off[i] + need;
    b->max_V = std::max<int64_t>(b->max_V, (int64_t)V);
  }
  auto fail = [&](coop_status st) {
    coop_batch_destroy(b);
    return st;
  };
  if (cuda_failed(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking), "capture stream") ||
      cuda_failed(cudaEventCreateWithFlags(&b->ran, cudaEventDisableTiming), "batch event"))
    return fail(COOP_ECUDA);
  if (cuda_failed(cudaMalloc(&b->scratch, std::max<size_t>(off[n], 256)), "batch scratch") ||
      cuda_failed(cudaMalloc((void **)&b->d_params, sizeof(Params) * n), "batch table") ||
      cuda_failed(cudaMalloc((void **)&b->d_first, sizeof(uint32_t) * n), "batch table"))
    return fail(COOP_ENOMEM);
  if (!set_traverse_attrs(batch_fn(c->nw), traverse_smem(MODE_SSSP, c->nw))) return fail(COOP_ECUDA);
  b->params.resize(n);
  for (int i = 0; i < n; ++i) {
    const coop_job &j = jobs[i];
    char *at = static_cast<char *>(b->scratch) + off[i];
    auto take = [&](size_t bytes) {
      char *q = at;
      at += al(bytes);
      return q;
    };
    const size_t V = (size_t)j.graph.num_vertices, X = (size_t)(j.graph.num_edges / kIndexEdges + 2);
    Params &p = b->params[i];
    p = Params{};
    p.ctl = reinterpret_cast<Ctl *>(take(sizeof(Ctl)));
    p.mbox = reinterpret_cast<Mailbox *>(take(sizeof(Mailbox)));
    if (j.kind == COOP_JOB_SSSP) p.ds = reinterpret_cast<unsigned long long *>(take(V * 8));
    else p.visited = reinterpret_cast<uint32_t *>(take((V + 31) / 32 * 4));
    for (int q = 0; q < 3; ++q) {
      p.qv[q] = reinterpret_cast<uint32_t *>(take(V * 4));
      p.qs[q] = reinterpret_cast<uint32_t *>(take(V * 4));
      p.qo[q] = reinterpret_cast<uint32_t *>(take(V * 4));
    }
    for (int q = 0; q < 3; ++q) p.qx[q] = reinterpret_cast<uint32_t *>(take(X * 4));
    p.row_off = j.graph.row_off;
    p.col = j.graph.col;
    p.V = j.graph.num_vertices;
    p.E = (uint32_t)j.graph.num_edges;
    p.src = j.source;
    p.mode = j.kind == COOP_JOB_SSSP ? MODE_SSSP : MODE_BFS;
    if (j.kind == COOP_JOB_SSSP) {
      p.w = j.d_weights;
      p.dist = static_cast<uint32_t *>(j.d_out);
    } else {
      p.level = static_cast<int32_t *>(j.d_out);
    }
    p.timeout_ns = (uint64_t)std::max<int64_t>(c->timeout_us, 1) * 1000ull;
    p.run = 1u;
    p.coop = 1u;
  }
  b->ctas = apportion(b->jobs, 1.0, c->N, c->N);
  const coop_status st = batch_layout(b);
  if (st != COOP_OK) return fail(st);
  *out = b;
  return COOP_OK;
}

coop_status coop_batch_set_ctas(coop_batch *b, const int32_t *ctas) {
  if (!b || !ctas) return COOP_EINVAL;
  for (int i = 0; i < b->n; ++i)
    if (ctas[i] < 1 || ctas[i] > kMaxCtas) return COOP_EINVAL;
  DeviceGuard guard(b->ctx->device);
  b->ctas.assign(ctas, ctas + b->n);
  return batch_layout(b);
}

coop_status coop_batch_run(coop_batch *b, coop_stream stream, int use_graph) {
  if (!b) return COOP_EINVAL;
  DeviceGuard guard(b->ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (!use_graph) {
    batch_enqueue(b, s);
    cudaEventRecord(b->ran, s);
    b->any_run = true;
    return cuda_failed(cudaGetLastError(), "batch launch") ? COOP_ECUDA : COOP_OK;
  }
  if (!b->graph_valid) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    // recorded on a private stream (the caller's may be the legacy default stream, which
    // cannot be captured), then launched on the caller's stream
    cudaGraph_t g = nullptr;
    if (cuda_failed(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal), "begin capture"))
      return COOP_ECUDA;
    batch_enqueue(b, b->capture);
    const cudaError_t e = cudaStreamEndCapture(b->capture, &g);
    if (cuda_failed(e, "end capture")) return COOP_ECUDA;
    const cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (cuda_failed(ie, "graph instantiate")) return COOP_ECUDA;
    b->graph_valid = true;
  }
  if (cuda_failed(cudaGraphLaunch(b->graph, s), "graph launch")) return COOP_ECUDA;
  cudaEventRecord(b->ran, s);
  b->any_run = true;
  return cuda_failed(cudaGetLastError(), "batch event") ? COOP_ECUDA : COOP_OK;
}

coop_status coop_batch_tune(coop_batch *b, coop_stream stream, int32_t *ctas_out) {
  if (!b) return COOP_EINVAL;
  coop_ctx *c = b->ctx;
  DeviceGuard guard(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cuda_failed(cudaEventCreate(&e0), "event") || cuda_failed(cudaEventCreate(&e1), "event")) return COOP_ECUDA;
  // candidate rules: blocks proportional to edges^alpha, `waves` x N blocks in total
  const double alphas[] = {0.5, 0.75, 1.0};
  const int waves[] = {1, 2, 4};
  float best = 1e30f;
  std::vector<int32_t> best_ctas = b->ctas;
  coop_status st = COOP_OK;
  for (double a : alphas)
    for (int wv : waves) {
      b->ctas = apportion(b->jobs, a, wv * c->N, c->N);
      if ((st = batch_layout(b)) != COOP_OK) break;
      float ms = 0.f, tot = 0.f;
      for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, s);
        batch_enqueue(b, s);
        cudaEventRecord(e1, s);
        cudaEventRecord(b->ran, s);
        b->any_run = true;
        if (cuda_failed(cudaEventSynchronize(e1), "tune run")) {
          st = COOP_ECUDA;
          break;
        }
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tot += ms;  // first run warms up
      }
      if (st != COOP_OK) break;
      if (tot < best) {
        best = tot;
        best_ctas = b->ctas;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != COOP_OK) return st;
  b->ctas = best_ctas;
  st = batch_layout(b);
  if (ctas_out) std::copy(b->ctas.begin(), b->ctas.end(), ctas_out);
  return st;
}

coop_status coop_batch_get_stats(coop_batch *b, coop_stats *per_job) {
  if (!b || !per_job) return COOP_EINVAL;
  DeviceGuard guard(b->ctx->device);
  if (cuda_failed(cudaDeviceSynchronize(), "batch sync")) return COOP_ECUDA;
  coop_status worst = COOP_OK;
  for (int i = 0; i < b->n; ++i) {
    Mailbox m;
    if (cuda_failed(cudaMemcpy(&m, b->params[i].mbox, sizeof(Mailbox), cudaMemcpyDeviceToHost), "batch stats"))
      return COOP_ECUDA;
    coop_stats &st = per_job[i];
    memset(&st, 0, sizeof(st));
    st.levels = m.levels;
    st.barriers = m.barriers;
    st.kills = m.kills;
    st.forks = m.forks;
    st.min_active = m.min_active;
    st.max_active = m.max_active;
    st.initial_active = m.initial_active;
    st.ctas_launched = m.ctas_launched;
    st.joined = m.joined;
    st.edges_scanned = (int64_t)m.edges_scanned;
    st.frontier_total = (int64_t)m.frontier_total;
    st.vertices_reached = (int64_t)m.reached;
    st.reached_edges = (int64_t)m.reached_edges;
    st.status = m.err != 0 ? m.err : (m.run_done == b->params[i].run ? m.status : (int32_t)COOP_ETIMEOUT);
    if (st.status != COOP_OK && worst == COOP_OK) worst = (coop_status)st.status;
  }
  return worst;
}

coop_status coop_batch_destroy(coop_batch *b) {
  if (!b) return COOP_OK;
  DeviceGuard guard(b->ctx->device);
  cudaDeviceSynchronize();
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->capture) cudaStreamDestroy(b->capture);
  if (b->ran) cudaEventDestroy(b->ran);
  if (b->scratch) cudaFree(b->scratch);
  if (b->d_params) cudaFree(b->d_params);
  if (b->d_first) cudaFree(b->d_first);
  (void)cudaGetLastError();
  delete b;
  return COOP_OK;
}

}  // extern "C"

// ===================================================================== serving loop
//
// A request loop with continuous batching.  Queries (BFS or SSSP from a source on one of
// the registered, device-resident graphs) are admitted in arrival order whenever a slot is
// free and the HBM budget allows; each admitted query runs as its own cooperative
// traversal in its slot (a context of its own, its own stream).  Queries that arrive
// while others run overlap with them: the dispatcher shrinks the running traversals
// (coop_request_resources, i.e. offer_kill at their next chunk boundary) so that every
// running query holds an equal share of the CTAs, and when a query finishes its CTAs are
// returned to the survivors (coop_release, i.e. request_fork).  A co-runner can take CTAs
// from the whole server the same way.

struct coop_server {
  int device = 0;
  int N = 0;           // CTAs of the GPU (one per SM)
  int min_share = 1;   // a running query never drops below this many CTAs
  size_t budget = 0, per_slot = 0;
  size_t resident = 0;  // device bytes of the registered graphs (CSR and weights)
  struct Slot {
    coop_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int64_t req = -1;  // running request, -1 when idle
    int share = 0;     // CTAs the dispatcher means this query to hold
  };
  std::vector<Slot> slots;
  struct Graph {
    coop_csr g;
    const uint32_t *w;
  };
  std::vector<Graph> graphs;
  struct Req {
    int graph, kind;
    int32_t src;
    void *out;
    double t_submit = 0, t_start = 0, t_done = 0;
    int status = 1;  // 1 = pending / running
    int slot = -1, ctas = 0;
    coop_stats st{};
  };
  std::unordered_map<uint64_t, Req> reqs;
  std::deque<uint64_t> queue;
  uint64_t next_ticket = 1;
  int corunner_held = 0;  // CTAs lent to a co-runner
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false, started = false;
};

namespace {

double now_us() {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// CTAs a slot's context can still lend: CTA 0 is never surrendered.
int lendable(coop_ctx *c) {
  std::lock_guard<std::mutex> lk(c->mu);
  return std::max(0, c->N - 1 - (int)(c->kill_req - c->returned));
}

int running_count(const coop_server *sv) {
  int n = 0;
  for (const auto &sl : sv->slots) n += sl.req >= 0;
  return n;
}

// Give every running query an equal share of the CTAs not held by a co-runner: take CTAs
// from queries above the share (they leave at their next offer_kill point) and return CTAs
// to queries below it (forked into them).
void rebalance_locked(coop_server *sv) {
  const int run = running_count(sv);
  if (run == 0) return;
  const int avail = std::max(run * sv->min_share, sv->N - sv->corunner_held);
  const int share = std::max(sv->min_share, avail / run);
  for (auto &sl : sv->slots) {
    if (sl.req < 0) continue;
    if (sl.share > share) {
      const int take = std::min(sl.share - share, lendable(sl.ctx));
      int freed = 0;
      if (take > 0) coop_request_resources(sl.ctx, take, 1, &freed);  // posts the request; does not wait
      sl.share -= take;
    } else if (sl.share < share) {
      int lent = 0;
      coop_query(sl.ctx, nullptr, nullptr, nullptr, &lent);
      const int give = std::min(share - sl.share, lent);
      if (give > 0 && coop_release(sl.ctx, give) == COOP_OK) sl.share += give;
    }
  }
}

void dispatcher(coop_server *sv) {
  DeviceGuard guard(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    bool changed = false;
    // completions
    for (size_t i = 0; i < sv->slots.size(); ++i) {
      auto &sl = sv->slots[i];
      if (sl.req < 0 || cudaEventQuery(sl.done) != cudaSuccess) continue;
      auto &r = sv->reqs[(uint64_t)sl.req];
      r.t_done = now_us();
      const coop_status st = coop_get_stats(sl.ctx, &r.st);
      r.status = (int)st;
      sl.req = -1;
      sl.share = 0;
      changed = true;
    }
    // admissions, in arrival order
    while (!sv->queue.empty()) {
      int free_slot = -1;
      for (size_t i = 0; i < sv->slots.size(); ++i)
        if (sv->slots[i].req < 0) {
          free_slot = (int)i;
          break;
        }
      if (free_slot < 0) break;
      const uint64_t t = sv->queue.front();
      sv->queue.pop_front();
      auto &r = sv->reqs[t];
      auto &sl = sv->slots[(size_t)free_slot];
      const int run = running_count(sv) + 1;
      const int avail = std::max(run * sv->min_share, sv->N - sv->corunner_held);
      const int share = std::max(sv->min_share, avail / run);
      // the new query starts with `share` CTAs: lend the rest of its slot's CTAs away
      int lent = 0;
      coop_query(sl.ctx, nullptr, nullptr, nullptr, &lent);
      const int want_lent = sv->N - share;
      if (lent < want_lent) coop_request_resources(sl.ctx, want_lent - lent, 0, nullptr);  // idle: immediate
      else if (lent > want_lent) coop_release(sl.ctx, lent - want_lent);
      sl.req = (int64_t)t;
      sl.share = share;
      r.slot = free_slot;
      r.ctas = share;
      r.t_start = now_us();
      const auto &G = sv->graphs[(size_t)r.graph];
      coop_status st = r.kind == COOP_JOB_SSSP
                           ? coop_sssp(sl.ctx, &G.g, G.w, r.src, static_cast<uint32_t *>(r.out), sl.stream, nullptr)
                           : coop_bfs(sl.ctx, &G.g, r.src, static_cast<int32_t *>(r.out), sl.stream, nullptr);
      if (st == COOP_OK) st = cuda_failed(cudaEventRecord(sl.done, sl.stream), "query event") ? COOP_ECUDA : COOP_OK;
      if (st != COOP_OK) {
        r.status = (int)st;
        r.t_done = now_us();
        sl.req = -1;
      }
      changed = true;
    }
    if (changed) {
      rebalance_locked(sv);
      sv->cv.notify_all();
    }
    if (sv->stop && sv->queue.empty() && running_count(sv) == 0) break;
    if (!changed) sv->cv.wait_for(lk, std::chrono::microseconds(running_count(sv) ? 5 : 200));
  }
  sv->cv.notify_all();
}

}  // namespace

extern "C" {

coop_status coop_server_create(int device, int slots, size_t hbm_budget_bytes, coop_server **out) {
  if (!out) return COOP_EINVAL;
  *out = nullptr;
  if (slots < 1 || slots > 64) return COOP_EINVAL;
  coop_server *sv = new coop_server();
  sv->device = device;
  sv->budget = hbm_budget_bytes;
  for (int i = 0; i < slots; ++i) {
    coop_server::Slot sl;
    coop_status st = coop_init(device, 0, 0, &sl.ctx);
    if (st != COOP_OK) {
      coop_server_destroy(sv);
      return st;
    }
    DeviceGuard guard(device);
    if (cuda_failed(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking), "slot stream") ||
        cuda_failed(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming), "slot event")) {
      sv->slots.push_back(sl);
      coop_server_destroy(sv);
      return COOP_ECUDA;
    }
    sv->slots.push_back(sl);
  }
  coop_query(sv->slots[0].ctx, &sv->N, nullptr, nullptr, nullptr);
  *out = sv;
  return COOP_OK;
}

coop_status coop_server_add_graph(coop_server *sv, const coop_csr *g, const uint32_t *d_weights, int *graph_id) {
  if (!sv || !graph_id || check_graph(g, 0) != COOP_OK) return COOP_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->started) return COOP_EBUSY;  // graphs are registered before the first query
  // every slot must be able to serve the graph: size its scratch now, before serving,
  // since an allocation while queries run would wait for them.  The budget covers every
  // slot's scratch (bitmap, three queues of three words per vertex, the packed distance
  // words, three chunk indexes) and the graphs registered so far.
  const size_t V = (size_t)g->num_vertices, E = (size_t)g->num_edges;
  const size_t per = V * 4 * 11 + (V + 31) / 32 * 4 + (E / kIndexEdges + 2) * 4 * 3 + (1u << 20);
  const size_t graph = (V + 1) * 4 + E * 4 + (d_weights ? E * 4 : 0);
  const size_t per_slot = std::max(sv->per_slot, per);
  if (sv->budget && per_slot * sv->slots.size() + sv->resident + graph > sv->budget) return COOP_ENOMEM;
  for (auto &sl : sv->slots) {
    DeviceGuard guard(sv->device);
    std::lock_guard<std::mutex> lk2(sl.ctx->mu);
    const coop_status st = ensure_scratch(sl.ctx, g->num_vertices, g->num_edges);
    if (st != COOP_OK) return st;
  }
  sv->per_slot = per_slot;
  sv->resident += graph;
  sv->graphs.push_back({*g, d_weights});
  *graph_id = (int)sv->graphs.size() - 1;
  return COOP_OK;
}

coop_status coop_server_submit(coop_server *sv, int graph_id, int kind, int32_t source, void *d_out,
                               uint64_t *ticket) {
  if (!sv || !ticket || !d_out || (kind != COOP_JOB_BFS && kind != COOP_JOB_SSSP)) return COOP_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (graph_id < 0 || graph_id >= (int)sv->graphs.size()) return COOP_EINVAL;
  const auto &G = sv->graphs[(size_t)graph_id];
  if (source < 0 || source >= G.g.num_vertices) return COOP_EINVAL;
  if (kind == COOP_JOB_SSSP && G.g.num_edges > 0 && !G.w) return COOP_EINVAL;
  if (!sv->started) {
    sv->started = true;
    sv->worker = std::thread(dispatcher, sv);
  }
  coop_server::Req r;
  r.graph = graph_id;
  r.kind = kind;
  r.src = source;
  r.out = d_out;
  r.t_submit = now_us();
  const uint64_t t = sv->next_ticket++;
  sv->reqs[t] = r;
  sv->queue.push_back(t);
  *ticket = t;
  sv->cv.notify_all();
  return COOP_OK;
}

coop_status coop_server_wait(coop_server *sv, uint64_t ticket, int timeout_us, coop_query_result *res) {
  if (!sv) return COOP_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return COOP_EINVAL;
  auto done = [&] { return it->second.status != 1; };
  if (timeout_us > 0) {
    if (!sv->cv.wait_for(lk, std::chrono::microseconds(timeout_us), done)) return COOP_ETIMEOUT;
  } else {
    sv->cv.wait(lk, done);
  }
  const auto &r = it->second;
  if (res) {
    res->status = r.status;
    res->slot = r.slot;
    res->ctas = r.ctas;
    res->queue_us = r.t_start - r.t_submit;
    res->latency_us = r.t_done - r.t_submit;
    res->stats = r.st;
  }
  const int st = r.status;
  sv->reqs.erase(it);
  return (coop_status)st;
}

coop_status coop_server_request_resources(coop_server *sv, int n_ctas, int timeout_us, int *n_freed) {
  if (n_freed) *n_freed = 0;
  if (!sv || n_ctas < 1) return COOP_EINVAL;
  struct Ask {
    coop_ctx *ctx;
    int n;
    uint32_t target;
    bool granted;
    uint32_t run;
  };
  std::vector<Ask> asks;
  int from_idle = 0;
  coop_status worst = COOP_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->corunner_held + n_ctas > sv->N - sv->min_share) return COOP_EINVAL;
    // CTAs that neither a running query nor the co-runner holds are free already
    int held = sv->corunner_held;
    std::vector<size_t> idx;
    for (size_t i = 0; i < sv->slots.size(); ++i)
      if (sv->slots[i].req >= 0) {
        idx.push_back(i);
        held += sv->slots[i].share;
      }
    from_idle = std::min(n_ctas, std::max(0, sv->N - held));
    // The rest from the running queries in proportion to what each can lend, so that every
    // query keeps the same fraction of its share.  CTAs taken from a query leave at its
    // next offer_kill point, but CTAs given back join it only at its next barrier: a query
    // cut down to its master CTA in the middle of a wide level would finish that level
    // alone, long after the co-runner has returned the CTAs.
    std::sort(idx.begin(), idx.end(), [&](size_t x, size_t y) { return sv->slots[x].share > sv->slots[y].share; });
    std::vector<int> room(idx.size()), take(idx.size(), 0);
    int total = 0;
    for (size_t j = 0; j < idx.size(); ++j) {
      const auto &sl = sv->slots[idx[j]];
      room[j] = std::max(0, std::min(sl.share - sv->min_share, lendable(sl.ctx)));
      total += room[j];
    }
    const int need = std::min(n_ctas - from_idle, total);
    int left = need;
    for (size_t j = 0; j < idx.size() && total > 0; ++j) {
      take[j] = (int)((int64_t)need * room[j] / total);
      left -= take[j];
    }
    // the remainder one CTA at a time, largest shares first (need <= total: it ends)
    for (size_t j = 0; left > 0; j = (j + 1) % idx.size())
      if (take[j] < room[j]) {
        ++take[j];
        --left;
      }
    // every request is posted before any is waited for: the queries free their CTAs
    // concurrently, within one deadline
    for (size_t j = 0; j < idx.size(); ++j) {
      if (take[j] <= 0) continue;
      auto &sl = sv->slots[idx[j]];
      Ask a{sl.ctx, take[j], 0u, false, 0u};
      double lock_us = 0.0;
      const coop_status st = post_kill(sl.ctx, a.n, &a.target, &a.granted, &lock_us, &a.run);
      if (st != COOP_OK) {
        if (worst == COOP_OK) worst = st;
        continue;
      }
      sl.share -= take[j];
      asks.push_back(a);
    }
    sv->corunner_held += n_ctas;
  }
  int got = from_idle;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(std::max(0, timeout_us));
  for (auto &a : asks) {
    int f = a.n;
    const coop_status st =
        a.granted ? COOP_OK : wait_kill(a.ctx, a.target, a.n, a.run, timeout_us > 0, deadline, &f);
    got += f;
    if (st != COOP_OK && worst == COOP_OK) worst = st;
  }
  if (n_freed) *n_freed = got;
  if (worst == COOP_OK && got < n_ctas) worst = COOP_ETIMEOUT;  // fewer CTAs could be taken
  return worst;
}

coop_status coop_server_release(coop_server *sv, int n_ctas) {
  if (!sv || n_ctas < 1) return COOP_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (n_ctas > sv->corunner_held) return COOP_EINVAL;
  sv->corunner_held -= n_ctas;
  rebalance_locked(sv);
  return COOP_OK;
}

coop_status coop_server_destroy(coop_server *sv) {
  if (!sv) return COOP_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->cv.notify_all();
  }
  if (sv->worker.joinable()) sv->worker.join();
  DeviceGuard guard(sv->device);
  for (auto &sl : sv->slots) {
    if (sl.ctx) coop_destroy(sl.ctx);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  (void)cudaGetLastError();
  delete sv;
  return COOP_OK;
}

}  // extern "C"

// ===================================================================== allocation-free BFS
//
// coop_bfs_noalloc runs the same cooperative BFS kernels as coop_bfs, but takes its
// scratch (control block, mailbox, visited bitmap, both frontier queues) from one static
// device array compiled into this library instead of memory allocated at run time.  It
// serves callers that must not allocate device memory: processes that reserve their
// whole device-memory budget up front through their own pool, code running inside an
// allocator's or a memory pool's callbacks (which must not re-enter the allocator), and
// latency-critical loops that cannot take cudaMalloc's implicit device synchronisation
// (which would also wait for any traversal still running).

namespace {

constexpr int64_t kNoAllocMaxVertices = (int64_t)1 << 20;
constexpr int64_t kNoAllocMaxEdges = (int64_t)1 << 25;
constexpr size_t na_align(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kNaMboxOff = na_align(sizeof(Ctl));
constexpr size_t kNaBitmapOff = kNaMboxOff + na_align(sizeof(Mailbox));
constexpr size_t kNaQueueOff = kNaBitmapOff + na_align((size_t)(kNoAllocMaxVertices + 31) / 32 * 4);
constexpr size_t kNaQueueBytes = na_align((size_t)kNoAllocMaxVertices * 4);
constexpr size_t kNaIndexOff = kNaQueueOff + 6 * kNaQueueBytes;
constexpr size_t kNaIndexBytes = na_align((size_t)(kNoAllocMaxEdges / kIndexEdges + 2) * 4);
constexpr size_t kNaBytes = kNaIndexOff + 2 * kNaIndexBytes;  // about 25 MB

// The scratch of coop_bfs_noalloc.  Every GPU that loads the library holds it until the
// process exits.  In host code this name is only a stand-in: the device address comes
// from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Final status of an allocation-free run: its sticky error, else its published status,
// else (the run never published) a timeout.
__global__ void coop_noalloc_status_kernel(const Mailbox *m, uint32_t run, int32_t *out) {
  const int32_t e = *(volatile const int32_t *)&m->err;
  const uint32_t finished = *(volatile const uint32_t *)&m->run_done;
  *out = e != 0 ? e : (finished == run ? *(volatile const int32_t *)&m->status : (int32_t)COOP_ETIMEOUT);
}

struct NoAllocDevice {
  bool ready = false;
  unsigned char *base = nullptr;  // device address of g_noalloc_scratch on this device
  int ctas = 0;
  int sms = 0;
  uint32_t run = 0;
};
constexpr int kNoAllocDevices = 64;
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc[kNoAllocDevices];

}  // namespace

extern "C" coop_status coop_bfs_noalloc(const coop_csr *g, int32_t source, int32_t *d_levels, int32_t *d_status,
                                        coop_stream stream) {
  if (!d_levels) return COOP_EINVAL;
  const coop_status st = check_graph(g, source);
  if (st != COOP_OK) return st;
  if ((int64_t)g->num_vertices > kNoAllocMaxVertices || g->num_edges > kNoAllocMaxEdges) {
    snprintf(g_last_error, sizeof(g_last_error),
             "coop_bfs_noalloc: %d vertices / %lld edges exceed the static scratch limit of %lld vertices and "
             "%lld edges",
             g->num_vertices, (long long)g->num_edges, (long long)kNoAllocMaxVertices, (long long)kNoAllocMaxEdges);
    return COOP_EINVAL;
  }
  int dev = -1;
  if (cuda_failed(cudaGetDevice(&dev), "current device")) return COOP_ECUDA;
  if (dev < 0 || dev >= kNoAllocDevices) return COOP_EINVAL;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoAllocDevice &d = g_noalloc[dev];
  if (!d.ready) {
    // one-time set-up on this device (the current one): the scratch's device address,
    // the kernel's shared-memory attribute and the CTA count.  Nothing is allocated.
    void *ptr = nullptr;
    if (cuda_failed(cudaGetSymbolAddress(&ptr, g_noalloc_scratch), "scratch symbol address")) return COOP_ECUDA;
    const void *k = traverse_fn<MODE_BFS>(kDefaultWorkerWarps);
    if (!set_traverse_attrs(k, traverse_smem(MODE_BFS, kDefaultWorkerWarps))) return COOP_ECUDA;
    int nb = 0, sms = 0;
    if (cuda_failed(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "sm count") ||
        cuda_failed(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, (kDefaultWorkerWarps + 1) * 32,
                                                                  traverse_smem(MODE_BFS, kDefaultWorkerWarps)),
                    "occupancy"))
      return COOP_ECUDA;
    if (nb < 1) {
      snprintf(g_last_error, sizeof(g_last_error), "traversal kernel cannot be resident (%d per SM)", nb);
      return COOP_ECUDA;
    }
    d.base = static_cast<unsigned char *>(ptr);
    d.ctas = std::min(nb * sms, kMaxCtas);
    d.sms = sms;
    d.ready = true;
  }
  Params p{};
  p.row_off = g->row_off;
  p.col = g->col;
  p.V = g->num_vertices;
  p.E = (uint32_t)g->num_edges;
  p.level = d_levels;
  p.ctl = reinterpret_cast<Ctl *>(d.base);
  p.mbox = reinterpret_cast<Mailbox *>(d.base + kNaMboxOff);
  p.visited = reinterpret_cast<uint32_t *>(d.base + kNaBitmapOff);
  for (int i = 0; i < 2; ++i) {
    p.qo[i] = reinterpret_cast<uint32_t *>(d.base + kNaQueueOff + (size_t)(3 * i + 0) * kNaQueueBytes);
    p.qs[i] = reinterpret_cast<uint32_t *>(d.base + kNaQueueOff + (size_t)(3 * i + 1) * kNaQueueBytes);
    p.qv[i] = reinterpret_cast<uint32_t *>(d.base + kNaQueueOff + (size_t)(3 * i + 2) * kNaQueueBytes);
    p.qx[i] = reinterpret_cast<uint32_t *>(d.base + kNaIndexOff + (size_t)i * kNaIndexBytes);
  }
  p.src = source;
  p.N = d.ctas;
  p.launched = (uint32_t)d.ctas;
  p.timeout_ns = 2000000000ull;
  p.run = ++d.run;
  p.coop = 1u;
  cudaStream_t s = (cudaStream_t)stream;
  // The array keeps the previous call's contents: clear the mailbox (scheduler requests,
  // error, statistics) here; the init kernel clears the control block and the bitmap.
  if (cuda_failed(cudaMemsetAsync(p.mbox, 0, sizeof(Mailbox), s), "clear mailbox")) return COOP_ECUDA;
  coop_init_kernel<MODE_BFS><<<d.sms * 4, 512, 0, s>>>(p);
  launch_traverse<MODE_BFS>(kDefaultWorkerWarps, d.ctas, p, 0, s);
  if (d_status) coop_noalloc_status_kernel<<<1, 1, 0, s>>>(p.mbox, p.run, d_status);
  if (cuda_failed(cudaGetLastError(), "allocation-free launch")) return COOP_ECUDA;
  return COOP_OK;
}

// ===================================================================== octree host side
namespace {

// Octree scratch for n points: 2 x 4 arrays of n words (coordinates and point index),
// the queue headers, the task slots and the control block; grown to the largest n.
coop_status ensure_oct_scratch(coop_ctx *c, int64_t n) {
  if (n <= c->oct_cap && c->oct_scratch) return COOP_OK;
  if (c->oct_scratch) {
    if (c->launched) cudaEventSynchronize(c->ev_done);
    cudaFree(c->oct_scratch);
    c->oct_scratch = nullptr;
    c->oct_cap = 0;
  }
  const int64_t cap = std::max<int64_t>(n, 1024);
  const size_t words = ((size_t)cap * 4 + 255) & ~(size_t)255;
  const size_t total = 8 * words + sizeof(OctQueue) * kOctQueues + sizeof(OctTask) * kOctQueues * kOctQueueCap +
                       sizeof(OctCtl) + 4 * kPreCells * sizeof(uint32_t) + 1024;
  if (cudaMalloc(&c->oct_scratch, total) != cudaSuccess) {
    (void)cudaGetLastError();
    c->oct_scratch = nullptr;
    return COOP_ENOMEM;
  }
  c->oct_cap = cap;
  return COOP_OK;
}

}  // namespace

extern "C" {

coop_status coop_octree(coop_ctx *c, const uint32_t *d_x, const uint32_t *d_y, const uint32_t *d_z, int32_t n,
                        int32_t leaf_cap, int32_t max_depth, uint64_t *d_leaf_code, uint32_t *d_leaf_begin,
                        uint32_t *d_leaf_count, int32_t max_leaves, uint32_t *d_perm, int32_t *d_n_leaves,
                        coop_stream stream, coop_stats *stats) {
  if (!c || n < 0 || leaf_cap < 1 || max_depth < 0 || max_depth > 21 || !d_n_leaves) return COOP_EINVAL;
  if (n > 0 && (!d_x || !d_y || !d_z || !d_leaf_code || !d_leaf_begin || !d_leaf_count || !d_perm ||
                max_leaves < 1))
    return COOP_EINVAL;
  DeviceGuard guard(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> launch_lk(c->launch_mu);
  if (c->launched) cudaEventSynchronize(c->ev_done);
  OctParams p{};
  {
    std::lock_guard<std::mutex> lk(c->mu);
    finalize_locked(c);
    if (n == 0) {
      if (cuda_failed(cudaMemsetAsync(d_n_leaves, 0, sizeof(int32_t), s), "octree: empty")) return COOP_ECUDA;
      if (stats) {
        if (cudaStreamSynchronize(s) != cudaSuccess) return COOP_ECUDA;
        memset(stats, 0, sizeof(*stats));
      }
      return COOP_OK;
    }
    coop_status st = ensure_oct_scratch(c, n);
    if (st != COOP_OK) return st;
    char *base = static_cast<char *>(c->oct_scratch);
    const size_t words = ((size_t)c->oct_cap * 4 + 255) & ~(size_t)255;
    uint32_t *w[8];
    for (int i = 0; i < 8; ++i) w[i] = reinterpret_cast<uint32_t *>(base + (size_t)i * words);
    char *at = base + 8 * words;
    p.queues = reinterpret_cast<OctQueue *>(at);
    at += sizeof(OctQueue) * kOctQueues;
    p.tasks = reinterpret_cast<OctTask *>(at);
    at += sizeof(OctTask) * kOctQueues * kOctQueueCap;
    p.ctl = reinterpret_cast<OctCtl *>(((uintptr_t)at + 127) & ~(uintptr_t)127);
    uint32_t *cells = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(p.ctl) + sizeof(OctCtl));
    p.cell_count = cells;
    p.cell_begin = cells + kPreCells;
    p.cell_cursor = cells + 2 * kPreCells;
    p.cell_leaf = cells + 3 * kPreCells;
    p.pre = ((uint32_t)n >= kPreMinPoints && (uint32_t)max_depth >= kPreDepth && n > leaf_cap) ? 1u : 0u;
    for (int b = 0; b < 2; ++b) {
      p.bx[b] = w[4 * b];
      p.by[b] = w[4 * b + 1];
      p.bz[b] = w[4 * b + 2];
      p.bi[b] = w[4 * b + 3];
    }
    p.x = d_x;
    p.y = d_y;
    p.z = d_z;
    p.n = (uint32_t)n;
    p.leaf_cap = (uint32_t)leaf_cap;
    p.max_depth = (uint32_t)max_depth;
    p.perm = d_perm;
    p.leaf_code = reinterpret_cast<unsigned long long *>(d_leaf_code);
    p.leaf_begin = d_leaf_begin;
    p.leaf_count = d_leaf_count;
    p.n_leaves = d_n_leaves;
    p.max_leaves = (uint32_t)max_leaves;
    p.mbox = c->mbox_d;
    // a run id of its own: a request posted while the octree is built waits for its CTAs
    // (or for the build's end, which the finish kernel publishes)
    p.run = ++c->run;
    c->cur.run = p.run;
    const int held = (int)(c->served - c->returned);
    p.launched = (uint32_t)std::max(1, c->N - held);
    p.kill_base = c->served;
    p.fork_base = c->fork_req;
    p.coop = 1u;
    p.timeout_ns = (uint64_t)std::max<int64_t>(c->timeout_us, 1) * 1000ull;
    c->mbox->err = 0;
    store_release(&c->mbox->freed, c->served);
    store_release(&c->mbox->kill_req, c->kill_req);
    store_release(&c->mbox->fork_req, c->fork_req);
    coop_octree_init<<<c->sm_count * 4, 512, 0, s>>>(p);
    if (c->timing) cudaEventRecord(c->ev_t0, s);
    if (p.pre) {
      coop_octree_pre_hist<<<c->sm_count * 4, 512, 0, s>>>(p);
      coop_octree_pre_plan<<<1, kPreCells, 0, s>>>(p);
      coop_octree_pre_scatter<<<c->sm_count * 4, 512, 0, s>>>(p);
    }
    switch (c->nw) {
      case 31: coop_octree_kernel<31><<<p.launched, 32 * 32, kTraverseSmemMin, s>>>(p, 0); break;
      case 23: coop_octree_kernel<23><<<p.launched, 24 * 32, kTraverseSmemMin, s>>>(p, 0); break;
      default: coop_octree_kernel<15><<<p.launched, 16 * 32, kTraverseSmemMin, s>>>(p, 0); break;
    }
    if (c->timing) cudaEventRecord(c->ev_t1, s);
    coop_octree_finish<<<1, 1, 0, s>>>(p);
    cudaEventRecord(c->ev_done, s);
    if (cuda_failed(cudaGetLastError(), "octree launch")) return COOP_ECUDA;
    c->launched = true;
    c->gather_us_max = 0.0;
  }
  if (!stats) return COOP_OK;
  if (cuda_failed(cudaEventSynchronize(c->ev_done), "octree")) return COOP_ECUDA;
  OctCtl h{};
  if (cuda_failed(cudaMemcpy(&h, p.ctl, sizeof(h), cudaMemcpyDeviceToHost), "octree stats")) return COOP_ECUDA;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    finalize_locked(c);
  }
  memset(stats, 0, sizeof(*stats));
  stats->kills = (int32_t)h.killed.v;
  stats->forks = (int32_t)(h.launched.v - p.launched);
  stats->initial_active = (int32_t)p.launched;
  stats->ctas_launched = (int32_t)h.launched.v;
  stats->frontier_total = (int64_t)h.tasks;
  stats->edges_scanned = (int64_t)h.steals;
  stats->vertices_reached = (int64_t)h.leaves.v;
  stats->reached_edges = (int64_t)h.moved;
  if (c->timing) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev_t0, c->ev_t1) == cudaSuccess) stats->kernel_us = ms * 1e3;
  }
  int32_t status = (int32_t)h.err.v;
  if (status == 0 && h.leaves.v > (uint32_t)max_leaves) status = COOP_EOVERFLOW;
  stats->status = status;
  return (coop_status)status;
}

}  // extern "C"
