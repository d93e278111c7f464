// gg_common.cuh -- shared device/host definitions of the frontier SSSP library.
//
// Data layout in HBM (one graph handle):
//   ro      u32[n+1]   CSR row offsets (push direction)
//   edges   uint2[m]   {col, weight} interleaved: one 8-byte load per edge, or
//   edges4  u32[m]     the packed form (col << wbits) | weight, used whenever the
//                      column bits of n-1 plus the bits of the largest weight
//                      fit in 32 (halves the edge stream; e.g. RMAT-22 with
//                      weights <= 255 uses 22 + 10 bits)
//   t_ro / t_edges(4)  the transpose (CSC) for pull; aliases ro/edges when the
//                      graph is symmetric
//   pv, ps  u32[np]    vertices with a non-empty CSC row and that row's start
//                      (the entry list of the pull sweep)
// Workspace of one SSSP run:
//   fv/fr/fs[2]  u32[n]  sparse frontier, ping-pong by superstep parity:
//                        vertex, its CSR row start, and the exclusive prefix
//                        of frontier out-degrees (the merge-path coordinate)
//   bm[3]   u32[ceil(n/32)]  dense frontier bitmaps, rotating by superstep:
//                        current (read), next (test-and-set dedup), old
//                        (cleared)
//   ctl     Ctl          counters and the superstep state machine
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gg.h"

namespace gg {

constexpr uint32_t kInf = 0xFFFFFFFFu;
constexpr uint32_t kSat = 0xFFFFFFFEu;   // saturated (overflowed) finite distance
constexpr uint32_t kFltMaxBits = 0x7F7FFFFFu;   // FLT_MAX: "unreached" for binary32 distances

// How a relaxation adds an edge weight (per run): unsigned integers, IEEE
// binary32 bit patterns (the paper's float weights), or unit weights (BFS).
enum : uint32_t { WM_U32 = 0, WM_F32 = 1, WM_UNIT = 2 };

// MODE_HEAVY_PULL_TAIL: a heavy pull after which bucketing ends; it writes the
// plain tail's first frontier itself (no split step follows)
enum : uint32_t { MODE_PUSH = 0, MODE_PULL = 1, MODE_SPLIT = 2, MODE_HEAVY = 3, MODE_HEAVY_PULL = 4,
                  MODE_HEAVY_PULL_TAIL = 5 };
enum : uint32_t { DIR_AUTO = 0, DIR_PUSH = 1, DIR_PULL = 2 };

// device-status bits, mapped to gg_status on the host
enum : uint32_t { DS_OVERFLOW = 1u, DS_ITER_CAP = 2u, DS_TIMEOUT = 4u, DS_INTERNAL = 8u };

// Buffers of the light/heavy bucket variant (allocated on first use by a
// graph; see Ctl::lh).  Rows of lh_edges hold the same edges as the graph's
// own array, light ones (weight < delta) first: the light edges of v are
// [ro[v], lend[v]) and its heavy edges [lend[v], ro[v+1]).
struct LhBufs {
  const void* edges;   // uint2[m] or packed u32[m], rows partitioned by weight < delta
  const uint32_t* lend;
  uint32_t* rv[2];     // R lists by epoch parity: vertex, heavy row start, heavy-edge prefix
  uint32_t* rr[2];
  uint32_t* rs[2];
  uint32_t* bm_r[2];   // R membership bitmaps by epoch parity
};

struct Ctl {
  unsigned long long cnt[2];   // (count << 32) | edge total of the frontier being built, by parity
  uint32_t iter;               // superstep index
  uint32_t done_ctas;          // arrival counter for the last-CTA finalize
  uint32_t status;             // DS_* bits
  uint32_t mode;               // MODE_PUSH / MODE_PULL of the current superstep
  uint32_t clear_prev;         // bm[(iter+2)%3] must be zeroed during this superstep
  uint32_t src;
  uint32_t max_iter;
  uint32_t dir;                // DIR_*
  uint32_t alpha, beta;        // direction switch thresholds
  uint32_t running;            // 1 while the frontier is non-empty
  uint32_t pull_iters;
  uint32_t* dist;              // caller's distance array for this run
  uint32_t* trace;             // optional per-superstep trace (4 u32 per superstep)
  uint32_t trace_cap;
  uint32_t max_frontier;
  uint32_t warp_thr, cta_thr;  // degree bins of the binned push advance
  uint32_t wmode;              // WM_*: how relaxations add edge weights in this run
  // near-far split of the frontier (priority buckets of width delta): vertices
  // improved to a distance < t_cur join the next frontier, the others wait in
  // the far pile far[fp] until the near frontier empties and a split step
  // raises the threshold
  uint32_t t_cur, t_prev, delta, fp;
  uint32_t far_cnt[2];
  uint32_t far_min;            // lower bound of the distances recorded in the far pile
  uint32_t splits;
  // persistent bulk-synchronous kernel: counters rotate over three slots so
  // that one grid barrier per superstep suffices
  unsigned long long cnt3[3];
  uint32_t fm3[3];             // smallest far distance recorded in a superstep
  uint32_t fcnt3[3];           // far-pile append positions (pile rotates with each split step)
  uint32_t fadd3[3];           // far entries appended in a superstep (what decisions read)
  uint32_t bar_count, bar_gen, abort;
  unsigned long long t_start;  // %globaltimer at init (watchdog)
  unsigned long long watchdog_ns;
  unsigned long long edges_scanned;
  unsigned long long frontier_total;
  // light/heavy buckets (Meyer-Sanders delta-stepping on top of the near-far
  // split): near supersteps relax only the light edges of their vertices; a
  // vertex that drops below t_cur joins the R list of the current epoch once,
  // and when the near frontier is empty one heavy superstep relaxes the heavy
  // edges of R (each heavy edge once per settled vertex) and starts the next
  // epoch.  Vertices of a bucket whose distance is final before its heavy
  // superstep never re-scan heavy edges, which is where plain near-far and
  // Bellman-Ford spend most of their re-relaxations.
  uint32_t lh;                       // 1: this run uses light/heavy buckets
  uint32_t epoch;                    // heavy supersteps completed
  unsigned long long rcnt[2];        // (count << 32) | heavy-edge total of R[0], R[1]
  uint32_t drain_div;                // unsettled heavy edges < m / drain_div end bucketing
  // heavy superstep by pull (symmetric graphs): chosen when R's heavy edges
  // outnumber those of the vertices not yet settled
  uint32_t heavy_pull_ok;
  unsigned long long heavy_total;    // heavy edges of the graph
  unsigned long long heavy_done;     // heavy edges of the vertices settled so far
  // once bucketing ends (the threshold becomes infinite) the rest of the run
  // is plain push over all edges of each vertex: with one bucket left, the
  // light/heavy alternation only adds supersteps
  uint32_t lh_tail;
};

struct DevGraph {
  uint32_t n, m, np, nwords;
  const uint32_t* ro;
  const void* edges;       // uint2[m] or, when packed, u32[m]
  const uint32_t* t_ro;
  const void* t_edges;
  const uint32_t* pv;
  const uint32_t* ps;
  uint32_t packed;         // 1: edges are (col << wbits) | weight
  uint32_t wbits;
  uint32_t sinks;          // 1: some vertex has in-edges but no out-edges
};

struct Frontier {
  uint32_t* fv[2];
  uint32_t* fr[2];
  uint32_t* fs[2];
  uint32_t* bm[3];
  uint32_t* far[3];    // far pile (vertex ids): ping-pong across split steps (three
                       // rotating piles in the persistent kernel)
  uint32_t* bm_far;    // far-pile membership (dedup)
};

#ifdef __CUDACC__
// Arrival at the end of a superstep, by one thread of each CTA after a CTA
// barrier; true in the CTA that arrives last.  One acquire-release atomic: the
// CTA's writes (ordered before by the barrier) are visible before its arrival
// counts, and the last arrival sees those of every other CTA.  (Measured
// against a full fence followed by a relaxed atomic: 7 % faster on a
// high-diameter grid of 10,000 supersteps.)
__device__ __forceinline__ bool arrive_last(uint32_t* done, uint32_t ctas) {
  uint32_t old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(done) : "memory");
  return old == ctas - 1u;
}

// Relaxed loads at L2 (no L1 copy): the counters that the CTAs of a superstep
// update with atomics, read by the last CTA after its acquire.
__device__ __forceinline__ uint32_t ld_rlx(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_rlx(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// L2-coherent load (bypasses L1): used for values other CTAs update with atomics.
__device__ __forceinline__ uint32_t ld_cg(const uint32_t* p) { return __ldcg(p); }

// Element i of a small kernel-parameter array without dynamic indexing
// (which would copy the whole parameter struct to local memory).
template <class T>
__device__ __forceinline__ T pick2(const T (&a)[2], uint32_t i) { return i ? a[1] : a[0]; }
template <class T>
__device__ __forceinline__ T pick3(const T (&a)[3], uint32_t i) { return i == 0 ? a[0] : (i == 1 ? a[1] : a[2]); }

// One edge as {col, weight} from either edge encoding.
template <bool PK>
__device__ __forceinline__ uint2 load_edge(const void* base, uint32_t e, uint32_t wbits) {
  if (PK) {
    const uint32_t x = __ldg(static_cast<const uint32_t*>(base) + e);
    return make_uint2(x >> wbits, x & ((1u << wbits) - 1u));
  } else {
    return __ldg(static_cast<const uint2*>(base) + e);
  }
}

// N consecutive edges (N = 2, 4 or 8) starting at e (e a multiple of N,
// buffer 256-byte aligned) with 8- or 16-byte vector loads.
template <bool PK, int N>
__device__ __forceinline__ void load_edges_run(const void* base, uint32_t e, uint32_t wbits, uint32_t* col,
                                               uint32_t* w) {
  static_assert(N == 2 || N == 4 || N == 8, "runs of 2, 4 or 8 edges");
  if (PK && N == 2) {
    const uint2 q = __ldg(reinterpret_cast<const uint2*>(static_cast<const uint32_t*>(base) + e));
    const uint32_t mask = (1u << wbits) - 1u;
    col[0] = q.x >> wbits;
    w[0] = q.x & mask;
    col[1] = q.y >> wbits;
    w[1] = q.y & mask;
  } else if (PK) {
    const uint4* p = reinterpret_cast<const uint4*>(static_cast<const uint32_t*>(base) + e);
    const uint32_t mask = (1u << wbits) - 1u;
#pragma unroll
    for (int h = 0; h < N / 4; ++h) {
      const uint4 q = __ldg(p + h);
      const uint32_t x[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        col[4 * h + k] = x[k] >> wbits;
        w[4 * h + k] = x[k] & mask;
      }
    }
  } else {
    const uint4* p = reinterpret_cast<const uint4*>(static_cast<const uint2*>(base) + e);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      const uint4 q = __ldg(p + k);
      col[2 * k] = q.x;
      w[2 * k] = q.y;
      col[2 * k + 1] = q.z;
      w[2 * k + 1] = q.w;
    }
  }
}

// saturating distance add; flags overflow when the sum does not fit below kInf.
__device__ __forceinline__ uint32_t add_sat(uint32_t d, uint32_t w, bool& ovf) {
  unsigned long long s = (unsigned long long)d + w;
  if (s >= kInf) { ovf = true; return kSat; }
  return (uint32_t)s;
}

// d + w for the run's weight mode.  WM_F32: nonnegative binary32 bit patterns
// order like the floats they encode, so the round-to-nearest sum's bits feed
// the same unsigned compare and atomicMin; an overflow rounds to +inf, which
// never improves on FLT_MAX.  WM_UNIT: every edge counts 1 (hop distance).
__device__ __forceinline__ uint32_t relax_add(uint32_t d, uint32_t w, bool& ovf, uint32_t wmode) {
  if (wmode == WM_F32) return __float_as_uint(__fadd_rn(__uint_as_float(d), __uint_as_float(w)));
  return add_sat(d, wmode == WM_UNIT ? 1u : w, ovf);
}

// Largest j in [0, F) with S[j] <= x, for S strictly increasing with S[0] <= x.
// Executed by a full warp (32-ary search: ceil(log32 F) dependent rounds).
__device__ __forceinline__ uint32_t warp_search_le(const uint32_t* S, uint32_t F, uint32_t x) {
  const int lane = threadIdx.x & 31;
  uint32_t lo = 0, hi = F;
  while (hi - lo > 32) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint32_t p = lo + lane * step;
    const bool pred = (p < hi) && (S[p] <= x);
    const unsigned b = __ballot_sync(0xFFFFFFFFu, pred);
    const int last = 31 - __clz(b);
    lo = lo + last * step;
    hi = min(hi, lo + step);
  }
  const uint32_t p = lo + lane;
  const bool pred = (p < hi) && (S[p] <= x);
  const unsigned b = __ballot_sync(0xFFFFFFFFu, pred);
  return lo + (31 - __clz(b));
}

// Exclusive scan in place of data[0..count) held in shared memory, by a
// whole CTA of BLOCK threads; returns the total.  wsum: BLOCK/32 words of smem.
template <int BLOCK>
__device__ __forceinline__ uint32_t block_scan_excl(uint32_t* data, uint32_t count, uint32_t* wsum) {
  constexpr int NW = BLOCK / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t items = (count + BLOCK - 1) / BLOCK;
  const uint32_t beg = min((uint32_t)tid * items, count), end = min(beg + items, count);
  uint32_t local = 0;
  for (uint32_t i = beg; i < end; ++i) local += data[i];
  uint32_t x = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < NW ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < NW) wsum[lane] = s;
  }
  __syncthreads();
  uint32_t run = x - local + (warp ? wsum[warp - 1] : 0);
  const uint32_t total = wsum[NW - 1];
  for (uint32_t i = beg; i < end; ++i) {
    const uint32_t d = data[i];
    data[i] = run;
    run += d;
  }
  __syncthreads();
  return total;
}

// Inclusive prefix sum in place of the BLOCK*ITEMS u16 shared array a, by a
// whole CTA (thread t owns ITEMS consecutive elements); wsum: BLOCK/32 words.
template <int BLOCK, int ITEMS>
__device__ __forceinline__ void block_incl_scan_u16(uint16_t* a, uint32_t* wsum) {
  constexpr int NW = BLOCK / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t v[ITEMS];
  uint32_t run = 0;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    run += a[tid * ITEMS + i];
    v[i] = run;
  }
  uint32_t x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < NW ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < NW) wsum[lane] = s;
  }
  __syncthreads();
  const uint32_t base = x - run + (warp ? wsum[warp - 1] : 0);
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) a[tid * ITEMS + i] = (uint16_t)(base + v[i]);
  __syncthreads();
}

// Index of the last element <= x in the strictly increasing smem array a[0..n).
__device__ __forceinline__ uint32_t smem_upper_bound_minus1(const uint32_t* a, uint32_t n, uint32_t x) {
  uint32_t lo = 0, len = n;
  while (len > 0) {
    const uint32_t half = len >> 1;
    if (a[lo + half] <= x) { lo += half + 1; len -= half + 1; }
    else len = half;
  }
  return lo - 1;
}
#endif

}  // namespace gg
