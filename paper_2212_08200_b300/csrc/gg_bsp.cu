// gg_bsp.cu -- bulk-synchronous frontier SSSP (the execution::par policy).
//
// The paper's SSSP (Listing 4) repeats   f = neighbors_expand(par, g, f, cond)
// while f is non-empty, where the expand operator (Listing 3) visits every
// out-edge (v, n, w) of every active vertex v and adds n to the output
// frontier when   cond = (dist[v] + w  <  atomic_min(&dist[n], dist[v] + w)).
//
// Here one superstep is ONE kernel, k_superstep, that fuses:
//   advance  push: every frontier out-edge relaxed with atomicMin on dist,
//            load-balanced by a merge-path split of the frontier's edge
//            prefix sums (equal edge ranges per CTA, whatever the degrees);
//            or pull: a sweep of the transpose where each vertex takes the
//            minimum over its in-edges from active vertices (dense bitmap
//            frontier), then one atomicMin per destination row segment;
//   filter   each improved vertex is test-and-set in the next bitmap (dedup),
//            collected in shared memory, block-scanned and appended to the
//            next sparse frontier with ONE 64-bit atomicAdd per CTA tile that
//            returns both its queue position and its edge-prefix base, so the
//            next frontier comes out already carrying its merge-path
//            coordinates (no separate scan pass);
//   loop     the last CTA to arrive (one acquire-release atomic per CTA)
//            reads the counters in one batch of loads, picks the next
//            superstep's kind (push, pull, near-far split, heavy push or
//            pull), and sets the CUDA-graph conditional (work left), so the
//            whole loop runs on the device; the graph's loop body holds eight
//            superstep kernels per evaluation of the condition.
// On skewed graphs the default is light/heavy buckets (Meyer-Sanders
// delta-stepping over the near-far split): push supersteps relax only the
// light edges of a light-first copy of the edges, and each vertex that settles
// into the current bucket has its heavy edges relaxed once, by a heavy
// superstep that pushes from the settled vertices or pulls into the unsettled
// ones; once the unsettled vertices hold few heavy edges the buckets end and
// the rest of the run is the plain push loop.  Every relaxation is the same
// atomicMin with the strict < test, so the distances are those of the plain
// loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "gg_host.h"

#ifndef GG_EPT
#define GG_EPT 4   // edges per thread per tile of the superstep kernels
#endif
#ifndef GG_WU
#define GG_WU 2    // 32-edge chunks per step of the warp-streaming advance
#endif
#ifndef GG_WARP_MINB
#define GG_WARP_MINB 5   // resident CTAs per SM the warp-streaming kernels are compiled for
#endif
#ifndef GG_HEAVY_PULL
#define GG_HEAVY_PULL 1   // allow heavy supersteps by pull on symmetric graphs
#endif
#ifndef GG_DEFER_DEDUP
#define GG_DEFER_DEDUP 1   // warp streaming: next-frontier test-and-set at the queue flush
#endif
#ifndef GG_SPARSE_PER_SM
#define GG_SPARSE_PER_SM 2   // superstep CTAs per SM on low-degree graphs (see superstep_grid)
#endif
#ifndef GG_SPARSE_PER_SM_P
#define GG_SPARSE_PER_SM_P 1   // persistent kernel CTAs per SM on low-degree graphs (4096^2 grid: 96 ms at 1, 116 at 2, 232 at 5)
#endif
#ifndef GG_BODY_UNROLL
#define GG_BODY_UNROLL 8   // supersteps per iteration of the CUDA-graph loop (measured: 1 -> 8 saves
#endif                     // 12 % on RMAT-20, 6 % on RMAT-22, 23 % on the 4096^2 grid; 16 adds nothing)
#ifndef GG_PULL_WU
#define GG_PULL_WU 4   // 32-edge chunks per step of the heavy pull (gathers in flight per lane)
#endif
#ifndef GG_FAR_Q
#define GG_FAR_Q 1     // heavy pull: park far vertices through a per-warp queue
#endif
#ifndef GG_FAR_Q_SPLIT
#define GG_FAR_Q_SPLIT 0   // the same in the split step (measured: 2 % slower on the 4096^2 grid)
#endif
#ifndef GG_LH_TAIL
#define GG_LH_TAIL 1   // light/heavy: plain push once bucketing has ended
#endif
#ifndef GG_WARP_MIN_EDGES
#define GG_WARP_MIN_EDGES 32   // warp streaming: smallest edge share per warp (0: every warp takes a share)
#endif
#ifndef GG_CTA_FLUSH
#define GG_CTA_FLUSH 1   // warp streaming: the near queues left at the end go out in one append per CTA
#endif
#ifndef GG_PULL_SEGMIN
#define GG_PULL_SEGMIN 1   // heavy pull: per-owner minimum by a segmented shuffle scan (0: match + reduce)
#endif
#ifndef GG_WARP_BALLOT_OWNER
#define GG_WARP_BALLOT_OWNER 1   // warp streaming: each edge's window entry from one ballot and one OR-reduction
#endif                           // (0: a 5-step shuffle search)
#ifndef GG_EARLY_TAIL_DIV
#define GG_EARLY_TAIL_DIV 256   // a light frontier of at most n / this many vertices may end the buckets early (0: never)
#endif
#ifndef GG_PULL_TAIL
#define GG_PULL_TAIL 1   // a heavy pull after which bucketing ends writes the plain tail's frontier
#endif
#ifndef GG_LOCAL_ROUNDS
#define GG_LOCAL_ROUNDS 16   // warp-local rounds per superstep (load balance GG_LB_LOCAL; 4096^2 grid: 43 ms at 4, 36 at 8, 34 at 16)
#endif
#ifndef GG_LOCAL_MAX_DEG
#define GG_LOCAL_MAX_DEG 32   // vertices with more out-edges leave local rounds for the next frontier
#endif
#ifndef GG_LH_DRAIN
#define GG_LH_DRAIN 8    // light/heavy: bucketing ends once the unsettled vertices hold
#endif                   // fewer than m / GG_LH_DRAIN heavy edges

namespace gg {

namespace {

__device__ __forceinline__ uint32_t lanemask_le() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
  return m;
}

// push load-balancing schemes (template argument of the superstep kernels)
constexpr int LB_TILE = 0;   // merge-path tiles of BLOCK*EPT edges per CTA
constexpr int LB_BINS = 1;   // degree bins: thread / warp / CTA per vertex
constexpr int LB_WARP = 2;   // warp streaming over equal edge shares
constexpr int LB_LOCAL = 3;  // warp streaming, then warp-local rounds over the near vertices each warp improved

// resident CTAs per SM each superstep kernel is register-limited to
constexpr int superstep_min_blocks(int lb, int ept) {
  return (lb == LB_WARP || lb == LB_LOCAL) ? GG_WARP_MINB : ept == 2 ? 8 : ept == 4 ? 6 : 4;
}

template <int BLOCK, int EPT>
struct MPSmem {
  static constexpr int TILE = BLOCK * EPT;
  static constexpr int ECAP = TILE + 1;
  uint32_t es[ECAP];   // entry: first merge-path coordinate
  uint32_t eb[ECAP];   // push: CSR row start;   pull: vertex id
  uint32_t ec[ECAP];   // push: dist of source;  pull: running min candidate
  uint32_t qv[ECAP];   // filter output queue: near vertices from the front, far ones from the back
  uint32_t qr[ECAP];   //                      CSR row start (near)
  uint32_t qd[ECAP];   //                      out-degree (near; scanned in place)
  uint32_t wsum[BLOCK / 32];
  uint32_t qn;         // near entries
  uint32_t qfn;        // far entries
  uint32_t fmin;       // smallest distance sent to the far pile
  uint32_t j;
  uint32_t last;
  uint32_t ovf;
  unsigned long long base;
  uint32_t fbase;
  uint32_t ledges;     // edges relaxed in warp-local rounds or scanned by a heavy pull (statistics)
  uint32_t wq[BLOCK / 32][5];   // warp streaming, end flush: per warp (entries, edges) of both lists and the
                                //   far-queue length, then the bases
  uint16_t own[TILE];  // push: entry that owns each edge slot of the tile
};

struct StepArgs {
  DevGraph g;
  Frontier fr;
  Ctl* ctl;
  LhBufs lb;   // light/heavy buffers (valid in light/heavy runs): kernel parameters, so
               // the relaxation loop holds none of these pointers in registers
};

// Where the filter writes: the next (near) frontier and the far pile.
struct FilterOut {
  const uint32_t* ro;
  uint32_t sinks;                 // graph has sinks: check the out-degree before the dedup
  uint32_t* bm_next;
  uint32_t* bm_far;
  uint32_t t_cur;                 // near threshold
  unsigned long long* cnt_next;   // (count << 32) | edges of the next frontier
  uint32_t *nfv, *nfr, *nfs;
  uint32_t* far;                  // far pile being appended to
  uint32_t* far_cnt;              // its append position
  uint32_t* far_add;              // per-superstep count of far appends (or NULL)
  uint32_t wmode;                 // WM_*: how relaxations add edge weights
  // light/heavy buckets (lh != 0): a near vertex v joins the next frontier
  // with its light edges [ro[v], lend[v]) and, once per epoch, the R list
  // R[lh - 1] with its heavy edges [lend[v], ro[v+1]); vertices without edges
  // of a kind are left out of that list
  uint32_t lh;
};

// Append of up to 32 near vertices, one per lane (have = lane holds one) to
// the next frontier (LHM: their light edges, plus their heavy edges to the R
// list of the epoch): one 64-bit atomicAdd per list returns the list position
// and the edge-prefix base of the warp's entries.  Vertices without edges of
// a kind are left out of that list.  to_frontier = false: the R list only
// (warp-local rounds expand the light edges themselves).
template <bool LHM>
__device__ __forceinline__ void append32(const StepArgs& a, const FilterOut& fo, bool have, uint32_t v,
                                         bool to_frontier = true) {
  const unsigned FULL = 0xFFFFFFFFu;
  const uint32_t lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t rj = fo.lh - 1u;
  uint32_t rs = 0, le = 0, re = 0;
  bool lgt = false, hvy = false;
  if (have) {
    rs = __ldg(fo.ro + v);
    re = __ldg(fo.ro + v + 1);
    le = LHM ? __ldg(a.lb.lend + v) : re;
    lgt = le > rs;
    if (LHM && re > le) {
      const uint32_t bit = 1u << (v & 31);
      hvy = !(atomicOr(pick2(a.lb.bm_r, rj) + (v >> 5), bit) & bit);
    }
  }
#pragma unroll
  for (int list = 0; list < (LHM ? 2 : 1); ++list) {
    const bool mine = list == 0 ? (lgt && to_frontier) : hvy;
    const unsigned b = __ballot_sync(FULL, mine);
    if (b == 0u) continue;   // warp-uniform
    const uint32_t d = mine ? (list == 0 ? le - rs : re - le) : 0u;
    uint32_t x = d;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    const uint32_t tot = __shfl_sync(FULL, x, 31);
    unsigned long long base = 0;
    if (lane == 0)
      base = atomicAdd(list == 0 ? fo.cnt_next : &a.ctl->rcnt[rj], ((unsigned long long)__popc(b) << 32) | tot);
    base = __shfl_sync(FULL, base, 0);
    if (mine) {
      const uint32_t pos = (uint32_t)(base >> 32) + __popc(b & lt);
      const uint32_t coord = (uint32_t)base + x - d;
      if (list == 0) {
        fo.nfv[pos] = v;
        fo.nfr[pos] = rs;
        fo.nfs[pos] = coord;
      } else {
        pick2(a.lb.rv, rj)[pos] = v;
        pick2(a.lb.rr, rj)[pos] = le;
        pick2(a.lb.rs, rj)[pos] = coord;
      }
    }
  }
}

// Filter: vertex v whose distance just dropped to nd.  Vertices without
// out-edges have nothing to expand and are skipped.  nd < t_cur: the next
// frontier (once, by test-and-set on its bitmap); otherwise the far pile
// (once, by its own bitmap).
template <int BLOCK, int EPT>
__device__ __forceinline__ void filter_candidate(MPSmem<BLOCK, EPT>& sm, const FilterOut& fo, uint32_t v,
                                                 uint32_t nd) {
  if (!fo.sinks) {
    // every reached vertex has out-edges: dedup first, read the row at flush time
    const uint32_t bit = 1u << (v & 31);
    if (nd < fo.t_cur) {
      if (!(atomicOr(fo.bm_next + (v >> 5), bit) & bit)) {
        const uint32_t q = atomicAdd(&sm.qn, 1u);
        sm.qv[q] = v;
        sm.qd[q] = kInf;   // row read in filter_flush
      }
    } else {
      atomicMin(&sm.fmin, nd);
      if (!(atomicOr(fo.bm_far + (v >> 5), bit) & bit)) {
        const uint32_t q = MPSmem<BLOCK, EPT>::ECAP - 1 - atomicAdd(&sm.qfn, 1u);
        sm.qv[q] = v;
      }
    }
    return;
  }
  const uint32_t rs = __ldg(fo.ro + v), re = __ldg(fo.ro + v + 1);
  if (re > rs) {
    const uint32_t bit = 1u << (v & 31);
    if (nd < fo.t_cur) {
      if (!(atomicOr(fo.bm_next + (v >> 5), bit) & bit)) {
        const uint32_t q = atomicAdd(&sm.qn, 1u);
        sm.qv[q] = v;
        sm.qr[q] = rs;
        sm.qd[q] = re - rs;
      }
    } else {
      atomicMin(&sm.fmin, nd);
      if (!(atomicOr(fo.bm_far + (v >> 5), bit) & bit)) {
        const uint32_t q = MPSmem<BLOCK, EPT>::ECAP - 1 - atomicAdd(&sm.qfn, 1u);
        sm.qv[q] = v;
      }
    }
  }
}

// Append the CTA's collected vertices to the next frontier (one 64-bit
// atomicAdd returns queue position and edge-prefix base) and to the far pile.
// TRAIL: end with a barrier.  Callers whose next step writes the queue
// without an intervening barrier need it; the merge-path tile loop does not
// (its next tile's staging barrier comes first).
template <int BLOCK, int EPT, bool TRAIL = true>
__device__ __forceinline__ void filter_flush(MPSmem<BLOCK, EPT>& sm, const StepArgs& a, const FilterOut& fo) {
  constexpr uint32_t ECAP = MPSmem<BLOCK, EPT>::ECAP;
  __syncthreads();
  const uint32_t qn = sm.qn, qfn = sm.qfn;
  if (qn == 0 && qfn == 0) return;   // uniform
  if (fo.lh) {
    // every warp appends 32-entry chunks of the near queue to both lists
    for (uint32_t c0 = threadIdx.x & ~31u; c0 < qn; c0 += BLOCK) {
      const uint32_t i = c0 + (threadIdx.x & 31);
      append32<true>(a, fo, i < qn, i < qn ? sm.qv[i] : 0u);
    }
    if (qfn && threadIdx.x == 0) {
      sm.fbase = atomicAdd(fo.far_cnt, qfn);
      if (fo.far_add) atomicAdd(fo.far_add, qfn);
    }
    __syncthreads();
    const uint32_t fb = sm.fbase;
    if (threadIdx.x == 0) {   // every thread has read the counts by now
      sm.qn = 0;
      sm.qfn = 0;
    }
    for (uint32_t i = threadIdx.x; i < qfn; i += BLOCK) fo.far[fb + i] = sm.qv[ECAP - 1 - i];
    if (TRAIL) __syncthreads();
    return;
  }
  if (qn && !fo.sinks) {
    for (uint32_t i = threadIdx.x; i < qn; i += BLOCK) {
      const uint32_t v = sm.qv[i];
      const uint32_t rs = __ldg(fo.ro + v);
      sm.qr[i] = rs;
      sm.qd[i] = __ldg(fo.ro + v + 1) - rs;
    }
    __syncthreads();
  }
  if (qn) {
    const uint32_t tot = block_scan_excl<BLOCK>(sm.qd, qn, sm.wsum);
    if (threadIdx.x == 0) sm.base = atomicAdd(fo.cnt_next, ((unsigned long long)qn << 32) | tot);
  }
  if (qfn && threadIdx.x == 0) {
    sm.fbase = atomicAdd(fo.far_cnt, qfn);
    if (fo.far_add) atomicAdd(fo.far_add, qfn);
  }
  __syncthreads();
  const unsigned long long b = sm.base;
  const uint32_t pos0 = (uint32_t)(b >> 32), eb0 = (uint32_t)b;
  const uint32_t fb = sm.fbase;
  if (threadIdx.x == 0) {   // every thread has read the counts by now
    sm.qn = 0;
    sm.qfn = 0;
  }
  for (uint32_t i = threadIdx.x; i < qn; i += BLOCK) {
    fo.nfv[pos0 + i] = sm.qv[i];
    fo.nfr[pos0 + i] = sm.qr[i];
    fo.nfs[pos0 + i] = eb0 + sm.qd[i];
  }
  for (uint32_t i = threadIdx.x; i < qfn; i += BLOCK) fo.far[fb + i] = sm.qv[ECAP - 1 - i];
  if (TRAIL) __syncthreads();
}

// Merge-path advance over entries (S strictly increasing edge coordinates,
// F entries, Etot edges), fused with the filter.  CTA b takes the edge range
// [split(b), split(b+1)), split rounded down to 32 edges so that in pull
// (where the coordinate is the edge index itself) every thread's 8-edge run
// is one aligned vector load.
template <int BLOCK, int EPT, bool PULL, bool PK>
__device__ __forceinline__ void mp_advance(MPSmem<BLOCK, EPT>& sm, const StepArgs& a, uint32_t F, uint32_t Etot,
                                           const uint32_t* __restrict__ S, const uint32_t* __restrict__ B,
                                           const uint32_t* __restrict__ V, const void* __restrict__ edges,
                                           uint32_t* __restrict__ dist, uint32_t* __restrict__ bm_cur,
                                           const FilterOut& fo) {
  static_assert(!PULL || EPT == 2 || EPT == 4 || EPT == 8, "pull uses 2-, 4- or 8-edge vector runs");
  constexpr uint32_t TILE = MPSmem<BLOCK, EPT>::TILE;
  const uint32_t tid = threadIdx.x;
  const uint32_t G = gridDim.x;
  const uint32_t wbits = a.g.wbits;
  const uint32_t e0 = (uint32_t)(((unsigned long long)blockIdx.x * Etot) / G) & ~31u;
  const uint32_t e1 =
      blockIdx.x + 1 == G ? Etot : (uint32_t)(((unsigned long long)(blockIdx.x + 1) * Etot) / G) & ~31u;
  if (e0 >= e1) return;   // uniform per CTA
  if (tid < 32) {
    const uint32_t j = warp_search_le(S, F, e0);
    if (tid == 0) sm.j = j;
  }
  __syncthreads();
  uint32_t j = sm.j;
  bool ovf = false;
  for (uint32_t t0 = e0; t0 < e1; t0 += TILE) {
    const uint32_t t1 = min(t0 + TILE, e1);
    // stage the entries overlapping [t0, t1)
    uint32_t nent = 0;
    if (!PULL) {
#pragma unroll
      for (int k = 0; k < EPT; ++k) sm.own[k * BLOCK + tid] = 0;   // the owner marks of this tile
    }
    for (;;) {
      const uint32_t idx = j + nent + tid;
      bool valid = false;
      uint32_t s = 0;
      uint32_t ev = 0, eb = 0;
      if (idx < F) {
        // all three loads issue together; the range test waits only for S
        s = S[idx];
        ev = V[idx];
        if (!PULL) eb = B[idx];
        valid = s < t1;
      }
      if (valid) {
        const uint32_t slot = nent + tid;
        sm.es[slot] = s;
        if (!PULL) {
          sm.eb[slot] = eb;
          sm.ec[slot] = ld_cg(dist + ev);
          bm_cur[ev >> 5] = 0u;   // the current bitmap is not read in push: clear as we go
        } else {
          sm.eb[slot] = ev;
          sm.ec[slot] = kInf;
        }
      }
      const int c = __syncthreads_count(valid);
      nent += (uint32_t)c;
      if (c < BLOCK) break;
    }
    if (!PULL) {
      // push: consecutive threads take consecutive edge coordinates (coalesced
      // rows).  Owner map instead of a per-edge search: every entry after the
      // first marks the tile slot where its edges start, and an inclusive
      // prefix sum over the marks gives each slot its entry.
      const uint32_t len = t1 - t0;
      for (uint32_t jj = 1 + tid; jj < nent; jj += BLOCK) sm.own[sm.es[jj] - t0] = 1;
      __syncthreads();
      block_incl_scan_u16<BLOCK, EPT>(sm.own, sm.wsum);
      uint2 ed[EPT];
      uint32_t ej[EPT];
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const uint32_t o = k * BLOCK + tid;
        ej[k] = kInf;
        if (o < len) {
          const uint32_t jj = sm.own[o];
          ej[k] = jj;
          ed[k] = load_edge<PK>(edges, sm.eb[jj] + (t0 + o - sm.es[jj]), wbits);
        }
      }
      uint32_t nd[EPT], cur[EPT];
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        if (ej[k] != kInf) {
          nd[k] = relax_add(sm.ec[ej[k]], ed[k].y, ovf, fo.wmode);
          cur[k] = ld_cg(dist + ed[k].x);
        }
      }
      // nd < cur read just before: after the atomic dist[v] <= nd < cur, so v
      // improved in this superstep and belongs in the next frontier; the
      // atomic's old value is not needed (fire-and-forget reduction)
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        if (ej[k] != kInf && nd[k] < cur[k]) {
          atomicMin(dist + ed[k].x, nd[k]);
          filter_candidate(sm, fo, ed[k].x, nd[k]);
        }
      }
    } else {
      // pull: each thread owns an aligned run of 8 in-edges, keeps a running
      // minimum per destination row in a register and folds it into the
      // row's shared slot only when the row changes
      const uint32_t g0 = t0 + tid * EPT;
      if (g0 < t1) {
        uint32_t col[EPT], wt[EPT];
        if (g0 + EPT <= t1) {
          load_edges_run<PK, EPT>(edges, g0, wbits, col, wt);
        } else {
#pragma unroll
          for (int k = 0; k < EPT; ++k) {
            if (g0 + k < t1) {
              const uint2 ed = load_edge<PK>(edges, g0 + k, wbits);
              col[k] = ed.x;
              wt[k] = ed.y;
            }
          }
        }
        uint32_t jj = smem_upper_bound_minus1(sm.es, nent, g0);
        uint32_t nxt = jj + 1 < nent ? sm.es[jj + 1] : 0xFFFFFFFFu;
        uint32_t acc = kInf;
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          const uint32_t gidx = g0 + k;
          if (gidx < t1) {
            if (gidx >= nxt) {
              if (acc != kInf) atomicMin(&sm.ec[jj], acc);
              acc = kInf;
              do {
                ++jj;
                nxt = jj + 1 < nent ? sm.es[jj + 1] : 0xFFFFFFFFu;
              } while (gidx >= nxt);
            }
            const uint32_t u = col[k];
            if ((bm_cur[u >> 5] >> (u & 31)) & 1u) acc = min(acc, relax_add(dist[u], wt[k], ovf, fo.wmode));
          }
        }
        if (acc != kInf) atomicMin(&sm.ec[jj], acc);
      }
      __syncthreads();
      for (uint32_t i = tid; i < nent; i += BLOCK) {
        const uint32_t c = sm.ec[i];
        if (c != kInf) {
          const uint32_t v = sm.eb[i];
          if (c < ld_cg(dist + v)) {
            const uint32_t old = atomicMin(dist + v, c);
            if (c < old) filter_candidate(sm, fo, v, c);
          }
        }
      }
    }
    filter_flush<BLOCK, EPT, PULL>(sm, a, fo);   // push: the next staging barrier protects the queue
    j = j + nent - 1;
  }
  if (ovf) sm.ovf = 1u;
}

// Degree-binned push advance (thread / warp / CTA per vertex).  Each CTA
// takes chunks of BLOCK frontier vertices; vertices of degree >= cta_thr are
// expanded by the whole CTA one at a time, degree >= warp_thr by one warp,
// the rest by their own thread.  Every round relaxes at most BLOCK*EPT edges,
// then the filter queue is flushed, so the shared queue never overflows.
template <int BLOCK, int EPT, bool PK>
__device__ __forceinline__ void bins_advance(MPSmem<BLOCK, EPT>& sm, const StepArgs& a, uint32_t F, uint32_t Etot,
                                             const uint32_t* __restrict__ fv, const uint32_t* __restrict__ fr,
                                             const uint32_t* __restrict__ fs, uint32_t* __restrict__ dist,
                                             uint32_t* __restrict__ bm_cur, const FilterOut& fo,
                                             uint32_t warp_thr, uint32_t cta_thr, const void* __restrict__ edges) {
  constexpr uint32_t NW = BLOCK / 32;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t wbits = a.g.wbits;
  bool ovf = false;
  auto relax = [&](uint32_t e, uint32_t du) {
    const uint2 ed = load_edge<PK>(edges, e, wbits);
    const uint32_t nd = relax_add(du, ed.y, ovf, fo.wmode);
    if (nd < ld_cg(dist + ed.x)) {
      const uint32_t old = atomicMin(dist + ed.x, nd);
      if (nd < old) filter_candidate(sm, fo, ed.x, nd);
    }
  };
  const uint32_t nchunks = (F + BLOCK - 1) / BLOCK;
  for (uint32_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const uint32_t i = c * BLOCK + tid;
    uint32_t row = 0, deg = 0, du = 0;
    if (tid == 0) { sm.j = 0; sm.last = 0; }   // large / medium list lengths
    __syncthreads();
    if (i < F) {
      const uint32_t v = fv[i];
      row = fr[i];
      deg = (i + 1 < F ? fs[i + 1] : Etot) - fs[i];
      du = ld_cg(dist + v);
      bm_cur[v >> 5] = 0u;
      if (deg >= cta_thr) {
        const uint32_t k = atomicAdd(&sm.j, 1u);
        sm.es[k] = row; sm.eb[k] = deg; sm.ec[k] = du;
        deg = 0;
      } else if (deg >= warp_thr) {
        const uint32_t k = BLOCK + atomicAdd(&sm.last, 1u);
        sm.es[k] = row; sm.eb[k] = deg; sm.ec[k] = du;
        deg = 0;
      }
    }
    __syncthreads();
    const uint32_t nl = sm.j, nm = sm.last;
    // CTA per vertex
    for (uint32_t k = 0; k < nl; ++k) {
      const uint32_t r = sm.es[k], d = sm.eb[k], u = sm.ec[k];
      for (uint32_t base = 0; base < d; base += BLOCK * EPT) {
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
          const uint32_t o = base + q * BLOCK + tid;
          if (o < d) relax(r + o, u);
        }
        filter_flush(sm, a, fo);
      }
    }
    // warp per vertex
    uint32_t mi = warp, moff = 0;
    while (__syncthreads_or(mi < nm)) {
      if (mi < nm) {
        const uint32_t r = sm.es[BLOCK + mi], d = sm.eb[BLOCK + mi], u = sm.ec[BLOCK + mi];
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
          const uint32_t o = moff + q * 32 + lane;
          if (o < d) relax(r + o, u);
        }
        moff += 32 * EPT;
        if (moff >= d) { mi += NW; moff = 0; }
      }
      filter_flush(sm, a, fo);
    }
    // thread per vertex
    uint32_t off = 0;
    while (__syncthreads_or(off < deg)) {
#pragma unroll
      for (int q = 0; q < EPT; ++q)
        if (off + q < deg) relax(row + off + q, du);
      off += EPT;
      filter_flush(sm, a, fo);
    }
  }
  if (ovf) sm.ovf = 1u;
}

// Warp-streaming push advance, with no block barriers.  Every warp of the
// grid takes an equal contiguous share of the frontier's edge coordinates and
// walks it in chunks of 32 edges, up to WU chunks per step.  The frontier
// entries covering the current chunks sit in a sliding window of 32 entries,
// one per lane (first coordinate, row start, distance); a lane finds its
// edge's entry with a 5-step shuffle search over the window.  Improved
// vertices pass the filter's dedup into a per-warp shared-memory queue that is
// appended to the next frontier with one 64-bit atomicAdd per flush (queue
// position and edge-prefix base), like the CTA queue of the tile advance.
// LOCAL (load balance GG_LB_LOCAL; push supersteps other than the heavy
// one): near vertices a warp improves are not deduplicated into the next
// frontier but kept in a per-warp local queue, and after its share of the
// frontier the warp runs up to GG_LOCAL_ROUNDS local rounds over that queue:
// each queued vertex (read with its current distance) relaxes its out-edges,
// and the near vertices those improve form the next local queue.  Every
// relaxation that lowers a distance below the threshold queues the vertex (a
// queue entry per improvement, no bitmap), so a vertex is expanded after its
// last decrease.  What the rounds leave (and what overflows a queue, and rows
// longer than GG_LOCAL_MAX_DEG) goes to the next frontier through the bitmap
// as usual.  With light/heavy buckets the rounds expand light rows, and every
// queued vertex joins the epoch's R list once (by its R bitmap) as in the
// plain filter.  On a high-diameter graph this advances the wavefront several
// hops per superstep.
template <int BLOCK, int EPT, bool PK, bool LOCAL = false>
__device__ __forceinline__ void warp_advance(MPSmem<BLOCK, EPT>& sm, const StepArgs& a, uint32_t F, uint32_t Etot,
                                             const uint32_t* __restrict__ S, const uint32_t* __restrict__ R,
                                             const uint32_t* __restrict__ V, const void* __restrict__ edges,
                                             uint32_t* __restrict__ dist, uint32_t* __restrict__ bm_cur,
                                             const FilterOut& fo) {
  constexpr uint32_t NW = BLOCK / 32;
  constexpr uint32_t QW = 128;   // per-warp queue slots
  constexpr int WU = GG_WU;      // chunks of 32 edges per step
  static_assert(NW * QW <= (uint32_t)MPSmem<BLOCK, EPT>::ECAP, "per-warp queues fit the shared arrays");
  const unsigned FULL = 0xFFFFFFFFu;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  uint32_t* qv = sm.qv + warp * QW;   // near queue: vertex, row start, degree (then its prefix)
  uint32_t* qr = sm.qr + warp * QW;
  uint32_t* qd = sm.qd + warp * QW;
  uint32_t* fq = sm.es + warp * QW;   // far queue (the entry arrays are unused here)
  uint32_t qn = 0, fn = 0;            // warp-uniform queue lengths
  // LOCAL: two local queues of QL (vertex, distance it was queued with)
  // entries: vertices in [0, QL), distances in [QL, 2 QL) of the unused entry
  // arrays eb / ec; the near queue keeps the distance in qr
  constexpr uint32_t QL = QW / 2;
  uint32_t* const lqa = sm.eb + warp * QW;
  uint32_t* const lqb = sm.ec + warp * QW;
  uint32_t* lq_next = lqa;
  uint32_t lqn = 0;                   // warp-uniform: entries in lq_next
  // one entry per lane (have) into the next frontier: test-and-set, append the winners
  auto handoff_lane = [&](bool have, uint32_t v) {
    bool win = false;
    if (have) {
      const uint32_t bit = 1u << (v & 31);
      win = !(atomicOr(fo.bm_next + (v >> 5), bit) & bit);
    }
    if (fo.lh) append32<true>(a, fo, win, v);   // warp-uniform
    else append32<false>(a, fo, win, v);
  };
  uint32_t fmin = kInf;
  bool ovf = false;
  const uint32_t wbits = a.g.wbits;
  // equal edge shares of at least GG_WARP_MIN_EDGES: a small superstep runs
  // on fewer warps (spread one per CTA first), so fewer of them pay the
  // per-warp fixed work and the appends' counter atomics
  const unsigned long long Wall = (unsigned long long)gridDim.x * NW;
  // (not with local rounds, whose work grows with the warps that stream)
  constexpr uint32_t kMinShare = LOCAL ? 0u : (uint32_t)GG_WARP_MIN_EDGES;
  const unsigned long long Wneed = kMinShare > 0 ? ((unsigned long long)Etot + kMinShare - 1) / kMinShare : Wall;
  const bool reduced = Wneed < Wall;
  const unsigned long long W = reduced ? (Wneed > 0 ? Wneed : 1ull) : Wall;
  const unsigned long long gw = reduced ? (unsigned long long)warp * gridDim.x + blockIdx.x
                                        : (unsigned long long)blockIdx.x * NW + warp;
  const bool wact = gw < W;
  const uint32_t w0 = wact ? (uint32_t)((Etot * gw) / W) : 0u, w1 = wact ? (uint32_t)((Etot * (gw + 1)) / W) : 0u;

  // Near-queue appends with deferred dedup (sink-free graphs): collect
  // test-and-sets the next-frontier bitmap (and, with buckets, the epoch's R
  // bitmap) for the whole queue and reads the rows, all in flight together
  // (none waits on another: a vertex without heavy edges may set its R bit,
  // which only ever keeps it out of an R list it has nothing to bring to),
  // marks each entry's lists and returns the warp's entries and edges per
  // list; emit writes the marked entries from the given list positions and
  // edge bases.
  uint32_t* const qe = sm.eb + warp * QW;   // row end (the entry arrays are unused without local rounds)
  uint32_t* const qf = sm.ec + warp * QW;   // 1: the frontier (light or plain edges), 2: the R list
  auto near_collect = [&](uint32_t& nl, uint32_t& el, uint32_t& nh, uint32_t& eh) {
    static_assert(QW == 128, "four queue entries per lane");
    const bool lhm = fo.lh != 0u;
    const uint32_t rj = fo.lh - 1u;
    __syncwarp();
    uint32_t vq[4], rs[4], le[4], re[4];
    bool kp[4], hv[4];
    // the next-frontier and R test-and-sets and the row reads of the whole
    // queue, all in flight together (none waits on another: a vertex without
    // heavy edges may set its R bit, which only ever keeps it out of an R list
    // it has nothing to bring to)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint32_t i = 32u * c + lane;
      vq[c] = i < qn ? qv[i] : 0u;
      kp[c] = hv[c] = false;
      rs[c] = le[c] = re[c] = 0u;
      if (i < qn) {
        const uint32_t bit = 1u << (vq[c] & 31);
        kp[c] = !(atomicOr(fo.bm_next + (vq[c] >> 5), bit) & bit);
        if (lhm) hv[c] = !(atomicOr(pick2(a.lb.bm_r, rj) + (vq[c] >> 5), bit) & bit);
        rs[c] = __ldg(fo.ro + vq[c]);
        re[c] = __ldg(fo.ro + vq[c] + 1);
        le[c] = lhm ? __ldg(a.lb.lend + vq[c]) : re[c];
      }
    }
    nl = el = nh = eh = 0;   // warp totals
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint32_t i = 32u * c + lane;
      uint32_t fl = 0;
      if (kp[c] && le[c] > rs[c]) fl |= 1u;
      if (hv[c] && re[c] > le[c]) fl |= 2u;
      if (fl) {
        qr[i] = rs[c];
        qd[i] = le[c];
        qe[i] = re[c];
      }
      if (i < qn) qf[i] = fl;
      nl += __popc(__ballot_sync(FULL, fl & 1u));
      nh += __popc(__ballot_sync(FULL, (fl & 2u) != 0u));
      el += __reduce_add_sync(FULL, (fl & 1u) ? le[c] - rs[c] : 0u);
      eh += __reduce_add_sync(FULL, (fl & 2u) ? re[c] - le[c] : 0u);
    }
  };
  auto near_emit = [&](uint32_t pl, uint32_t ol, uint32_t ph, uint32_t oh) {
    const uint32_t rj = fo.lh - 1u;
    __syncwarp();
    for (uint32_t i0 = 0; i0 < qn; i0 += 32) {
      const uint32_t i = i0 + lane;
      const uint32_t fl = i < qn ? qf[i] : 0u;
      uint32_t v = 0, r0 = 0, r1 = 0, r2 = 0;
      if (fl) {
        v = qv[i];
        r0 = qr[i];
        r1 = qd[i];
        r2 = qe[i];
      }
#pragma unroll
      for (int list = 0; list < 2; ++list) {
        const bool mine = (fl & (list == 0 ? 1u : 2u)) != 0u;
        const unsigned mb = __ballot_sync(FULL, mine);
        if (mb == 0u) continue;   // warp-uniform
        const uint32_t d = mine ? (list == 0 ? r1 - r0 : r2 - r1) : 0u;
        uint32_t x = d;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(FULL, x, o);
          if (lane >= (uint32_t)o) x += y;
        }
        uint32_t& pp = list == 0 ? pl : ph;
        uint32_t& oo = list == 0 ? ol : oh;
        if (mine) {
          const uint32_t pos = pp + __popc(mb & lt);
          const uint32_t coord = oo + x - d;
          if (list == 0) {
            fo.nfv[pos] = v;
            fo.nfr[pos] = r0;
            fo.nfs[pos] = coord;
          } else {
            pick2(a.lb.rv, rj)[pos] = v;
            pick2(a.lb.rr, rj)[pos] = r1;
            pick2(a.lb.rs, rj)[pos] = coord;
          }
        }
        pp += __popc(mb);
        oo += __shfl_sync(FULL, x, 31);
      }
    }
    qn = 0;
    __syncwarp();
  };
  auto flush_near = [&]() {
    __syncwarp();
    if (LOCAL) {
      // light/heavy buckets: every near vertex joins the epoch's R list once
      // (its heavy edges wait for the heavy superstep); the light edges are
      // expanded by the local rounds or, after a hand-off, the next frontier
      if (fo.lh)
        for (uint32_t i0 = 0; i0 < qn; i0 += 32)
          append32<true>(a, fo, i0 + lane < qn, i0 + lane < qn ? qv[i0 + lane] : 0u, false);
      // into the local queue; what does not fit goes to the next frontier
      const uint32_t take = min(QL - lqn, qn);
      for (uint32_t i = lane; i < take; i += 32) {
        lq_next[lqn + i] = qv[i];
        lq_next[QL + lqn + i] = qr[i];
      }
      for (uint32_t i0 = take; i0 < qn; i0 += 32) handoff_lane(i0 + lane < qn, i0 + lane < qn ? qv[i0 + lane] : 0u);
      lqn += take;
      qn = 0;
      __syncwarp();
      return;
    }
    if (GG_DEFER_DEDUP && !fo.sinks) {
      // deferred dedup: the queue holds every improved near vertex (repeats
      // included); collect test-and-sets them all, then one counter atomic
      // per list places the warp's winners
      uint32_t nl, el, nh, eh;
      near_collect(nl, el, nh, eh);
      unsigned long long b0 = 0, b1 = 0;
      if (lane == 0) {
        if (nl) b0 = atomicAdd(fo.cnt_next, ((unsigned long long)nl << 32) | el);
        if (nh) b1 = atomicAdd(&a.ctl->rcnt[fo.lh - 1u], ((unsigned long long)nh << 32) | eh);
      }
      b0 = __shfl_sync(FULL, b0, 0);
      b1 = __shfl_sync(FULL, b1, 0);
      near_emit((uint32_t)(b0 >> 32), (uint32_t)b0, (uint32_t)(b1 >> 32), (uint32_t)b1);
      return;
    }
    if (fo.lh) {
      for (uint32_t i0 = 0; i0 < qn; i0 += 32) {
        const uint32_t i = i0 + lane;
        append32<true>(a, fo, i < qn, i < qn ? qv[i] : 0u);
      }
      qn = 0;
      __syncwarp();
      return;
    }
    uint32_t run = 0;
    for (uint32_t i0 = 0; i0 < qn; i0 += 32) {
      const uint32_t i = i0 + lane;
      uint32_t d = 0;
      if (i < qn) {
        if (!fo.sinks) {   // row read deferred to here
          const uint32_t v = qv[i];
          const uint32_t rs = __ldg(fo.ro + v);
          d = __ldg(fo.ro + v + 1) - rs;
          qr[i] = rs;
        } else {
          d = qd[i];
        }
      }
      uint32_t x = d;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= (uint32_t)o) x += y;
      }
      if (i < qn) qd[i] = run + x - d;
      run += __shfl_sync(FULL, x, 31);
    }
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(fo.cnt_next, ((unsigned long long)qn << 32) | run);
    b = __shfl_sync(FULL, b, 0);
    __syncwarp();
    const uint32_t pos0 = (uint32_t)(b >> 32), eb0 = (uint32_t)b;
    for (uint32_t i = lane; i < qn; i += 32) {
      fo.nfv[pos0 + i] = qv[i];
      fo.nfr[pos0 + i] = qr[i];
      fo.nfs[pos0 + i] = eb0 + qd[i];
    }
    qn = 0;
    __syncwarp();
  };
  // End flush for the whole CTA (deferred dedup only; CTA-uniform): every warp
  // test-and-sets its queued vertices and reads their rows, then one 64-bit
  // counter atomic per list and CTA places the winners of all warps, and one
  // more the far queues (per-warp flushes would make each of the grid's warps
  // hit the same counters).
  const bool cta_end = GG_CTA_FLUSH && !LOCAL && GG_DEFER_DEDUP && !fo.sinks;
  auto cta_flush = [&]() {
    uint32_t nl, el, nh, eh;
    near_collect(nl, el, nh, eh);
    const uint32_t rj = fo.lh - 1u;
    if (lane == 0) {
      sm.wq[warp][0] = nl;
      sm.wq[warp][1] = el;
      sm.wq[warp][2] = nh;
      sm.wq[warp][3] = eh;
      sm.wq[warp][4] = fn;
    }
    __syncthreads();
    if (threadIdx.x == 32) {   // the far pile (another warp than the lists' threads)
      uint32_t tot = 0;
      for (uint32_t w = 0; w < NW; ++w) tot += sm.wq[w][4];
      uint32_t b = 0;
      if (tot) {
        b = atomicAdd(fo.far_cnt, tot);
        if (fo.far_add) atomicAdd(fo.far_add, tot);
      }
      for (uint32_t w = 0; w < NW; ++w) {
        const uint32_t c = sm.wq[w][4];
        sm.wq[w][4] = b;
        b += c;
      }
    }
    if (threadIdx.x < 2) {   // thread t: list t (the frontier; the R list)
      const uint32_t t = threadIdx.x;
      uint32_t cn = 0, ce = 0;
      for (uint32_t w = 0; w < NW; ++w) {
        cn += sm.wq[w][2 * t];
        ce += sm.wq[w][2 * t + 1];
      }
      unsigned long long b = 0;
      if (cn) b = atomicAdd(t == 0 ? fo.cnt_next : &a.ctl->rcnt[rj], ((unsigned long long)cn << 32) | ce);
      uint32_t pn = (uint32_t)(b >> 32), pe = (uint32_t)b;
      for (uint32_t w = 0; w < NW; ++w) {   // exclusive prefix over the warps, in place
        const uint32_t n_w = sm.wq[w][2 * t], e_w = sm.wq[w][2 * t + 1];
        sm.wq[w][2 * t] = pn;
        sm.wq[w][2 * t + 1] = pe;
        pn += n_w;
        pe += e_w;
      }
    }
    __syncthreads();
    near_emit(sm.wq[warp][0], sm.wq[warp][1], sm.wq[warp][2], sm.wq[warp][3]);
    const uint32_t fb = sm.wq[warp][4];
    for (uint32_t i = lane; i < fn; i += 32) fo.far[fb + i] = fq[i];
    fn = 0;
  };
  auto flush_far = [&]() {
    __syncwarp();
    uint32_t b = 0;
    if (lane == 0) {
      b = atomicAdd(fo.far_cnt, fn);
      if (fo.far_add) atomicAdd(fo.far_add, fn);
    }
    b = __shfl_sync(FULL, b, 0);
    for (uint32_t i = lane; i < fn; i += 32) fo.far[b + i] = fq[i];
    fn = 0;
    __syncwarp();
  };

  if (w0 < w1) {   // warp-uniform
    uint32_t j = warp_search_le(S, F, w0);
    uint32_t ws = 0, wr = 0, wd = 0, wend = 0;
    auto load_window = [&]() {
      const uint32_t idx = j + lane;
      ws = 0xFFFFFFFFu;
      if (idx < F) {
        ws = S[idx];
        wr = R[idx];
        const uint32_t v = V[idx];
        wd = ld_cg(dist + v);
        // the current bitmap is not read in push: clear as we go (null: the
        // next superstep's prologue clears it whole, as in light/heavy runs)
        if (bm_cur != nullptr) bm_cur[v >> 5] = 0u;
      }
      wend = j + 32 < F ? S[j + 32] : Etot;   // first coordinate past the window
    };
    load_window();
    for (uint32_t b = w0; b < w1;) {
      // slide until the window holds chunk [b, b+32): S[j] <= b and the
      // chunk's last coordinate is below wend (at most two slides)
      for (int guard = 0; guard < 4 && min(b + 31, w1 - 1) >= wend; ++guard) {
        const unsigned le = __ballot_sync(FULL, ws <= b);
        if (le == 0u) break;   // cannot happen while S[j] <= b holds
        const uint32_t adv = (le == FULL && wend <= b) ? 32u : 31u - (uint32_t)__clz(le);
        j += adv;
        load_window();
      }
      // chunks [b + 32u, b + 32u + 32) that the window covers
      int nc = 1;
#pragma unroll
      for (int u = 1; u < WU; ++u)
        if (nc == u && b + 32u * u < w1 && min(b + 32u * u + 31u, w1 - 1) < wend) nc = u + 1;
      uint2 ed[WU];
      uint32_t nd[WU], cur[WU];
      bool act[WU];
#pragma unroll
      for (int u = 0; u < WU; ++u) {
        const uint32_t g = b + 32u * u + lane;
        act[u] = u < nc && g < w1;
        uint32_t k = 0;
        if (GG_WARP_BALLOT_OWNER) {
          // the chunk's first edge belongs to the last window entry starting at
          // or before it; each entry that starts later inside the chunk moves the
          // owner of the edges from its offset on by one (first coordinates
          // increase strictly: every entry has edges)
          const uint32_t cb = b + 32u * u;
          const unsigned le0 = __ballot_sync(FULL, ws <= cb);
          const uint32_t k0 = le0 ? 31u - (uint32_t)__clz(le0) : 0u;
          const uint32_t off = ws - cb;   // entries before the chunk wrap to large values
          const uint32_t starts = __reduce_or_sync(FULL, off - 1u < 31u ? 1u << off : 0u);
          k = k0 + (uint32_t)__popc(starts & lanemask_le());
        } else {
#pragma unroll
          for (int step = 16; step; step >>= 1) {
            const uint32_t sv = __shfl_sync(FULL, ws, k + step);
            if (sv <= g) k += step;
          }
        }
        const uint32_t ks = __shfl_sync(FULL, ws, k);
        const uint32_t kr = __shfl_sync(FULL, wr, k);
        const uint32_t kd = __shfl_sync(FULL, wd, k);
        const uint32_t kn = __shfl_sync(FULL, ws, (k + 1) & 31u);
        // the entry's range [ks, ke) holds g whenever S increases strictly; the
        // test keeps every edge read inside the entry's row regardless
        const uint32_t ke = k == 31 ? wend : kn;
        act[u] = act[u] && ks <= g && g < ke;
        nd[u] = kd;
        if (act[u]) ed[u] = load_edge<PK>(edges, kr + (g - ks), wbits);
      }
#pragma unroll
      for (int u = 0; u < WU; ++u) {
        if (act[u]) {
          nd[u] = relax_add(nd[u], ed[u].y, ovf, fo.wmode);
          cur[u] = ld_cg(dist + ed[u].x);
        }
      }
#pragma unroll
      for (int u = 0; u < WU; ++u) {
        bool near = false, far = false;
        uint32_t rs = 0, deg = 0;
        const uint32_t v = ed[u].x;
        if (act[u] && nd[u] < cur[u]) {
          // dist[v] <= nd < cur after the atomic: v improved this superstep
          atomicMin(dist + v, nd[u]);
          bool ok = true;
          if (fo.sinks) {
            rs = __ldg(fo.ro + v);
            deg = __ldg(fo.ro + v + 1) - rs;
            ok = deg > 0;
          }
          if (ok) {
            const uint32_t bit = 1u << (v & 31);
            if (nd[u] < fo.t_cur) {
              // with deferred dedup the bitmap is tested at the flush
              near = (LOCAL || (GG_DEFER_DEDUP && !fo.sinks)) ? true : !(atomicOr(fo.bm_next + (v >> 5), bit) & bit);
            } else {
              fmin = min(fmin, nd[u]);
              far = !(atomicOr(fo.bm_far + (v >> 5), bit) & bit);
            }
          }
        }
        const unsigned nb = __ballot_sync(FULL, near);
        if (nb) {
          if (near) {
            const uint32_t off = qn + __popc(nb & lt);
            qv[off] = v;
            qr[off] = LOCAL ? nd[u] : rs;   // LOCAL: the distance v is queued with
            qd[off] = deg;
          }
          qn += __popc(nb);
          if (qn > QW - 32) flush_near();
        }
        const unsigned fb = __ballot_sync(FULL, far);
        if (fb) {
          if (far) fq[fn + __popc(fb & lt)] = v;
          fn += __popc(fb);
          if (fn > QW - 32) flush_far();
        }
      }
      b += 32u * nc;
    }
    if (qn && !cta_end) flush_near();
    if (fn && !cta_end) flush_far();
  }
  if (cta_end) cta_flush();
  if (LOCAL) {
    uint32_t ledges = 0;   // warp-uniform
    for (int r = 0; r < GG_LOCAL_ROUNDS && lqn > 0; ++r) {   // warp-uniform
      uint32_t* const cur = lq_next;
      const uint32_t ncur = lqn;
      lq_next = cur == lqa ? lqb : lqa;
      lqn = 0;
      __syncwarp();
      for (uint32_t i0 = 0; i0 < ncur; i0 += 32) {   // warp-uniform
        const uint32_t i = i0 + lane;
        uint32_t v = 0, du = 0, rs = 0, deg = 0;
        if (i < ncur) {
          v = cur[i];
          du = ld_cg(dist + v);
          rs = __ldg(fo.ro + v);
          deg = (fo.lh ? __ldg(a.lb.lend + v) : __ldg(fo.ro + v + 1)) - rs;   // light/heavy: light row
          // a later improvement queued v again with a smaller distance: that
          // entry expands it, this one is stale
          if (du < cur[QL + i]) deg = 0;
        }
        const bool big = deg > GG_LOCAL_MAX_DEG;   // long rows: the next frontier's balanced advance
        if (__any_sync(FULL, big)) handoff_lane(big, v);
        if (big) deg = 0;
        const uint32_t dmax = __reduce_max_sync(FULL, deg);
        ledges += __reduce_add_sync(FULL, deg);
        for (uint32_t k = 0; k < dmax; k += 4) {   // warp-uniform; four edges per lane in flight
          uint2 ed[4];
          uint32_t nd[4], cv[4];
          bool act[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            act[q] = k + q < deg;
            if (act[q]) ed[q] = load_edge<PK>(edges, rs + k + q, wbits);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (act[q]) {
              nd[q] = relax_add(du, ed[q].y, ovf, fo.wmode);
              cv[q] = ld_cg(dist + ed[q].x);
            }
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            bool near = false, far = false;
            const uint32_t t = ed[q].x;
            if (act[q] && nd[q] < cv[q]) {
              atomicMin(dist + t, nd[q]);
              bool ok = true;
              if (fo.sinks) ok = __ldg(fo.ro + t + 1) > __ldg(fo.ro + t);
              if (ok) {
                if (nd[q] < fo.t_cur) {
                  near = true;
                } else {
                  const uint32_t bit = 1u << (t & 31);
                  fmin = min(fmin, nd[q]);
                  far = !(atomicOr(fo.bm_far + (t >> 5), bit) & bit);
                }
              }
            }
            const unsigned nb = __ballot_sync(FULL, near);
            if (nb) {
              if (near) {
                qv[qn + __popc(nb & lt)] = t;
                qr[qn + __popc(nb & lt)] = nd[q];
              }
              qn += __popc(nb);
              if (qn > QW - 32) flush_near();
            }
            const unsigned fb = __ballot_sync(FULL, far);
            if (fb) {
              if (far) fq[fn + __popc(fb & lt)] = t;
              fn += __popc(fb);
              if (fn > QW - 32) flush_far();
            }
          }
        }
      }
      if (qn) flush_near();
      if (fn) flush_far();
    }
    __syncwarp();
    for (uint32_t i0 = 0; i0 < lqn; i0 += 32)   // what the rounds leave: the next frontier
      handoff_lane(i0 + lane < lqn, i0 + lane < lqn ? lq_next[i0 + lane] : 0u);
    lqn = 0;
    if (lane == 0 && ledges) atomicAdd(&sm.ledges, ledges);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) fmin = min(fmin, __shfl_xor_sync(FULL, fmin, o));
  if (lane == 0 && fmin != kInf) atomicMin(&sm.fmin, fmin);
  if (__any_sync(FULL, ovf) && lane == 0) sm.ovf = 1u;
}

// Per-warp far queue: parked vertices gather in shared memory and reach the
// far pile in runs of up to kFarQ, one counter atomic per run instead of one
// per 32 entries (every warp of the grid appends to the same counter).
constexpr uint32_t kFarQ = 128;

__device__ __forceinline__ void far_q_flush(uint32_t* fq, uint32_t& fn, const FilterOut& fo) {
  const uint32_t lane = threadIdx.x & 31;
  __syncwarp();
  uint32_t b = 0;
  if (lane == 0) {
    b = atomicAdd(fo.far_cnt, fn);
    if (fo.far_add) atomicAdd(fo.far_add, fn);
  }
  b = __shfl_sync(0xFFFFFFFFu, b, 0);
  for (uint32_t i = lane; i < fn; i += 32) fo.far[b + i] = fq[i];
  fn = 0;
  __syncwarp();
}

// Appends the lanes with `mine` set (ballot `mb`, non-zero) to the queue.
__device__ __forceinline__ void far_q_push(uint32_t* fq, uint32_t& fn, const FilterOut& fo, bool mine, uint32_t v,
                                           unsigned mb) {
  const uint32_t lane = threadIdx.x & 31;
  if (mine) fq[fn + __popc(mb & ((1u << lane) - 1u))] = v;
  fn += __popc(mb);
  if (fn > kFarQ - 32) far_q_flush(fq, fn, fo);
}

// Split step of the near-far frontier, run when the near frontier is empty:
// every far-pile vertex v is re-examined against the raised threshold.
//   dist[v] <  t_prev  it was improved below the old threshold after it was
//                      parked, so the near phase already expanded it: drop
//   dist[v] <  t_cur   move it to the next (near) frontier
//   otherwise          keep it in the other far pile
// Warp-level: 32 entries per step, one append per warp and list, no CTA barriers.
template <int BLOCK, int EPT>
__device__ __forceinline__ void far_split(MPSmem<BLOCK, EPT>& sm, const StepArgs& a, const FilterOut& fo,
                                          uint32_t* __restrict__ dist, const uint32_t* __restrict__ far_in,
                                          uint32_t nfar, uint32_t t_prev) {
  const unsigned FULL = 0xFFFFFFFFu;
  const uint32_t lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t W = gridDim.x * (BLOCK / 32);
  uint32_t fmin = kInf;
  static_assert((BLOCK / 32) * kFarQ <= (uint32_t)MPSmem<BLOCK, EPT>::ECAP, "per-warp far queues fit");
  uint32_t* fq = sm.es + (threadIdx.x >> 5) * kFarQ;   // per-warp far queue
  uint32_t fn = 0;
  for (uint32_t base = (blockIdx.x * (BLOCK / 32) + (threadIdx.x >> 5)) * 32u; base < nfar; base += W * 32u) {
    const uint32_t i = base + lane;
    uint32_t v = 0;
    bool near = false, keep = false;
    if (i < nfar) {
      v = far_in[i];
      const uint32_t d = ld_cg(dist + v);
      const uint32_t bit = 1u << (v & 31);
      if (d < fo.t_cur) {
        // once the threshold is infinite nothing is parked again: the far
        // bits no longer matter
        if (fo.t_cur != kInf) atomicAnd(fo.bm_far + (v >> 5), ~bit);
        // a split step relaxes nothing and the pile holds each vertex once,
        // so its near vertices need no dedup; they still enter the bitmap,
        // which a pull superstep reads as the frontier (no result: no wait)
        near = d >= t_prev;
        if (near) atomicOr(fo.bm_next + (v >> 5), bit);
      } else {
        keep = true;   // its far bit stays set
        fmin = min(fmin, d);
      }
    }
    const unsigned kb = __ballot_sync(FULL, keep);
    if (GG_FAR_Q_SPLIT) {
      if (kb) far_q_push(fq, fn, fo, keep, v, kb);
    } else if (kb) {
      uint32_t b = 0;
      if (lane == 0) {
        b = atomicAdd(fo.far_cnt, (uint32_t)__popc(kb));
        if (fo.far_add) atomicAdd(fo.far_add, (uint32_t)__popc(kb));
      }
      b = __shfl_sync(FULL, b, 0);
      if (keep) fo.far[b + __popc(kb & lt)] = v;
    }
    if (__any_sync(FULL, near)) {
      if (fo.lh) append32<true>(a, fo, near, v);
      else append32<false>(a, fo, near, v);
    }
  }
  if (GG_FAR_Q_SPLIT && fn) far_q_flush(fq, fn, fo);
#pragma unroll
  for (int o = 16; o; o >>= 1) fmin = min(fmin, __shfl_xor_sync(FULL, fmin, o));
  if (lane == 0 && fmin != kInf) atomicMin(&sm.fmin, fmin);
}

// Heavy superstep by pull (symmetric graphs, bucket no wider than delta).
// Every vertex v not yet settled (dist[v] >= t_cur) takes the minimum of
// dist[u] + w over its heavy edges (u, w) from settled vertices
// (dist[u] < t_cur); in a symmetric graph these are exactly the heavy edges
// into v.  Heavy edges of vertices settled in earlier buckets were relaxed
// then and cannot improve v again, so the minimum covers the heavy edges of
// the current R list, and every improvement is >= t_cur (far pile).  A warp
// takes 32 consecutive vertices and walks their heavy edges as one list, 32
// edges per step; each v is written by its own lane only (no atomics on
// dist).  Chosen over the push form when R's heavy edges outnumber those of
// the unsettled vertices (the dense core settles first on skewed graphs).
// TAIL: bucketing ends after this step (threshold infinite, plain push over
// all edges).  The unsettled vertices with a finite distance are then exactly
// the vertices the split would move from the far pile into the frontier, so
// they go straight to the next frontier (all edges of their rows, through a
// per-warp queue) and the split step is skipped.
template <int BLOCK, int EPT, bool PK, bool TAIL>
__device__ __forceinline__ void heavy_pull(MPSmem<BLOCK, EPT>& sm, const StepArgs& a, const FilterOut& fo,
                                           uint32_t* __restrict__ dist, uint32_t* __restrict__ bm_r_old,
                                           const uint32_t* __restrict__ lfv, uint32_t lf) {
  const unsigned FULL = 0xFFFFFFFFu;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t t_cur = fo.t_cur, wbits = a.g.wbits;
  const void* __restrict__ edges = a.lb.edges;
  const uint32_t* __restrict__ lend = a.lb.lend;
  uint32_t* wbest = sm.ec + warp * 32;
  static_assert((BLOCK / 32) * kFarQ <= (uint32_t)MPSmem<BLOCK, EPT>::ECAP, "per-warp far queues fit");
  uint32_t* fq = sm.es + warp * kFarQ;   // per-warp far queue
  uint32_t fn = 0;
  // TAIL: per-warp queue of next-frontier entries (vertex, row start, degree
  // and then its prefix), one counter atomic per run of up to kTailQ
  constexpr uint32_t kTailQ = 128;
  static_assert((BLOCK / 32) * kTailQ <= (uint32_t)MPSmem<BLOCK, EPT>::ECAP, "per-warp tail queues fit");
  uint32_t* tqv = sm.qv + warp * kTailQ;
  uint32_t* tqr = sm.qr + warp * kTailQ;
  uint32_t* tqd = sm.qd + warp * kTailQ;
  uint32_t tqn = 0;   // warp-uniform
  auto tail_flush = [&]() {
    __syncwarp();
    uint32_t run = 0;
    for (uint32_t i0 = 0; i0 < tqn; i0 += 32) {
      const uint32_t i = i0 + lane;
      const uint32_t d = i < tqn ? tqd[i] : 0u;
      uint32_t x = d;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= (uint32_t)o) x += y;
      }
      if (i < tqn) tqd[i] = run + x - d;
      run += __shfl_sync(FULL, x, 31);
    }
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(fo.cnt_next, ((unsigned long long)tqn << 32) | run);
    b = __shfl_sync(FULL, b, 0);
    __syncwarp();
    const uint32_t pos0 = (uint32_t)(b >> 32), eb0 = (uint32_t)b;
    for (uint32_t i = lane; i < tqn; i += 32) {
      fo.nfv[pos0 + i] = tqv[i];
      fo.nfr[pos0 + i] = tqr[i];
      fo.nfs[pos0 + i] = eb0 + tqd[i];
    }
    tqn = 0;
    __syncwarp();
  };
  // the consumed R list is not read: clear its membership bitmap outright
  for (uint32_t i = blockIdx.x * BLOCK + threadIdx.x; i < a.g.nwords; i += gridDim.x * BLOCK) bm_r_old[i] = 0u;
  const uint32_t W = gridDim.x * (BLOCK / 32);
  uint32_t fmin = kInf;
  unsigned long long scanned = 0;
  bool ovf = false;
  // the vertices with edges, in id order (the pull list; isolated vertices,
  // 40 % of an RMAT graph, have nothing to pull)
  const uint32_t np = a.g.np;
  const uint32_t* __restrict__ pv = a.g.pv;
  // the next group's vertex and distance are read while this one is worked on
  uint32_t base = (blockIdx.x * (BLOCK / 32) + warp) * 32u;
  uint32_t nv = base + lane < np ? __ldg(pv + base + lane) : 0u;
  uint32_t ndv = base + lane < np ? ld_cg(dist + nv) : 0u;
  for (; base < np; base += W * 32u) {
    const bool have = base + lane < np;
    const uint32_t v = nv;
    uint32_t dv = ndv, hs = 0, deg = 0, rsv = 0;
    if (have && dv >= t_cur) {
      hs = __ldg(lend + v);
      deg = __ldg(fo.ro + v + 1) - hs;
      if (TAIL) rsv = __ldg(fo.ro + v);   // the row start a join needs
    }
    {
      const uint32_t nb = base + W * 32u + lane;
      nv = nb < np ? __ldg(pv + nb) : 0u;
      if (nb < np) ndv = ld_cg(dist + nv);
    }
    uint32_t x = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    const uint32_t T = __shfl_sync(FULL, x, 31);
    if (!TAIL && T == 0) continue;   // warp-uniform
    const uint32_t ex = x - deg;   // first list position of this lane's edges
    wbest[lane] = kInf;
    __syncwarp();
    constexpr int PU = GG_PULL_WU;
    for (uint32_t c = 0; c < T; c += 32u * PU) {
      // PU chunks per step: their edge loads, then their distance gathers, in flight together
      uint32_t k[PU];
      uint2 ed[PU];
#pragma unroll
      for (int u = 0; u < PU; ++u) {
        const uint32_t j = c + 32u * u + lane;
        // owner: the last lane whose first position is <= j (lanes without edges
        // share their successor's position and come before it)
        k[u] = 0;
#pragma unroll
        for (int step = 16; step; step >>= 1) {
          const uint32_t sv = __shfl_sync(FULL, ex, k[u] + step);
          if (sv <= j) k[u] += step;
        }
        const uint32_t ks = __shfl_sync(FULL, hs, k[u]), kx = __shfl_sync(FULL, ex, k[u]);
        if (j < T) ed[u] = load_edge<PK>(edges, ks + (j - kx), wbits);
      }
      uint32_t cand[PU];
#pragma unroll
      for (int u = 0; u < PU; ++u) {
        cand[u] = kInf;
        if (c + 32u * u + lane < T) {
          const uint32_t du = ld_cg(dist + ed[u].x);
          if (du < t_cur) cand[u] = add_sat(du, ed[u].y, ovf);
        }
      }
#pragma unroll
      for (int u = 0; u < PU; ++u) {
        if (u == 0 || c + 32u * u < T) {   // warp-uniform
          if (GG_PULL_SEGMIN) {
            // owners are non-decreasing over the lanes: a segmented minimum by
            // shuffles leaves each owner's minimum in its first lane
            uint32_t r = cand[u];
            const uint32_t kk = k[u];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const uint32_t rd = __shfl_down_sync(FULL, r, o);
              const uint32_t kd = __shfl_down_sync(FULL, kk, o);
              if (lane + (uint32_t)o < 32u && kd == kk) r = min(r, rd);
            }
            const uint32_t kp = __shfl_up_sync(FULL, kk, 1);
            if (r != kInf && (lane == 0 || kp != kk)) atomicMin(&wbest[kk], r);
          } else {
            const unsigned same = __match_any_sync(FULL, k[u]);
            const uint32_t r = __reduce_min_sync(same, cand[u]);
            if (r != kInf && lane == (uint32_t)(__ffs(same) - 1)) atomicMin(&wbest[k[u]], r);
          }
        }
      }
    }
    __syncwarp();
    const uint32_t best = wbest[lane];
    if (TAIL) {
      bool join = false;
      uint32_t rs = 0, full = 0;
      if (have && dv >= t_cur) {
        if (best < dv) dist[v] = best;
        if (min(best, dv) != kInf) {
          rs = rsv;
          full = hs + deg - rs;   // the whole row: [ro[v], ro[v+1])
          join = full > 0;
        }
      }
      const unsigned jb = __ballot_sync(FULL, join);
      if (jb) {   // warp-uniform
        if (join) {
          const uint32_t off = tqn + __popc(jb & lt);
          tqv[off] = v;
          tqr[off] = rs;
          tqd[off] = full;
        }
        tqn += __popc(jb);
        if (tqn > kTailQ - 32) tail_flush();
      }
      scanned += T;
      __syncwarp();
      continue;
    }
    bool far = false;
    if (have && best < dv) {
      dist[v] = best;
      fmin = min(fmin, best);
      const uint32_t bit = 1u << (v & 31);
      far = !(atomicOr(fo.bm_far + (v >> 5), bit) & bit);
    }
    const unsigned fb = __ballot_sync(FULL, far);
    if (GG_FAR_Q) {
      if (fb) far_q_push(fq, fn, fo, far, v, fb);
    } else if (fb) {
      uint32_t b = 0;
      if (lane == 0) b = atomicAdd(fo.far_cnt, (uint32_t)__popc(fb));
      b = __shfl_sync(FULL, b, 0);
      if (far) fo.far[b + __popc(fb & lt)] = v;
    }
    scanned += T;
    __syncwarp();
  }
  if (TAIL) {
    // the light frontier of a pull that ends the buckets early (its vertices
    // are below the threshold, so the loop above did not take them): whole rows
    for (uint32_t b0 = (blockIdx.x * (BLOCK / 32) + warp) * 32u; b0 < lf; b0 += W * 32u) {
      const uint32_t i = b0 + lane;
      uint32_t v = 0, rs = 0, full = 0;
      if (i < lf) {
        v = __ldg(lfv + i);
        rs = __ldg(fo.ro + v);
        full = __ldg(fo.ro + v + 1) - rs;
      }
      const bool join = full > 0u;
      const unsigned jb = __ballot_sync(FULL, join);
      if (jb) {   // warp-uniform
        if (join) {
          const uint32_t off = tqn + __popc(jb & lt);
          tqv[off] = v;
          tqr[off] = rs;
          tqd[off] = full;
        }
        tqn += __popc(jb);
        if (tqn > kTailQ - 32) tail_flush();
      }
    }
  }
  if (GG_FAR_Q && fn) far_q_flush(fq, fn, fo);
  if (TAIL && tqn) tail_flush();
#pragma unroll
  for (int o = 16; o; o >>= 1) fmin = min(fmin, __shfl_xor_sync(FULL, fmin, o));
  if (lane == 0) {
    if (fmin != kInf) atomicMin(&sm.fmin, fmin);
    // per CTA (the finalize adds it once): one global atomic per CTA, not per warp
    if (scanned) atomicAdd(&sm.ledges, (uint32_t)scanned);
  }
  if (__any_sync(FULL, ovf) && lane == 0) sm.ovf = 1u;
}

// Shared prologue: reset the CTA's queue, clear the bitmap left by a pull step.
template <int BLOCK, int EPT>
__device__ __forceinline__ void superstep_prologue(MPSmem<BLOCK, EPT>& sm, const StepArgs& a, uint32_t it,
                                                   bool clear_prev) {
  if (threadIdx.x == 0) {
    sm.qn = 0;
    sm.qfn = 0;
    sm.fmin = kInf;
    sm.ovf = 0;
    sm.ledges = 0;
  }
  if (clear_prev) {
    uint32_t* bm_old = a.fr.bm[(it + 2) % 3];
    for (uint32_t i = blockIdx.x * BLOCK + threadIdx.x; i < a.g.nwords; i += gridDim.x * BLOCK) bm_old[i] = 0u;
  }
  __syncthreads();
}

__device__ __forceinline__ unsigned long long bsp_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// The last CTA to arrive closes the superstep: counters, trace, the next
// step's kind (push, pull, or a near-far split) and the loop condition.  It
// sits between every two supersteps, so its one thread reads everything it
// needs in one batch of independent loads, decides in registers, and only then
// stores (no load waits on another).
template <int BLOCK, int EPT>
__device__ __forceinline__ void superstep_finalize(MPSmem<BLOCK, EPT>& sm, const StepArgs& a, uint32_t it, uint32_t f,
                                                   uint32_t E, uint32_t mode, cudaGraphConditionalHandle cond,
                                                   int use_cond) {
  Ctl* ctl = a.ctl;
  const uint32_t p = it & 1u;
  __syncthreads();
  if (threadIdx.x == 0) {
    if (sm.ovf) atomicOr(&ctl->status, DS_OVERFLOW);
    if (sm.fmin != kInf) atomicMin(&ctl->far_min, sm.fmin);
    if (sm.ledges) atomicAdd(&ctl->edges_scanned, (unsigned long long)sm.ledges);   // local rounds, heavy pull
    sm.last = arrive_last(&ctl->done_ctas, gridDim.x) ? 1u : 0u;
  }
  __syncthreads();
  if (sm.last && threadIdx.x == 0) {
    // counters of this superstep (atomics of every CTA)
    const unsigned long long cn = ld_rlx(&ctl->cnt[p ^ 1u]);
    const uint32_t fc0 = ld_rlx(&ctl->far_cnt[0]), fc1 = ld_rlx(&ctl->far_cnt[1]);
    const unsigned long long rc0 = ld_rlx(&ctl->rcnt[0]), rc1 = ld_rlx(&ctl->rcnt[1]);
    const uint32_t far_min = ld_rlx(&ctl->far_min);
    const uint32_t status = ld_rlx(&ctl->status);
    // run state (written by this finalize only)
    uint32_t fp = ctl->fp;
    const uint32_t lh = ctl->lh, lh_tail = ctl->lh_tail, splits = ctl->splits;
    uint32_t epoch = ctl->epoch;
    uint32_t* trace = ctl->trace;
    const uint32_t trace_cap = ctl->trace_cap;
    const uint32_t heavy_pull_ok = ctl->heavy_pull_ok, t_cur = ctl->t_cur, delta = ctl->delta;
    const uint32_t drain_div = ctl->drain_div, dir = ctl->dir, alpha = ctl->alpha, beta = ctl->beta;
    const uint32_t max_iter = ctl->max_iter, max_frontier = ctl->max_frontier, pull_iters = ctl->pull_iters;
    const unsigned long long heavy_total = ctl->heavy_total, frontier_total = ctl->frontier_total;
    unsigned long long heavy_done = ctl->heavy_done;
    const unsigned long long t_start = ctl->t_start, watchdog_ns = ctl->watchdog_ns;

    const uint32_t fn = (uint32_t)(cn >> 32), En = (uint32_t)cn;
    if (mode == MODE_SPLIT) fp ^= 1u;   // the kept entries were written to the other pile
    // a pull that ended bucketing consumed the far pile into the next frontier
    const bool pulled_tail = mode == MODE_HEAVY_PULL_TAIL;
    const uint32_t nfar = pulled_tail ? 0u : fp ? fc1 : fc0;
    const bool heavy = mode == MODE_HEAVY || mode == MODE_HEAVY_PULL || pulled_tail;
    const bool lhb = lh && !lh_tail;   // bucketed light/heavy supersteps
    bool tail = false;
    uint32_t rn = 0;   // R list of the epoch the next superstep works in
    unsigned long long rE = 0;   // and its heavy edges
    if (lhb) {
      if (heavy) {   // R[epoch] is consumed: the next epoch begins
        heavy_done += E;
        epoch += 1u;
      }
      const unsigned long long r = (epoch & 1u) ? rc1 : rc0;
      rn = (uint32_t)(r >> 32);
      rE = (uint32_t)r;
    }
    uint32_t nm;
    uint32_t t_next = t_cur;
    if (lhb && !pulled_tail && (fn > 0 || rn > 0)) {
      // light edges of the near frontier first; when it is empty, one heavy
      // superstep over the vertices that settled since the last one
      nm = fn > 0 ? MODE_PUSH : MODE_HEAVY;
      // a light frontier of at most n / GG_EARLY_TAIL_DIV vertices may end the
      // buckets early: if the pull that ends them is due on the current R
      // list, it runs now and takes the light frontier into the plain push's
      // first frontier (whole rows), whose pushes do what the bucket's last
      // light supersteps would
      const bool early = GG_EARLY_TAIL_DIV != 0 && fn > 0 &&
                         (unsigned long long)fn * (unsigned long long)GG_EARLY_TAIL_DIV <= a.g.n;
      if ((nm == MODE_HEAVY || early) && heavy_pull_ok && t_cur != kInf) {
        // pull when R's heavy edges outnumber those still unsettled (plus the
        // cost of the dense pass over the distances)
        const unsigned long long left = heavy_total > heavy_done + rE ? heavy_total - heavy_done - rE : 0ull;
        if (rE > left + a.g.n / 8) {
          if (nm == MODE_HEAVY) nm = MODE_HEAVY_PULL;
          // the split after this pull would end bucketing (the drain rule
          // below, on the heavy edges left once R's are relaxed): the pull
          // writes the plain tail's first frontier itself
          if (GG_PULL_TAIL && GG_LH_TAIL && drain_div && left * drain_div < (unsigned long long)a.g.m)
            nm = MODE_HEAVY_PULL_TAIL;
        }
      }
    } else if (fn == 0 && nfar > 0) {
      // near frontier exhausted: raise the threshold past the smallest parked distance
      nm = MODE_SPLIT;
      const unsigned long long t1 = (unsigned long long)t_cur + delta;
      const unsigned long long t2 = (unsigned long long)far_min + 1;
      unsigned long long tn = t1 > t2 ? t1 : t2;
      // light/heavy: once the vertices not yet settled hold only a small share
      // of the heavy edges, the rest of the run is one bucket (the sparse tail
      // of a skewed graph costs more in supersteps than in re-relaxations);
      // the R list is empty here, and that bucket is plain push from the split on
      if (lhb && drain_div && (heavy_total - min(heavy_done, heavy_total)) * drain_div < (unsigned long long)a.g.m) {
        tn = kInf;
        tail = GG_LH_TAIL != 0;
      }
      t_next = tn >= kInf ? kInf : (uint32_t)tn;
    } else if (dir == DIR_PUSH) {
      nm = MODE_PUSH;
    } else if (dir == DIR_PULL) {
      nm = MODE_PULL;
    } else if (mode != MODE_PULL) {
      nm = ((unsigned long long)En * alpha > a.g.m) ? MODE_PULL : MODE_PUSH;
    } else {
      nm = ((unsigned long long)fn * beta < a.g.np) ? MODE_PUSH : MODE_PULL;
    }
    bool more = fn != 0 || nfar != 0 || rn != 0;
    uint32_t st = 0;
    if (more && it + 1 >= max_iter) {
      st |= DS_ITER_CAP;
      more = false;
    }
    // signed difference: %globaltimer on this SM may lag the start stamp slightly
    if (more && (long long)(bsp_globaltimer() - t_start) > (long long)watchdog_ns) {
      st |= DS_TIMEOUT;
      more = false;
    }

    // stores
    if (mode == MODE_SPLIT) {
      ctl->far_cnt[fp ^ 1u] = 0u;
      ctl->fp = fp;
      ctl->splits = splits + 1u;
    }
    if (tail || pulled_tail) ctl->lh_tail = 1u;
    if (pulled_tail) {
      ctl->far_cnt[0] = 0u;
      ctl->far_cnt[1] = 0u;
    }
    if (lhb && heavy) {
      ctl->heavy_done = heavy_done;
      ctl->rcnt[(epoch - 1u) & 1u] = 0ull;
      ctl->epoch = epoch;
    }
    if (trace && it < trace_cap) {
      uint32_t* t = trace + 4ull * it;
      t[0] = f;
      t[1] = (mode == MODE_PUSH || heavy) ? E : mode == MODE_PULL ? a.g.m : 0u;
      t[2] = mode;
      t[3] = fn;
    }
    if (f > 0 && mode != MODE_SPLIT) {
      // a pull heavy step counts the edges it scans itself (atomically: add to it)
      const unsigned long long sc = (mode == MODE_PUSH || mode == MODE_HEAVY) ? E : mode == MODE_PULL ? a.g.m : 0u;
      if (sc) atomicAdd(&ctl->edges_scanned, sc);
      ctl->frontier_total = frontier_total + f;
      ctl->max_frontier = max(max_frontier, f);
      if (mode == MODE_PULL) ctl->pull_iters = pull_iters + 1u;
    }
    ctl->cnt[p] = 0ull;
    ctl->done_ctas = 0u;
    // light/heavy: vertices without light edges are marked in the next
    // bitmap but never enter the frontier, so the old bitmap is always cleared
    ctl->clear_prev = (mode == MODE_PULL || lh) ? 1u : 0u;
    if (nm == MODE_SPLIT) {
      ctl->t_prev = t_cur;
      ctl->t_cur = t_next;
      ctl->far_min = kInf;
    } else if (pulled_tail) {   // one unbounded bucket from here on
      ctl->t_prev = t_cur;
      ctl->t_cur = kInf;
      ctl->far_min = kInf;
    }
    ctl->mode = nm;
    ctl->iter = it + 1;
    if (st) ctl->status = status | st;
    ctl->running = more ? 1u : 0u;
    if (use_cond) cudaGraphSetConditional(cond, more ? 1u : 0u);
  }
}

// One superstep; LB selects the push advance (merge-path tiles, degree bins
// or warp streaming) (pull is the same merge-path sweep in both); a split step
// refills the near frontier from the far pile.
template <int BLOCK, int EPT, int LB, bool PK, int WMV>
__global__ void __launch_bounds__(BLOCK, superstep_min_blocks(LB, EPT)) k_superstep(StepArgs a, cudaGraphConditionalHandle cond,
                                                                       int use_cond) {
  // WMV: the weight mode, or kWmU32Lh for integer weights with light/heavy buckets
  constexpr bool LH = WMV == kWmU32Lh;
  constexpr int WM = LH ? (int)WM_U32 : WMV;
  extern __shared__ __align__(16) unsigned char smraw[];
  MPSmem<BLOCK, EPT>& sm = *reinterpret_cast<MPSmem<BLOCK, EPT>*>(smraw);
  Ctl* ctl = a.ctl;
  // the CUDA-graph loop body holds GG_BODY_UNROLL supersteps, which may run
  // past the last one: those return at once, and each also clears the loop
  // condition, so a run that starts finished (a source without out-edges)
  // ends after one iteration instead of looping on the condition's default
  // the step's state in one batch of independent loads (no load waits on
  // another: both parities of each counter are read and selected after)
  const uint32_t running = ctl->running, it = ctl->iter, mode = ctl->mode, fp = ctl->fp;
  const unsigned long long c0 = ctl->cnt[0], c1 = ctl->cnt[1];
  uint32_t* dist = ctl->dist;
  const uint32_t t_cur = ctl->t_cur, t_prev = ctl->t_prev, clear_prev = ctl->clear_prev;
  const uint32_t fc0 = ctl->far_cnt[0], fc1 = ctl->far_cnt[1];
  const uint32_t ep = LH ? ctl->epoch : 0u, lh_tail = LH ? ctl->lh_tail : 0u;
  const unsigned long long r0 = LH ? ctl->rcnt[0] : 0ull, r1 = LH ? ctl->rcnt[1] : 0ull;
  if (GG_BODY_UNROLL > 1 && use_cond && running == 0u) {
    if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
    return;
  }
  const uint32_t p = it & 1u;
  const unsigned long long c = p ? c1 : c0;
  const uint32_t f = (uint32_t)(c >> 32), E = (uint32_t)c;
  uint32_t* bm_cur = a.fr.bm[it % 3];
  FilterOut fo;
  fo.ro = a.g.ro;
  fo.sinks = a.g.sinks;
  fo.bm_next = a.fr.bm[(it + 1) % 3];
  fo.bm_far = a.fr.bm_far;
  fo.t_cur = t_cur;
  fo.cnt_next = &ctl->cnt[p ^ 1u];
  fo.nfv = a.fr.fv[p ^ 1u];
  fo.nfr = a.fr.fr[p ^ 1u];
  fo.nfs = a.fr.fs[p ^ 1u];
  // a split step reads far[fp] and keeps entries in far[fp^1]; other steps append to far[fp]
  fo.far = a.fr.far[mode == MODE_SPLIT ? fp ^ 1u : fp];
  fo.far_cnt = &ctl->far_cnt[mode == MODE_SPLIT ? fp ^ 1u : fp];
  fo.far_add = nullptr;
  fo.wmode = WM;   // compile-time: relax_add folds to one arithmetic path
  fo.lh = 0u;
  const void* edges = a.g.edges;
  const uint32_t* fS = a.fr.fs[p];
  const uint32_t* fR = a.fr.fr[p];
  const uint32_t* fV = a.fr.fv[p];
  uint32_t fw = f, Ew = E;   // entries and edges this superstep works on
  if (LH) {
    // new near vertices join the R list of the current epoch, or of the next
    // one while the heavy superstep consumes the current list
    const bool hv = mode == MODE_HEAVY || mode == MODE_HEAVY_PULL || mode == MODE_HEAVY_PULL_TAIL;
    const uint32_t rj = (hv ? ep + 1u : ep) & 1u;
    // the light/heavy append checks both degrees itself; after bucketing the
    // appends are plain (all edges of a row of the light-first copy), with the
    // plain loop's own handling of vertices without out-edges
    fo.sinks = lh_tail ? a.g.sinks : 0u;
    fo.lh = lh_tail ? 0u : 1u + rj;
    edges = a.lb.edges;
    if (hv) {
      const uint32_t rc = ep & 1u;
      const unsigned long long r = rc ? r1 : r0;
      fw = (uint32_t)(r >> 32);
      Ew = (uint32_t)r;
      fS = pick2(a.lb.rs, rc);
      fR = pick2(a.lb.rr, rc);
      fV = pick2(a.lb.rv, rc);
      bm_cur = pick2(a.lb.bm_r, rc);   // R entries clear their membership words as they are loaded
    }
  }
  superstep_prologue(sm, a, it, clear_prev != 0);
  if (mode == MODE_SPLIT) {
    far_split(sm, a, fo, dist, a.fr.far[fp], fp ? fc1 : fc0, t_prev);
  } else if (LH && mode == MODE_HEAVY_PULL) {
    heavy_pull<BLOCK, EPT, PK, false>(sm, a, fo, dist, pick2(a.lb.bm_r, ep & 1u), nullptr, 0u);
  } else if (LH && mode == MODE_HEAVY_PULL_TAIL) {
    // f: the light frontier a pull that ends the buckets early takes along
    heavy_pull<BLOCK, EPT, PK, true>(sm, a, fo, dist, pick2(a.lb.bm_r, ep & 1u), a.fr.fv[p], f);
  } else if (fw > 0) {
    if (mode == MODE_PUSH || mode == MODE_HEAVY) {
      if (LB == LB_BINS)
        bins_advance<BLOCK, EPT, PK>(sm, a, fw, Ew, fV, fR, fS, dist, bm_cur, fo, ctl->warp_thr, ctl->cta_thr,
                                     edges);
      else if ((LB == LB_WARP || LB == LB_LOCAL) && LH && mode == MODE_HEAVY)   // separate copies keep the
        warp_advance<BLOCK, EPT, PK>(sm, a, fw, Ew, fS, fR, fV, edges, dist, bm_cur, fo);   // pointer selects out
      else if (LB == LB_WARP || LB == LB_LOCAL)                                              // of the loop
        warp_advance<BLOCK, EPT, PK, LB == LB_LOCAL>(sm, a, f, E, a.fr.fs[p], a.fr.fr[p], a.fr.fv[p], edges, dist,
                                                     LH ? nullptr : a.fr.bm[it % 3], fo);
      else
        mp_advance<BLOCK, EPT, false, PK>(sm, a, fw, Ew, fS, fR, fV, edges, dist, bm_cur, fo);
    } else {
      mp_advance<BLOCK, EPT, true, PK>(sm, a, a.g.np, a.g.m, a.g.ps, a.g.ps, a.g.pv, a.g.t_edges, dist, bm_cur,
                                       fo);
    }
  }
  superstep_finalize(sm, a, it, fw, Ew, mode, cond, use_cond);
}

// Bounded grid barrier for the persistent kernel: generation counter, the
// last CTA to arrive bumps it.  Waits give up at the run's deadline (or when
// another CTA has aborted) and raise `abort`, so no CTA spins forever.
__device__ __forceinline__ void grid_barrier(Ctl* ctl, unsigned long long deadline) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t* gen = &ctl->bar_gen;
    const uint32_t g = *gen;
    __threadfence();
    if (atomicAdd(&ctl->bar_count, 1u) == gridDim.x - 1) {
      ctl->bar_count = 0u;
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      uint32_t spins = 0;
      while (*gen == g) {
        if (*(volatile uint32_t*)&ctl->abort) break;
        if ((++spins & 63u) == 0 && bsp_globaltimer() > deadline) {
          atomicOr(&ctl->status, DS_TIMEOUT);
          atomicExch(&ctl->abort, 1u);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// All supersteps of one run in one cooperative launch (grid <= co-resident
// CTAs).  Each superstep is the same work as k_superstep; instead of a kernel
// boundary, one grid barrier separates supersteps, after which every CTA reads
// the same final counters and takes the same decision (next step's kind,
// thresholds, termination) in its own registers.  Counters rotate over three
// slots (a slot is reset two supersteps after its last reader passed a
// barrier); the far pile rotates over three piles, one per split step.
template <int BLOCK, int EPT, int LB, bool PK, int WM>
__global__ void __launch_bounds__(BLOCK, superstep_min_blocks(LB, EPT)) k_bsp_persistent(StepArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  MPSmem<BLOCK, EPT>& sm = *reinterpret_cast<MPSmem<BLOCK, EPT>*>(smraw);
  Ctl* ctl = a.ctl;
  uint32_t* dist = ctl->dist;
  const unsigned long long deadline = ctl->t_start + ctl->watchdog_ns;
  const uint32_t dir = ctl->dir, alpha = ctl->alpha, beta = ctl->beta, delta = ctl->delta;
  const uint32_t max_iter = ctl->max_iter;
  uint32_t it = 0, mode = ctl->mode, t_cur = ctl->t_cur, t_prev = 0, splits = 0, run_fmin = kInf;
  uint32_t nfar = 0;   // far-pile size, tracked identically by every CTA
  bool clear = false;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  unsigned long long edges_scanned = 0, frontier_total = 0;
  uint32_t max_frontier = 0, pull_iters = 0;
  for (;;) {
    const uint32_t s0 = it % 3, s1 = (it + 1) % 3, s2 = (it + 2) % 3;
    const uint32_t pile = splits % 3, pile_out = (splits + 1) % 3;
    const unsigned long long c = *(volatile unsigned long long*)&ctl->cnt3[s0];
    const uint32_t f = (uint32_t)(c >> 32), E = (uint32_t)c;
    const uint32_t p = it & 1u;
    uint32_t* bm_cur = a.fr.bm[s0];
    FilterOut fo;
    fo.ro = a.g.ro;
    fo.sinks = a.g.sinks;
    fo.bm_next = a.fr.bm[s1];
    fo.bm_far = a.fr.bm_far;
    fo.t_cur = t_cur;
    fo.cnt_next = &ctl->cnt3[s1];
    fo.nfv = a.fr.fv[p ^ 1u];
    fo.nfr = a.fr.fr[p ^ 1u];
    fo.nfs = a.fr.fs[p ^ 1u];
    fo.far = a.fr.far[mode == MODE_SPLIT ? pile_out : pile];
    fo.far_cnt = &ctl->fcnt3[mode == MODE_SPLIT ? pile_out : pile];
    fo.far_add = &ctl->fadd3[s0];
    fo.wmode = WM;   // compile-time: relax_add folds to one arithmetic path
    fo.lh = 0u;      // light/heavy buckets run in the launched-superstep policies only
    superstep_prologue(sm, a, it, clear);
    if (lead) {
      ctl->cnt3[s2] = 0ull;      // written next superstep; its readers are two barriers back
      ctl->fm3[s1] = kInf;       // written next superstep
      ctl->fadd3[s1] = 0u;
      if (mode == MODE_SPLIT) ctl->fcnt3[(splits + 2) % 3] = 0u;   // output pile of the next split
    }
    if (mode == MODE_SPLIT) {
      far_split(sm, a, fo, dist, a.fr.far[pile], nfar, t_prev);
    } else if (f > 0) {
      if (mode == MODE_PUSH) {
        if (LB == LB_BINS)
          bins_advance<BLOCK, EPT, PK>(sm, a, f, E, a.fr.fv[p], a.fr.fr[p], a.fr.fs[p], dist, bm_cur, fo,
                                       ctl->warp_thr, ctl->cta_thr, a.g.edges);
        else if (LB == LB_WARP || LB == LB_LOCAL)
          warp_advance<BLOCK, EPT, PK>(sm, a, f, E, a.fr.fs[p], a.fr.fr[p], a.fr.fv[p], a.g.edges, dist, bm_cur,
                                       fo);
        else
          mp_advance<BLOCK, EPT, false, PK>(sm, a, f, E, a.fr.fs[p], a.fr.fr[p], a.fr.fv[p], a.g.edges, dist,
                                            bm_cur, fo);
      } else {
        mp_advance<BLOCK, EPT, true, PK>(sm, a, a.g.np, a.g.m, a.g.ps, a.g.ps, a.g.pv, a.g.t_edges, dist,
                                         bm_cur, fo);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (sm.ovf) atomicOr(&ctl->status, DS_OVERFLOW);
      if (sm.fmin != kInf) atomicMin(&ctl->fm3[s0], sm.fmin);
      if (blockIdx.x == 0 && bsp_globaltimer() > deadline) {
        atomicOr(&ctl->status, DS_TIMEOUT);
        atomicExch(&ctl->abort, 1u);
      }
    }
    grid_barrier(ctl, deadline);
    // every CTA takes the same decision from the same final counters
    const unsigned long long cn = *(volatile unsigned long long*)&ctl->cnt3[s1];
    const uint32_t fn = (uint32_t)(cn >> 32), En = (uint32_t)cn;
    // far-pile size: a split keeps fadd3 entries; other steps add fadd3 entries
    const uint32_t added = *(volatile uint32_t*)&ctl->fadd3[s0];
    if (mode == MODE_SPLIT) {
      ++splits;
      nfar = added;
    } else {
      nfar += added;
    }
    run_fmin = min(run_fmin, *(volatile uint32_t*)&ctl->fm3[s0]);
    if (lead) {
      if (ctl->trace && it < ctl->trace_cap) {
        uint32_t* t = ctl->trace + 4ull * it;
        t[0] = f;
        t[1] = mode == MODE_PUSH ? E : mode == MODE_PULL ? a.g.m : 0u;
        t[2] = mode;
        t[3] = fn;
      }
      if (f > 0 && mode != MODE_SPLIT) {
        edges_scanned += mode == MODE_PUSH ? E : a.g.m;
        frontier_total += f;
        max_frontier = max(max_frontier, f);
        pull_iters += mode == MODE_PULL ? 1u : 0u;
      }
    }
    uint32_t nm;
    if (fn == 0 && nfar > 0) {
      nm = MODE_SPLIT;
      const unsigned long long t1 = (unsigned long long)t_cur + delta;
      const unsigned long long t2 = (unsigned long long)run_fmin + 1;
      const unsigned long long tn = t1 > t2 ? t1 : t2;
      t_prev = t_cur;
      t_cur = tn >= kInf ? kInf : (uint32_t)tn;
      run_fmin = kInf;
    } else if (dir == DIR_PUSH) {
      nm = MODE_PUSH;
    } else if (dir == DIR_PULL) {
      nm = MODE_PULL;
    } else if (mode != MODE_PULL) {
      nm = ((unsigned long long)En * alpha > a.g.m) ? MODE_PULL : MODE_PUSH;
    } else {
      nm = ((unsigned long long)fn * beta < a.g.np) ? MODE_PUSH : MODE_PULL;
    }
    clear = mode == MODE_PULL;
    mode = nm;
    ++it;
    const bool more = fn != 0 || nfar != 0;
    const bool aborted = *(volatile uint32_t*)&ctl->abort != 0;
    if (!more || aborted || it >= max_iter) {
      if (lead) {
        if (more && !aborted) atomicOr(&ctl->status, DS_ITER_CAP);
        ctl->iter = it;
        ctl->mode = mode;
        ctl->splits = splits;
        ctl->edges_scanned = edges_scanned;
        ctl->frontier_total = frontier_total;
        ctl->max_frontier = max_frontier;
        ctl->pull_iters = pull_iters;
        ctl->running = 0u;
      }
      break;
    }
  }
}

// Per-run parameters written into the control block by k_init_tail.
struct RunParams {
  uint32_t src;
  uint32_t* dist;
  uint32_t dir, alpha, beta, max_iter;
  uint32_t* trace;
  uint32_t trace_cap;
  uint32_t warp_thr, cta_thr;
  uint32_t delta;                  // near-far bucket width (kInf: no split)
  uint32_t wmode;                  // WM_*
  unsigned long long watchdog_ns;
  uint32_t lh;                     // light/heavy buckets (StepArgs::lb holds the buffers)
  uint32_t drain_div;
  uint32_t heavy_pull_ok;
  unsigned long long heavy_total;
};

// dist := the unreached value everywhere (INF, or FLT_MAX for binary32
// distances; vectorised 16-byte stores when aligned); bitmaps := 0.
__global__ void k_init(StepArgs a, uint32_t* dist, uint32_t unreached, uint32_t* bm_r0, uint32_t* bm_r1) {
  const uint32_t n = a.g.n;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((reinterpret_cast<uintptr_t>(dist) & 15u) == 0) {
    const uint64_t n4 = n / 4;
    uint4* d4 = reinterpret_cast<uint4*>(dist);
    for (uint64_t i = t; i < n4; i += stride) d4[i] = make_uint4(unreached, unreached, unreached, unreached);
    for (uint64_t i = n4 * 4 + t; i < n; i += stride) dist[i] = unreached;
  } else {
    for (uint64_t i = t; i < n; i += stride) dist[i] = unreached;
  }
  for (uint64_t i = t; i < a.g.nwords; i += stride) {
    a.fr.bm[0][i] = 0u;
    a.fr.bm[1][i] = 0u;
    a.fr.bm[2][i] = 0u;
    a.fr.bm_far[i] = 0u;
    if (bm_r0) {
      bm_r0[i] = 0u;
      bm_r1[i] = 0u;
    }
  }
}

// dist[src] := 0, frontier := {src} (when src has out-edges), counters reset.
// Light/heavy runs: src's light edges form the first frontier and its heavy
// edges the first R list (a source without light edges starts with the heavy
// superstep).
__global__ void k_init_tail(StepArgs a, RunParams rp) {
  Ctl* ctl = a.ctl;
  const uint32_t src = rp.src;
  rp.dist[src] = 0u;
  const uint32_t rs = a.g.ro[src], re = a.g.ro[src + 1];
  const uint32_t le = rp.lh ? a.lb.lend[src] : re;   // end of the edges the first frontier relaxes
  if (le > rs) {
    a.fr.fv[0][0] = src;
    a.fr.fr[0][0] = rs;
    a.fr.fs[0][0] = 0u;
    a.fr.bm[0][src >> 5] = 1u << (src & 31);
    ctl->cnt[0] = (1ull << 32) | (le - rs);
  } else {
    ctl->cnt[0] = 0ull;
  }
  ctl->rcnt[0] = 0ull;
  ctl->rcnt[1] = 0ull;
  const bool heavy0 = rp.lh && re > le;
  if (heavy0) {
    a.lb.rv[0][0] = src;
    a.lb.rr[0][0] = le;
    a.lb.rs[0][0] = 0u;
    a.lb.bm_r[0][src >> 5] = 1u << (src & 31);
    ctl->rcnt[0] = (1ull << 32) | (re - le);
  }
  ctl->lh = rp.lh;
  ctl->epoch = 0;
  ctl->drain_div = rp.drain_div;
  ctl->heavy_pull_ok = rp.heavy_pull_ok;
  ctl->heavy_total = rp.heavy_total;
  ctl->heavy_done = 0ull;
  ctl->lh_tail = 0u;
  ctl->cnt[1] = 0ull;
  ctl->iter = 0;
  ctl->done_ctas = 0;
  ctl->status = 0;
  ctl->mode = rp.dir == DIR_PULL ? MODE_PULL : (le == rs && heavy0) ? MODE_HEAVY : MODE_PUSH;
  ctl->clear_prev = 0;
  ctl->src = src;
  ctl->max_iter = rp.max_iter;
  ctl->dir = rp.dir;
  ctl->alpha = rp.alpha;
  ctl->beta = rp.beta;
  ctl->running = re > rs ? 1u : 0u;
  ctl->pull_iters = 0;
  ctl->dist = rp.dist;
  ctl->trace = rp.trace;
  ctl->trace_cap = rp.trace ? rp.trace_cap : 0u;
  ctl->max_frontier = 0;
  ctl->warp_thr = rp.warp_thr;
  ctl->cta_thr = rp.cta_thr;
  ctl->wmode = rp.wmode;
  ctl->delta = rp.delta;
  ctl->t_cur = rp.delta;           // the first bucket is [0, delta)
  ctl->t_prev = 0;
  ctl->fp = 0;
  ctl->far_cnt[0] = 0;
  ctl->far_cnt[1] = 0;
  ctl->far_min = kInf;
  ctl->splits = 0;
  ctl->watchdog_ns = rp.watchdog_ns;
  ctl->cnt3[0] = ctl->cnt[0];
  ctl->cnt3[1] = 0ull;
  ctl->cnt3[2] = 0ull;
  for (int i = 0; i < 3; ++i) {
    ctl->fm3[i] = kInf;
    ctl->fcnt3[i] = 0u;
    ctl->fadd3[i] = 0u;
  }
  ctl->bar_count = 0u;
  ctl->bar_gen = 0u;
  ctl->abort = 0u;
  ctl->t_start = bsp_globaltimer();
  ctl->edges_scanned = 0;
  ctl->frontier_total = 0;
}

constexpr int kBlock = 256;
constexpr int kEpt = GG_EPT;
// kernel variants: (load balance x packed edges) x (weight mode, or integer
// weights with light/heavy buckets)
constexpr int kVariants = kBspVariants;
static_assert(kVariants == 4 * 2 * 4, "variant table");

constexpr int variant_of(int lb, bool packed, uint32_t wmode, bool lh) {
  return (lb * 2 + (packed ? 1 : 0)) * 4 + (lh ? kWmU32Lh : (int)wmode);
}

template <int LB, bool PK, int WM>
void* superstep_ptr() { return reinterpret_cast<void*>(&k_superstep<kBlock, kEpt, LB, PK, WM>); }
// the persistent policy has no light/heavy form: its slot holds the plain integer kernel
template <int LB, bool PK, int WM>
void* persistent_ptr() {
  return reinterpret_cast<void*>(&k_bsp_persistent<kBlock, kEpt, LB, PK, WM == kWmU32Lh ? 0 : WM>);
}

#define GG_VARIANT_ROW(F, LBV, PKV) F<LBV, PKV, 0>(), F<LBV, PKV, 1>(), F<LBV, PKV, 2>(), F<LBV, PKV, kWmU32Lh>()
#define GG_VARIANT_TABLE(F)                                                                   \
  {GG_VARIANT_ROW(F, LB_TILE, false), GG_VARIANT_ROW(F, LB_TILE, true), GG_VARIANT_ROW(F, LB_BINS, false), \
   GG_VARIANT_ROW(F, LB_BINS, true),  GG_VARIANT_ROW(F, LB_WARP, false), GG_VARIANT_ROW(F, LB_WARP, true),  \
   GG_VARIANT_ROW(F, LB_LOCAL, false), GG_VARIANT_ROW(F, LB_LOCAL, true)}

void* superstep_fn(int variant) {
  static void* const table[kVariants] = GG_VARIANT_TABLE(superstep_ptr);
  return table[variant];
}

size_t superstep_smem(int) { return sizeof(MPSmem<kBlock, kEpt>); }

void* persistent_fn(int variant) {
  static void* const table[kVariants] = GG_VARIANT_TABLE(persistent_ptr);
  return table[variant];
}

// co-resident grid of the persistent kernel (cooperative launch limit),
// capped like the superstep grid on low-degree graphs (fewer CTAs at each
// grid barrier)
int persistent_grid(const gg_graph* g, int variant) {
  static int cached[kVariants] = {};
  if (!cached[variant]) {
    int per_sm = 0;
    void* fn = persistent_fn(variant);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)superstep_smem(variant));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, superstep_smem(variant));
    cached[variant] = per_sm < 1 ? 1 : per_sm;
  }
  int per_sm = cached[variant];
  if (g->low_degree && per_sm > GG_SPARSE_PER_SM_P) per_sm = GG_SPARSE_PER_SM_P;
  return per_sm * device_info().num_sms;
}

gg_status ensure_workspace(gg_graph* g, cudaStream_t s) {
  BspWorkspace& w = g->bsp;
  if (w.block) return GG_OK;
  const size_t n = g->n;
  const size_t nw = (n + 31) / 32;
  const size_t fbytes = sizeof(uint32_t) * std::max<size_t>(n, 1);
  auto r256 = [](size_t b) { return (b + 255) & ~size_t(255); };
  // every sub-buffer starts on a 256-byte boundary
  const size_t total = 9 * r256(fbytes) + 4 * r256(sizeof(uint32_t) * nw) + r256(sizeof(Ctl));
  char* p = nullptr;
  GG_CK(dev_malloc(&p, total, s));
  GG_CK(cudaMemsetAsync(p, 0, total, s));
  w.block = p;
  w.bytes = total;
  size_t off = 0;
  auto take = [&](size_t b) { char* q = p + off; off += r256(b); return q; };
  for (int i = 0; i < 2; ++i) {
    w.fr.fv[i] = reinterpret_cast<uint32_t*>(take(fbytes));
    w.fr.fr[i] = reinterpret_cast<uint32_t*>(take(fbytes));
    w.fr.fs[i] = reinterpret_cast<uint32_t*>(take(fbytes));
  }
  for (int i = 0; i < 3; ++i) w.fr.bm[i] = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * nw));
  for (int i = 0; i < 3; ++i) w.fr.far[i] = reinterpret_cast<uint32_t*>(take(fbytes));
  w.fr.bm_far = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * nw));
  w.ctl = reinterpret_cast<Ctl*>(take(sizeof(Ctl)));
  if (off != total) return fail(GG_ERR_INTERNAL, "workspace layout");
  return GG_OK;
}

// Superstep grid: every resident CTA on skewed graphs, whose large supersteps
// need the occupancy to hide memory latency; GG_SPARSE_PER_SM CTAs per SM on
// low-degree graphs (mean degree < 8: grids, paths), whose thousands of
// mid-size supersteps are bound by the per-launch cost, which grows with the
// grid (measured on the 4096^2 grid: 139 ms at 2 per SM, 162 ms at 5).
int superstep_grid(const gg_graph* g, int variant) {
  static int cached[kVariants] = {};
  if (!cached[variant]) {
    int per_sm = 0;
    void* fn = superstep_fn(variant);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)superstep_smem(variant));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, superstep_smem(variant));
    cached[variant] = per_sm < 1 ? 1 : per_sm;
  }
  int per_sm = cached[variant];
  if (g->low_degree && per_sm > GG_SPARSE_PER_SM) per_sm = GG_SPARSE_PER_SM;
  return per_sm * device_info().num_sms;
}

gg_status build_graph_exec(gg_graph* g, int variant) {
  BspWorkspace& w = g->bsp;
  if (w.exec[variant]) return GG_OK;
  cudaGraph_t graph = nullptr;
  GG_CK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle h;
  GG_CK(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wnode;
  GG_CK(cudaGraphAddNode(&wnode, graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  StepArgs a{g->dg, w.fr, w.ctl, g->lhb};   // light/heavy variants are built after lh_prepare
  int use_cond = 1;
  void* args[] = {&a, &h, &use_cond};
  cudaKernelNodeParams kp = {};
  kp.func = superstep_fn(variant);
  kp.gridDim = dim3(superstep_grid(g, variant));
  kp.blockDim = dim3(kBlock);
  kp.sharedMemBytes = (unsigned)superstep_smem(variant);
  kp.kernelParams = args;
  // GG_BODY_UNROLL supersteps per loop iteration: the loop condition is
  // evaluated once per iteration (about 3 us each), and a superstep past the
  // last one returns at once
  cudaGraphNode_t prev = nullptr;
  for (int u = 0; u < GG_BODY_UNROLL; ++u) {
    cudaGraphNode_t knode;
    GG_CK(cudaGraphAddKernelNode(&knode, body, prev ? &prev : nullptr, prev ? 1 : 0, &kp));
    prev = knode;
  }
  cudaGraphExec_t exec = nullptr;
  GG_CK(cudaGraphInstantiate(&exec, graph, 0));
  w.graph[variant] = graph;
  w.exec[variant] = exec;
  w.grid[variant] = superstep_grid(g, variant);
  return GG_OK;
}

}  // namespace

gg_status bsp_run(gg_graph* g, uint32_t src, uint32_t* dist, const gg_options& o, cudaStream_t s, uint32_t wmode) {
  gg_status st = ensure_workspace(g, s);
  if (st != GG_OK) return st;
  // automatic choice: warp streaming (measured faster than merge-path tiles on
  // RMAT, equal on grids), with warp-local rounds on low-degree graphs (the
  // 4096^2 grid: 95 -> 34-36 ms, a tenth of the supersteps)
  const int lb = o.lb_mode == GG_LB_BINS ? LB_BINS : o.lb_mode == GG_LB_MERGE_PATH ? LB_TILE
               : o.lb_mode == GG_LB_LOCAL ? LB_LOCAL : o.lb_mode == GG_LB_WARP ? LB_WARP
               : g->low_degree ? LB_LOCAL : LB_WARP;
  BspWorkspace& w = g->bsp;
  RunParams rp;
  rp.src = src;
  rp.dist = dist;
  rp.dir = o.direction == GG_DIR_PUSH ? DIR_PUSH : o.direction == GG_DIR_PULL ? DIR_PULL : DIR_AUTO;
  rp.alpha = o.pull_alpha ? o.pull_alpha : 4u;
  rp.beta = o.pull_beta ? o.pull_beta : 24u;
  // near-far: with buckets the superstep count is bounded by about 3n (every
  // phase finalises at least one vertex and runs at most its bucket's size + 2
  // steps); without, by n + 1
  // buckets are integer distance ranges: binary32 and hop-count runs go without
  // light/heavy buckets: launched-superstep policies, push, integer weights,
  // and a width that leaves some edge heavy; the graph's own default width is
  // the light/heavy one where it has one
  const bool lh_ok = (o.policy == GG_POLICY_BSP_GRAPH || o.policy == GG_POLICY_BSP_HOST) &&
                     o.light_heavy != GG_LH_OFF && rp.dir == DIR_PUSH && wmode == WM_U32 && g->m > 0;
  if (o.delta == GG_DELTA_NONE || wmode != WM_U32) rp.delta = kInf;
  else if (o.delta) rp.delta = o.delta;
  else rp.delta = (lh_ok && g->default_delta_lh != GG_DELTA_NONE) ? g->default_delta_lh : g->default_delta;
  rp.wmode = wmode;
  rp.lh = (lh_ok && rp.delta != kInf && rp.delta <= g->wmax) ? 1u : 0u;
  rp.drain_div = GG_LH_DRAIN;
  rp.heavy_pull_ok = 0u;
  rp.heavy_total = 0ull;
  if (rp.lh) {
    st = lh_prepare(g, rp.delta, s);
    if (st != GG_OK) return st;
    // a symmetric graph's heavy in-edges are its heavy out-edges
    rp.heavy_pull_ok = (g->symmetric && GG_HEAVY_PULL) ? 1u : 0u;
    rp.heavy_total = g->lh_heavy_total;
  }
  const int variant = variant_of(lb, g->dg.packed != 0, wmode, rp.lh != 0);
  // a light/heavy run adds at most one heavy superstep per settled vertex
  const unsigned long long cap = rp.delta == kInf ? (unsigned long long)g->n + 2
                                 : rp.lh ? 6ull * g->n + 16 : 4ull * g->n + 16;
  rp.max_iter = o.max_iterations ? o.max_iterations : (cap >= 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)cap);
  rp.watchdog_ns = o.watchdog_ns ? o.watchdog_ns : 60000000000ull;
  rp.trace = o.trace;
  rp.trace_cap = o.trace_cap;
  rp.warp_thr = o.warp_threshold ? o.warp_threshold : 32u;
  rp.cta_thr = o.cta_threshold ? o.cta_threshold : 1024u;
  if (rp.cta_thr < rp.warp_thr) rp.cta_thr = rp.warp_thr;
  const uint32_t max_iter = rp.max_iter;
  StepArgs a{g->dg, w.fr, w.ctl, g->lhb};
  const DeviceInfo di = device_info();
  const uint64_t work = std::max<uint64_t>(g->n / 4, g->dg.nwords);
  unsigned ib = (unsigned)std::min<uint64_t>((work + 255) / 256, (uint64_t)di.num_sms * 8);
  if (ib == 0) ib = 1;
  k_init<<<ib, 256, 0, s>>>(a, dist, wmode == WM_F32 ? kFltMaxBits : kInf, rp.lh ? g->lhb.bm_r[0] : nullptr,
                            rp.lh ? g->lhb.bm_r[1] : nullptr);
  GG_CK(cudaGetLastError());
  k_init_tail<<<1, 1, 0, s>>>(a, rp);
  GG_CK(cudaGetLastError());
  if (o.policy == GG_POLICY_BSP_PERSISTENT) {
    void* args[] = {&a};
    GG_CK(cudaLaunchCooperativeKernel(persistent_fn(variant), dim3(persistent_grid(g, variant)), dim3(kBlock), args,
                                      superstep_smem(variant), s));
  } else if (o.policy == GG_POLICY_BSP_GRAPH) {
    st = build_graph_exec(g, variant);
    if (st != GG_OK) return st;
    GG_CK(cudaGraphLaunch(w.exec[variant], s));
  } else {
    const int grid = superstep_grid(g, variant);
    const size_t smem = superstep_smem(variant);
    cudaGraphConditionalHandle none = 0;
    int zero = 0;
    if (!g->h_ctl) GG_CK(cudaMallocHost(&g->h_ctl, sizeof(Ctl)));   // pinned mirror, on first use
    uint32_t* h_running = &g->h_ctl->running;
    uint32_t launched = 0;
    uint32_t check_every = 1;
    for (;;) {
      for (uint32_t k = 0; k < check_every; ++k) {
        void* args[] = {&a, &none, &zero};
        GG_CK(cudaLaunchKernel(superstep_fn(variant), dim3(grid), dim3(kBlock), args, smem, s));
        ++launched;
      }
      GG_CK(cudaGetLastError());
      GG_CK(cudaMemcpyAsync(h_running, &w.ctl->running, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
      GG_CK(cudaStreamSynchronize(s));
      if (*h_running == 0) break;
      if (launched > max_iter + 16) break;
      check_every = std::min<uint32_t>(check_every * 2, 16);
    }
  }
  return GG_OK;
}

gg_status bsp_read_ctl(gg_graph* g, cudaStream_t s) {
  if (!g->h_ctl) {   // pinned mirror, allocated on first use
    GG_CK(cudaMallocHost(&g->h_ctl, sizeof(Ctl)));
    memset(g->h_ctl, 0, sizeof(Ctl));
  }
  if (!g->bsp.ctl) return GG_OK;
  GG_CK(cudaMemcpyAsync(g->h_ctl, g->bsp.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  GG_CK(cudaStreamSynchronize(s));
  return GG_OK;
}

gg_status bsp_release(gg_graph* g) {
  BspWorkspace& w = g->bsp;
  for (int i = 0; i < kVariants; ++i) {
    if (w.exec[i]) cudaGraphExecDestroy(w.exec[i]);
    if (w.graph[i]) cudaGraphDestroy(w.graph[i]);
    w.exec[i] = nullptr;
    w.graph[i] = nullptr;
  }
  dev_free(w.block, 0);   // the handle's work has been synchronised
  w.block = nullptr;
  w.ctl = nullptr;
  return GG_OK;
}

}  // namespace gg
