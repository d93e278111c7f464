// gg_batch.cu -- batched multi-source SSSP: k independent single-source runs
// of the paper's frontier loop (Listing 4) fused into one bulk-synchronous
// loop over a shared frontier.
//
// Distance matrix: dist[v*k + s] (vertex-major), so the up-to-64 distances of
// one vertex row are contiguous: lane l of a warp owns sources l and l+32 of
// the current 64-source group, and every relaxation of an edge (u, v) reads
// and updates v's row with two coalesced 128-byte accesses.  The col/weight
// stream of an edge is read once for all sources whose distance at u
// improved.
//
// Frontier entry = vertex u + a 64-bit mask of the sources whose dist[u][s]
// decreased in the previous superstep (only those sources are relaxed from
// u).  The mask array M_next is accumulated with atomicOr; the edge that takes
// a vertex's mask from 0 to non-zero appends the vertex to the next sparse
// frontier, with the same block-aggregated append (one 64-bit atomicAdd per
// CTA tile returning queue position and edge-prefix base) as the
// single-source filter.  Candidacy comes from the pre-check  nd < dist[v][s]
// read before the atomicMin: after the atomic, dist[v][s] <= nd < that value,
// so v did improve in this superstep and belongs in the next frontier; the
// atomic itself is fire-and-forget.
//
// Three rotating frontier queues and mask arrays: superstep t reads F_t and
// M_t, builds F_{t+1}/M_{t+1}, and zeroes the masks of F_{t-1}'s vertices
// (their list is intact in the third queue).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "gg_host.h"

namespace gg {

struct BatchCtl {
  unsigned long long cnt[3];
  uint32_t iter, done_ctas, status, running, max_iter;
  uint32_t k, col0, kg;
  uint32_t max_frontier;
  uint32_t* dist;
  unsigned long long edges_scanned, frontier_total;
  // near-far buckets over (vertex, source) pairs: a pair improved to a
  // distance >= t_cur is parked as a bit of fmask[v]; the vertices with
  // parked bits form the far list far_v[fsel]
  uint32_t t_cur, t_prev, delta, fsel, fcnt[2], far_min, mode, splits;
  // light-first rounds (lh = 1; mode 2 = heavy superstep): light supersteps
  // relax only the light edges (weight < the graph's light/heavy width) of
  // their (vertex, sources) entries; every pair that improves is also ORed
  // into the R mask of the epoch, and when the light frontier empties one
  // heavy superstep relaxes the heavy edges of the R entries for their R
  // masks and starts the next epoch.  No distance thresholds: the rounds are a
  // label-correcting loop in which a heavy edge is scanned once per epoch
  // that improved its source vertex.  R buffers rotate over three epochs;
  // the masks of a consumed R list are cleared one superstep later.
  uint32_t lh, epoch, zero_pending, zero_par;
  unsigned long long rcnt[3];
  // normalised buckets (nb = 1, light-first rounds only): one shared bucket
  // threshold over the pairs' distances shifted by sh[s] = max_s' o_s' - o_s,
  // where o_s is the source's distance from the graph's highest-degree vertex
  // (the hub).  A pair (v, s) is near while dist[v][s] + sh[s] < t_cur; near
  // pairs relax their light edges and join the R mask, far ones are parked in
  // fmask.  Sources reach the dense core at about the same shifted distance,
  // so one bucket holds the same vertices for most sources and each edge read
  // still serves many of them.  Bucketing ends (tail = 1: plain push over all
  // edges of every improved pair) once the unsettled pairs hold fewer than
  // heavy_total_k / drain_div heavy edges.
  uint32_t nb, tail, width, drain_div;
  uint32_t* trace;      // optional: per superstep (kind | tail << 4, entries, edges, next frontier size)
  uint32_t trace_cap;
  // heavy superstep by pull (mode 4; symmetric graphs, bucket width <= the
  // light/heavy width): chosen when the pairs settled since the last heavy
  // superstep hold more heavy edges than the pairs not yet settled
  uint32_t pull_ok;
  unsigned long long settled_mark;   // heavy_settled at the last heavy superstep
  unsigned long long pull_edges;     // heavy edges the pull scanned (statistics)
  unsigned long long heavy_total_k;   // heavy edges of the graph x sources of the group
  unsigned long long heavy_settled;   // heavy edges of the pairs that settled into a bucket
  uint32_t sh[64];
};

struct BatchBufs {
  uint32_t* fv[3];
  uint32_t* fr[3];
  uint32_t* fs[3];
  unsigned long long* mask[3];
  unsigned long long* fmask;
  uint32_t* far_v[2];
  BatchCtl* ctl;
  // light-first rounds: the graph's light-first edge copy and the R lists
  const void* ledges;
  const uint32_t* lend;
  uint32_t* rv[3];
  uint32_t* rr[3];
  uint32_t* rs[3];
  unsigned long long* rmask[3];
  const uint32_t* hubd;   // distances from the hub (normalised buckets)
};

namespace {

constexpr int kBB = 256;
constexpr int kBNW = kBB / 32;
constexpr int kBTile = 1024;
constexpr int kBCap = kBTile + 1;
constexpr uint32_t kBQW = 128;   // per-warp queue slots of the warp-streaming relaxation
static_assert(kBNW * kBQW <= (uint32_t)kBCap, "per-warp queues fit the CTA queue arrays");
#ifndef GG_BMINB
#define GG_BMINB 6   // resident CTAs per SM the batch superstep is compiled for (40 registers)
#endif
#ifndef GG_NB_WIDTH
#define GG_NB_WIDTH 1   // normalised buckets: bucket width in light/heavy widths
#endif
#ifndef GG_NB_DRAIN
#define GG_NB_DRAIN 8   // normalised buckets end once the unsettled pairs hold < 1/GG_NB_DRAIN of the heavy edges
#endif
#ifndef GG_BATCH_PULL_TAIL
#define GG_BATCH_PULL_TAIL 1   // normalised buckets: a pull after which the buckets end writes the tail's frontier
#endif
#ifndef GG_BATCH_PULL
#define GG_BATCH_PULL 1   // normalised buckets: heavy supersteps by pull on symmetric graphs
#endif
#ifndef GG_BATCH_UNROLL
#define GG_BATCH_UNROLL 4   // superstep kernels per iteration of the batch's CUDA-graph loop
#endif

struct BSmem {
  uint32_t qv[kBCap], qr[kBCap], qd[kBCap];   // split step: CTA queue; otherwise kBQW per warp
  // per warp, per edge of the current 32-edge chunk: target vertex and the
  // sources it improved (near, far), appended together after the chunk
  unsigned long long pm[kBNW][32], pf[kBNW][32];
  uint32_t pv[kBNW][32];
  uint32_t rq[kBNW * kBQW];   // light-first rounds: per-warp queue of new R entries
  uint32_t wsum[kBNW];
  // per source of the group: near limit max(t_cur - sh, 0), split floor
  // max(t_prev - sh, 0) and the shift itself (all sh = 0 without normalised buckets)
  uint32_t tabs[64], tprev[64], shs[64];
  uint32_t qn, j, last, ovf;
  unsigned long long base;
  // per-CTA sums of what every warp reports (one global atomic per CTA at the end)
  unsigned long long hacc, pedges;   // heavy edges of newly settled pairs; edges a pull scanned
  uint32_t fmin;                     // smallest shifted distance parked
};

// Eight consecutive distances row[0..7] into d[], read only where bit q of
// `on` is set (the other entries are left unspecified and must not be used).
// VEC: the row is 16-byte aligned and read as two 16-byte vectors, each only
// when one of its four bits is set (a set bit implies the whole vector lies
// inside the matrix: groups are 4-aligned when VEC).
template <bool VEC>
__device__ __forceinline__ void load_row8(const uint32_t* row, uint32_t on, uint32_t (&d)[8]) {
  if (VEC) {
    uint4 a, b;
    if (on & 0x0Fu) a = __ldcg(reinterpret_cast<const uint4*>(row));
    if (on & 0xF0u) b = __ldcg(reinterpret_cast<const uint4*>(row) + 1);
    d[0] = a.x;
    d[1] = a.y;
    d[2] = a.z;
    d[3] = a.w;
    d[4] = b.x;
    d[5] = b.y;
    d[6] = b.z;
    d[7] = b.w;
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if ((on >> q) & 1u) d[q] = ld_cg(row + q);
  }
}

// Append of up to 32 vertices, one per lane (have), to the list (fv, fr, fs)
// whose counter is cnt: each brings the edges [rs, re) of its row, read here
// (start[v], end[v]); vertices without such edges are left out.  One 64-bit
// atomicAdd returns the list position and the edge-prefix base.
__device__ __forceinline__ void b_append32(bool have, uint32_t v, const uint32_t* __restrict__ start,
                                           const uint32_t* __restrict__ end, unsigned long long* cnt,
                                           uint32_t* fv, uint32_t* fr, uint32_t* fs) {
  const unsigned FULL = 0xFFFFFFFFu;
  const uint32_t lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  uint32_t rs = 0, d = 0;
  if (have) {
    rs = __ldg(start + v);
    d = __ldg(end + v) - rs;
  }
  const bool keep = d > 0;
  const unsigned b = __ballot_sync(FULL, keep);
  if (b == 0u) return;
  uint32_t x = d;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  const uint32_t tot = __shfl_sync(FULL, x, 31);
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(cnt, ((unsigned long long)__popc(b) << 32) | tot);
  base = __shfl_sync(FULL, base, 0);
  if (keep) {
    const uint32_t pos = (uint32_t)(base >> 32) + __popc(b & lt);
    fv[pos] = v;
    fr[pos] = rs;
    fs[pos] = (uint32_t)base + x - d;
  }
}

template <bool PK, bool VEC, bool LH>
__global__ void __launch_bounds__(kBB, GG_BMINB) k_batch_superstep(DevGraph g, BatchBufs w, cudaGraphConditionalHandle cond,
                                                         int use_cond) {
  __shared__ BSmem sm;
  BatchCtl* ctl = w.ctl;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (ctl->running == 0u) {   // a superstep node past the end of the loop (unrolled graph body)
    if (use_cond && blockIdx.x == 0 && tid == 0) cudaGraphSetConditional(cond, 0u);
    return;
  }
  const uint32_t it = ctl->iter;
  const uint32_t pc = it % 3, pn = (it + 1) % 3, po = (it + 2) % 3;
  const uint32_t bmode0 = ctl->mode;
  const uint32_t ep = LH ? ctl->epoch : 0u;
  // heavy superstep by pull (normalised buckets); mode 5: a pull after which
  // the buckets end, which writes the tail's first frontier itself
  const bool pull = LH && (bmode0 == 4u || bmode0 == 5u);
  const bool pull_tail = LH && bmode0 == 5u;
  const bool heavy = LH && (bmode0 == 2u || pull);
  const unsigned long long c = heavy ? ctl->rcnt[ep % 3] : ctl->cnt[pc];
  const uint32_t F = (uint32_t)(c >> 32), E = (uint32_t)c;
  const uint32_t K = ctl->k, col0 = ctl->col0;
  uint32_t* dist = ctl->dist;
  // the entries' source masks: the frontier's, or the R list's in a heavy superstep
  const unsigned long long* Mc = heavy ? pick3(w.rmask, ep % 3) : pick3(w.mask, pc);
  unsigned long long* Mn = pick3(w.mask, pn);
  const uint32_t wbits = g.wbits;
  const uint32_t T = ctl->t_cur, fsel = ctl->fsel, bmode = heavy ? 0u : bmode0;
  const bool tailm = LH && ctl->tail != 0u;   // normalised buckets ended: full rows, no R
  const bool nbm = LH && ctl->nb != 0u;
  if (tid < 64) {
    const uint32_t sh = ctl->sh[tid], tp = ctl->t_prev;
    sm.shs[tid] = sh;
    sm.tabs[tid] = T == kInf ? kInf : (T > sh ? T - sh : 0u);
    sm.tprev[tid] = tp > sh ? tp - sh : 0u;
  }
  // new R entries join the epoch in progress (the next one during a heavy superstep)
  const uint32_t rj = (heavy ? ep + 1u : ep) % 3;
  // zero the masks of F_{t-1}
  {
    const uint32_t Fo = (uint32_t)(ctl->cnt[po] >> 32);
    const uint32_t* fvo = pick3(w.fv, po);
    unsigned long long* Mo = pick3(w.mask, po);
    for (uint32_t i = blockIdx.x * kBB + tid; i < Fo; i += gridDim.x * kBB) Mo[fvo[i]] = 0ull;
  }
  // and those of the R list the last heavy superstep consumed
  if (LH && ctl->zero_pending) {
    const uint32_t zp = ctl->zero_par;
    const uint32_t Ro = (uint32_t)(ctl->rcnt[zp] >> 32);
    const uint32_t* rvo = pick3(w.rv, zp);
    unsigned long long* RMo = pick3(w.rmask, zp);
    for (uint32_t i = blockIdx.x * kBB + tid; i < Ro; i += gridDim.x * kBB) RMo[rvo[i]] = 0ull;
  }
  if (tid == 0) {
    sm.qn = 0;
    sm.ovf = 0;
    sm.hacc = 0ull;
    sm.pedges = 0ull;
    sm.fmin = kInf;
  }
  __syncthreads();
  bool ovf = false;
  if (pull) {
    // Heavy superstep by pull (symmetric graphs: the heavy in-edges of v are
    // its heavy out-edges): every vertex with an unsettled pair (dist[v][s]
    // at or above its source's threshold) takes, for each such source, the
    // minimum of dist[u][s] + w over its heavy edges (u, w) from the pairs of
    // the epoch's R masks.  One vertex per warp, lane l holds sources l and
    // l + 32; four edges' distance rows in flight at a time.  A settled pair
    // is never written and an unsettled one is only written by its own
    // vertex's warp, so no atomics on dist.  With the bucket no wider than
    // the light/heavy width every improvement is at or above the threshold:
    // it is parked (far mask and list).
    const unsigned FULL = 0xFFFFFFFFu;
    const unsigned long long* Rm = pick3(w.rmask, ep % 3);
    const uint32_t kgv = ctl->kg;
    const bool vlo = lane < kgv, vhi = lane + 32 < kgv;
    const uint32_t tc_lo = sm.tabs[lane], tc_hi = sm.tabs[lane + 32];
    const uint32_t sh_lo = sm.shs[lane], sh_hi = sm.shs[lane + 32];
    uint32_t* fq = sm.qd + warp * kBQW;
    uint32_t fqn = 0;   // warp-uniform
    uint32_t wfm = kInf;
    unsigned long long scanned = 0ull;
    // pull_tail: the tail's frontier queue (vertices with whole rows)
    uint32_t* tq = sm.qv + warp * kBQW;
    uint32_t tqn = 0;   // warp-uniform
    unsigned long long* Mn_t = pick3(w.mask, pn);
    auto tflush = [&]() {
      __syncwarp();
      for (uint32_t j0 = 0; j0 < tqn; j0 += 32)
        b_append32(j0 + lane < tqn, j0 + lane < tqn ? tq[j0 + lane] : 0u, g.ro, g.ro + 1, &ctl->cnt[pn],
                   pick3(w.fv, pn), pick3(w.fr, pn), pick3(w.fs, pn));
      tqn = 0;
      __syncwarp();
    };
    if (pull_tail) {
      // the other two frontier mask arrays are cleared whole (a vertex
      // without light edges may hold bits no list carries); the next
      // frontier's mask is written for every vertex below
      for (uint32_t i = blockIdx.x * kBB + tid; i < g.n; i += gridDim.x * kBB) {
        pick3(w.mask, pc)[i] = 0ull;
        pick3(w.mask, po)[i] = 0ull;
      }
    }
    auto ffl = [&]() {
      __syncwarp();
      uint32_t pos = 0;
      if (lane == 0) pos = atomicAdd(&ctl->fcnt[fsel], fqn);
      pos = __shfl_sync(FULL, pos, 0);
      for (uint32_t j = lane; j < fqn; j += 32) pick2(w.far_v, fsel)[pos + j] = fq[j];
      fqn = 0;
      __syncwarp();
    };
    const uint32_t nwarps = gridDim.x * kBNW;
    for (uint32_t v = blockIdx.x * kBNW + warp; v < g.n; v += nwarps) {   // warp-uniform
      const uint32_t hs = __ldg(w.lend + v), he = __ldg(g.ro + v + 1);
      if (pull_tail) {
        if (__ldg(g.ro + v) >= he) {   // no edges: nothing to expand
          if (lane == 0) Mn_t[v] = 0ull;
          continue;
        }
      } else if (hs >= he) {
        continue;
      }
      uint32_t* vrow = dist + (size_t)v * K + col0;
      const uint32_t dlo = vlo ? ld_cg(vrow + lane) : 0u, dhi = vhi ? ld_cg(vrow + lane + 32) : 0u;
      const unsigned Ulo = __ballot_sync(FULL, vlo && dlo >= tc_lo), Uhi = __ballot_sync(FULL, vhi && dhi >= tc_hi);
      if ((Ulo | Uhi) == 0u) {
        if (pull_tail && lane == 0) Mn_t[v] = 0ull;
        continue;
      }
      const unsigned long long U = ((unsigned long long)Uhi << 32) | Ulo;
      scanned += he - hs;
      uint32_t clo = dlo, chi = dhi;
      for (uint32_t e0 = hs; e0 < he; e0 += 32) {
        const uint32_t e = e0 + lane;
        uint32_t u = 0, wt = 0;
        unsigned long long r = 0ull;
        if (e < he) {
          const uint2 ed = load_edge<PK>(w.ledges, e, wbits);
          u = ed.x;
          wt = ed.y;
          r = __ldcg(Rm + u) & U;
        }
        unsigned rb = __ballot_sync(FULL, r != 0ull);
        while (rb) {   // warp-uniform
          uint32_t xl[4], xh[4], ww[4];
          bool bl[4], bh[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const bool have = rb != 0u;
            const uint32_t j = have ? (uint32_t)(__ffs(rb) - 1) : 0u;
            rb &= rb - 1u;
            const uint32_t uj = __shfl_sync(FULL, u, j);
            ww[q] = __shfl_sync(FULL, wt, j);
            const uint32_t rl = __shfl_sync(FULL, (uint32_t)r, j), rh = __shfl_sync(FULL, (uint32_t)(r >> 32), j);
            bl[q] = have && ((rl >> lane) & 1u);
            bh[q] = have && ((rh >> lane) & 1u);
            const uint32_t* urow = dist + (size_t)uj * K + col0;
            xl[q] = bl[q] ? ld_cg(urow + lane) : 0u;
            xh[q] = bh[q] ? ld_cg(urow + lane + 32) : 0u;
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (bl[q]) clo = min(clo, add_sat(xl[q], ww[q], ovf));
            if (bh[q]) chi = min(chi, add_sat(xh[q], ww[q], ovf));
          }
        }
      }
      const bool il = clo < dlo, ih = chi < dhi;
      if (il) {
        vrow[lane] = clo;
        wfm = min(wfm, (uint32_t)min(0xFFFFFFFFull, (unsigned long long)clo + sh_lo));
      }
      if (ih) {
        vrow[lane + 32] = chi;
        wfm = min(wfm, (uint32_t)min(0xFFFFFFFFull, (unsigned long long)chi + sh_hi));
      }
      if (pull_tail) {
        // the tail's first frontier: every pair not settled (at or above the
        // threshold) with a finite distance (the pairs a split would release
        // from the far masks), with whole rows
        const unsigned Tl = __ballot_sync(FULL, vlo && clo >= tc_lo && clo != kInf);
        const unsigned Th = __ballot_sync(FULL, vhi && chi >= tc_hi && chi != kInf);
        const unsigned long long tb = ((unsigned long long)Th << 32) | Tl;
        if (lane == 0) Mn_t[v] = tb;
        if (tb) {
          if (lane == 0) tq[tqn] = v;
          if (++tqn == kBQW) tflush();
        }
        continue;
      }
      const unsigned Il = __ballot_sync(FULL, il), Ih = __ballot_sync(FULL, ih);
      if (Il | Ih) {   // park the improved pairs
        bool fapp = false;
        if (lane == 0) fapp = atomicOr(w.fmask + v, ((unsigned long long)Ih << 32) | Il) == 0ull;
        if (__shfl_sync(FULL, fapp, 0)) {
          if (lane == 0) fq[fqn] = v;
          if (++fqn == kBQW) ffl();
        }
      }
    }
    if (fqn) ffl();
    if (tqn) tflush();
#pragma unroll
    for (int o = 16; o; o >>= 1) wfm = min(wfm, __shfl_xor_sync(FULL, wfm, o));
    if (lane == 0 && wfm != kInf && !pull_tail) atomicMin(&sm.fmin, wfm);
    if (lane == 0 && scanned) atomicAdd(&sm.pedges, scanned);
  } else if (bmode == 3) {
    // before the tail's split: clear the three frontier mask arrays.  A vertex
    // without light edges may hold mask bits that no frontier list carries
    // (nothing clears them), which would keep it out of the tail's frontier.
    for (uint32_t i = blockIdx.x * kBB + tid; i < g.n; i += gridDim.x * kBB) {
      w.mask[0][i] = 0ull;
      w.mask[1][i] = 0ull;
      w.mask[2][i] = 0ull;
    }
  } else if (bmode == 1) {
    // split step: every parked (vertex, source) bit is re-examined against
    // the raised threshold: below the previous threshold it was expanded
    // already (drop), below the new one it joins the next frontier (and, in
    // light-first rounds with buckets, the epoch's R mask), otherwise it stays
    // parked.  One far vertex per warp; lane l holds sources l and l + 32.
    const unsigned FULL = 0xFFFFFFFFu;
    const uint32_t nfar = ctl->fcnt[fsel];
    const uint32_t* fend = (LH && !tailm) ? w.lend : g.ro + 1;   // frontier rows: light edges, or all
    const uint32_t rj = ep % 3;
    uint32_t* qv = sm.qv + warp * kBQW;
    uint32_t* rq = sm.rq + warp * kBQW;
    uint32_t qn = 0, rqn = 0;   // warp-uniform
    unsigned long long hacc = 0ull;   // lane 0: heavy edges of the pairs settling here
    const uint32_t tp_lo = sm.tprev[lane], tp_hi = sm.tprev[lane + 32];
    const uint32_t tc_lo = sm.tabs[lane], tc_hi = sm.tabs[lane + 32];
    const uint32_t sh_lo = sm.shs[lane], sh_hi = sm.shs[lane + 32];
    uint32_t wfm = kInf;
    uint32_t* kq = sm.qd + warp * kBQW;   // vertices that keep parked bits
    uint32_t kqn = 0;                     // warp-uniform
    auto kflush = [&]() {
      __syncwarp();
      uint32_t pos = 0;
      if (lane == 0) pos = atomicAdd(&ctl->fcnt[fsel ^ 1u], kqn);
      pos = __shfl_sync(FULL, pos, 0);
      for (uint32_t j = lane; j < kqn; j += 32) pick2(w.far_v, fsel ^ 1u)[pos + j] = kq[j];
      kqn = 0;
      __syncwarp();
    };
    // the next far vertex and its parked bits are read while this one is worked on
    const uint32_t* far_in = pick2(w.far_v, fsel);
    const uint32_t wstride = gridDim.x * kBNW;
    uint32_t nv = 0, ni = blockIdx.x * kBNW + warp;
    unsigned long long nbits = 0ull;
    if (ni < nfar) {
      nv = far_in[ni];
      nbits = w.fmask[nv];
    }
    for (uint32_t i = blockIdx.x * kBNW + warp; i < nfar; i += wstride) {   // warp-uniform
      const uint32_t v = nv;
      const unsigned long long bits = nbits;
      const uint32_t* vrow = dist + (size_t)v * K + col0;
      const bool lo = (bits >> lane) & 1ull, hi = (bits >> (lane + 32)) & 1ull;
      const uint32_t dlo = lo ? ld_cg(vrow + lane) : 0u, dhi = hi ? ld_cg(vrow + lane + 32) : 0u;
      ni = i + wstride;
      if (ni < nfar) nv = far_in[ni];
      const bool mlo = lo && dlo >= tp_lo && dlo < tc_lo, mhi = hi && dhi >= tp_hi && dhi < tc_hi;
      const bool klo = lo && dlo >= tc_lo, khi = hi && dhi >= tc_hi;
      const unsigned nb_lo = __ballot_sync(FULL, mlo), nb_hi = __ballot_sync(FULL, mhi);
      const unsigned kb_lo = __ballot_sync(FULL, klo), kb_hi = __ballot_sync(FULL, khi);
      if (ni < nfar) nbits = w.fmask[nv];   // far-list entries are distinct: not this vertex's word
      // smallest shifted distance left parked (one atomic per warp at the end)
      if (klo) wfm = min(wfm, (uint32_t)min(0xFFFFFFFFull, (unsigned long long)dlo + sh_lo));
      if (khi) wfm = min(wfm, (uint32_t)min(0xFFFFFFFFull, (unsigned long long)dhi + sh_hi));
      bool app = false, rapp = false;
      if (kb_lo | kb_hi) {   // stays on the (other) far list: per-warp queue
        if (lane == 0) kq[kqn] = v;
        if (++kqn == kBQW) kflush();
      }
      if (lane == 0) {
        const unsigned long long kb = (unsigned long long)kb_lo | ((unsigned long long)kb_hi << 32);
        const unsigned long long nb = (unsigned long long)nb_lo | ((unsigned long long)nb_hi << 32);
        w.fmask[v] = kb;
        if (nb) {
          app = atomicOr(Mn + v, nb) == 0ull;
          if (LH && !tailm) {
            const unsigned long long old = atomicOr(pick3(w.rmask, rj) + v, nb);
            rapp = old == 0ull;
            const unsigned long long nw = nb & ~old;
            if (nbm && nw) hacc += (unsigned long long)__popcll(nw) * (__ldg(g.ro + v + 1) - __ldg(w.lend + v));
          }
        }
      }
      app = __shfl_sync(FULL, app, 0);
      rapp = __shfl_sync(FULL, rapp, 0);
      if (app) {
        if (lane == 0) qv[qn] = v;
        if (++qn == kBQW) {
          __syncwarp();
          for (uint32_t j0 = 0; j0 < qn; j0 += 32)
            b_append32(j0 + lane < qn, j0 + lane < qn ? qv[j0 + lane] : 0u, g.ro, fend, &ctl->cnt[pn],
                       pick3(w.fv, pn), pick3(w.fr, pn), pick3(w.fs, pn));
          qn = 0;
          __syncwarp();
        }
      }
      if (LH && rapp) {
        if (lane == 0) rq[rqn] = v;
        if (++rqn == kBQW) {
          __syncwarp();
          for (uint32_t j0 = 0; j0 < rqn; j0 += 32)
            b_append32(j0 + lane < rqn, j0 + lane < rqn ? rq[j0 + lane] : 0u, w.lend, g.ro + 1, &ctl->rcnt[rj],
                       pick3(w.rv, rj), pick3(w.rr, rj), pick3(w.rs, rj));
          rqn = 0;
          __syncwarp();
        }
      }
    }
    __syncwarp();
    for (uint32_t j0 = 0; j0 < qn; j0 += 32)
      b_append32(j0 + lane < qn, j0 + lane < qn ? qv[j0 + lane] : 0u, g.ro, fend, &ctl->cnt[pn], pick3(w.fv, pn),
                 pick3(w.fr, pn), pick3(w.fs, pn));
    if (LH)
      for (uint32_t j0 = 0; j0 < rqn; j0 += 32)
        b_append32(j0 + lane < rqn, j0 + lane < rqn ? rq[j0 + lane] : 0u, w.lend, g.ro + 1, &ctl->rcnt[rj],
                   pick3(w.rv, rj), pick3(w.rr, rj), pick3(w.rs, rj));
    if (kqn) kflush();
#pragma unroll
    for (int o = 16; o; o >>= 1) wfm = min(wfm, __shfl_xor_sync(FULL, wfm, o));
    if (lane == 0 && wfm != kInf) atomicMin(&sm.fmin, wfm);
    if (lane == 0 && hacc) atomicAdd(&sm.hacc, hacc);
  } else if (F > 0) {
    // Warp streaming, no block barriers: every warp of the grid takes an
    // equal contiguous share of the frontier's edge coordinates and walks it
    // 32 edges at a time.  The frontier entries covering the current edges
    // sit in a sliding window of 32 entries, one per lane (first coordinate,
    // row start, vertex, source mask); a lane finds its edge's entry with a
    // 5-step shuffle search.  The warp then relaxes the 32 edges four at a
    // time, one per 8-lane group: lane l8 of a group holds the eight
    // consecutive sources 8*l8 .. 8*l8+7 of the 64-source group, one 32-byte
    // sector of a distance row (two 16-byte vectors when VEC).
    const unsigned FULL = 0xFFFFFFFFu;
    const uint32_t* S = heavy ? pick3(w.rs, ep % 3) : pick3(w.fs, pc);
    const uint32_t* R = heavy ? pick3(w.rr, ep % 3) : pick3(w.fr, pc);
    const uint32_t* V = heavy ? pick3(w.rv, ep % 3) : pick3(w.fv, pc);
    const void* edges = LH ? w.ledges : g.edges;
    constexpr uint32_t QW = kBQW;
    uint32_t* rq = sm.rq + warp * QW;   // light-first rounds: new R entries
    uint32_t rqn = 0;                   // warp-uniform
    uint32_t* qv = sm.qv + warp * QW;   // this warp's queue of new frontier vertices
    uint32_t* qr = sm.qr + warp * QW;
    uint32_t* qd = sm.qd + warp * QW;
    uint32_t qn = 0;                    // warp-uniform
    unsigned long long hacc = 0ull;     // warp-uniform: heavy edges of pairs that settled (normalised buckets)
    uint32_t wfm = kInf;                // smallest shifted distance this lane parked
    uint32_t* fq = sm.qd + warp * QW;   // light-first rounds: this warp's queue of new far-list vertices
    uint32_t fqn = 0;                   // warp-uniform
    const uint32_t g4 = lane >> 3, l8 = lane & 7;
    const unsigned lt = (1u << lane) - 1u;
    const bool buckets = T != kInf;     // uniform
    const unsigned long long Wn = (unsigned long long)gridDim.x * kBNW;
    const unsigned long long gw = (unsigned long long)blockIdx.x * kBNW + warp;
    const uint32_t w0 = (uint32_t)((E * gw) / Wn), w1 = (uint32_t)((E * (gw + 1)) / Wn);

    auto flush = [&]() {
      // rows (deferred on sink-free graphs), warp scan of the degrees, one
      // 64-bit atomic for the queue position and the edge-prefix base
      __syncwarp();
      if (LH) {   // light edges [ro[v], lend[v]) (all edges in the tail); vertices without any are left out
        const uint32_t* fend = tailm ? g.ro + 1 : w.lend;
        for (uint32_t i0 = 0; i0 < qn; i0 += 32) {
          const uint32_t i = i0 + lane;
          b_append32(i < qn, i < qn ? qv[i] : 0u, g.ro, fend, &ctl->cnt[pn], pick3(w.fv, pn), pick3(w.fr, pn),
                     pick3(w.fs, pn));
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
          if (!g.sinks) {
            const uint32_t rs = __ldg(g.ro + qv[i]);
            d = __ldg(g.ro + qv[i] + 1) - rs;
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
      unsigned long long bse = 0;
      if (lane == 0) bse = atomicAdd(&ctl->cnt[pn], ((unsigned long long)qn << 32) | run);
      bse = __shfl_sync(FULL, bse, 0);
      __syncwarp();
      const uint32_t pos0 = (uint32_t)(bse >> 32), eb0 = (uint32_t)bse;
      for (uint32_t i = lane; i < qn; i += 32) {
        pick3(w.fv, pn)[pos0 + i] = qv[i];
        pick3(w.fr, pn)[pos0 + i] = qr[i];
        pick3(w.fs, pn)[pos0 + i] = eb0 + qd[i];
      }
      qn = 0;
      __syncwarp();
    };
    auto ffl = [&]() {   // the warp's new far-list vertices, one atomicAdd
      __syncwarp();
      uint32_t pos = 0;
      if (lane == 0) pos = atomicAdd(&ctl->fcnt[fsel], fqn);
      pos = __shfl_sync(FULL, pos, 0);
      for (uint32_t i = lane; i < fqn; i += 32) pick2(w.far_v, fsel)[pos + i] = fq[i];
      fqn = 0;
      __syncwarp();
    };
    auto rflush = [&]() {   // heavy edges [lend[v], ro[v+1]) of new R entries
      __syncwarp();
      for (uint32_t i0 = 0; i0 < rqn; i0 += 32) {
        const uint32_t i = i0 + lane;
        b_append32(i < rqn, i < rqn ? rq[i] : 0u, w.lend, g.ro + 1, &ctl->rcnt[rj], pick3(w.rv, rj),
                   pick3(w.rr, rj), pick3(w.rs, rj));
      }
      rqn = 0;
      __syncwarp();
    };

    if (w0 < w1) {   // warp-uniform
      uint32_t j = warp_search_le(S, F, w0);
      uint32_t ws = 0, wr = 0, wv = 0, wend = 0;
      unsigned long long wm = 0ull;
      auto load_window = [&]() {
        const uint32_t idx = j + lane;
        ws = 0xFFFFFFFFu;
        wm = 0ull;
        if (idx < F) {
          ws = S[idx];
          wr = R[idx];
          wv = V[idx];
          wm = Mc[wv];
        }
        wend = j + 32 < F ? S[j + 32] : E;   // first coordinate past the window
      };
      load_window();
      uint32_t cur_j = 0xFFFFFFFFu, amask = 0u, dmax = 0u;
      uint32_t du[8];   // the current source row, where amask has a bit
      for (uint32_t b = w0; b < w1; b += 32) {
        // slide until the window holds chunk [b, b+32) (at most two slides)
        for (int guard = 0; guard < 4 && min(b + 31, w1 - 1) >= wend; ++guard) {
          const unsigned le = __ballot_sync(FULL, ws <= b);
          if (le == 0u) break;   // cannot happen while S[j] <= b holds
          const uint32_t adv = (le == FULL && wend <= b) ? 32u : 31u - (uint32_t)__clz(le);
          j += adv;
          load_window();
          cur_j = 0xFFFFFFFFu;   // window positions changed
        }
        // each lane loads one edge of the chunk and notes its window entry
        const uint32_t gidx = b + lane;
        uint32_t k = 0;
#pragma unroll
        for (int step = 16; step; step >>= 1) {
          const uint32_t sv = __shfl_sync(FULL, ws, k + step);
          if (sv <= gidx) k += step;
        }
        const uint32_t ks = __shfl_sync(FULL, ws, k);
        const uint32_t kr = __shfl_sync(FULL, wr, k);
        const uint32_t kn = __shfl_sync(FULL, ws, (k + 1) & 31u);
        const uint32_t ke = k == 31 ? wend : kn;
        // [ks, ke) holds gidx whenever S increases strictly; the test keeps
        // every edge read inside the entry's row regardless
        const bool valid = gidx < w1 && ks <= gidx && gidx < ke;
        uint32_t vv = 0, ww = 0;
        if (valid) {
          const uint2 ed = load_edge<PK>(edges, kr + (gidx - ks), wbits);
          vv = ed.x;
          ww = ed.y;
        }
        const unsigned vm = __ballot_sync(FULL, valid);
        const int nvalid = __popc(vm);   // valid edges are a prefix of the lanes
        for (int i0 = 0; i0 < nvalid; i0 += 4) {
          const int i = i0 + (int)g4;
          const bool live = i < nvalid;
          const int isrc = live ? i : nvalid - 1;
          const uint32_t ji = __shfl_sync(FULL, k, isrc);
          const uint32_t vi = __shfl_sync(FULL, vv, isrc);
          const uint32_t wi = __shfl_sync(FULL, ww, isrc);
          const bool need = live && ji != cur_j;
          if (__any_sync(FULL, need)) {
            const uint32_t uu = __shfl_sync(FULL, wv, ji);
            const uint32_t mlo = __shfl_sync(FULL, (uint32_t)wm, ji);
            const uint32_t mhi = __shfl_sync(FULL, (uint32_t)(wm >> 32), ji);
            if (need) {   // uniform within the group
              cur_j = ji;
              amask = ((l8 < 4 ? mlo : mhi) >> (8 * (l8 & 3))) & 0xFFu;
              load_row8<VEC>(dist + (size_t)uu * K + col0 + 8 * l8, amask, du);
              dmax = 0u;
#pragma unroll
              for (int q = 0; q < 8; ++q)
                if ((amask >> q) & 1u) dmax = max(dmax, du[q]);
            }
          }
          const uint32_t am = live ? amask : 0u;
          uint32_t* vrow = dist + (size_t)vi * K + col0 + 8 * l8;
          uint32_t cv[8];
          load_row8<VEC>(vrow, am, cv);
          uint32_t near = 0u, far = 0u, fm = kInf;
          // fast path: no buckets and no sum of this row can reach kInf (the
          // largest active source distance plus w fits), so plain adds suffice
          if (!buckets && __all_sync(FULL, am == 0u || dmax < kInf - wi)) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              if ((am >> q) & 1u) {
                const uint32_t nd = du[q] + wi;
                if (nd < cv[q]) {
                  atomicMin(vrow + q, nd);
                  near |= 1u << q;
                }
              }
            }
          } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              if ((am >> q) & 1u) {
                const uint32_t nd = add_sat(du[q], wi, ovf);
                if (nd < cv[q]) {
                  atomicMin(vrow + q, nd);
                  // near bits (new distance below the source's threshold) join
                  // the next frontier's mask; the others are parked in the far
                  // mask, and the smallest shifted distance parked is kept
                  if (nd < sm.tabs[8 * l8 + q]) {
                    near |= 1u << q;
                  } else {
                    far |= 1u << q;
                    fm = min(fm, (uint32_t)min(0xFFFFFFFFull, (unsigned long long)nd + sm.shs[8 * l8 + q]));
                  }
                }
              }
            }
          }
          // the group's 64-bit masks: OR of the lanes' bytes over the 8-lane group
          unsigned long long nmask = (unsigned long long)near << (8 * l8);
          unsigned long long fmask = (unsigned long long)far << (8 * l8);
          if (__any_sync(FULL, near != 0u)) {   // most late relaxations improve nothing
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) nmask |= __shfl_xor_sync(FULL, nmask, o);
          }
          if (buckets) {   // uniform: only with buckets can anything be parked
            const unsigned anyf = __ballot_sync(FULL, far != 0u);
            if (anyf) {
#pragma unroll
              for (int o = 1; o < 8; o <<= 1) fmask |= __shfl_xor_sync(FULL, fmask, o);
            }
          }
          wfm = min(wfm, fm);   // one atomic per warp at the end of the pass, not per group of edges
          if (l8 == 0 && live) {
            sm.pv[warp][i] = vi;
            sm.pm[warp][i] = nmask;
            sm.pf[warp][i] = fmask;
          }
        }
        // the chunk's appends, one edge per lane, their atomics in flight together
        __syncwarp();
        bool app = false, fapp = false, rapp = false;
        uint32_t vi = 0, rs = 0, re = 1;
        unsigned long long hset = 0ull;
        if (lane < (uint32_t)nvalid) {
          const unsigned long long nb = sm.pm[warp][lane], fb = sm.pf[warp][lane];
          if (nb | fb) {
            vi = sm.pv[warp][lane];
            // vertices without out-edges are never appended; on a graph
            // without such sinks (and in light-first rounds, whose appends
            // check both degrees) the row is read at the flush instead
            if (g.sinks && !LH) {
              rs = __ldg(g.ro + vi);
              re = __ldg(g.ro + vi + 1);
            }
            if (re > rs) {
              app = nb && atomicOr(Mn + vi, nb) == 0ull;
              fapp = fb && atomicOr(w.fmask + vi, fb) == 0ull;
              if (LH && !tailm && nb) {
                const unsigned long long old = atomicOr(pick3(w.rmask, rj) + vi, nb);
                rapp = old == 0ull;
                const unsigned long long nw = nb & ~old;
                if (nbm && nw) hset = (unsigned long long)__popcll(nw) * (__ldg(g.ro + vi + 1) - __ldg(w.lend + vi));
              }
            }
          }
        }
        if (nbm && __any_sync(FULL, hset != 0ull)) {   // pairs that settled into the bucket: their heavy edges
#pragma unroll
          for (int o = 16; o; o >>= 1) hset += __shfl_xor_sync(FULL, hset, o);
          hacc += hset;
          hset = 0ull;
        }
        if (LH) {
          const unsigned rb = __ballot_sync(FULL, rapp);
          if (rb) {
            if (rapp) rq[rqn + __popc(rb & lt)] = vi;
            rqn += __popc(rb);
            if (rqn > QW - 32) rflush();
          }
        }
        const unsigned ab = __ballot_sync(FULL, app);
        if (ab) {
          if (app) {
            const uint32_t off = qn + __popc(ab & lt);
            qv[off] = vi;
            if (!LH) {   // light-first rounds read the rows at the flush
              qr[off] = rs;
              qd[off] = re - rs;
            }
          }
          qn += __popc(ab);
          if (qn > QW - 32) flush();
        }
        const unsigned fbal = __ballot_sync(FULL, fapp);
        if (fbal) {
          if (LH) {   // per-warp far queue, one atomic per flush
            if (fapp) fq[fqn + __popc(fbal & lt)] = vi;
            fqn += __popc(fbal);
            if (fqn > QW - 32) ffl();
          } else {    // far list: one atomic per warp
            uint32_t pos = 0;
            if (lane == 0) pos = atomicAdd(&ctl->fcnt[fsel], (uint32_t)__popc(fbal));
            pos = __shfl_sync(FULL, pos, 0);
            if (fapp) pick2(w.far_v, fsel)[pos + __popc(fbal & lt)] = vi;
          }
        }
        __syncwarp();
      }
      if (LH && fqn) ffl();
      if (qn) flush();
      if (LH && rqn) rflush();
    }
    if (lane == 0 && hacc) atomicAdd(&sm.hacc, hacc);
    if (buckets) {
#pragma unroll
      for (int o = 16; o; o >>= 1) wfm = min(wfm, __shfl_xor_sync(FULL, wfm, o));
      if (lane == 0 && wfm != kInf) atomicMin(&sm.fmin, wfm);
    }
  }
  if (ovf) sm.ovf = 1u;
  __syncthreads();
  if (tid == 0) {
    if (sm.ovf) atomicOr(&ctl->status, DS_OVERFLOW);
    if (sm.fmin != kInf) atomicMin(&ctl->far_min, sm.fmin);
    if (sm.hacc) atomicAdd(&ctl->heavy_settled, sm.hacc);
    if (sm.pedges) atomicAdd(&ctl->pull_edges, sm.pedges);
    sm.last = arrive_last(&ctl->done_ctas, gridDim.x) ? 1u : 0u;
  }
  __syncthreads();
  if (sm.last && tid == 0) {
    const unsigned long long cn = atomicAdd(&ctl->cnt[pn], 0ull);
    const uint32_t fn = (uint32_t)(cn >> 32);
    if (ctl->trace && it < ctl->trace_cap) {
      uint32_t* t = ctl->trace + 4ull * it;
      t[0] = bmode0 | (tailm ? 16u : 0u);
      t[1] = F;
      t[2] = E;
      t[3] = fn;
    }
    if (pull) {
      ctl->edges_scanned += ctl->pull_edges;
      ctl->pull_edges = 0ull;
      ctl->frontier_total += F;
    } else if (F > 0 && bmode == 0) {
      ctl->edges_scanned += E;
      ctl->frontier_total += F;
      ctl->max_frontier = max(ctl->max_frontier, F);
    }
    if (LH) {
      ctl->cnt[po] = 0ull;
      ctl->done_ctas = 0u;
      ctl->iter = it + 1;
      if (ctl->zero_pending) {   // this superstep cleared that list's masks
        ctl->rcnt[ctl->zero_par] = 0ull;
        ctl->zero_pending = 0u;
      }
      if (heavy) {
        ctl->zero_pending = 1u;
        ctl->zero_par = ep % 3;
        ctl->epoch = ep + 1u;
      }
      const uint32_t rn = (uint32_t)(atomicAdd(&ctl->rcnt[ctl->epoch % 3], 0ull) >> 32);
      uint32_t mode_next = fn > 0 ? 0u : 2u;
      bool more = fn != 0 || rn != 0;
      if (ctl->nb) {
        uint32_t fs_now = fsel;
        if (bmode == 1) {   // the pairs kept parked went to the other list
          ctl->fcnt[fsel] = 0u;
          fs_now = fsel ^ 1u;
          ctl->fsel = fs_now;
          ctl->splits += 1;
        }
        const uint32_t nfar = atomicAdd(&ctl->fcnt[fs_now], 0u);
        if (mode_next == 2u && fn == 0 && rn > 0) {
          // heavy superstep: pull when the pairs settled since the last one
          // hold more heavy edges than the pairs not settled yet
          const unsigned long long done = atomicAdd(&ctl->heavy_settled, 0ull);
          const unsigned long long hk = ctl->heavy_total_k;
          const unsigned long long open = hk > done ? hk - done : 0ull;
          if (ctl->pull_ok && done - ctl->settled_mark > open) mode_next = 4u;
          // a pull settles no pair, so the drain rule holds after it exactly
          // when it holds now: the split after it would end the buckets, so
          // the pull writes the tail's first frontier itself
          if (mode_next == 4u && GG_BATCH_PULL_TAIL && open < hk / ctl->drain_div) mode_next = 5u;
          ctl->settled_mark = done;
        }
        if (bmode0 == 5u) {   // the pull ended the buckets: plain push from its frontier on
          ctl->tail = 1u;
          ctl->t_prev = ctl->t_cur;
          ctl->t_cur = kInf;
          ctl->far_min = kInf;
          ctl->fcnt[0] = 0u;
          ctl->fcnt[1] = 0u;
          mode_next = 0u;
          more = fn != 0;
        } else if (bmode == 3) {   // masks cleared: the tail's split follows
          mode_next = 1u;
          more = true;
        } else if (!more && nfar > 0) {
          // the bucket is settled (no near pair, no heavy edge left): raise the
          // shared threshold to the next occupied bucket, or end bucketing once
          // the unsettled pairs hold few heavy edges (the rest is plain push)
          const unsigned long long hk = ctl->heavy_total_k;
          const unsigned long long done = atomicAdd(&ctl->heavy_settled, 0ull);
          const unsigned long long open = hk > done ? hk - done : 0ull;
          const unsigned long long t1 = (unsigned long long)ctl->t_cur + ctl->width;
          const unsigned long long t2 = (unsigned long long)atomicAdd(&ctl->far_min, 0u) + 1ull;
          unsigned long long tn = t1 > t2 ? t1 : t2;
          mode_next = 1u;
          if (open < hk / ctl->drain_div || tn >= (unsigned long long)kInf) {
            ctl->tail = 1u;
            tn = kInf;
            mode_next = 3u;   // clear the masks first
          }
          ctl->t_prev = ctl->t_cur;
          ctl->t_cur = (uint32_t)tn;
          ctl->far_min = kInf;
          more = true;
        }
      }
      ctl->mode = mode_next;
      if (more && it + 1 >= ctl->max_iter) {
        ctl->status |= DS_ITER_CAP;
        more = false;
      }
      ctl->running = more ? 1u : 0u;
      if (use_cond) cudaGraphSetConditional(cond, more ? 1u : 0u);
      return;
    }
    uint32_t fs_now = fsel;
    if (bmode == 1) {   // the kept vertices went to the other list
      ctl->fcnt[fsel] = 0u;
      fs_now = fsel ^ 1u;
      ctl->fsel = fs_now;
      ctl->splits += 1;
    }
    const uint32_t nfar = atomicAdd(&ctl->fcnt[fs_now], 0u);
    if (fn == 0 && nfar > 0) {
      const unsigned long long t1 = (unsigned long long)ctl->t_cur + ctl->delta;
      const unsigned long long t2 = (unsigned long long)atomicAdd(&ctl->far_min, 0u) + 1;
      const unsigned long long tn = t1 > t2 ? t1 : t2;
      ctl->t_prev = ctl->t_cur;
      ctl->t_cur = tn >= kInf ? kInf : (uint32_t)tn;
      ctl->far_min = kInf;
      ctl->mode = 1u;
    } else {
      ctl->mode = 0u;
    }
    ctl->cnt[po] = 0ull;
    ctl->done_ctas = 0u;
    ctl->iter = it + 1;
    bool more = fn != 0 || nfar != 0;
    if (more && it + 1 >= ctl->max_iter) {
      ctl->status |= DS_ITER_CAP;
      more = false;
    }
    ctl->running = more ? 1u : 0u;
    if (use_cond) cudaGraphSetConditional(cond, more ? 1u : 0u);
  }
}

// every entry of the n x k matrix := INF
__global__ void k_batch_fill(uint32_t* dist, unsigned long long count) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if ((reinterpret_cast<uintptr_t>(dist) & 15u) == 0) {
    uint4* d4 = reinterpret_cast<uint4*>(dist);
    const unsigned long long c4 = count / 4;
    for (unsigned long long i = t; i < c4; i += stride) d4[i] = make_uint4(kInf, kInf, kInf, kInf);
    for (unsigned long long i = c4 * 4 + t; i < count; i += stride) dist[i] = kInf;
  } else {
    for (unsigned long long i = t; i < count; i += stride) dist[i] = kInf;
  }
}

// group start: dist[src_s][col0+s] := 0; initial frontier = distinct sources
// with out-edges, each carrying the mask of its columns.  With normalised
// buckets each source's shift sh[s] = max o - o_s comes from its hub distance
// o_s (unreached from the hub: 0), and a source whose shift is not below the
// first threshold starts parked.  One CTA of 64.
__global__ void k_batch_seed(DevGraph g, BatchBufs w, const uint32_t* srcs, uint32_t k, uint32_t col0,
                             uint32_t kg, uint32_t* dist, uint32_t max_iter, uint32_t delta, uint32_t lh,
                             uint32_t nb, uint32_t width, uint32_t drain_div, unsigned long long heavy_total,
                             uint32_t* trace, uint32_t trace_cap, uint32_t pull_ok) {
  __shared__ uint32_t so[64];
  BatchCtl* ctl = w.ctl;
  const uint32_t s = threadIdx.x;
  uint32_t o = 0;
  if (nb && s < kg) {
    o = w.hubd[srcs[col0 + s]];
    if (o == kInf) o = 0;
  }
  so[s] = o;
  __syncthreads();
  uint32_t omax = 0;
  for (uint32_t i = 0; i < kg; ++i) omax = max(omax, so[i]);
  const uint32_t sh = s < kg ? omax - o : 0u;
  const uint32_t t0 = nb ? width : (lh ? kInf : delta);
  if (s == 0) {
    ctl->cnt[0] = 0ull;
    ctl->cnt[1] = 0ull;
    ctl->cnt[2] = 0ull;
    ctl->iter = 0;
    ctl->done_ctas = 0;
    ctl->status = 0;
    ctl->max_iter = max_iter;
    ctl->k = k;
    ctl->col0 = col0;
    ctl->kg = kg;
    ctl->dist = dist;
    ctl->max_frontier = 0;
    ctl->edges_scanned = 0;
    ctl->frontier_total = 0;
    ctl->t_cur = t0;
    ctl->t_prev = 0;
    ctl->delta = delta;
    ctl->fsel = 0;
    ctl->fcnt[0] = 0;
    ctl->fcnt[1] = 0;
    ctl->far_min = kInf;
    ctl->mode = 0;
    ctl->splits = 0;
    ctl->lh = lh;
    ctl->epoch = 0;
    ctl->zero_pending = 0;
    ctl->zero_par = 0;
    ctl->rcnt[0] = 0ull;
    ctl->rcnt[1] = 0ull;
    ctl->rcnt[2] = 0ull;
    ctl->nb = nb;
    ctl->tail = 0;
    ctl->width = width;
    ctl->drain_div = max(drain_div, 1u);
    ctl->heavy_total_k = heavy_total * kg;
    ctl->heavy_settled = 0ull;
    ctl->trace = trace;
    ctl->trace_cap = trace ? trace_cap : 0u;
    ctl->pull_ok = pull_ok;
    ctl->settled_mark = 0ull;
    ctl->pull_edges = 0ull;
  }
  ctl->sh[s] = sh;
  __syncthreads();
  if (s < kg) {
    const uint32_t v = srcs[col0 + s];
    dist[(size_t)v * k + col0 + s] = 0u;
    const uint32_t rs = g.ro[v], re = g.ro[v + 1];
    if (nb && sh >= t0) {   // parked until the threshold reaches its shift
      if (re > rs) {
        if (atomicOr(w.fmask + v, 1ull << s) == 0ull) {
          const uint32_t pos = atomicAdd(&ctl->fcnt[0], 1u);
          w.far_v[0][pos] = v;
        }
        atomicMin(&ctl->far_min, sh);
      }
    } else {
      // light-first rounds: the light edges form the first frontier, the heavy
      // ones the first R list
      const uint32_t le = lh ? w.lend[v] : re;
      if (le > rs) {
        if (atomicOr(w.mask[0] + v, 1ull << s) == 0ull) {
          const unsigned long long b = atomicAdd(&ctl->cnt[0], (1ull << 32) | (le - rs));
          const uint32_t pos = (uint32_t)(b >> 32);
          w.fv[0][pos] = v;
          w.fr[0][pos] = rs;
          w.fs[0][pos] = (uint32_t)b;
        }
      }
      if (lh && re > le) {
        if (nb) atomicAdd(&ctl->heavy_settled, (unsigned long long)(re - le));
        if (atomicOr(w.rmask[0] + v, 1ull << s) == 0ull) {
          const unsigned long long b = atomicAdd(&ctl->rcnt[0], (1ull << 32) | (re - le));
          const uint32_t pos = (uint32_t)(b >> 32);
          w.rv[0][pos] = v;
          w.rr[0][pos] = le;
          w.rs[0][pos] = (uint32_t)b;
        }
      }
    }
  }
  __syncthreads();
  if (s == 0) {
    const bool work = ctl->cnt[0] != 0ull || ctl->rcnt[0] != 0ull;
    ctl->running = (work || ctl->fcnt[0] != 0u) ? 1u : 0u;
    if (ctl->cnt[0] == 0ull && ctl->rcnt[0] != 0ull) ctl->mode = 2u;   // sources without light edges
    if (!work && ctl->fcnt[0] != 0u) {   // every source parked: open the bucket of the nearest
      ctl->t_prev = 0;
      ctl->t_cur = ctl->far_min + 1u;
      ctl->far_min = kInf;
      ctl->mode = 1u;
    }
  }
}

// The vertex of largest out-degree (lowest id on ties) into *best as
// (degree << 32) | ~v.
__global__ void k_max_degree(uint32_t n, const uint32_t* __restrict__ ro, unsigned long long* best) {
  unsigned long long b = 0ull;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    b = max(b, ((unsigned long long)(ro[v + 1] - ro[v]) << 32) | (uint32_t)~v);
#pragma unroll
  for (int o = 16; o; o >>= 1) b = max(b, __shfl_xor_sync(0xFFFFFFFFu, b, o));
  if ((threadIdx.x & 31) == 0 && b) atomicMax(best, b);
}

}  // namespace

struct BatchWorkspace {
  void* block = nullptr;
  size_t bytes = 0;
  BatchBufs b{};
  uint32_t* srcs = nullptr;
  uint32_t srcs_cap = 0;
  // per row-read mode (scalar, 16-byte vectors) x light-first rounds
  cudaGraph_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  cudaGraphExec_t exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  int grid = 0;
  BatchCtl* h_ctl = nullptr;
  // normalised buckets: distances from the hub (the highest-degree vertex),
  // a per-graph index computed by the first call that needs it
  uint32_t* hubd = nullptr;
  bool hub_ready = false;
  uint32_t hub = 0;
};

// the superstep kernel for the edge format, the row-read mode and the rounds
template <bool LH>
static void* batch_fn_lh(bool packed, bool vec) {
  if (packed) return vec ? reinterpret_cast<void*>(&k_batch_superstep<true, true, LH>)
                         : reinterpret_cast<void*>(&k_batch_superstep<true, false, LH>);
  return vec ? reinterpret_cast<void*>(&k_batch_superstep<false, true, LH>)
             : reinterpret_cast<void*>(&k_batch_superstep<false, false, LH>);
}
static void* batch_fn(bool packed, bool vec, bool lh) {
  return lh ? batch_fn_lh<true>(packed, vec) : batch_fn_lh<false>(packed, vec);
}

static gg_status batch_ws(gg_graph* g, BatchWorkspace** out) {
  if (!g->batch) {
    BatchWorkspace* w = new BatchWorkspace();
    const size_t n = std::max<uint32_t>(g->n, 1);
    auto r256 = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t total = 21 * r256(4 * n) + 7 * r256(8 * n) + r256(sizeof(BatchCtl));
    char* p = nullptr;
    cudaError_t e = cudaMalloc(&p, total);
    if (e != cudaSuccess) { delete w; return cuda_fail(e, "cudaMalloc(batch workspace)"); }
    w->block = p;
    w->bytes = total;
    size_t off = 0;
    auto take = [&](size_t b) { char* q = p + off; off += r256(b); return q; };
    for (int i = 0; i < 3; ++i) {
      w->b.fv[i] = reinterpret_cast<uint32_t*>(take(4 * n));
      w->b.fr[i] = reinterpret_cast<uint32_t*>(take(4 * n));
      w->b.fs[i] = reinterpret_cast<uint32_t*>(take(4 * n));
    }
    for (int i = 0; i < 3; ++i) w->b.mask[i] = reinterpret_cast<unsigned long long*>(take(8 * n));
    w->b.fmask = reinterpret_cast<unsigned long long*>(take(8 * n));
    for (int i = 0; i < 2; ++i) w->b.far_v[i] = reinterpret_cast<uint32_t*>(take(4 * n));
    for (int i = 0; i < 3; ++i) {
      w->b.rv[i] = reinterpret_cast<uint32_t*>(take(4 * n));
      w->b.rr[i] = reinterpret_cast<uint32_t*>(take(4 * n));
      w->b.rs[i] = reinterpret_cast<uint32_t*>(take(4 * n));
    }
    for (int i = 0; i < 3; ++i) w->b.rmask[i] = reinterpret_cast<unsigned long long*>(take(8 * n));
    w->hubd = reinterpret_cast<uint32_t*>(take(4 * n));
    w->b.hubd = w->hubd;
    w->b.ctl = reinterpret_cast<BatchCtl*>(take(sizeof(BatchCtl)));
    if (off != total) { cudaFree(p); delete w; return fail(GG_ERR_INTERNAL, "batch workspace layout"); }
    e = cudaMallocHost(&w->h_ctl, sizeof(BatchCtl));
    if (e != cudaSuccess) { cudaFree(p); delete w; return cuda_fail(e, "cudaMallocHost"); }
    void* fn = batch_fn(g->dg.packed, false, false);
    int per_sm = 0;
    GG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBB, 0));
    w->grid = std::max(1, per_sm) * device_info().num_sms;
    g->batch = w;
  }
  *out = g->batch;
  return GG_OK;
}

static gg_status batch_exec(gg_graph* g, BatchWorkspace* w, bool vec, bool lh) {
  if (w->exec[vec][lh]) return GG_OK;
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
  DevGraph dg = g->dg;
  BatchBufs b = w->b;
  int use_cond = 1;
  void* args[] = {&dg, &b, &h, &use_cond};
  cudaKernelNodeParams kp = {};
  kp.func = batch_fn(g->dg.packed, vec, lh);
  kp.gridDim = dim3(w->grid);
  kp.blockDim = dim3(kBB);
  kp.kernelParams = args;
  // GG_BATCH_UNROLL supersteps per evaluation of the loop condition; a
  // superstep that finds the loop ended returns at once and clears it
  cudaGraphNode_t prev = nullptr;
  for (int u = 0; u < GG_BATCH_UNROLL; ++u) {
    cudaGraphNode_t knode;
    GG_CK(cudaGraphAddKernelNode(&knode, cp.conditional.phGraph_out[0], prev ? &prev : nullptr, prev ? 1 : 0, &kp));
    prev = knode;
  }
  GG_CK(cudaGraphInstantiate(&w->exec[vec][lh], graph, 0));
  w->graph[vec][lh] = graph;
  return GG_OK;
}

gg_status batch_run(gg_graph* g, const uint32_t* srcs, uint32_t k, uint32_t* dist, const gg_options& o,
                    cudaStream_t s) {
  BatchWorkspace* w = nullptr;
  gg_status st = batch_ws(g, &w);
  if (st != GG_OK) return st;
  if (w->srcs_cap < k) {
    if (w->srcs) GG_CK(cudaFree(w->srcs));
    w->srcs = nullptr;
    w->srcs_cap = 0;
    GG_CK(cudaMalloc(&w->srcs, sizeof(uint32_t) * k));
    w->srcs_cap = k;
  }
  GG_CK(cudaMemcpyAsync(w->srcs, srcs, sizeof(uint32_t) * k, cudaMemcpyHostToDevice, s));
  // 16-byte row reads need 16-byte aligned rows: k a multiple of 4 and an aligned matrix
  const bool vec = (k % 4u) == 0u && (reinterpret_cast<uintptr_t>(dist) & 15u) == 0u;
  // light-first rounds on graphs with a light/heavy width (skewed graphs,
  // integer weights): delta 0 takes the graph's width, a delta up to the
  // largest weight is the width itself.  The light-first edge copy is shared
  // with the single-source loop and is in place before the rounds' graph runs.
  const bool lh_graph = o.light_heavy != GG_LH_OFF && g->default_delta_lh != GG_DELTA_NONE && g->m > 0;
  const uint32_t lh_width = o.delta == 0 ? g->default_delta_lh : o.delta;
  const bool lh = lh_graph && o.delta != GG_DELTA_NONE && lh_width <= g->wmax;
  // normalised buckets (the default with light-first rounds): the sources'
  // distances from the hub align their buckets; computed once per graph, by
  // the single-source loop with its default options (before the light-first
  // copy is partitioned for this call's width)
  const bool nb = lh && o.light_heavy != GG_LH_ROUNDS;
  if (nb && !w->hub_ready) {
    unsigned long long* best = w->b.fmask;   // scratch word (the masks are cleared below)
    GG_CK(cudaMemsetAsync(best, 0, sizeof(unsigned long long), s));
    k_max_degree<<<std::max(1, std::min<int>((int)((g->n + 255) / 256), device_info().num_sms * 4)), 256, 0, s>>>(
        g->n, g->ro, best);
    GG_CK(cudaGetLastError());
    unsigned long long hb = 0;
    GG_CK(cudaMemcpyAsync(&hb, best, sizeof(hb), cudaMemcpyDeviceToHost, s));
    GG_CK(cudaStreamSynchronize(s));
    w->hub = ~(uint32_t)hb;
    gg_options ho;
    gg_options_default(&ho);
    st = bsp_run(g, w->hub, w->hubd, ho, s, WM_U32);
    if (st != GG_OK) return st;
    w->hub_ready = true;
  }
  if (lh) {
    st = lh_prepare(g, lh_width, s);
    if (st != GG_OK) return st;
    w->b.ledges = g->lhb.edges;
    w->b.lend = g->lhb.lend;
  }
  st = batch_exec(g, w, vec, lh);
  if (st != GG_OK) return st;
  const unsigned long long count = (unsigned long long)g->n * k;
  const unsigned fb = (unsigned)std::max<unsigned long long>(
      1, std::min<unsigned long long>((count / 4 + 255) / 256, (unsigned long long)device_info().num_sms * 8));
  k_batch_fill<<<fb, 256, 0, s>>>(dist, count);
  GG_CK(cudaGetLastError());
  // near-far buckets for the batch only on request: a vertex whose sources sit
  // in different buckets is re-expanded once per bucket, which on the measured
  // RMAT workloads cost far more edge scans than the buckets saved
  const uint32_t delta = (o.delta == GG_DELTA_NONE || o.delta == 0) ? kInf : o.delta;
  // a light-first round adds at most one heavy superstep per improving vertex
  const unsigned long long cap = nb ? 8ull * g->n + 64 : lh ? 3ull * g->n + 16
                                : delta == kInf ? (unsigned long long)g->n + 2 : 4ull * g->n + 16;
  const uint32_t nb_width = (uint32_t)std::min<uint64_t>((uint64_t)lh_width * GG_NB_WIDTH, kInf - 1u);
  const uint32_t max_iter = o.max_iterations ? o.max_iterations : (cap >= 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)cap);
  for (uint32_t col0 = 0; col0 < k; col0 += 64) {
    const uint32_t kg = std::min<uint32_t>(64, k - col0);
    // the previous group (or call) may leave the masks of its last frontier set
    for (int i = 0; i < 3; ++i) GG_CK(cudaMemsetAsync(w->b.mask[i], 0, 8 * (size_t)g->n, s));
    GG_CK(cudaMemsetAsync(w->b.fmask, 0, 8 * (size_t)g->n, s));
    if (lh)
      for (int i = 0; i < 3; ++i) GG_CK(cudaMemsetAsync(w->b.rmask[i], 0, 8 * (size_t)g->n, s));
    k_batch_seed<<<1, 64, 0, s>>>(g->dg, w->b, w->srcs, k, col0, kg, dist, max_iter, lh ? kInf : delta, lh ? 1u : 0u,
                                  nb ? 1u : 0u, nb_width, GG_NB_DRAIN, (unsigned long long)g->lh_heavy_total,
                                  col0 == 0 ? o.trace : nullptr, o.trace_cap,
                                  (nb && g->symmetric && GG_BATCH_PULL && nb_width <= lh_width) ? 1u : 0u);
    GG_CK(cudaGetLastError());
    if (o.policy == GG_POLICY_BSP_HOST) {
      // supersteps launched one by one, the loop flag read back after each
      DevGraph dg = g->dg;
      BatchBufs b = w->b;
      cudaGraphConditionalHandle none = 0;
      int zero = 0;
      void* fn = batch_fn(g->dg.packed, vec, lh);
      for (uint32_t it = 0;; ++it) {
        void* args[] = {&dg, &b, &none, &zero};
        GG_CK(cudaLaunchKernel(fn, dim3(w->grid), dim3(kBB), args, 0, s));
        GG_CK(cudaMemcpyAsync(&w->h_ctl->running, &w->b.ctl->running, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        GG_CK(cudaStreamSynchronize(s));
        if (w->h_ctl->running == 0u || it >= max_iter) break;
      }
    } else {
      GG_CK(cudaGraphLaunch(w->exec[vec][lh], s));
    }
    if (o.stats) {
      GG_CK(cudaMemcpyAsync(w->h_ctl, w->b.ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
      GG_CK(cudaStreamSynchronize(s));
      o.stats->iterations += w->h_ctl->iter;
      o.stats->pull_iterations += 0;
      o.stats->edges_scanned += w->h_ctl->edges_scanned;
      o.stats->frontier_total += w->h_ctl->frontier_total;
      o.stats->max_frontier = std::max(o.stats->max_frontier, w->h_ctl->max_frontier);
      o.stats->device_status |= w->h_ctl->status;
    }
  }
  return GG_OK;
}

gg_status batch_status(gg_graph* g, uint32_t* ds) {
  *ds = 0;
  if (!g->batch) return GG_OK;
  GG_CK(cudaMemcpyAsync(g->batch->h_ctl, g->batch->b.ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, g->last_stream));
  GG_CK(cudaStreamSynchronize(g->last_stream));
  *ds = g->batch->h_ctl->status;
  return GG_OK;
}

void batch_release(gg_graph* g) {
  BatchWorkspace* w = g->batch;
  if (!w) return;
  for (int i = 0; i < 2; ++i) {
    for (int j = 0; j < 2; ++j) {
      if (w->exec[i][j]) cudaGraphExecDestroy(w->exec[i][j]);
      if (w->graph[i][j]) cudaGraphDestroy(w->graph[i][j]);
    }
  }
  if (w->block) cudaFree(w->block);
  if (w->srcs) cudaFree(w->srcs);
  if (w->h_ctl) cudaFreeHost(w->h_ctl);
  delete w;
  g->batch = nullptr;
}

size_t batch_bytes(const gg_graph* g) { return g->batch ? g->batch->bytes : 0; }

}  // namespace gg
