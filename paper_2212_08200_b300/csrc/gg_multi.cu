// gg_multi.cu -- many single-source queries on many graphs in one launch
// sequence: the "slot" engine behind gg_sssp_multi and the query server.
//
// Each query occupies a slot {graph, source, caller's distance array, its own
// two dedup bitmaps}.  All slots share ONE union frontier whose entries are
// (slot, vertex, CSR row start, edge-prefix coordinate), so a superstep is
// still one kernel: the merge-path advance of the single-source path splits
// the union's edges evenly over the CTAs whatever mix of large and small
// graphs is active, and the fused filter appends improved vertices with their
// slot.  Per-slot counters of the next frontier tell the closing CTA which
// queries have converged: it marks them done (slot state and, for the
// server, words in host-mapped memory) so that new queries can take their
// slots between supersteps -- continuous batching at superstep granularity.
// Push only.  Each slot runs its own near-far buckets: improved vertices at or
// above the slot's threshold are parked in the slot's far pile; when a slot's
// near frontier empties, the closing CTA raises its threshold and the next
// superstep re-examines that pile (edge-balanced over all CTAs, alongside the
// other slots' advance).
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>

#include "gg_host.h"
#include "gg_multi.h"

namespace gg {
namespace {

constexpr int kMB = 256;
constexpr int kMEpt = 4;
constexpr int kMTile = kMB * kMEpt;
constexpr int kMCap = kMTile + 1;
#ifndef GG_MULTI_LOCAL_ROUNDS
#define GG_MULTI_LOCAL_ROUNDS 8   // CTA-local rounds per superstep (0: none)
#endif
constexpr uint32_t kMLocalCap = 256;      // entries of each CTA-local queue
constexpr uint32_t kMLocalMaxDeg = 4;     // longer rows go to the union next frontier

struct MSmem {
  uint32_t es[kMCap], eb[kMCap], ec[kMCap], eq[kMCap];
  uint32_t qv[kMCap], qr[kMCap], qd[kMCap], qq[kMCap];
  uint32_t wsum[kMB / 32];
  uint32_t qn, j, last;
  // CTA-local rounds: two queues of (vertex, distance it was queued with, slot)
  uint32_t lv[2][kMLocalCap], ld[2][kMLocalCap], lq[2][kMLocalCap];
  uint32_t ln[2];
  unsigned long long base;
};

__device__ __forceinline__ uint32_t* lq_v(MSmem& sm, uint32_t k) { return sm.lv[k]; }
__device__ __forceinline__ uint32_t* lq_d(MSmem& sm, uint32_t k) { return sm.ld[k]; }
__device__ __forceinline__ uint32_t* lq_q(MSmem& sm, uint32_t k) { return sm.lq[k]; }

__device__ __forceinline__ uint2 slot_edge(const MultiSlot& s, uint32_t e) {
  if (s.packed) {
    const uint32_t x = __ldg(static_cast<const uint32_t*>(s.edges) + e);
    return make_uint2(x >> s.wbits, x & ((1u << s.wbits) - 1u));
  }
  return __ldg(static_cast<const uint2*>(s.edges) + e);
}

// Filter of the slot engine: vertex v of slot q just dropped to nd.  Below
// the slot's threshold it joins the union next frontier (once per slot, by its
// near bitmap); otherwise it is parked in the slot's far pile (once, by its
// far bitmap).  Vertices without out-edges are skipped.
__device__ __forceinline__ void m_filter(MSmem& sm, const MultiBufs& b, MultiSlot* slots, uint32_t q,
                                         const MultiSlot& sl, uint32_t p, uint32_t v, uint32_t nd) {
  const uint32_t rs = __ldg(sl.ro + v), re = __ldg(sl.ro + v + 1);
  if (re <= rs) return;
  const uint32_t bit = 1u << (v & 31);
  if (nd < sl.t_cur) {
    if (!(atomicOr(b.bm_pool + sl.bm_off[p ^ 1u] + (v >> 5), bit) & bit)) {
      const uint32_t i = atomicAdd(&sm.qn, 1u);
      sm.qv[i] = v;
      sm.qr[i] = rs;
      sm.qd[i] = re - rs;
      sm.qq[i] = q;
    }
  } else {
    atomicMin(&slots[q].far_min, nd);
    if (!(atomicOr(b.bm_pool + sl.bm_off[2] + (v >> 5), bit) & bit)) {
      const uint32_t pile = sl.fpp;
      const uint32_t pos = atomicAdd(&slots[q].far_cnt[pile], 1u);
      b.far_pool[sl.far_off[pile] + pos] = v;
    }
  }
}

// Filter with CTA-local rounds: a near vertex goes to local queue k (no
// bitmap: one entry per improvement, with the distance it was improved to)
// while there is room, else through the bitmap to the union next frontier;
// far vertices are parked as in m_filter.
__device__ __forceinline__ void m_filter_local(MSmem& sm, const MultiBufs& b, MultiSlot* slots, uint32_t q,
                                               const MultiSlot& sl, uint32_t p, uint32_t v, uint32_t nd, uint32_t k) {
  if (nd < sl.t_cur) {
    const uint32_t i = atomicAdd(&sm.ln[k], 1u);
    if (i < kMLocalCap) {
      lq_v(sm, k)[i] = v;
      lq_d(sm, k)[i] = nd;
      lq_q(sm, k)[i] = q;
      return;
    }
  }
  m_filter(sm, b, slots, q, sl, p, v, nd);
}

// Appends the CTA's queued (slot, vertex) entries to the union next frontier.
__device__ __forceinline__ void m_flush(MSmem& sm, const MultiBufs& b, MultiCtl* ctl, uint32_t p) {
  __syncthreads();
  const uint32_t qn = sm.qn;
  if (qn) {
    const uint32_t tid = threadIdx.x;
    for (uint32_t i = tid; i < qn; i += kMB) atomicAdd(&b.slot_cnt[sm.qq[i]], 1u);
    const uint32_t tot = block_scan_excl<kMB>(sm.qd, qn, sm.wsum);
    if (tid == 0) sm.base = atomicAdd(&ctl->cnt[p ^ 1u], ((unsigned long long)qn << 32) | tot);
    __syncthreads();
    const uint32_t pos0 = (uint32_t)(sm.base >> 32), eb0 = (uint32_t)sm.base;
    for (uint32_t i = tid; i < qn; i += kMB) {
      b.fv[p ^ 1u][pos0 + i] = sm.qv[i];
      b.fr[p ^ 1u][pos0 + i] = sm.qr[i];
      b.fs[p ^ 1u][pos0 + i] = eb0 + sm.qd[i];
      b.fq[p ^ 1u][pos0 + i] = sm.qq[i];
    }
    __syncthreads();
    if (tid == 0) sm.qn = 0;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kMB) k_multi_superstep(MultiBufs b, cudaGraphConditionalHandle cond,
                                                         int use_cond) {
  __shared__ MSmem sm;
  MultiCtl* ctl = b.ctl;
  const uint32_t tid = threadIdx.x;
  const uint32_t it = ctl->iter, p = it & 1u;
  const unsigned long long c = ctl->cnt[p];
  const uint32_t F = (uint32_t)(c >> 32), E = (uint32_t)c;
  MultiSlot* slots = b.slots;
  if (tid == 0) {
    sm.qn = 0;
    sm.ln[0] = 0;
    sm.ln[1] = 0;
  }
  __syncthreads();
  const uint32_t e0 = (uint32_t)(((unsigned long long)blockIdx.x * E) / gridDim.x);
  const uint32_t e1 = (uint32_t)(((unsigned long long)(blockIdx.x + 1) * E) / gridDim.x);
  if (F > 0 && e0 < e1) {
    const uint32_t* S = b.fs[p];
    if (tid < 32) {
      const uint32_t j = warp_search_le(S, F, e0);
      if (tid == 0) sm.j = j;
    }
    __syncthreads();
    uint32_t j = sm.j;
    for (uint32_t t0 = e0; t0 < e1; t0 += kMTile) {
      const uint32_t t1 = min(t0 + (uint32_t)kMTile, e1);
      uint32_t nent = 0;
      for (;;) {
        const uint32_t idx = j + nent + tid;
        bool valid = false;
        uint32_t s = 0;
        if (idx < F) {
          s = S[idx];
          valid = s < t1;
        }
        if (valid) {
          const uint32_t q = b.fq[p][idx], v = b.fv[p][idx];
          const MultiSlot& sl = slots[q];
          sm.es[nent + tid] = s;
          sm.eb[nent + tid] = b.fr[p][idx];
          sm.ec[nent + tid] = ld_cg(sl.dist + v);
          sm.eq[nent + tid] = q;
          b.bm_pool[sl.bm_off[p] + (v >> 5)] = 0u;   // the current bitmap is not read: clear as we go
        }
        const int cnt = __syncthreads_count(valid);
        nent += (uint32_t)cnt;
        if (cnt < kMB) break;
      }
#pragma unroll
      for (int k = 0; k < kMEpt; ++k) {
        const uint32_t gidx = t0 + k * kMB + tid;
        if (gidx < t1) {
          const uint32_t jj = smem_upper_bound_minus1(sm.es, nent, gidx);
          const uint32_t q = sm.eq[jj];
          const MultiSlot& sl = slots[q];
          const uint2 ed = slot_edge(sl, sm.eb[jj] + (gidx - sm.es[jj]));
          bool ovf = false;
          const uint32_t nd = add_sat(sm.ec[jj], ed.y, ovf);
          if (ovf) atomicOr(&slots[q].status, DS_OVERFLOW);
          if (nd < ld_cg(sl.dist + ed.x)) {
            atomicMin(sl.dist + ed.x, nd);
            if (GG_MULTI_LOCAL_ROUNDS) m_filter_local(sm, b, slots, q, sl, p, ed.x, nd, 0);
            else m_filter(sm, b, slots, q, sl, p, ed.x, nd);
          }
        }
      }
      m_flush(sm, b, ctl, p);
      j = j + nent - 1;
    }
  }
  // CTA-local rounds: the near vertices this CTA improved are expanded here,
  // up to GG_MULTI_LOCAL_ROUNDS times, before the rest joins the union next
  // frontier.  An entry whose vertex has dropped below the distance it was
  // queued with is stale (the later decrease queued it again); rows longer
  // than kMLocalMaxDeg go to the next frontier through the bitmap.  On
  // high-diameter graphs a superstep covers several hops.
  if (GG_MULTI_LOCAL_ROUNDS) {
    uint32_t k = 0;
    for (int r = 0; r < GG_MULTI_LOCAL_ROUNDS; ++r) {
      __syncthreads();
      const uint32_t n_cur = min(sm.ln[k], kMLocalCap);
      if (n_cur == 0) break;   // CTA-uniform
      __syncthreads();
      if (tid == 0) sm.ln[k ^ 1u] = 0;
      __syncthreads();
      for (uint32_t base = 0; base < n_cur; base += kMB) {   // CTA-uniform
        const uint32_t i = base + tid;
        if (i < n_cur) {
          const uint32_t v = sm.lv[k][i], nq = sm.ld[k][i], q = sm.lq[k][i];
          const MultiSlot& sl = slots[q];
          const uint32_t du = ld_cg(sl.dist + v);
          if (du >= nq) {
            const uint32_t rs = __ldg(sl.ro + v), re = __ldg(sl.ro + v + 1);
            if (re - rs > kMLocalMaxDeg) {
              m_filter(sm, b, slots, q, sl, p, v, du);
            } else {
              for (uint32_t e = rs; e < re; ++e) {
                const uint2 ed = slot_edge(sl, e);
                bool ovf = false;
                const uint32_t nd = add_sat(du, ed.y, ovf);
                if (ovf) atomicOr(&slots[q].status, DS_OVERFLOW);
                if (nd < ld_cg(sl.dist + ed.x)) {
                  atomicMin(sl.dist + ed.x, nd);
                  m_filter_local(sm, b, slots, q, sl, p, ed.x, nd, k ^ 1u);
                }
              }
            }
          }
        }
        m_flush(sm, b, ctl, p);
      }
      k ^= 1u;
    }
    __syncthreads();
    // what the rounds leave: the union next frontier, through the bitmap
    const uint32_t n_left = min(sm.ln[k], kMLocalCap);
    for (uint32_t base = 0; base < n_left; base += kMB) {   // CTA-uniform
      const uint32_t i = base + tid;
      if (i < n_left) {
        const uint32_t v = sm.lv[k][i], q = sm.lq[k][i];
        const MultiSlot& sl = slots[q];
        m_filter(sm, b, slots, q, sl, p, v, ld_cg(sl.dist + v));
      }
      m_flush(sm, b, ctl, p);
    }
  }
  // split work: the far piles of the slots flagged by the previous superstep,
  // spread evenly over the CTAs
  {
    const uint32_t S = ctl->split_total, ns = ctl->nsplit;
    const uint32_t s0 = (uint32_t)(((unsigned long long)blockIdx.x * S) / gridDim.x);
    const uint32_t s1 = (uint32_t)(((unsigned long long)(blockIdx.x + 1) * S) / gridDim.x);
    for (uint32_t base = s0; base < s1; base += kMB) {
      const uint32_t i = base + tid;
      if (i < s1) {
        uint32_t lo = 0, len = ns;   // last k with split_pref[k] <= i
        while (len > 0) {
          const uint32_t half = len >> 1;
          if (ctl->split_pref[lo + half] <= i) { lo += half + 1; len -= half + 1; }
          else len = half;
        }
        const uint32_t k = lo - 1;
        const uint32_t q = ctl->split_slot[k];
        const MultiSlot& sl = slots[q];
        const uint32_t v = b.far_pool[sl.far_off[sl.fpp] + (i - ctl->split_pref[k])];
        const uint32_t d = ld_cg(sl.dist + v);
        const uint32_t bit = 1u << (v & 31);
        if (d < sl.t_cur) {
          // below the raised threshold: leave the pile; expand unless already expanded below t_prev
          atomicAnd(b.bm_pool + sl.bm_off[2] + (v >> 5), ~bit);
          if (d >= sl.t_prev) m_filter(sm, b, slots, q, sl, p, v, d);
        } else {
          atomicMin(&slots[q].far_min, d);
          const uint32_t pile = sl.fpp ^ 1u;
          const uint32_t pos = atomicAdd(&slots[q].far_cnt[pile], 1u);
          b.far_pool[sl.far_off[pile] + pos] = v;
        }
      }
      m_flush(sm, b, ctl, p);
    }
  }
  __syncthreads();
  if (tid == 0) {
    sm.last = arrive_last(&ctl->done_ctas, gridDim.x) ? 1u : 0u;
  }
  __syncthreads();
  if (sm.last) {
    // the closing CTA: a slot with nothing in the next frontier either splits
    // its far pile next superstep (threshold raised past its smallest parked
    // distance) or, with an empty pile, has converged
    __threadfence();
    // the next frontier's count and the budget are loaded first; their wait
    // overlaps the slot pass
    unsigned long long cn = 0;
    uint32_t budget = 0;
    if (tid == 0) {
      sm.j = 0;
      cn = ld_rlx(&ctl->cnt[p ^ 1u]);
      budget = ctl->budget_left;
    }
    __syncthreads();
    for (uint32_t q = tid; q < b.nslots; q += kMB) {
      MultiSlot& sl = slots[q];
      if (sl.state == kSlotRunning) {
        sl.supersteps += 1;
        if (sl.split) {   // this superstep consumed pile fpp and kept the rest in the other pile
          sl.far_cnt[sl.fpp] = 0u;
          sl.fpp ^= 1u;
          sl.split = 0u;
        }
        const uint32_t fc = sl.far_cnt[sl.fpp];
        if (b.slot_cnt[q] == 0) {
          if (fc > 0) {
            const unsigned long long t1 = (unsigned long long)sl.t_cur + sl.delta;
            const unsigned long long t2 = (unsigned long long)sl.far_min + 1;
            const unsigned long long tn = t1 > t2 ? t1 : t2;
            sl.t_prev = sl.t_cur;
            sl.t_cur = tn >= kInf ? kInf : (uint32_t)tn;
            sl.far_min = kInf;
            sl.split = 1u;
            const uint32_t k = atomicAdd(&sm.j, 1u);
            sm.qv[k] = q;
            sm.qd[k] = fc;   // its pile's size: the prefix below reads no slot again
          } else {
            sl.state = kSlotDone;
            if (b.done_flags) {
              b.done_status[q] = sl.status;
              __threadfence_system();
              reinterpret_cast<volatile uint32_t*>(b.done_flags)[q] = sl.ticket;
            }
          }
        }
      }
      b.slot_cnt[q] = 0u;
    }
    __syncthreads();
    if (tid == 0) {
      const uint32_t ns = sm.j;
      uint32_t run = 0;
      for (uint32_t k = 0; k < ns; ++k) {
        ctl->split_slot[k] = sm.qv[k];
        ctl->split_pref[k] = run;
        run += sm.qd[k];
      }
      ctl->split_pref[ns] = run;
      ctl->nsplit = ns;
      ctl->split_total = run;
      ctl->cnt[p] = 0ull;
      ctl->done_ctas = 0u;
      ctl->iter = it + 1;
      ctl->supersteps_run += 1;
      const bool nonempty = (cn >> 32) != 0 || ns != 0;
      const uint32_t left = budget > 0 ? budget - 1 : 0;
      ctl->budget_left = left;
      ctl->running = nonempty ? 1u : 0u;
      if (use_cond) cudaGraphSetConditional(cond, (nonempty && left > 0) ? 1u : 0u);
    }
  }
}

// dist := INF and bitmaps := 0 for every slot in `starting` (blockIdx.y walks the list)
__global__ void k_multi_fill(MultiBufs b, const uint32_t* starting, uint32_t nstart) {
  for (uint32_t i = blockIdx.y; i < nstart; i += gridDim.y) {
    const MultiSlot& sl = b.slots[starting[i]];
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < sl.n; v += stride) sl.dist[v] = kInf;
    const uint32_t nw = (sl.n + 31) / 32;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nw; v += stride) {
      b.bm_pool[sl.bm_off[0] + v] = 0u;
      b.bm_pool[sl.bm_off[1] + v] = 0u;
      b.bm_pool[sl.bm_off[2] + v] = 0u;
    }
  }
}

// seed the starting slots into the union frontier of the current parity
__global__ void k_multi_seed(MultiBufs b, const uint32_t* starting, uint32_t nstart) {
  MultiCtl* ctl = b.ctl;
  const uint32_t p = ctl->iter & 1u;
  for (uint32_t i = threadIdx.x; i < nstart; i += blockDim.x) {
    const uint32_t q = starting[i];
    MultiSlot& sl = b.slots[q];
    const uint32_t src = sl.src;
    sl.dist[src] = 0u;
    const uint32_t rs = sl.ro[src], re = sl.ro[src + 1];
    if (re > rs) {
      sl.state = kSlotRunning;
      const unsigned long long base = atomicAdd(&ctl->cnt[p], (1ull << 32) | (re - rs));
      const uint32_t pos = (uint32_t)(base >> 32);
      b.fv[p][pos] = src;
      b.fr[p][pos] = rs;
      b.fs[p][pos] = (uint32_t)base;
      b.fq[p][pos] = q;
    } else {
      sl.state = kSlotDone;   // nothing to expand: dist is final already
      if (b.done_flags) {
        b.done_status[q] = sl.status;
        __threadfence_system();
        reinterpret_cast<volatile uint32_t*>(b.done_flags)[q] = sl.ticket;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) ctl->running = ctl->cnt[p] != 0ull ? 1u : 0u;
}

__global__ void k_multi_budget(MultiCtl* ctl, uint32_t budget) { ctl->budget_left = budget; }

}  // namespace

void multi_slot_buckets(MultiSlot& s, uint32_t delta, uint32_t far0, uint32_t far1) {
  s.delta = delta;
  s.t_cur = delta;   // first bucket [0, delta); kInf: no buckets
  s.t_prev = 0;
  s.far_off[0] = far0;
  s.far_off[1] = far1;
  s.far_cnt[0] = s.far_cnt[1] = 0;
  s.fpp = 0;
  s.far_min = kInf;
  s.split = 0;
}

gg_status multi_engine_init(MultiEngine* e, uint32_t max_slots, uint64_t max_vertices, uint64_t max_bitmap_words,
                            uint64_t max_far, bool mapped_flags) {
  if (max_slots > (uint32_t)kMaxSplitSlots) return fail(GG_ERR_INVALID_ARG, "at most 1024 slots");
  e->max_slots = max_slots;
  e->cap_vertices = max_vertices;
  e->cap_words = max_bitmap_words;
  e->cap_far = max_far;
  auto r256 = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t fb = r256(4 * std::max<uint64_t>(max_vertices, 1));
  const size_t total = 8 * fb + r256(sizeof(MultiSlot) * max_slots) + 2 * r256(4 * (size_t)max_slots) +
                       r256(4 * std::max<uint64_t>(max_bitmap_words, 1)) + r256(4 * std::max<uint64_t>(max_far, 1)) +
                       r256(sizeof(MultiCtl));
  char* p = nullptr;
  GG_CK(cudaMalloc(&p, total));
  e->block = p;
  e->bytes = total;
  GG_CK(cudaMemset(p, 0, total));
  size_t off = 0;
  auto take = [&](size_t bytes) { char* q = p + off; off += r256(bytes); return q; };
  for (int i = 0; i < 2; ++i) {
    e->b.fv[i] = reinterpret_cast<uint32_t*>(take(fb));
    e->b.fr[i] = reinterpret_cast<uint32_t*>(take(fb));
    e->b.fs[i] = reinterpret_cast<uint32_t*>(take(fb));
    e->b.fq[i] = reinterpret_cast<uint32_t*>(take(fb));
  }
  e->b.slots = reinterpret_cast<MultiSlot*>(take(sizeof(MultiSlot) * max_slots));
  e->b.slot_cnt = reinterpret_cast<uint32_t*>(take(4 * (size_t)max_slots));
  e->starting = reinterpret_cast<uint32_t*>(take(4 * (size_t)max_slots));
  e->b.bm_pool = reinterpret_cast<uint32_t*>(take(4 * std::max<uint64_t>(max_bitmap_words, 1)));
  e->b.far_pool = reinterpret_cast<uint32_t*>(take(4 * std::max<uint64_t>(max_far, 1)));
  e->b.ctl = reinterpret_cast<MultiCtl*>(take(sizeof(MultiCtl)));
  e->b.nslots = max_slots;
  if (off != total) return fail(GG_ERR_INTERNAL, "multi workspace layout");
  GG_CK(cudaMallocHost(&e->h_slots, sizeof(MultiSlot) * max_slots));
  GG_CK(cudaMallocHost(&e->h_ctl, sizeof(MultiCtl)));
  GG_CK(cudaMallocHost(&e->h_start, 4 * (size_t)max_slots));
  memset(e->h_slots, 0, sizeof(MultiSlot) * max_slots);
  e->b.done_flags = nullptr;
  e->b.done_status = nullptr;
  if (mapped_flags) {
    GG_CK(cudaHostAlloc(&e->h_done, 4 * (size_t)max_slots, cudaHostAllocMapped));
    GG_CK(cudaHostAlloc(&e->h_done_status, 4 * (size_t)max_slots, cudaHostAllocMapped));
    memset(e->h_done, 0, 4 * (size_t)max_slots);
    memset(e->h_done_status, 0, 4 * (size_t)max_slots);
    GG_CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&e->b.done_flags), e->h_done, 0));
    GG_CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&e->b.done_status), e->h_done_status, 0));
  }
  int per_sm = 0;
  GG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi_superstep, kMB, 0));
  e->grid = std::max(1, per_sm) * device_info().num_sms;
  // CUDA graph: WHILE (union frontier non-empty and budget left) { superstep }
  GG_CK(cudaGraphCreate(&e->graph, 0));
  cudaGraphConditionalHandle h;
  GG_CK(cudaGraphConditionalHandleCreate(&h, e->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wnode;
  GG_CK(cudaGraphAddNode(&wnode, e->graph, nullptr, nullptr, 0, &cp));
  MultiBufs b = e->b;
  int use_cond = 1;
  void* args[] = {&b, &h, &use_cond};
  cudaKernelNodeParams kp = {};
  kp.func = reinterpret_cast<void*>(&k_multi_superstep);
  kp.gridDim = dim3(e->grid);
  kp.blockDim = dim3(kMB);
  kp.kernelParams = args;
  cudaGraphNode_t knode;
  GG_CK(cudaGraphAddKernelNode(&knode, cp.conditional.phGraph_out[0], nullptr, 0, &kp));
  GG_CK(cudaGraphInstantiate(&e->exec, e->graph, 0));
  return GG_OK;
}

void multi_engine_free(MultiEngine* e) {
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->graph) cudaGraphDestroy(e->graph);
  if (e->block) cudaFree(e->block);
  if (e->h_slots) cudaFreeHost(e->h_slots);
  if (e->h_ctl) cudaFreeHost(e->h_ctl);
  if (e->h_start) cudaFreeHost(e->h_start);
  if (e->h_done) cudaFreeHost(e->h_done);
  if (e->h_done_status) cudaFreeHost(e->h_done_status);
  *e = MultiEngine{};
}

gg_status multi_engine_reset(MultiEngine* e, cudaStream_t s) {
  GG_CK(cudaMemsetAsync(e->b.ctl, 0, sizeof(MultiCtl), s));
  GG_CK(cudaMemsetAsync(e->b.slot_cnt, 0, 4 * (size_t)e->max_slots, s));
  return GG_OK;
}

gg_status multi_engine_start(MultiEngine* e, const uint32_t* slots, uint32_t count, cudaStream_t s) {
  if (count == 0) return GG_OK;
  uint32_t nmax = 1;
  for (uint32_t i = 0; i < count; ++i) {
    const uint32_t q = slots[i];
    e->h_start[i] = q;
    nmax = std::max(nmax, e->h_slots[q].n);
    GG_CK(cudaMemcpyAsync(e->b.slots + q, e->h_slots + q, sizeof(MultiSlot), cudaMemcpyHostToDevice, s));
  }
  GG_CK(cudaMemcpyAsync(e->starting, e->h_start, 4 * (size_t)count, cudaMemcpyHostToDevice, s));
  dim3 grid((unsigned)std::min<uint32_t>((nmax + 255) / 256, 512), (unsigned)std::min<uint32_t>(count, 1024));
  k_multi_fill<<<grid, 256, 0, s>>>(e->b, e->starting, count);
  GG_CK(cudaGetLastError());
  k_multi_seed<<<1, 256, 0, s>>>(e->b, e->starting, count);
  GG_CK(cudaGetLastError());
  return GG_OK;
}

gg_status multi_engine_run(MultiEngine* e, uint32_t budget, cudaStream_t s) {
  k_multi_budget<<<1, 1, 0, s>>>(e->b.ctl, budget ? budget : 0xFFFFFFFFu);
  GG_CK(cudaGetLastError());
  GG_CK(cudaGraphLaunch(e->exec, s));
  return GG_OK;
}

}  // namespace gg
