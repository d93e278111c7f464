// gg_async.cu -- asynchronous frontier SSSP (the execution::par_nosync policy).
//
// The paper's asynchronous variant of neighbors_expand drops the barrier
// between expansions (Listing 3's par_nosync overload and the "Timing Model
// and Parallelism" box) and represents the frontier as an asynchronous queue
// that passes active vertices as messages (Sec. III-B and the "Asynchrony and
// Message-Passing" box).  Here that is ONE persistent kernel:
//
//   queue    a ring of 64-bit slots {tag, vertex} with per-slot sequence tags
//            (a bounded multi-producer multi-consumer ring): the producer of
//            position p waits for tag 2*lap, writes {2*lap+1, v}; the
//            consumer waits for 2*lap+1, takes v and writes 2*lap+2.
//   dedup    an in-queue bitmap: a vertex is enqueued only if its bit was
//            clear; the consumer clears it before reading dist[v], so any
//            later improvement re-enqueues it.  At most n vertices are queued
//            at once.  A producer whose slot still holds the previous lap's
//            item waits for it, and while it waits its warp takes the items
//            at its own reserved positions, so no warp waits on itself.
//   work     each warp reserves 32 consecutive positions, takes whichever
//            arrive, and expands the taken vertices' edges together
//            (warp-level merge-path over their degree prefix sums).
//   stop     sharded counters: items published (counted before publishing)
//            and items expanded (counted after expanding).  A warp reads all
//            expanded shards, then all published shards; equal sums mean
//            nothing is queued or running, which no later step can undo, so
//            the warp exits.
//   watchdog every wait is bounded by a %globaltimer budget; when it runs
//            out the kernel raises `abort`, records GG_ERR_TIMEOUT and every
//            warp returns.  Nothing spins without a limit.
//   buckets  near-far priority without barriers: an improved vertex whose new
//            distance is >= the threshold t_cur is parked in a far pile
//            (deduplicated by a bitmap).  When nothing is queued or running,
//            one idle warp raises the threshold and idle warps split the
//            pile chunk by chunk: entries below the old threshold were
//            expanded already and are dropped, entries below the new one are
//            queued, the rest move to the other pile.  Termination: nothing
//            queued or running, no split in progress, empty pile.
#include <cuda_runtime.h>

#include <algorithm>

#include "gg_host.h"

namespace gg {

constexpr int kAShards = 32;   // termination counter shards, one cache line each (one per lane)
static_assert(kAShards == 32, "warp_quiescent reads one shard per lane");

struct AsyncCtl {
  // the counters every warp updates live on cache lines of their own
  alignas(128) unsigned long long head;
  alignas(128) unsigned long long tail;
  // termination counting, sharded over cache lines: a warp adds the items it
  // publishes to pushed[its shard] before publishing them and the items it
  // expanded to done[its shard] after expanding them; everything is drained
  // when a read of all done shards followed by a read of all pushed shards
  // gives equal sums (both only grow, and done never passes pushed)
  alignas(128) unsigned long long pushed[kAShards * 16];
  alignas(128) unsigned long long done[kAShards * 16];
  alignas(128) uint32_t far_cnt[2];
  alignas(128) uint32_t far_min;
  alignas(128) uint32_t split_cursor;
  uint32_t split_done;
  alignas(128) unsigned long long pops;
  unsigned long long edges;
  unsigned long long watchdog_ns;
  unsigned long long t_start;
  uint32_t status;
  uint32_t abort;
  uint32_t* dist;
  // near-far buckets: vertices improved to a distance >= t_cur are parked in
  // the far pile far[sel]; when nothing is queued or running, idle warps split
  // the pile against a raised threshold (drop / queue / keep)
  uint32_t t_cur, t_prev, delta, sel;
  uint32_t phase;          // 0 none, 1 starting, 2 split running
  uint32_t epoch;          // split starts so far
  uint32_t split_src, split_total;
  uint32_t* far[2];
  uint32_t* bm_far;
  uint32_t* trace;         // per split: split number, new threshold, pile size, microseconds since start
  uint32_t trace_cap;
  uint32_t wmode;          // WM_*: how relaxations add edge weights
};

namespace {

constexpr int kABlock = 256;
constexpr int kAWarps = kABlock / 32;

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Time since t_start beyond `limit` ns?  The difference is taken as signed:
// %globaltimer read on another SM can lag the start stamp by a little, and an
// unsigned difference would wrap to a huge value and fire the watchdog at once.
__device__ __forceinline__ bool past_watchdog(unsigned long long t_start, unsigned long long limit) {
  return (long long)(globaltimer() - t_start) > (long long)limit;
}

__device__ __forceinline__ uint32_t shard_of_warp() {
  return (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % kAShards;
}

// Whole warp: true when every published item has been expanded.  All done
// shards are read (and ordered by a fence and the warp barrier) before any
// pushed shard.  Since done <= pushed at every instant and both only grow,
// equal sums mean that at the moment between the two reads nothing was
// queued or being expanded, and nothing can be published after that (only a
// near-far split adds work, and splits are excluded by the caller).
__device__ __forceinline__ bool warp_quiescent(const AsyncCtl* ctl, uint32_t lane) {
  unsigned long long d = *(volatile const unsigned long long*)&ctl->done[16 * lane];
  __threadfence();
  __syncwarp();
  unsigned long long p = *(volatile const unsigned long long*)&ctl->pushed[16 * lane];
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    d += __shfl_xor_sync(0xFFFFFFFFu, d, o);
    p += __shfl_xor_sync(0xFFFFFFFFu, p, o);
  }
  return d == p;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) { return *(volatile const uint32_t*)p; }

struct AsyncArgs {
  DevGraph g;
  unsigned long long* Q;
  uint32_t logcap;
  uint32_t* inq;
  AsyncCtl* ctl;
};

// Warp-aggregated far-pile append: one atomicMin on far_min (the warp's
// smallest parked distance fd, skipped when it cannot lower the minimum) and
// one atomicAdd on the pile's count for the lanes with app == true.
__device__ __forceinline__ void far_append_warp(AsyncCtl* ctl, bool app, uint32_t v, uint32_t fd, uint32_t lane) {
  uint32_t m = fd;
#pragma unroll
  for (int o = 16; o; o >>= 1) m = min(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
  const unsigned am = __ballot_sync(0xFFFFFFFFu, app);
  uint32_t sel = 0, base = 0;
  if (lane == 0) {
    if (m != kInf && m < ld_volatile_u32(&ctl->far_min)) atomicMin(&ctl->far_min, m);
    if (am) {
      sel = ld_volatile_u32(&ctl->sel);
      base = atomicAdd(&ctl->far_cnt[sel], (uint32_t)__popc(am));
    }
  }
  if (!am) return;
  sel = __shfl_sync(0xFFFFFFFFu, sel, 0);
  base = __shfl_sync(0xFFFFFFFFu, base, 0);
  if (app) ctl->far[sel][base + __popc(am & ((1u << lane) - 1u))] = v;
}

// A lane's consumer state: the queue position it reserved (have), and an
// item it already took from the ring but has not expanded yet (held).
struct Taker {
  unsigned long long pos;
  uint32_t held_v;
  bool have, held;
};

// Take the item at the lane's reserved position if it has been published:
// mark the slot consumed for this lap, clear the vertex's in-queue bit (a
// later improvement re-enqueues it) and order that before the dist read.
__device__ __forceinline__ bool try_take(const AsyncArgs& a, Taker& tk, uint32_t& v) {
  unsigned long long* slot = a.Q + (tk.pos & ((1ull << a.logcap) - 1));
  const uint32_t lap = (uint32_t)(tk.pos >> a.logcap);
  const unsigned long long val = ld_acquire_u64(slot);
  if ((uint32_t)(val >> 32) != 2 * lap + 1) return false;
  v = (uint32_t)val;
  tk.have = false;
  st_release_u64(slot, (unsigned long long)(2 * lap + 2) << 32);
  atomicAnd(a.inq + (v >> 5), ~(1u << (v & 31)));
  __threadfence();
  return true;
}

// Enqueue the improved vertices held by the lanes with want == true (new
// distance nd): below the threshold into the ring queue, otherwise into the
// far pile (once, by the far bitmap).
__device__ __forceinline__ void push_warp(const AsyncArgs& a, bool want, uint32_t v, uint32_t nd, uint32_t lane,
                                          Taker& tk) {
  if (!__any_sync(0xFFFFFFFFu, want)) return;
  bool mine = false, fnew = false;
  uint32_t fd = kInf;
  if (want) {
    const uint32_t rs = __ldg(a.g.ro + v), re = __ldg(a.g.ro + v + 1);
    if (re > rs) {
      __threadfence();   // the dist update is visible before the in-queue / far bit
      const uint32_t bit = 1u << (v & 31);
      if (nd < ld_volatile_u32(&a.ctl->t_cur)) {
        mine = !(atomicOr(a.inq + (v >> 5), bit) & bit);
      } else {
        fd = nd;
        fnew = !(atomicOr(a.ctl->bm_far + (v >> 5), bit) & bit);
      }
    }
  }
  far_append_warp(a.ctl, fnew, v, fd, lane);
  const unsigned mm = __ballot_sync(0xFFFFFFFFu, mine);
  if (!mm) return;
  const uint32_t cnt = __popc(mm);
  const uint32_t leader = __ffs(mm) - 1;
  unsigned long long base = 0;
  if (lane == leader) {
    atomicAdd(&a.ctl->pushed[16 * shard_of_warp()], (unsigned long long)cnt);
    base = atomicAdd(&a.ctl->tail, (unsigned long long)cnt);
  }
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  // Publish.  A slot is free once its previous lap was consumed.  The whole
  // warp waits together and meanwhile takes the items published at its own
  // reserved positions (held for its next round), so a warp never waits on a
  // slot that only it could free, and every waiting warp keeps freeing slots.
  const unsigned long long pos = base + __popc(mm & ((1u << lane) - 1));
  unsigned long long* slot = a.Q + (pos & ((1ull << a.logcap) - 1));
  const uint32_t want_tag = (uint32_t)(2 * (pos >> a.logcap));
  bool todo = mine;
  uint32_t spins = 0;
  for (;;) {
    if (todo && (uint32_t)(ld_acquire_u64(slot) >> 32) == want_tag) {
      st_release_u64(slot, ((unsigned long long)(want_tag + 1) << 32) | v);
      todo = false;
    }
    if (!__any_sync(0xFFFFFFFFu, todo)) break;
    if (tk.have && !tk.held) {
      uint32_t hv;
      if (try_take(a, tk, hv)) {
        tk.held = true;
        tk.held_v = hv;
      }
    }
    int stop = 0;
    if (lane == 0) {
      if (ld_volatile_u32(&a.ctl->abort)) {
        stop = 1;
      } else if (++spins > (1u << 22) || past_watchdog(a.ctl->t_start, a.ctl->watchdog_ns)) {
        atomicOr(&a.ctl->status, DS_TIMEOUT);
        atomicExch(&a.ctl->abort, 1u);
        stop = 1;
      }
    }
    if (__shfl_sync(0xFFFFFFFFu, stop, 0)) return;
    __nanosleep(64);
  }
}

template <bool PK>
__global__ void __launch_bounds__(kABlock) k_async(AsyncArgs a) {
  __shared__ uint32_t s_pref[kAWarps][33];
  __shared__ uint32_t s_row[kAWarps][32];
  __shared__ uint32_t s_du[kAWarps][32];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  AsyncCtl* ctl = a.ctl;
  uint32_t* dist = ctl->dist;
  const uint32_t wmode = ctl->wmode;
  Taker tk{0ull, 0u, false, false};
  uint32_t backoff = 32, idle_rounds = 0;
  unsigned long long pops = 0, edges = 0;
  bool ovf = false;
  for (;;) {
    if (!__any_sync(0xFFFFFFFFu, tk.have)) {
      unsigned long long h = 0;
      if (lane == 0) h = atomicAdd(&ctl->head, 32ull);
      h = __shfl_sync(0xFFFFFFFFu, h, 0);
      tk.pos = h + lane;
      tk.have = true;
    }
    bool got = false;
    uint32_t v = 0;
    if (tk.held) {   // taken while this warp waited to publish
      v = tk.held_v;
      tk.held = false;
      got = true;
    } else if (tk.have) {
      got = try_take(a, tk, v);
    }
    const unsigned gm = __ballot_sync(0xFFFFFFFFu, got);
    if (gm) {
      backoff = 32;
      idle_rounds = 0;
      uint32_t deg = 0, rs = 0, du = 0;
      if (got) {
        rs = __ldg(a.g.ro + v);
        deg = __ldg(a.g.ro + v + 1) - rs;
        du = ld_cg(dist + v);
      }
      uint32_t x = deg;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
      }
      const uint32_t total = __shfl_sync(0xFFFFFFFFu, x, 31);
      s_pref[wid][lane] = x - deg;
      s_row[wid][lane] = rs;
      s_du[wid][lane] = du;
      __syncwarp();
      for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t gidx = base + lane;
        bool want = false;
        uint32_t dst = 0, ndv = 0;
        if (gidx < total) {
          // last lane whose prefix is <= gidx (lanes without an item repeat the next prefix)
          uint32_t lo = 0, len = 32;
          while (len > 0) {
            const uint32_t half = len >> 1;
            if (s_pref[wid][lo + half] <= gidx) { lo += half + 1; len -= half + 1; }
            else len = half;
          }
          const uint32_t k = lo - 1;
          const uint2 ed = load_edge<PK>(a.g.edges, s_row[wid][k] + (gidx - s_pref[wid][k]), a.g.wbits);
          const uint32_t nd = relax_add(s_du[wid][k], ed.y, ovf, wmode);
          dst = ed.x;
          ndv = nd;
          if (nd < ld_cg(dist + dst)) {
            const uint32_t old = atomicMin(dist + dst, nd);
            want = nd < old;
          }
        }
        push_warp(a, want, dst, ndv, lane, tk);
      }
      pops += got ? 1 : 0;
      edges += got ? deg : 0;
      __threadfence();
      __syncwarp();
      if (lane == 0) atomicAdd(&ctl->done[16 * shard_of_warp()], (unsigned long long)__popc(gm));
      if (ld_volatile_u32(&ctl->abort)) break;
    } else {
      // idle: re-poll the own reserved slots (distinct lines) most of the
      // time; only every 8th idle round read the shared state to stop, start
      // or join a far-pile split -- thousands of idle warps polling the same
      // counters would otherwise serialise the working warps' atomics on them
      if ((++idle_rounds & 7u) != 0u) {
        __nanosleep(backoff);
        backoff = min(backoff * 2, 1024u);
        continue;
      }
      int act = 0;   // 0 back off, 1 stop, 2 split work, 3 split lock taken
      uint32_t e1 = 0, ph = 0;
      if (lane == 0) {
        if (ld_volatile_u32(&ctl->abort)) {
          act = 1;
        } else if (past_watchdog(ctl->t_start, ctl->watchdog_ns)) {
          atomicOr(&ctl->status, DS_TIMEOUT);
          atomicExch(&ctl->abort, 1u);
          act = 1;
        } else {
          e1 = ld_volatile_u32(&ctl->epoch);
          ph = ld_volatile_u32(&ctl->phase);
          if (ph == 2) act = 2;
        }
      }
      act = __shfl_sync(0xFFFFFFFFu, act, 0);
      ph = __shfl_sync(0xFFFFFFFFu, ph, 0);
      if (act == 0 && ph == 0) {
        // quiescence is read between two reads of the split epoch, so no
        // split can have started and ended unseen in between
        const bool quiet = warp_quiescent(ctl, lane);
        if (lane == 0 && quiet) {
          const uint32_t nfar = ld_volatile_u32(&ctl->far_cnt[ld_volatile_u32(&ctl->sel)]);
          const uint32_t e2 = ld_volatile_u32(&ctl->epoch);
          if (e1 == e2 && ld_volatile_u32(&ctl->phase) == 0) {
            if (nfar == 0) {
              act = 1;   // nothing queued, running or parked: done
            } else if (atomicCAS(&ctl->phase, 0u, 1u) == 0u) {
              act = 3;
            }
          }
        }
        act = __shfl_sync(0xFFFFFFFFu, act, 0);
        if (act == 3) {
          // split lock held: start a split if still nothing is in flight
          __threadfence();
          const bool still = warp_quiescent(ctl, lane);
          if (lane == 0) {
            const uint32_t src = ctl->sel;
            const uint32_t total = ld_volatile_u32(&ctl->far_cnt[src]);
            if (!still || total == 0) {
              atomicExch(&ctl->phase, 0u);
              act = 0;
            } else {
              const unsigned long long t1 = (unsigned long long)ctl->t_cur + ctl->delta;
              const unsigned long long t2 = (unsigned long long)ctl->far_min + 1;
              const unsigned long long tn = t1 > t2 ? t1 : t2;
              ctl->t_prev = ctl->t_cur;
              ctl->t_cur = tn >= kInf ? kInf : (uint32_t)tn;
              ctl->far_min = kInf;
              ctl->split_src = src;
              ctl->split_total = total;
              ctl->split_cursor = 0;
              ctl->split_done = 0;
              ctl->sel = src ^ 1u;
              const uint32_t ep = ctl->epoch;
              if (ctl->trace && ep < ctl->trace_cap) {
                uint32_t* t = ctl->trace + 4ull * ep;
                t[0] = ep;
                t[1] = ctl->t_cur;
                t[2] = total;
                const long long el = (long long)(globaltimer() - ctl->t_start);
                t[3] = el > 0 ? (uint32_t)(el / 1000) : 0u;
              }
              ctl->epoch = ep + 1;
              __threadfence();
              atomicExch(&ctl->phase, 2u);
              act = 2;
            }
          }
        }
      }
      act = __shfl_sync(0xFFFFFFFFu, act, 0);
      if (act == 1) break;
      if (act == 2) {
        // one 32-entry chunk of the far pile being split
        uint32_t chunk = 0;
        if (lane == 0) chunk = atomicAdd(&ctl->split_cursor, 32u);
        chunk = __shfl_sync(0xFFFFFFFFu, chunk, 0);
        const uint32_t total = ld_volatile_u32(&ctl->split_total);
        if (chunk < total) {
          const uint32_t idx = chunk + lane;
          bool want = false, keep = false;
          uint32_t v = 0, d = 0;
          if (idx < total) {
            const uint32_t src = ld_volatile_u32(&ctl->split_src);
            v = ld_cg(ctl->far[src] + idx);
            d = ld_cg(dist + v);
            const uint32_t bit = 1u << (v & 31);
            if (d < ld_volatile_u32(&ctl->t_cur)) {
              atomicAnd(ctl->bm_far + (v >> 5), ~bit);
              want = d >= ld_volatile_u32(&ctl->t_prev);   // below t_prev: expanded already
            } else {
              keep = true;
            }
          }
          far_append_warp(ctl, keep, v, keep ? d : kInf, lane);
          push_warp(a, want, v, d, lane, tk);
          const uint32_t done = (uint32_t)min(32u, total - chunk);
          __threadfence();
          __syncwarp();
          if (lane == 0 && atomicAdd(&ctl->split_done, done) + done == total) {
            ctl->far_cnt[ld_volatile_u32(&ctl->split_src)] = 0u;
            __threadfence();
            atomicExch(&ctl->phase, 0u);
          }
          backoff = 32;
          continue;
        }
      }
      __nanosleep(backoff);
      backoff = min(backoff * 2, 1024u);
    }
  }
  // per-warp stats
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    pops += __shfl_down_sync(0xFFFFFFFFu, pops, o);
    edges += __shfl_down_sync(0xFFFFFFFFu, edges, o);
  }
  const unsigned ov = __ballot_sync(0xFFFFFFFFu, ovf);
  if (lane == 0) {
    atomicAdd(&ctl->pops, pops);
    atomicAdd(&ctl->edges, edges);
    if (ov) atomicOr(&ctl->status, DS_OVERFLOW);
  }
}

__global__ void k_async_init(DevGraph g, uint32_t* dist, uint32_t* inq, uint32_t* bm_far, uint32_t unreached) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (uint64_t i = t; i < g.n; i += stride) dist[i] = unreached;
  for (uint64_t i = t; i < g.nwords; i += stride) {
    inq[i] = 0u;
    bm_far[i] = 0u;
  }
}

__global__ void k_async_seed(DevGraph g, uint32_t src, uint32_t* dist, unsigned long long* Q, uint32_t* inq,
                             AsyncCtl* ctl, unsigned long long watchdog_ns, uint32_t delta, uint32_t* far0,
                             uint32_t* far1, uint32_t* bm_far, uint32_t* trace, uint32_t trace_cap,
                             uint32_t wmode) {
  dist[src] = 0u;
  ctl->t_cur = delta;
  ctl->t_prev = 0;
  ctl->delta = delta;
  ctl->sel = 0;
  ctl->far_cnt[0] = 0;
  ctl->far_cnt[1] = 0;
  ctl->far_min = kInf;
  ctl->phase = 0;
  ctl->epoch = 0;
  ctl->trace = trace;
  ctl->trace_cap = trace ? trace_cap : 0u;
  ctl->wmode = wmode;
  ctl->split_src = 0;
  ctl->split_total = 0;
  ctl->split_cursor = 0;
  ctl->split_done = 0;
  ctl->far[0] = far0;
  ctl->far[1] = far1;
  ctl->bm_far = bm_far;
  ctl->head = 0;
  ctl->pops = 0;
  ctl->edges = 0;
  ctl->status = 0;
  ctl->abort = 0;
  ctl->dist = dist;
  ctl->watchdog_ns = watchdog_ns;
  ctl->t_start = globaltimer();
  for (int i = 0; i < kAShards; ++i) {
    ctl->pushed[16 * i] = 0ull;
    ctl->done[16 * i] = 0ull;
  }
  if (g.ro[src + 1] > g.ro[src]) {
    Q[0] = (1ull << 32) | src;
    inq[src >> 5] = 1u << (src & 31);
    ctl->tail = 1;
    ctl->pushed[0] = 1ull;
  } else {
    ctl->tail = 0;
  }
}

}  // namespace

gg_status async_run(gg_graph* g, uint32_t src, uint32_t* dist, const gg_options& o, cudaStream_t s, uint32_t wmode) {
  AsyncWorkspace& w = g->async;
  const DeviceInfo di = device_info();
  if (!w.block) {
    // ring of >= 2n + (resident warps * 32) slots
    int per_sm = 0;
    GG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_async<false>, kABlock, 0));
    int per_sm_pk = 0;
    GG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_pk, k_async<true>, kABlock, 0));
    per_sm = std::min(per_sm, per_sm_pk);
    if (per_sm < 1) return fail(GG_ERR_INTERNAL, "async kernel does not fit on an SM");
    w.grid = per_sm * di.num_sms;
    const uint64_t need = 2ull * g->n + (uint64_t)w.grid * kAWarps * 32 + 1024;
    uint32_t logcap = 10;
    while ((1ull << logcap) < need) ++logcap;
    const size_t qbytes = sizeof(unsigned long long) << logcap;
    const size_t nw = (g->n + 31) / 32;
    const size_t r_bm = (sizeof(uint32_t) * nw + 255) & ~size_t(255);
    const size_t r_far = (sizeof(uint32_t) * std::max<size_t>(g->n, 1) + 255) & ~size_t(255);
    const size_t r_ctl = (sizeof(AsyncCtl) + 255) & ~size_t(255);
    const size_t total = qbytes + 2 * r_bm + 2 * r_far + r_ctl;
    char* p = nullptr;
    GG_CK(cudaMalloc(&p, total));
    w.block = p;
    w.bytes = total;
    w.queue = reinterpret_cast<uint32_t*>(p);
    w.cap = logcap;   // stored as log2 capacity
    w.inq = reinterpret_cast<uint32_t*>(p + qbytes);
    w.bm_far = reinterpret_cast<uint32_t*>(p + qbytes + r_bm);
    w.far[0] = reinterpret_cast<uint32_t*>(p + qbytes + 2 * r_bm);
    w.far[1] = reinterpret_cast<uint32_t*>(p + qbytes + 2 * r_bm + r_far);
    w.ctl = p + qbytes + 2 * r_bm + 2 * r_far;
    if (!g->h_async) GG_CK(cudaMallocHost(&g->h_async, sizeof(AsyncCtl)));
  }
  const uint32_t logcap = w.cap;
  unsigned long long* Q = reinterpret_cast<unsigned long long*>(w.queue);
  AsyncCtl* ctl = reinterpret_cast<AsyncCtl*>(w.ctl);
  GG_CK(cudaMemsetAsync(Q, 0, sizeof(unsigned long long) << logcap, s));
  unsigned ib = (unsigned)std::min<uint64_t>((g->n + 255) / 256, (uint64_t)di.num_sms * 8);
  if (ib == 0) ib = 1;
  k_async_init<<<ib, 256, 0, s>>>(g->dg, dist, w.inq, w.bm_far, wmode == WM_F32 ? kFltMaxBits : kInf);
  GG_CK(cudaGetLastError());
  const unsigned long long wd = o.watchdog_ns ? o.watchdog_ns : 10000000000ull;
  // buckets are integer distance ranges: binary32 and hop-count runs go without
  const uint32_t delta =
      (o.delta == GG_DELTA_NONE || wmode != WM_U32) ? kInf : (o.delta ? o.delta : g->default_delta);
  k_async_seed<<<1, 1, 0, s>>>(g->dg, src, dist, Q, w.inq, ctl, wd, delta, w.far[0], w.far[1], w.bm_far, o.trace,
                               o.trace_cap, wmode);
  GG_CK(cudaGetLastError());
  AsyncArgs a{g->dg, Q, logcap, w.inq, ctl};
  void* args[] = {&a};
  void* fn = g->dg.packed ? reinterpret_cast<void*>(&k_async<true>) : reinterpret_cast<void*>(&k_async<false>);
  GG_CK(cudaLaunchCooperativeKernel(fn, dim3(w.grid), dim3(kABlock), args, 0, s));
  return GG_OK;
}

gg_status async_status(gg_graph* g, uint32_t* ds, gg_stats* st) {
  if (!g->async.ctl) return GG_OK;
  AsyncCtl* h = reinterpret_cast<AsyncCtl*>(g->h_async);
  GG_CK(cudaMemcpyAsync(h, g->async.ctl, sizeof(AsyncCtl), cudaMemcpyDeviceToHost, g->last_stream));
  GG_CK(cudaStreamSynchronize(g->last_stream));
  *ds = h->status;
  if (st) {
    st->iterations = 0;
    st->pull_iterations = 0;
    st->edges_scanned = h->edges;
    st->frontier_total = h->pops;
    st->max_frontier = 0;
  }
  return GG_OK;
}

gg_status async_release(gg_graph* g) {
  if (g->async.block) cudaFree(g->async.block);
  g->async = AsyncWorkspace{};
  return GG_OK;
}

}  // namespace gg
