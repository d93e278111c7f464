// gg_server.cu -- gg_sssp_multi (many graphs, one source each, one launch
// sequence) and the query server (continuous batching of (graph, source)
// requests over the slot engine of gg_multi.cu).
//
// Server model:
//   submit   enqueues a request (thread-safe) and returns a ticket;
//   worker   one host thread per server owns a CUDA stream and loops:
//              admit    queued requests take free slots while the in-flight
//                       vertex budget allows: the engine's capacity (sized
//                       from free HBM at creation), re-derived at every
//                       admission round from the device's free HBM, so that
//                       memory other allocations take later defers admission;
//                       each admitted query's distances are reset and its
//                       source seeded straight into the running union frontier
//              run      a CUDA graph advances every in-flight query by up to
//                       `supersteps_per_launch` supersteps
//              retire   queries whose frontier emptied are flagged by the
//                       device in host-mapped memory; their slots are freed
//                       for the next admission round
//   poll     reports GG_ERR_NOT_READY until the request's distances are final.
// New queries therefore join while others are mid-flight and share every
// superstep launch with them; a query's result does not depend on what it
// shared the GPU with (distances are exact integers).
//
// Queries on graphs with a light/heavy width (skewed graphs with integer
// weights, when the server uses the graphs' default bucket widths) are
// coalesced per graph instead: the worker takes up to 64 queued sources of
// one graph (round robin over the graphs with queued queries) into one
// batched call (gg_sssp_batch_ex: normalised buckets, light-first rounds with
// a pulled heavy superstep) on a second stream, then copies each column of
// the distance matrix to its query's array.  Such a batch overlaps the slot
// engine's launches; queries arriving meanwhile wait for the next batch of
// their graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gg_host.h"
#include "gg_nvtx.h"
#include "gg_multi.h"

using namespace gg;
using Clock = std::chrono::steady_clock;

namespace {

#ifndef GG_MULTI_SKEW_DELTA
#define GG_MULTI_SKEW_DELTA 0   // multiple of the light/heavy width used as the slot's near-far width on
#endif                          // skewed graphs (0: the graph's own default, no buckets)

// Near-far width of a query slot when the caller asks for the graph's default.
uint32_t slot_default_delta(const gg_graph* g) {
  if (GG_MULTI_SKEW_DELTA && g->default_delta == GG_DELTA_NONE && g->default_delta_lh != GG_DELTA_NONE)
    return (uint32_t)std::min<uint64_t>((uint64_t)g->default_delta_lh * GG_MULTI_SKEW_DELTA, 0xFFFFFFFEull);
  return g->default_delta;
}

void fill_slot(MultiSlot& s, const gg_graph* g, uint32_t src, uint32_t* dist, uint32_t ticket, uint32_t off0,
               uint32_t off1, uint32_t off2, uint32_t far0, uint32_t far1, uint32_t delta) {
  s = MultiSlot{};
  s.ro = g->dg.ro;
  s.edges = g->dg.edges;
  s.dist = dist;
  s.n = g->n;
  s.packed = g->dg.packed;
  s.wbits = g->dg.wbits;
  s.src = src;
  s.bm_off[0] = off0;
  s.bm_off[1] = off1;
  s.bm_off[2] = off2;
  s.state = kSlotFree;
  s.ticket = ticket;
  multi_slot_buckets(s, delta == 0 ? slot_default_delta(g) : delta, far0, far1);
}

// ---- gg_sssp_multi: a process-wide engine per device, grown on demand -------
struct MultiCache {
  std::mutex mu;
  MultiEngine eng;
  cudaEvent_t ev = nullptr;
  bool ev_valid = false;
  cudaStream_t last = nullptr;
};
MultiCache g_multi[16];

}  // namespace

extern "C" gg_status gg_sssp_multi_ex(const gg_graph_t* graphs, const uint32_t* srcs, uint32_t count,
                                      uint32_t* const* dist_outs, uint32_t delta, cudaStream_t stream) {
  NvtxRange nvtx_range("gg_sssp_multi");
  if (!graphs || !srcs || !dist_outs) return fail(GG_ERR_INVALID_ARG, "graphs/srcs/dist_outs is NULL");
  if (count == 0) return fail(GG_ERR_INVALID_ARG, "count must be >= 1");
  int dev = 0;
  GG_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 16) return fail(GG_ERR_NOT_SUPPORTED, "device index out of range");
  uint64_t total_n = 0, words = 0;
  uint32_t nmax = 1;
  for (uint32_t i = 0; i < count; ++i) {
    const gg_graph* g = graphs[i];
    if (!g) return fail(GG_ERR_INVALID_ARG, "a graph is NULL");
    if (!dist_outs[i]) return fail(GG_ERR_INVALID_ARG, "a dist_out is NULL");
    if (g->device != dev) return fail(GG_ERR_INVALID_ARG, "a graph lives on another device");
    if (srcs[i] >= g->n) return fail(GG_ERR_INVALID_ARG, "a source is >= its graph's n");
    if (g->float_weights)
      return fail(GG_ERR_NOT_SUPPORTED, "binary32 weights: gg_sssp, gg_sssp_ex and gg_bfs only");
    total_n += g->n;
    words += 3ull * ((g->n + 31) / 32);
    nmax = std::max(nmax, g->n);
  }
  if (total_n >= 0xFFFFFFFFull || words >= 0xFFFFFFFFull)
    return fail(GG_ERR_INVALID_ARG, "the queries' vertex total must stay below 2^32");
  MultiCache& mc = g_multi[dev];
  std::lock_guard<std::mutex> lk(mc.mu);
  MultiEngine& e = mc.eng;
  if (mc.ev_valid) {
    if (mc.last != stream) GG_CK(cudaStreamWaitEvent(stream, mc.ev, 0));
  }
  if (count > (uint32_t)kMaxSplitSlots) return fail(GG_ERR_INVALID_ARG, "at most 1024 queries per call");
  if (!e.block || e.max_slots < count || e.cap_vertices < total_n || e.cap_words < words || e.cap_far < 2 * total_n) {
    if (mc.ev_valid) GG_CK(cudaEventSynchronize(mc.ev));
    if (e.block) multi_engine_free(&e);
    gg_status st = multi_engine_init(&e, std::max<uint32_t>(count, 64), std::max<uint64_t>(total_n, 1 << 16),
                                     std::max<uint64_t>(words, 4096), std::max<uint64_t>(2 * total_n, 1 << 17),
                                     false);
    if (st != GG_OK) { multi_engine_free(&e); return st; }
  }
  if (!mc.ev) GG_CK(cudaEventCreateWithFlags(&mc.ev, cudaEventDisableTiming));
  // the previous call's slot table may still be read by in-flight work on its stream
  if (mc.ev_valid) GG_CK(cudaEventSynchronize(mc.ev));
  gg_status st = multi_engine_reset(&e, stream);
  if (st != GG_OK) return st;
  std::vector<uint32_t> ids(count);
  uint32_t off = 0, foff = 0;
  for (uint32_t i = 0; i < count; ++i) {
    const uint32_t w = (graphs[i]->n + 31) / 32;
    const uint32_t nn = graphs[i]->n;
    fill_slot(e.h_slots[i], graphs[i], srcs[i], dist_outs[i], i + 1, off, off + w, off + 2 * w, foff, foff + nn,
              delta);
    off += 3 * w;
    foff += 2 * nn;
    ids[i] = i;
  }
  // slots beyond count stay free
  for (uint32_t q = count; q < e.max_slots; ++q) e.h_slots[q].state = kSlotFree;
  GG_CK(cudaMemcpyAsync(e.b.slots + count, e.h_slots + count, sizeof(MultiSlot) * (e.max_slots - count),
                        cudaMemcpyHostToDevice, stream));
  st = multi_engine_start(&e, ids.data(), count, stream);
  if (st != GG_OK) return st;
  // every query converges within about 3n supersteps with buckets (n + 1 without)
  st = multi_engine_run(&e, (uint32_t)std::min<uint64_t>(4ull * nmax + 16, 0xFFFFFFFEull), stream);
  if (st != GG_OK) return st;
  GG_CK(cudaEventRecord(mc.ev, stream));
  mc.ev_valid = true;
  mc.last = stream;
  return GG_OK;
}

extern "C" gg_status gg_sssp_multi(const gg_graph_t* graphs, const uint32_t* srcs, uint32_t count,
                                   uint32_t* const* dist_outs, cudaStream_t stream) {
  return gg_sssp_multi_ex(graphs, srcs, count, dist_outs, 0, stream);
}

// ---- server ------------------------------------------------------------------

struct gg_server {
  int device = 0;
  gg_server_config cfg{};
  MultiEngine eng;
  cudaStream_t stream = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  gg_status worker_error = GG_OK;
  std::string worker_msg;

  struct Req {
    gg_graph* g;
    uint32_t src;
    uint32_t* dist;
    Clock::time_point t_submit, t_done;
    gg_status status = GG_OK;
    int state = 0;   // 0 queued, 1 running, 2 done
  };
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Req> reqs;
  std::vector<uint64_t> slot_ticket;   // 0 = free
  uint64_t next_ticket = 1;
  uint64_t used_vertices = 0;
  uint64_t live_budget = 0;   // vertex budget of the last admission round
  uint32_t running = 0;
  std::vector<double> lat_us;
  gg_server_stats st{};
  // per-graph source batches (skewed graphs)
  std::unordered_map<gg_graph*, std::deque<uint64_t>> gq;   // queued tickets per graph
  std::deque<gg_graph*> gorder;                             // graphs with queued tickets, round robin
  cudaStream_t bstream = nullptr;
  cudaEvent_t bev = nullptr;
  std::vector<uint64_t> btickets;   // the batch in flight (empty: none)
  gg_graph* bgraph = nullptr;
  uint32_t* bmat = nullptr;         // its distance matrix (n x k) and the k output pointers after it
  uint32_t** h_bptr = nullptr;      // pinned staging of the output pointers
  uint32_t* h_bsrc = nullptr;       // pinned staging of the sources
};

namespace {

// Device bytes charged per in-flight vertex when the budget is re-derived
// from free HBM (frontier state, bitmaps and far piles, with headroom).
constexpr uint64_t kBytesPerFlightVertex = 32;

// The in-flight vertex budget in force now: the engine's capacity, capped by
// the vertices already in flight plus what the device's free HBM above the
// reserve would hold.  Other allocations on the device that leave less than
// the reserve free therefore stop admission until memory is released.
uint64_t live_budget(const gg_server* s) {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return s->used_vertices;   // defer on error
  const uint64_t head = free_b > s->cfg.hbm_reserve_bytes ? (free_b - s->cfg.hbm_reserve_bytes) / kBytesPerFlightVertex
                                                          : 0ull;
  return std::min<uint64_t>(s->eng.cap_vertices, s->used_vertices + head);
}

constexpr uint32_t kServerBatch = 64;

// Whether a query on g goes to a per-graph source batch.
bool batched_graph(const gg_server* s, const gg_graph* g) {
  return s->cfg.delta == 0 && g->default_delta_lh != GG_DELTA_NONE && g->m > 0 && !g->float_weights;
}

// out[s][v] := mat[v * k + s]: one thread per vertex, row read once, each
// column written coalesced across the warp
__global__ void k_scatter_columns(const uint32_t* __restrict__ mat, uint32_t n, uint32_t k,
                                  uint32_t* const* __restrict__ out) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const uint32_t* row = mat + (size_t)v * k;
    for (uint32_t c = 0; c < k; ++c) out[c][v] = row[c];
  }
}

// Starts the next per-graph batch on the batch stream when none is in flight
// and the free HBM above the reserve holds its distance matrix.  Called with
// the server lock held; returns false when nothing was started.
bool start_batch(gg_server* s) {
  if (!s->btickets.empty() || s->gorder.empty()) return false;
  gg_graph* g = s->gorder.front();
  std::deque<uint64_t>& q = s->gq[g];
  const uint32_t k = (uint32_t)std::min<size_t>(q.size(), kServerBatch);
  const uint64_t mat_bytes = 4ull * g->n * k + 8ull * kServerBatch + 256;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess || free_b < s->cfg.hbm_reserve_bytes + mat_bytes)
    return false;   // wait for memory (other work finishes first)
  s->gorder.pop_front();
  for (uint32_t i = 0; i < k; ++i) {
    const uint64_t t = q.front();
    q.pop_front();
    gg_server::Req& r = s->reqs[t];
    r.state = 1;
    s->btickets.push_back(t);
    s->h_bsrc[i] = r.src;
    s->h_bptr[i] = r.dist;
  }
  if (!q.empty()) s->gorder.push_back(g);   // more of this graph: after the other graphs
  else s->gq.erase(g);
  s->bgraph = g;
  gg_status st = GG_OK;
  char* buf = nullptr;
  cudaError_t e = dev_malloc(&buf, mat_bytes, s->bstream);
  if (e == cudaSuccess) {
    s->bmat = reinterpret_cast<uint32_t*>(buf);
    uint32_t** dptr = reinterpret_cast<uint32_t**>(buf + ((4ull * g->n * k + 255) & ~255ull));
    e = cudaMemcpyAsync(dptr, s->h_bptr, sizeof(uint32_t*) * k, cudaMemcpyHostToDevice, s->bstream);
    if (e == cudaSuccess) st = gg_sssp_batch_ex(g, s->h_bsrc, k, s->bmat, nullptr, s->bstream);
    if (e == cudaSuccess && st == GG_OK) {
      const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((g->n + 255) / 256, 4096));
      k_scatter_columns<<<grid, 256, 0, s->bstream>>>(s->bmat, g->n, k, dptr);
      e = cudaGetLastError();
    }
    dev_free(buf, s->bstream);
    s->bmat = nullptr;
  }
  if (e == cudaSuccess && st == GG_OK) e = cudaEventRecord(s->bev, s->bstream);
  if (e != cudaSuccess || st != GG_OK) {
    // the batch could not be launched: its queries fail with the error
    const gg_status fs = st != GG_OK ? st : GG_ERR_CUDA;
    const Clock::time_point now = Clock::now();
    for (uint64_t t : s->btickets) {
      gg_server::Req& r = s->reqs[t];
      r.state = 2;
      r.status = fs;
      r.t_done = now;
    }
    s->btickets.clear();
    s->cv_done.notify_all();
    return false;
  }
  return true;
}

// Retires the batch in flight once its event completed (wait: block for it).
// Called with the server lock held.
void finish_batch(gg_server* s, bool wait) {
  if (s->btickets.empty()) return;
  cudaError_t e = wait ? cudaEventSynchronize(s->bev) : cudaEventQuery(s->bev);
  if (e == cudaErrorNotReady) return;
  gg_status st = e == cudaSuccess ? gg_graph_check(s->bgraph) : GG_ERR_CUDA;
  const Clock::time_point now = Clock::now();
  for (uint64_t t : s->btickets) {
    gg_server::Req& r = s->reqs[t];
    r.state = 2;
    r.status = st;
    r.t_done = now;
    s->lat_us.push_back(std::chrono::duration<double, std::micro>(now - r.t_submit).count());
    s->st.completed += 1;
  }
  s->st.launches += 1;
  s->btickets.clear();
  s->bgraph = nullptr;
  s->cv_done.notify_all();
}

void server_loop(gg_server* s) {
  cudaSetDevice(s->device);
  const uint32_t words = (s->cfg.max_graph_vertices + 31) / 32;
  std::vector<uint32_t> admit;
  for (;;) {
    admit.clear();
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        // admission: free slot and room in the in-flight vertex budget in force
        if (!s->queue.empty()) s->live_budget = live_budget(s);
        while (!s->queue.empty()) {
          const uint64_t t = s->queue.front();
          gg_server::Req& r = s->reqs[t];
          if (s->used_vertices + r.g->n > s->live_budget) break;
          uint32_t q = 0;
          while (q < s->eng.max_slots && s->slot_ticket[q]) ++q;
          if (q == s->eng.max_slots) break;
          s->queue.pop_front();
          s->slot_ticket[q] = t;
          s->used_vertices += r.g->n;
          r.state = 1;
          const uint32_t maxn = s->cfg.max_graph_vertices;
          fill_slot(s->eng.h_slots[q], r.g, r.src, r.dist, (uint32_t)t, 3 * q * words, 3 * q * words + words,
                    3 * q * words + 2 * words, 2 * q * maxn, 2 * q * maxn + maxn, s->cfg.delta);
          s->eng.h_done[q] = 0;
          admit.push_back(q);
          ++s->running;
        }
        s->st.max_running = std::max(s->st.max_running, s->running);
        // per-graph batches: retire a finished one, start the next
        finish_batch(s, false);
        start_batch(s);
        s->st.max_running = std::max<uint32_t>(s->st.max_running, s->running + (uint32_t)s->btickets.size());
        if (s->running > 0 || !admit.empty()) break;
        if (!s->btickets.empty()) {   // only a batch in flight: wait for it without the lock
          lk.unlock();
          cudaEventSynchronize(s->bev);
          lk.lock();
          finish_batch(s, false);
          continue;
        }
        if (s->stop && s->gorder.empty()) return;
        s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
      }
    }
    gg_status e = multi_engine_start(&s->eng, admit.data(), (uint32_t)admit.size(), s->stream);
    if (e == GG_OK) e = multi_engine_run(&s->eng, s->cfg.supersteps_per_launch, s->stream);
    cudaError_t ce = cudaStreamSynchronize(s->stream);
    std::unique_lock<std::mutex> lk(s->mu);
    if (e != GG_OK || ce != cudaSuccess) {
      s->worker_error = e != GG_OK ? e : GG_ERR_CUDA;
      s->worker_msg = ce != cudaSuccess ? cudaGetErrorString(ce) : "slot engine launch failed";
      // fail every in-flight and queued request
      for (auto& kv : s->reqs) {
        if (kv.second.state != 2) {
          kv.second.state = 2;
          kv.second.status = s->worker_error;
          kv.second.t_done = Clock::now();
        }
      }
      s->queue.clear();
      s->cv_done.notify_all();
      return;
    }
    s->st.launches += 1;
    const Clock::time_point now = Clock::now();
    for (uint32_t q = 0; q < s->eng.max_slots; ++q) {
      const uint64_t t = s->slot_ticket[q];
      if (!t) continue;
      if (reinterpret_cast<volatile uint32_t*>(s->eng.h_done)[q] != (uint32_t)t) continue;
      gg_server::Req& r = s->reqs[t];
      r.state = 2;
      r.t_done = now;
      r.status = status_from_device(reinterpret_cast<volatile uint32_t*>(s->eng.h_done_status)[q]);
      s->lat_us.push_back(std::chrono::duration<double, std::micro>(now - r.t_submit).count());
      s->st.completed += 1;
      s->slot_ticket[q] = 0;
      s->used_vertices -= r.g->n;
      --s->running;
    }
    s->cv_done.notify_all();
  }
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double idx = p * (v.size() - 1);
  const size_t lo = (size_t)idx;
  const size_t hi = std::min(lo + 1, v.size() - 1);
  return v[lo] + (v[hi] - v[lo]) * (idx - lo);
}

}  // namespace

extern "C" {

void gg_server_config_default(gg_server_config* c) {
  if (!c) return;
  *c = gg_server_config{};
  c->struct_size = sizeof(gg_server_config);
  c->max_slots = 64;
  c->supersteps_per_launch = 8;
  c->hbm_reserve_bytes = 1ull << 30;
}

gg_status gg_server_create(const gg_server_config* cfg, gg_server_t* out) {
  if (!cfg || !out) return fail(GG_ERR_INVALID_ARG, "cfg/out is NULL");
  *out = nullptr;
  if (cfg->struct_size != sizeof(gg_server_config)) return fail(GG_ERR_INVALID_ARG, "struct_size mismatch");
  if (cfg->max_graph_vertices == 0) return fail(GG_ERR_INVALID_ARG, "max_graph_vertices must be set");
  gg_server* s = new gg_server();
  s->cfg = *cfg;
  if (!s->cfg.max_slots) s->cfg.max_slots = 64;
  if (!s->cfg.supersteps_per_launch) s->cfg.supersteps_per_launch = 8;
  if (s->cfg.max_slots > (uint32_t)kMaxSplitSlots) { delete s; return fail(GG_ERR_INVALID_ARG, "max_slots > 1024"); }
  const uint64_t words = 3ull * s->cfg.max_slots * ((s->cfg.max_graph_vertices + 31) / 32);
  const uint64_t far_entries = 2ull * s->cfg.max_slots * s->cfg.max_graph_vertices;
  uint64_t cap = s->cfg.max_vertices_in_flight ? s->cfg.max_vertices_in_flight
                                               : (uint64_t)s->cfg.max_slots * s->cfg.max_graph_vertices;
  cap = std::max<uint64_t>(cap, s->cfg.max_graph_vertices);
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) { delete s; return cuda_fail(e, "cudaGetDevice"); }
  // admission by free HBM: the in-flight vertex budget (16 bytes of frontier
  // state per vertex) must fit in the free memory minus the reserve
  size_t free_b = 0, total_b = 0;
  e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) { delete s; return cuda_fail(e, "cudaMemGetInfo"); }
  const uint64_t avail = free_b > s->cfg.hbm_reserve_bytes ? free_b - s->cfg.hbm_reserve_bytes : 0;
  const uint64_t fixed = 4 * words + 4 * far_entries + 1024ull * s->cfg.max_slots + (1 << 20);
  if (avail < fixed + 32ull * s->cfg.max_graph_vertices) {
    delete s;
    return fail(GG_ERR_OUT_OF_MEMORY, "not enough free HBM for the server's frontier budget");
  }
  cap = std::min<uint64_t>(cap, (avail - fixed) / 32);
  if (cap >= 0xFFFFFFFFull || words >= 0xFFFFFFFFull || far_entries >= 0xFFFFFFFFull) {
    delete s;
    return fail(GG_ERR_INVALID_ARG, "budget too large");
  }
  gg_status st = multi_engine_init(&s->eng, s->cfg.max_slots, cap, words, far_entries, true);
  if (st == GG_OK) {
    e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->bstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->bev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_bptr, sizeof(uint32_t*) * kServerBatch);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_bsrc, sizeof(uint32_t) * kServerBatch);
    if (e != cudaSuccess) st = cuda_fail(e, "server streams");
  }
  if (st == GG_OK) st = multi_engine_reset(&s->eng, s->stream);
  if (st == GG_OK) {
    for (uint32_t q = 0; q < s->eng.max_slots; ++q) s->eng.h_slots[q].state = kSlotFree;
    e = cudaMemcpyAsync(s->eng.b.slots, s->eng.h_slots, sizeof(MultiSlot) * s->eng.max_slots,
                        cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "server setup");
  }
  if (st != GG_OK) {
    multi_engine_free(&s->eng);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->bstream) cudaStreamDestroy(s->bstream);
    if (s->bev) cudaEventDestroy(s->bev);
    if (s->h_bptr) cudaFreeHost(s->h_bptr);
    if (s->h_bsrc) cudaFreeHost(s->h_bsrc);
    delete s;
    return st;
  }
  s->slot_ticket.assign(s->eng.max_slots, 0);
  s->live_budget = s->eng.cap_vertices;
  s->worker = std::thread(server_loop, s);
  *out = s;
  return GG_OK;
}

gg_status gg_server_submit(gg_server_t s, gg_graph_t g, uint32_t src, uint32_t* dist_out, uint64_t* ticket) {
  NvtxRange nvtx_range("gg_server_submit");
  if (!s || !g || !dist_out || !ticket) return fail(GG_ERR_INVALID_ARG, "NULL argument");
  if (src >= g->n) return fail(GG_ERR_INVALID_ARG, "src >= n");
  if (g->float_weights)
    return fail(GG_ERR_NOT_SUPPORTED, "binary32 weights: gg_sssp, gg_sssp_ex and gg_bfs only");
  if (g->device != s->device) return fail(GG_ERR_INVALID_ARG, "graph lives on another device");
  if (g->n > s->cfg.max_graph_vertices) return fail(GG_ERR_INVALID_ARG, "graph larger than max_graph_vertices");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->worker_error != GG_OK) return fail(s->worker_error, "server stopped: " + s->worker_msg);
  if (s->stop) return fail(GG_ERR_BUSY, "server is shutting down");
  const uint64_t t = s->next_ticket++;
  if ((uint32_t)t == 0) {   // 0 marks "not done" in the device flags; skip it
    ++s->next_ticket;
    return gg_server_submit(s, g, src, dist_out, ticket);
  }
  gg_server::Req r;
  r.g = g;
  r.src = src;
  r.dist = dist_out;
  r.t_submit = Clock::now();
  s->reqs[t] = r;
  if (batched_graph(s, g)) {   // per-graph source batch
    std::deque<uint64_t>& q = s->gq[g];
    if (q.empty()) s->gorder.push_back(g);
    q.push_back(t);
  } else {
    s->queue.push_back(t);
  }
  s->st.submitted += 1;
  *ticket = t;
  s->cv_work.notify_one();
  return GG_OK;
}

gg_status gg_server_poll(gg_server_t s, uint64_t ticket, gg_status* result) {
  if (!s || !result) return fail(GG_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(GG_ERR_INVALID_ARG, "unknown or already collected ticket");
  if (it->second.state != 2) return GG_ERR_NOT_READY;
  *result = it->second.status;
  s->reqs.erase(it);
  return GG_OK;
}

gg_status gg_server_wait(gg_server_t s, uint64_t ticket, uint32_t timeout_ms, gg_status* result) {
  if (!s || !result) return fail(GG_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
  for (;;) {
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(GG_ERR_INVALID_ARG, "unknown or already collected ticket");
    if (it->second.state == 2) {
      *result = it->second.status;
      s->reqs.erase(it);
      return GG_OK;
    }
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      auto it2 = s->reqs.find(ticket);
      if (it2 != s->reqs.end() && it2->second.state == 2) continue;
      return GG_ERR_NOT_READY;
    }
  }
}

gg_status gg_server_get_stats(gg_server_t s, gg_server_stats* out) {
  if (!s || !out) return fail(GG_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  gg_server_stats st = s->st;
  size_t gq = 0;
  for (const auto& kv : s->gq) gq += kv.second.size();
  st.queued = (uint32_t)(s->queue.size() + gq);
  st.running = s->running + (uint32_t)s->btickets.size();
  st.p50_us = percentile(s->lat_us, 0.50);
  st.p99_us = percentile(s->lat_us, 0.99);
  double sum = 0, mx = 0;
  for (double v : s->lat_us) { sum += v; mx = std::max(mx, v); }
  st.mean_us = s->lat_us.empty() ? 0.0 : sum / s->lat_us.size();
  st.max_us = mx;
  st.vertex_budget = s->live_budget;
  *out = st;
  return GG_OK;
}

gg_status gg_server_reset_stats(gg_server_t s) {
  if (!s) return fail(GG_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  s->lat_us.clear();
  const uint64_t sub = s->st.submitted - s->st.completed;
  s->st = gg_server_stats{};
  s->st.submitted = sub;
  return GG_OK;
}

gg_status gg_server_destroy(gg_server_t s) {
  if (!s) return fail(GG_ERR_INVALID_ARG, "NULL argument");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();   // drains queued and in-flight queries first
  cudaStreamSynchronize(s->stream);
  cudaStreamSynchronize(s->bstream);
  multi_engine_free(&s->eng);
  cudaStreamDestroy(s->stream);
  cudaStreamDestroy(s->bstream);
  cudaEventDestroy(s->bev);
  cudaFreeHost(s->h_bptr);
  cudaFreeHost(s->h_bsrc);
  delete s;
  return GG_OK;
}

}  // extern "C"
