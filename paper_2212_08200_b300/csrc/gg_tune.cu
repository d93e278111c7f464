// gg_tune.cu -- autotuners: time candidate option sets on the caller's graph
// and sample sources with CUDA events and return the fastest.
//   gg_autotune        single source: coordinate descent over policy, bucket
//                      width (the light/heavy width on skewed graphs, the
//                      near-far width otherwise), direction / switch
//                      threshold and load balancing (warp streaming with or
//                      without warp-local rounds, merge-path tiles, or degree
//                      bins with thresholds);
//   gg_autotune_batch  batched sources: schedule (normalised buckets or
//                      light-first rounds) and light/heavy width.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "gg_host.h"
#include "gg_nvtx.h"

using namespace gg;

namespace {

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// median over `reps` of the summed time of one run per sample source
gg_status time_options(gg_graph* g, const uint32_t* srcs, uint32_t nsrc, uint32_t* dist, const gg_options& o,
                       cudaStream_t s, Timer& t, int reps, float* ms) {
  std::vector<float> v;
  for (int r = 0; r < reps; ++r) {
    GG_CK(cudaEventRecord(t.a, s));
    for (uint32_t i = 0; i < nsrc; ++i) {
      gg_status st = gg_sssp_ex(g, srcs[i], dist, &o, s);
      if (st != GG_OK) return st;
    }
    GG_CK(cudaEventRecord(t.b, s));
    GG_CK(cudaEventSynchronize(t.b));
    float x = 0;
    GG_CK(cudaEventElapsedTime(&x, t.a, t.b));
    v.push_back(x);
  }
  std::sort(v.begin(), v.end());
  *ms = v[v.size() / 2];
  // a candidate that hit the watchdog or a cap is not a valid choice
  if (gg_graph_check(g) != GG_OK) *ms = 3.0e38f;
  return GG_OK;
}

// Candidate bucket widths for the graph (distinct, non-zero): light/heavy
// widths floor(K * w_max / mean degree) for K in 1.5 .. 4.5 on graphs that
// have a light/heavy default, near-far widths d0/8 .. 8 d0 otherwise, and
// GG_DELTA_NONE (no buckets).
std::vector<uint32_t> bucket_widths(const gg_graph* g) {
  std::vector<uint32_t> out{GG_DELTA_NONE};
  auto add = [&](uint64_t d) {
    if (d == 0 || d >= GG_DELTA_NONE) return;
    if (std::find(out.begin(), out.end(), (uint32_t)d) == out.end()) out.push_back((uint32_t)d);
  };
  if (g->default_delta_lh != GG_DELTA_NONE) {
    const double davg = g->n ? (double)g->m / g->n : 1.0;
    for (double k : {1.5, 2.0, 2.4, 2.7, 3.0, 3.5, 4.5})
      add((uint64_t)std::min<double>(std::max(1.0, std::floor(k * g->wmax / std::max(davg, 1e-9))), g->wmax));
  } else {
    const uint64_t d0 = std::max<uint32_t>(g->default_delta, 1);
    if (g->default_delta != GG_DELTA_NONE)
      for (uint64_t d : {d0 / 8, d0 / 2, d0, d0 * 2, d0 * 8}) add(d);
  }
  return out;
}

// median over `reps` of one batched call over all sources
gg_status time_batch(gg_graph* g, const uint32_t* srcs, uint32_t k, uint32_t* dist, const gg_options& o,
                     cudaStream_t s, Timer& t, int reps, float* ms) {
  std::vector<float> v;
  for (int r = 0; r < reps; ++r) {
    GG_CK(cudaEventRecord(t.a, s));
    gg_status st = gg_sssp_batch_ex(g, srcs, k, dist, &o, s);
    if (st != GG_OK) return st;
    GG_CK(cudaEventRecord(t.b, s));
    GG_CK(cudaEventSynchronize(t.b));
    float x = 0;
    GG_CK(cudaEventElapsedTime(&x, t.a, t.b));
    v.push_back(x);
  }
  std::sort(v.begin(), v.end());
  *ms = v[v.size() / 2];
  if (gg_graph_check(g) != GG_OK) *ms = 3.0e38f;
  return GG_OK;
}

}  // namespace

extern "C" gg_status gg_autotune_batch(gg_graph_t g, const uint32_t* srcs, uint32_t k, uint32_t* dist_scratch,
                                       gg_options* best, float* best_ms, cudaStream_t stream) {
  NvtxRange nvtx_range("gg_autotune_batch");
  if (!g || !srcs || !dist_scratch || !best) return fail(GG_ERR_INVALID_ARG, "NULL argument");
  if (k == 0) return fail(GG_ERR_INVALID_ARG, "k must be >= 1");
  for (uint32_t i = 0; i < k; ++i)
    if (srcs[i] >= g->n) return fail(GG_ERR_INVALID_ARG, "a source is >= n");
  Timer t;
  GG_CK(cudaEventCreate(&t.a));
  GG_CK(cudaEventCreate(&t.b));
  gg_options cur;
  gg_options_default(&cur);
  float cur_ms = 0;
  gg_status st = time_batch(g, srcs, k, dist_scratch, cur, stream, t, 1, &cur_ms);   // warm-up
  if (st != GG_OK) return st;
  st = time_batch(g, srcs, k, dist_scratch, cur, stream, t, 3, &cur_ms);
  if (st != GG_OK) return st;
  // schedule x width: both schedules at every candidate width
  for (uint32_t lh : {GG_LH_AUTO, GG_LH_ROUNDS}) {
    for (uint32_t d : bucket_widths(g)) {
      gg_options o;
      gg_options_default(&o);
      o.light_heavy = lh;
      o.delta = d;
      float x;
      st = time_batch(g, srcs, k, dist_scratch, o, stream, t, 3, &x);
      if (st != GG_OK) return st;
      if (x < cur_ms) {
        cur = o;
        cur_ms = x;
      }
    }
  }
  *best = cur;
  if (best_ms) *best_ms = cur_ms;
  return GG_OK;
}

extern "C" gg_status gg_autotune(gg_graph_t g, const uint32_t* srcs, uint32_t nsrc, uint32_t* dist_scratch,
                                 gg_options* best, float* best_ms, cudaStream_t stream) {
  NvtxRange nvtx_range("gg_autotune");
  if (!g || !srcs || !dist_scratch || !best) return fail(GG_ERR_INVALID_ARG, "NULL argument");
  if (nsrc == 0) return fail(GG_ERR_INVALID_ARG, "nsrc must be >= 1");
  for (uint32_t i = 0; i < nsrc; ++i)
    if (srcs[i] >= g->n) return fail(GG_ERR_INVALID_ARG, "a source is >= n");
  Timer t;
  GG_CK(cudaEventCreate(&t.a));
  GG_CK(cudaEventCreate(&t.b));
  gg_options cur;
  gg_options_default(&cur);
  cur.direction = GG_DIR_PUSH;
  cur.watchdog_ns = 20000000000ull;
  float cur_ms = 0;
  // warm-up (workspace, CUDA graphs)
  for (int pol : {GG_POLICY_BSP_GRAPH, GG_POLICY_BSP_PERSISTENT}) {
    gg_options w = cur;
    w.policy = (gg_policy)pol;
    float x;
    gg_status st = time_options(g, srcs, 1, dist_scratch, w, stream, t, 1, &x);
    if (st != GG_OK) return st;
  }
  gg_status st = time_options(g, srcs, nsrc, dist_scratch, cur, stream, t, 3, &cur_ms);
  if (st != GG_OK) return st;
  auto try_opt = [&](const gg_options& o) -> gg_status {
    float x;
    gg_status s2 = time_options(g, srcs, nsrc, dist_scratch, o, stream, t, 3, &x);
    if (s2 != GG_OK) return s2;
    if (x < cur_ms) {
      cur = o;
      cur_ms = x;
    }
    return GG_OK;
  };
  // 1. policy
  {
    gg_options o = cur;
    o.policy = GG_POLICY_BSP_PERSISTENT;
    if ((st = try_opt(o)) != GG_OK) return st;
  }
  // 2. bucket width: on skewed graphs the light/heavy width (light edges per
  //    vertex from 1.5 to 4.5 around the default 2.7), elsewhere the near-far
  //    width around the graph's default; and no buckets at all
  {
    const gg_options base = cur;
    for (uint32_t d : bucket_widths(g)) {
      gg_options o = base;
      o.delta = d;
      if ((st = try_opt(o)) != GG_OK) return st;
    }
  }
  // 3. direction: push/pull switching at a few thresholds
  {
    const gg_options base = cur;
    for (uint32_t alpha : {2u, 4u, 16u}) {
      gg_options o = base;
      o.direction = GG_DIR_AUTO;
      o.pull_alpha = alpha;
      if ((st = try_opt(o)) != GG_OK) return st;
    }
  }
  // 4. load balancing: warp streaming with and without warp-local rounds,
  //    merge-path tiles, or degree bins at a few thresholds
  {
    const gg_options base = cur;
    for (gg_lb_mode lb : {GG_LB_WARP, GG_LB_LOCAL, GG_LB_MERGE_PATH}) {
      gg_options o = base;
      o.lb_mode = lb;
      if ((st = try_opt(o)) != GG_OK) return st;
    }
  }
  {
    const gg_options base = cur;
    for (uint32_t w : {8u, 32u}) {
      for (uint32_t c : {256u, 4096u}) {
        gg_options o = base;
        o.lb_mode = GG_LB_BINS;
        o.warp_threshold = w;
        o.cta_threshold = c;
        if ((st = try_opt(o)) != GG_OK) return st;
      }
    }
  }
  cur.watchdog_ns = 0;
  *best = cur;
  if (best_ms) *best_ms = cur_ms / (float)nsrc;
  return GG_OK;
}
