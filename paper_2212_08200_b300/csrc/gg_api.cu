// gg_api.cu -- the extern "C" boundary: argument checks, error reporting,
// handle lifetime and policy dispatch.  No compute happens here; every step
// of an SSSP run is a kernel in gg_bsp.cu / gg_async.cu.
#include <cuda_runtime.h>
#include <stdio.h>

#include <new>
#include <string>

#include "gg_host.h"
#include "gg_nvtx.h"

namespace gg {

static thread_local std::string t_err;

void set_error(const std::string& msg) { t_err = msg; }

gg_status fail(gg_status s, const std::string& msg) {
  t_err = msg;
  return s;
}

gg_status cuda_fail(cudaError_t e, const char* what) {
  t_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  if (e == cudaErrorMemoryAllocation) return GG_ERR_OUT_OF_MEMORY;
  return GG_ERR_CUDA;
}

#ifndef GG_POOL_KEEP
#define GG_POOL_KEEP (8ull << 30)   // freed bytes the allocation pool keeps mapped
#endif

namespace {
cudaMemPool_t pool_for_current_device() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t keep = GG_POOL_KEEP;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = pool;
  }
  return pools[dev];
}
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool = pool_for_current_device();
  if (!pool) return cudaMallocAsync(p, bytes, s);
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

void dev_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

DeviceInfo device_info() {
  static thread_local DeviceInfo cache[16];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 16) dev = 0;
  DeviceInfo& d = cache[dev];
  if (d.device != dev) {
    d.device = dev;
    cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  return d;
}

gg_status status_from_device(uint32_t ds) {
  if (ds & DS_TIMEOUT) return GG_ERR_TIMEOUT;
  if (ds & DS_OVERFLOW) return GG_ERR_OVERFLOW;
  if (ds & (DS_ITER_CAP | DS_INTERNAL)) return GG_ERR_INTERNAL;
  return GG_OK;
}

gg_status bsp_read_ctl(gg_graph* g, cudaStream_t s);

}  // namespace gg

using namespace gg;

namespace {

gg_status order_after_previous(gg_graph* g, cudaStream_t s) {
  if (g->ev_valid && g->last_stream != s) GG_CK(cudaStreamWaitEvent(s, g->last_ev, 0));
  return GG_OK;
}

gg_status record_call(gg_graph* g, cudaStream_t s) {
  GG_CK(cudaEventRecord(g->last_ev, s));
  g->last_stream = s;
  g->ev_valid = true;
  return GG_OK;
}

}  // namespace

extern "C" {

uint32_t gg_abi_version(void) { return GG_ABI_VERSION; }

const char* gg_status_string(gg_status s) {
  switch (s) {
    case GG_OK: return "GG_OK";
    case GG_ERR_INVALID_ARG: return "GG_ERR_INVALID_ARG";
    case GG_ERR_OUT_OF_MEMORY: return "GG_ERR_OUT_OF_MEMORY";
    case GG_ERR_CUDA: return "GG_ERR_CUDA";
    case GG_ERR_TIMEOUT: return "GG_ERR_TIMEOUT";
    case GG_ERR_BUSY: return "GG_ERR_BUSY";
    case GG_ERR_NOT_READY: return "GG_ERR_NOT_READY";
    case GG_ERR_OVERFLOW: return "GG_ERR_OVERFLOW";
    case GG_ERR_INTERNAL: return "GG_ERR_INTERNAL";
    case GG_ERR_NOT_SUPPORTED: return "GG_ERR_NOT_SUPPORTED";
  }
  return "GG_UNKNOWN_STATUS";
}

const char* gg_last_error(void) { return t_err.c_str(); }

void gg_options_default(gg_options* o) {
  if (!o) return;
  *o = gg_options{};
  o->struct_size = sizeof(gg_options);
  o->policy = GG_POLICY_BSP_GRAPH;
  o->direction = GG_DIR_PUSH;   // measured faster than push/pull switching for SSSP on RMAT-20/22
  o->lb_mode = GG_LB_AUTO;
}

gg_status gg_graph_create_csr(uint32_t n, uint64_t m, const uint32_t* row_offsets, const uint32_t* col_indices,
                              const uint32_t* weights, uint32_t flags, cudaStream_t stream, gg_graph_t* out) {
  NvtxRange nvtx_range("gg_graph_create_csr");
  if (!out) return fail(GG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n == 0 || n >= 0xFFFFFFFFu) return fail(GG_ERR_INVALID_ARG, "n must be in [1, 2^32 - 2]");
  if (m >= 0xFFFFFFFFull) return fail(GG_ERR_INVALID_ARG, "m must be < 2^32 - 1 (uint32 row offsets)");
  if (!row_offsets) return fail(GG_ERR_INVALID_ARG, "row_offsets is NULL");
  if (m > 0 && (!col_indices || !weights)) return fail(GG_ERR_INVALID_ARG, "col_indices/weights is NULL");
  if (flags & ~(GG_DEVICE_PTRS | GG_SYMMETRIC | GG_NO_VALIDATE | GG_NO_PACK | GG_FLOAT_WEIGHTS))
    return fail(GG_ERR_INVALID_ARG, "unknown flag");
  gg_graph* g = new (std::nothrow) gg_graph();
  if (!g) return fail(GG_ERR_OUT_OF_MEMORY, "host allocation failed");
  gg_status st = graph_build(g, n, m, row_offsets, col_indices, weights, flags, stream);
  if (st == GG_OK) {
    cudaError_t e = cudaEventCreateWithFlags(&g->last_ev, cudaEventDisableTiming);
    // (the pinned control-block mirror is allocated on first use: bsp_read_ctl)
    if (e != cudaSuccess) st = cuda_fail(e, "graph handle setup");
  }
  if (st != GG_OK) {
    std::string msg = t_err;
    cudaStreamSynchronize(stream);
    graph_free(g);
    if (g->last_ev) cudaEventDestroy(g->last_ev);
    if (g->h_ctl) cudaFreeHost(g->h_ctl);
    delete g;
    t_err = msg;
    return st;
  }
  *out = g;
  return GG_OK;
}

gg_status gg_graph_destroy(gg_graph_t g) {
  NvtxRange nvtx_range("gg_graph_destroy");
  if (!g) return fail(GG_ERR_INVALID_ARG, "graph is NULL");
  {
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->ev_valid) cudaEventSynchronize(g->last_ev);
    bsp_release(g);
    async_release(g);
    batch_release(g);
    graph_free(g);
    if (g->last_ev) cudaEventDestroy(g->last_ev);
    if (g->h_ctl) cudaFreeHost(g->h_ctl);
    if (g->h_async) cudaFreeHost(g->h_async);
  }
  delete g;
  return GG_OK;
}

gg_status gg_graph_info(gg_graph_t g, uint32_t* n, uint64_t* m, uint64_t* device_bytes) {
  if (!g) return fail(GG_ERR_INVALID_ARG, "graph is NULL");
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (device_bytes) *device_bytes = g->bytes + g->bsp.bytes + g->async.bytes + batch_bytes(g) + g->lh_bytes;
  return GG_OK;
}

static gg_status collect(gg_graph* g, cudaStream_t s, gg_stats* st_out) {
  uint32_t ds = 0;
  gg_stats st{};
  if (g->last_policy == GG_POLICY_ASYNC_PERSISTENT) {
    gg_status r = async_status(g, &ds, &st);
    if (r != GG_OK) return r;
  } else if (g->last_policy == kLastBatch) {
    gg_status r = batch_status(g, &ds);
    if (r != GG_OK) return r;
  } else if (g->last_policy >= 0) {
    gg_status r = bsp_read_ctl(g, s);
    if (r != GG_OK) return r;
    const Ctl& c = *g->h_ctl;
    ds = c.status;
    st.iterations = c.iter;
    st.pull_iterations = c.pull_iters;
    st.edges_scanned = c.edges_scanned;
    st.frontier_total = c.frontier_total;
    st.max_frontier = c.max_frontier;
  }
  st.device_status = (uint32_t)status_from_device(ds);
  if (st_out) *st_out = st;
  return status_from_device(ds);
}

gg_status gg_graph_check(gg_graph_t g) {
  if (!g) return fail(GG_ERR_INVALID_ARG, "graph is NULL");
  std::lock_guard<std::mutex> lk(g->mu);
  if (!g->ev_valid) return GG_OK;
  GG_CK(cudaEventSynchronize(g->last_ev));
  gg_status r = collect(g, g->last_stream, nullptr);
  if (r != GG_OK && r != GG_ERR_CUDA && r != GG_ERR_OUT_OF_MEMORY) {
    const char* what = r == GG_ERR_OVERFLOW ? "a finite distance did not fit below 0xFFFFFFFF"
                       : r == GG_ERR_TIMEOUT ? "the asynchronous queue did not drain before the watchdog limit"
                                             : "superstep cap reached before the frontier emptied";
    set_error(what);
  }
  return r;
}

namespace {

// One single-source run in the given weight mode (WM_U32 / WM_F32 / WM_UNIT).
gg_status run_single(gg_graph_t g, uint32_t src, uint32_t* dist_out, const gg_options* opt, cudaStream_t stream,
                     uint32_t wmode) {
  if (!g) return fail(GG_ERR_INVALID_ARG, "graph is NULL");
  if (!dist_out) return fail(GG_ERR_INVALID_ARG, "dist_out is NULL");
  if (src >= g->n) return fail(GG_ERR_INVALID_ARG, "src >= n");
  gg_options o;
  gg_options_default(&o);
  if (opt) {
    if (opt->struct_size != sizeof(gg_options)) return fail(GG_ERR_INVALID_ARG, "gg_options.struct_size mismatch");
    o = *opt;
  }
  if ((unsigned)o.policy > 3u) return fail(GG_ERR_INVALID_ARG, "unknown policy");
  if ((unsigned)o.direction > 2u) return fail(GG_ERR_INVALID_ARG, "unknown direction");
  if ((unsigned)o.lb_mode > 4u) return fail(GG_ERR_INVALID_ARG, "unknown load-balance mode");
  if (o.light_heavy > GG_LH_ROUNDS) return fail(GG_ERR_INVALID_ARG, "unknown light_heavy mode");
  if (o.trace && o.trace_cap == 0) return fail(GG_ERR_INVALID_ARG, "trace without trace_cap");
  int dev = -1;
  GG_CK(cudaGetDevice(&dev));
  if (dev != g->device) return fail(GG_ERR_INVALID_ARG, "current device differs from the graph's device");
  std::lock_guard<std::mutex> lk(g->mu);
  gg_status st = order_after_previous(g, stream);
  if (st != GG_OK) return st;
  if (o.policy == GG_POLICY_ASYNC_PERSISTENT) st = async_run(g, src, dist_out, o, stream, wmode);
  else st = bsp_run(g, src, dist_out, o, stream, wmode);
  if (st != GG_OK) return st;
  g->last_policy = (int)o.policy;
  st = record_call(g, stream);
  if (st != GG_OK) return st;
  if (o.stats) {
    GG_CK(cudaStreamSynchronize(stream));
    st = collect(g, stream, o.stats);
    if (st != GG_OK && st != GG_ERR_CUDA) set_error("device status: " + std::string(gg_status_string(st)));
    return st;
  }
  return GG_OK;
}

}  // namespace

gg_status gg_sssp_ex(gg_graph_t g, uint32_t src, uint32_t* dist_out, const gg_options* opt, cudaStream_t stream) {
  NvtxRange nvtx_range("gg_sssp");
  return run_single(g, src, dist_out, opt, stream, g && g->float_weights ? WM_F32 : WM_U32);
}

gg_status gg_sssp(gg_graph_t g, uint32_t src, uint32_t* dist_out, cudaStream_t stream) {
  return gg_sssp_ex(g, src, dist_out, nullptr, stream);
}

gg_status gg_bfs_ex(gg_graph_t g, uint32_t src, uint32_t* depth_out, const gg_options* opt, cudaStream_t stream) {
  NvtxRange nvtx_range("gg_bfs");
  return run_single(g, src, depth_out, opt, stream, WM_UNIT);
}

gg_status gg_bfs(gg_graph_t g, uint32_t src, uint32_t* depth_out, cudaStream_t stream) {
  return gg_bfs_ex(g, src, depth_out, nullptr, stream);
}

gg_status gg_sssp_batch_ex(gg_graph_t g, const uint32_t* srcs, uint32_t k, uint32_t* dist_out,
                           const gg_options* opt, cudaStream_t stream) {
  NvtxRange nvtx_range("gg_sssp_batch");
  if (!g) return fail(GG_ERR_INVALID_ARG, "graph is NULL");
  if (!srcs || !dist_out) return fail(GG_ERR_INVALID_ARG, "srcs/dist_out is NULL");
  if (k == 0) return fail(GG_ERR_INVALID_ARG, "k must be >= 1");
  if (g->float_weights) return fail(GG_ERR_NOT_SUPPORTED, "binary32 weights: gg_sssp, gg_sssp_ex and gg_bfs only");
  for (uint32_t i = 0; i < k; ++i)
    if (srcs[i] >= g->n) return fail(GG_ERR_INVALID_ARG, "a source is >= n");
  gg_options o;
  gg_options_default(&o);
  if (opt) {
    if (opt->struct_size != sizeof(gg_options)) return fail(GG_ERR_INVALID_ARG, "gg_options.struct_size mismatch");
    o = *opt;
  }
  if (o.stats) *o.stats = gg_stats{};
  if (o.light_heavy > GG_LH_ROUNDS) return fail(GG_ERR_INVALID_ARG, "unknown light_heavy mode");
  int dev = -1;
  GG_CK(cudaGetDevice(&dev));
  if (dev != g->device) return fail(GG_ERR_INVALID_ARG, "current device differs from the graph's device");
  std::lock_guard<std::mutex> lk(g->mu);
  gg_status st = order_after_previous(g, stream);
  if (st != GG_OK) return st;
  st = batch_run(g, srcs, k, dist_out, o, stream);
  if (st != GG_OK) return st;
  g->last_policy = kLastBatch;
  st = record_call(g, stream);
  if (st != GG_OK) return st;
  if (o.stats) {
    const gg_status ds = status_from_device(o.stats->device_status);
    o.stats->device_status = (uint32_t)ds;
    if (ds != GG_OK) set_error("device status: " + std::string(gg_status_string(ds)));
    return ds;
  }
  return GG_OK;
}

gg_status gg_sssp_batch(gg_graph_t g, const uint32_t* srcs, uint32_t k, uint32_t* dist_out, cudaStream_t stream) {
  return gg_sssp_batch_ex(g, srcs, k, dist_out, nullptr, stream);
}

}  // extern "C"
