// gg_host.h -- host-side internals shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "gg.h"
#include "gg_common.cuh"

namespace gg {

// thread-local error message + status helper
void set_error(const std::string& msg);
gg_status fail(gg_status s, const std::string& msg);
gg_status cuda_fail(cudaError_t e, const char* what);

#define GG_CK(call)                                          \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return ::gg::cuda_fail(e_, #call); \
  } while (0)

// Device memory of graph handles and their workspaces comes from one
// stream-ordered pool per device that keeps up to GG_POOL_KEEP bytes of freed
// memory mapped, so that creating and destroying handles does not map and
// unmap memory (nor synchronise the device, as cudaFree does) each time.
cudaError_t dev_malloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);
template <class T>
cudaError_t dev_malloc(T** p, size_t bytes, cudaStream_t s) {
  return dev_malloc(reinterpret_cast<void**>(p), bytes, s);
}

struct DeviceInfo {
  int device = -1;
  int num_sms = 0;
  int max_smem_optin = 0;
};
DeviceInfo device_info();

// Superstep kernel variants: load balance (4) x edge packing (2) x weight
// mode (u32, binary32, unit, u32 with light/heavy buckets).
constexpr int kWmU32Lh = 3;
constexpr int kBspVariants = 4 * 2 * 4;

// Workspace of the bulk-synchronous path (allocated on first use).
struct BspWorkspace {
  Frontier fr{};
  Ctl* ctl = nullptr;
  void* block = nullptr;      // single device allocation backing fr and ctl
  size_t bytes = 0;
  // CUDA graph with a conditional WHILE node around one superstep kernel,
  // one per kernel variant.
  cudaGraph_t graph[kBspVariants] = {};
  cudaGraphExec_t exec[kBspVariants] = {};
  int grid[kBspVariants] = {};
};

// Workspace of the asynchronous persistent path.
struct AsyncWorkspace {
  void* block = nullptr;
  size_t bytes = 0;
  uint32_t* queue = nullptr;   // ring of vertex ids
  uint32_t cap = 0;            // power of two >= n
  uint32_t* inq = nullptr;     // in-queue bitmap
  uint32_t* bm_far = nullptr;  // far-pile bitmap
  uint32_t* far[2] = {nullptr, nullptr};
  void* ctl = nullptr;         // AsyncCtl
  int grid = 0;
};

struct BatchWorkspace;

}  // namespace gg

struct gg_graph {
  uint32_t n = 0;
  uint32_t m = 0;
  int device = -1;
  bool symmetric = false;
  gg::DevGraph dg{};
  // owned device buffers
  uint32_t* ro = nullptr;
  uint2* edges = nullptr;
  uint32_t* t_ro = nullptr;
  uint2* t_edges = nullptr;
  uint32_t* edges4 = nullptr;     // packed edges (replace edges/t_edges when used)
  uint32_t* t_edges4 = nullptr;
  uint32_t* pv = nullptr;
  uint32_t* ps = nullptr;
  size_t bytes = 0;
  std::mutex mu;
  gg::BspWorkspace bsp;
  gg::AsyncWorkspace async;
  gg::BatchWorkspace* batch = nullptr;
  cudaEvent_t last_ev = nullptr;
  cudaStream_t last_stream = nullptr;
  bool ev_valid = false;
  gg::Ctl* h_ctl = nullptr;      // pinned host mirror for status/stats reads
  void* h_async = nullptr;       // pinned host mirror of the async control block
  int last_policy = -1;
  uint32_t wmax = 0;            // largest edge weight (bit pattern)
  bool float_weights = false;   // weights and distances are IEEE binary32 bit patterns
  uint32_t default_delta = 0;   // near-far bucket width used when gg_options.delta == 0
  bool low_degree = false;      // mean degree < 8 (grids, paths): smaller superstep grid
  // light/heavy buckets of the single-source bulk-synchronous loop: bucket
  // width used when gg_options.delta == 0 (GG_DELTA_NONE: none), and the
  // light-first edge copy with its buffers (lh_delta = the width it is
  // partitioned for, 0 before the first light/heavy run)
  uint32_t default_delta_lh = GG_DELTA_NONE;
  uint32_t lh_delta = 0;
  uint64_t lh_heavy_total = 0;    // edges with weight >= lh_delta
  void* lh_block = nullptr;
  size_t lh_bytes = 0;
  gg::LhBufs lhb{};
};

namespace gg {
// gg_bsp.cu
gg_status bsp_run(gg_graph* g, uint32_t src, uint32_t* dist, const gg_options& o, cudaStream_t s, uint32_t wmode);
gg_status bsp_release(gg_graph* g);
// gg_async.cu
gg_status async_run(gg_graph* g, uint32_t src, uint32_t* dist, const gg_options& o, cudaStream_t s, uint32_t wmode);
gg_status async_release(gg_graph* g);
gg_status async_status(gg_graph* g, uint32_t* ds, gg_stats* st);
// gg_batch.cu
gg_status batch_run(gg_graph* g, const uint32_t* srcs, uint32_t k, uint32_t* dist, const gg_options& o,
                    cudaStream_t s);
gg_status batch_status(gg_graph* g, uint32_t* ds);
void batch_release(gg_graph* g);
size_t batch_bytes(const gg_graph* g);
constexpr int kLastBatch = 16;   // gg_graph::last_policy value after gg_sssp_batch
// gg_graph.cu
gg_status graph_build(gg_graph* g, uint32_t n, uint64_t m, const uint32_t* ro, const uint32_t* col,
                      const uint32_t* w, uint32_t flags, cudaStream_t s);
void graph_free(gg_graph* g);
// light-first edge copy partitioned for bucket width delta (and the R-list
// buffers), built on first use and re-partitioned when delta changes
gg_status lh_prepare(gg_graph* g, uint32_t delta, cudaStream_t s);
gg_status status_from_device(uint32_t ds);
}  // namespace gg
