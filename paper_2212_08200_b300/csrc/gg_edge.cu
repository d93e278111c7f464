// gg_edge.cu -- an edge-frontier program on the same graph, frontier and
// operator abstraction: the shortest-path DAG and a predecessor per vertex.
//
// Sec. III-C lets a frontier hold edges as well as vertices, and lets the
// operator apply the user's program to each {source, destination, edge}.
// This program runs two operators over one graph handle and a distance
// vector (from gg_sssp or any other source of shortest-path distances):
//
//   advance + filter (vertex frontier -> edge frontier): every out-edge
//     (u, v, w) of every reached vertex u is tested, and the edge joins the
//     output edge frontier when it is tight, dist[u] + w == dist[v] (exact
//     64-bit sum).  Tight edges are exactly the edges that lie on some
//     shortest path from the source.  Entries carry (u, edge id); the edge id
//     is the edge's position in the caller's CSR.
//   edge operator over that frontier: parent[v] := min(parent[v], u) by
//     atomicMin, so each reached vertex other than the source gets the
//     smallest vertex id among its tight in-edges, the source gets itself and
//     everything else GG_INF.
//
// The advance balances work by edges: thread t takes an equal contiguous
// share of the m edge slots, finds the row holding its first edge with one
// binary search of the row offsets, and walks its share, moving to the next
// row as each one ends; tight edges are appended per warp with one atomic.
#include <cuda_runtime.h>

#include <algorithm>

#include "gg_host.h"
#include "gg_nvtx.h"

namespace gg {
namespace {

constexpr int kEB = 256;

// the row holding edge slot e: the last u with ro[u] <= e (ro[0] = 0 <= e < m)
__device__ __forceinline__ uint32_t row_of(const uint32_t* __restrict__ ro, uint32_t n, uint32_t e) {
  uint32_t lo = 0, hi = n;   // invariant: ro[lo] <= e < ro[hi]
  while (hi - lo > 1) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (__ldg(ro + mid) <= e) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <bool PK>
__global__ void __launch_bounds__(kEB) k_tight_edges(DevGraph g, const uint32_t* __restrict__ dist, uint32_t* eu,
                                                    uint32_t* ee, unsigned long long* cnt, uint64_t cap) {
  const unsigned FULL = 0xFFFFFFFFu;
  const uint32_t lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const uint64_t T = (uint64_t)gridDim.x * kEB;
  const uint64_t t = (uint64_t)blockIdx.x * kEB + threadIdx.x;
  const uint32_t e0 = (uint32_t)((uint64_t)g.m * t / T), e1 = (uint32_t)((uint64_t)g.m * (t + 1) / T);
  const uint32_t share = e1 - e0;
  const uint32_t steps = __reduce_max_sync(FULL, share);   // the warp walks its longest share
  uint32_t u = 0, uend = 0, du = kInf;
  if (share) {
    u = row_of(g.ro, g.n, e0);
    uend = __ldg(g.ro + u + 1);
    du = __ldg(dist + u);
  }
  for (uint32_t i = 0; i < steps; ++i) {
    bool tight = false;
    const uint32_t e = e0 + i;
    if (i < share) {
      while (e >= uend) {   // rows end inside the share: move on (empty rows are skipped)
        ++u;
        uend = __ldg(g.ro + u + 1);
        du = (e < uend) ? __ldg(dist + u) : du;
      }
      if (du != kInf) {
        const uint2 ed = load_edge<PK>(g.edges, e, g.wbits);
        tight = (unsigned long long)du + ed.y == (unsigned long long)__ldg(dist + ed.x);
      }
    }
    const unsigned b = __ballot_sync(FULL, tight);
    if (b) {
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(cnt, (unsigned long long)__popc(b));
      base = __shfl_sync(FULL, base, 0);
      const unsigned long long pos = base + __popc(b & lt);
      if (tight && pos < cap) {
        eu[pos] = u;
        ee[pos] = e;
      }
    }
  }
}

// parent := INF everywhere, parent[src] := src
__global__ void k_parent_init(uint32_t n, uint32_t src, uint32_t* parent) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    parent[v] = v == src ? src : kInf;
}

// the edge operator: every tight edge (u, e) offers u as v's predecessor
template <bool PK>
__global__ void k_edge_parent(DevGraph g, uint32_t src, const uint32_t* __restrict__ eu,
                              const uint32_t* __restrict__ ee, const unsigned long long* cnt, uint64_t cap,
                              uint32_t* parent) {
  const uint64_t c = min((uint64_t)*cnt, cap);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < c; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t v = load_edge<PK>(g.edges, ee[i], g.wbits).x;
    if (v != src) atomicMin(parent + v, eu[i]);
  }
}

}  // namespace
}  // namespace gg

using namespace gg;

extern "C" gg_status gg_sssp_tree(gg_graph_t g, uint32_t src, const uint32_t* dist, uint32_t* parent_out,
                                  uint32_t* tight_out, uint64_t tight_cap, uint64_t* tight_count,
                                  cudaStream_t stream) {
  NvtxRange nvtx_range("gg_sssp_tree");
  if (!g || !dist || !parent_out) return fail(GG_ERR_INVALID_ARG, "graph/dist/parent_out is NULL");
  if (src >= g->n) return fail(GG_ERR_INVALID_ARG, "src >= n");
  if (tight_cap && !tight_out) return fail(GG_ERR_INVALID_ARG, "tight_cap > 0 with tight_out NULL");
  if (g->float_weights) return fail(GG_ERR_NOT_SUPPORTED, "binary32 weights: integer graphs only");
  int dev = -1;
  GG_CK(cudaGetDevice(&dev));
  if (dev != g->device) return fail(GG_ERR_INVALID_ARG, "current device differs from the graph's device");
  std::lock_guard<std::mutex> lk(g->mu);
  if (g->ev_valid) GG_CK(cudaStreamWaitEvent(stream, g->last_ev, 0));   // after the handle's last call
  // the edge frontier: (u, edge id) per tight edge, at most m entries; the
  // caller's array is used for the edge ids when it can hold them all
  const uint64_t m = g->m;
  const bool own_ids = tight_cap < m;
  // each array starts on a 256-byte boundary (the 8-byte counter must be aligned)
  const uint64_t slot = (std::max<uint64_t>(m, 1) + 63) / 64 * 64;   // u32 entries
  uint32_t* buf = nullptr;
  const size_t bytes = sizeof(uint32_t) * slot * (own_ids ? 2 : 1) + 256;
  GG_CK(dev_malloc(&buf, bytes, stream));
  uint32_t* eu = buf;
  uint32_t* ee = own_ids ? buf + slot : tight_out;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(buf + slot * (own_ids ? 2 : 1));
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), stream);
  const DeviceInfo di = device_info();
  const unsigned pg = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((g->n + 255) / 256, (uint64_t)di.num_sms * 8));
  if (e == cudaSuccess) {
    k_parent_init<<<pg, 256, 0, stream>>>(g->n, src, parent_out);
    if (m) {
      const unsigned eg = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((m + 8ull * kEB - 1) / (8ull * kEB),
                                                                              (uint64_t)di.num_sms * 16));
      if (g->dg.packed) {
        k_tight_edges<true><<<eg, kEB, 0, stream>>>(g->dg, dist, eu, ee, cnt, m);
        k_edge_parent<true><<<eg, kEB, 0, stream>>>(g->dg, src, eu, ee, cnt, m, parent_out);
      } else {
        k_tight_edges<false><<<eg, kEB, 0, stream>>>(g->dg, dist, eu, ee, cnt, m);
        k_edge_parent<false><<<eg, kEB, 0, stream>>>(g->dg, src, eu, ee, cnt, m, parent_out);
      }
    }
    e = cudaGetLastError();
  }
  unsigned long long count = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&count, cnt, sizeof(count), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  const uint64_t keep = std::min<uint64_t>(tight_cap, count);
  if (e == cudaSuccess && own_ids && keep) {
    e = cudaMemcpyAsync(tight_out, ee, sizeof(uint32_t) * keep, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  }
  dev_free(buf, stream);
  if (e != cudaSuccess) return cuda_fail(e, "gg_sssp_tree");
  if (tight_count) *tight_count = count;
  return GG_OK;
}
