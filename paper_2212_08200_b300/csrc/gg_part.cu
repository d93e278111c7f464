// gg_part.cu -- single-source SSSP over a 1D vertex partition (one part per
// rank, Sec. III-D and Table I: the graph split across processors by a
// random vertex partition), with a per-superstep exchange of boundary
// updates.
//
// Each rank holds the out-edges of the vertices it owns (columns stay
// global ids) and the distances of those vertices.  A superstep on a rank:
//   advance   every out-edge (u, v, w) of its frontier is relaxed: when it
//             owns v the update is applied at once (atomicMin, and a vertex
//             whose distance dropped joins the next frontier through a
//             test-and-set in the next bitmap); otherwise the pair (v's index
//             on its owner, dist[u] + w) goes to a send list, which is then
//             grouped by destination rank (a counting sort over the ranks);
//   exchange  the caller moves the groups between ranks (a collective);
//   apply     every received pair is relaxed the same way as a local one.
// The run ends when no rank has a frontier.  Every relaxation is the same
// atomicMin with the strict < test as in the one-GPU loop, so the distances
// are the same fixed point.
//
// Vertex routing: route[v] = (owner << 24) | (v's index among its owner's
// vertices), so at most 256 ranks and 2^24 vertices per rank.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "gg_host.h"
#include "gg_nvtx.h"

struct gg_part {
  int device = -1;
  uint32_t n_global = 0, rank = 0, nranks = 1, n_local = 0;
  uint64_t m_local = 0;
  uint32_t* route = nullptr;   // u32[n_global]
  uint32_t* ro = nullptr;      // u32[n_local + 1]
  uint32_t* col = nullptr;     // u32[m_local], global ids
  uint32_t* w = nullptr;       // u32[m_local]
  uint32_t* dist = nullptr;    // u32[n_local]
  uint32_t* fv[2] = {nullptr, nullptr};   // frontiers (local ids), by superstep parity
  uint32_t* bm[2] = {nullptr, nullptr};   // their dedup bitmaps
  uint32_t* skey = nullptr;    // unsorted send list: route word of the target
  uint32_t* sval = nullptr;    //                     and the offered distance
  uint32_t* ctl = nullptr;     // [0..1] frontier counts, [2] send count, [3] status, [4..4+nranks) per-rank counts/cursors
  void* block = nullptr;
  uint32_t parity = 0;
  uint32_t* h_ctl = nullptr;   // pinned mirror
};

namespace gg {
namespace {

constexpr int kPB = 256;
constexpr uint32_t kPartMaxRanks = 256;
constexpr uint32_t kPartMaxLocal = 1u << 24;

__global__ void k_part_init(uint32_t n, uint32_t* dist, uint32_t* bm0, uint32_t* bm1, uint32_t* ctl, uint32_t nctl) {
  const uint32_t nw = (n + 31) / 32;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < max(n, nw); i += gridDim.x * blockDim.x) {
    if (i < n) dist[i] = kInf;
    if (i < nw) {
      bm0[i] = 0u;
      bm1[i] = 0u;
    }
  }
  if (blockIdx.x == 0)
    for (uint32_t i = threadIdx.x; i < nctl; i += blockDim.x) ctl[i] = 0u;
}

__global__ void k_part_seed(uint32_t lv, uint32_t* dist, uint32_t* fv0, uint32_t* bm0, uint32_t* ctl) {
  dist[lv] = 0u;
  fv0[0] = lv;
  bm0[lv >> 5] = 1u << (lv & 31);
  ctl[0] = 1u;
}

// next-frontier candidate v (local): test-and-set in the next bitmap, and
// one append per warp for the lanes that won
__device__ __forceinline__ void part_candidate(bool cand, uint32_t v, uint32_t* bm_next, uint32_t* fv_next,
                                               uint32_t* cnt_next) {
  const unsigned FULL = 0xFFFFFFFFu;
  bool win = false;
  if (cand) {
    const uint32_t bit = 1u << (v & 31);
    win = !(atomicOr(bm_next + (v >> 5), bit) & bit);
  }
  const unsigned b = __ballot_sync(FULL, win);
  if (b) {
    const uint32_t lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(cnt_next, (uint32_t)__popc(b));
    base = __shfl_sync(FULL, base, 0);
    if (win) fv_next[base + __popc(b & ((1u << lane) - 1u))] = v;
  }
}

// One warp per frontier vertex; lanes stride its out-edges.
__global__ void __launch_bounds__(kPB) k_part_advance(gg_part p, uint32_t par) {
  const unsigned FULL = 0xFFFFFFFFu;
  const uint32_t lane = threadIdx.x & 31;
  uint32_t* ctl = p.ctl;
  const uint32_t F = ctl[par];
  const uint32_t* fv = p.fv[par];
  uint32_t* bm_cur = p.bm[par];
  uint32_t* bm_next = p.bm[par ^ 1u];
  uint32_t* fv_next = p.fv[par ^ 1u];
  bool ovf = false;
  const uint32_t nwarps = gridDim.x * (kPB / 32);
  for (uint32_t i = blockIdx.x * (kPB / 32) + (threadIdx.x >> 5); i < F; i += nwarps) {   // warp-uniform
    const uint32_t u = fv[i];
    if (lane == 0) atomicAnd(bm_cur + (u >> 5), ~(1u << (u & 31)));   // consumed: free the bit for later
    const uint32_t du = ld_cg(p.dist + u);
    const uint32_t e0 = p.ro[u], e1 = p.ro[u + 1];
    for (uint32_t eb = e0; eb < e1; eb += 32) {   // warp-uniform
      const uint32_t e = eb + lane;
      bool local_cand = false, remote = false;
      uint32_t lv = 0, rt = 0, nd = 0;
      if (e < e1) {
        const uint32_t v = p.col[e];
        nd = add_sat(du, p.w[e], ovf);
        rt = p.route[v];
        if ((rt >> 24) == p.rank) {
          lv = rt & 0xFFFFFFu;
          if (nd < ld_cg(p.dist + lv)) local_cand = nd < atomicMin(p.dist + lv, nd);
        } else {
          remote = true;
        }
      }
      part_candidate(local_cand, lv, bm_next, fv_next, &ctl[par ^ 1u]);
      const unsigned rb = __ballot_sync(FULL, remote);
      if (rb) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&ctl[2], (uint32_t)__popc(rb));
        base = __shfl_sync(FULL, base, 0);
        if (remote) {
          const uint32_t pos = base + __popc(rb & ((1u << lane) - 1u));
          p.skey[pos] = rt;
          p.sval[pos] = nd;
        }
      }
    }
  }
  if (ovf) atomicOr(&ctl[3], DS_OVERFLOW);
}

// per-destination counts of the send list (shared-memory histogram)
__global__ void k_part_count(gg_part p) {
  __shared__ uint32_t h[kPartMaxRanks];
  for (uint32_t i = threadIdx.x; i < p.nranks; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  const uint32_t S = p.ctl[2];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x)
    atomicAdd(&h[p.skey[i] >> 24], 1u);
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < p.nranks; i += blockDim.x)
    if (h[i]) atomicAdd(&p.ctl[4 + i], h[i]);
}

// scatter into the caller's buffer: pairs (index on the owner, distance),
// destination d's pairs from offs[d] on (ctl[4 + d] holds the cursor)
__global__ void k_part_scatter(gg_part p, const unsigned long long* offs, uint32_t* out) {
  const uint32_t S = p.ctl[2];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x) {
    const uint32_t k = p.skey[i], d = k >> 24;
    const unsigned long long pos = offs[d] + atomicAdd(&p.ctl[4 + d], 1u);
    out[2 * pos] = k & 0xFFFFFFu;
    out[2 * pos + 1] = p.sval[i];
  }
}

// received pairs relaxed like local ones
__global__ void k_part_apply(gg_part p, uint32_t par, const uint32_t* pairs, unsigned long long count) {
  uint32_t* bm_next = p.bm[par ^ 1u];
  uint32_t* fv_next = p.fv[par ^ 1u];
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long rounds = (count + stride - 1) / stride;   // every lane takes part in each round
  for (unsigned long long r = 0; r < rounds; ++r) {
    const unsigned long long i = r * stride + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool cand = false;
    uint32_t lv = 0;
    if (i < count) {
      lv = pairs[2 * i];
      const uint32_t nd = pairs[2 * i + 1];
      if (lv < p.n_local && nd < ld_cg(p.dist + lv)) cand = nd < atomicMin(p.dist + lv, nd);
    }
    part_candidate(cand, lv, bm_next, fv_next, &p.ctl[par ^ 1u]);
  }
}

unsigned grid_of(uint64_t work, unsigned per_block) {
  const uint64_t g = (work + per_block - 1) / per_block;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(g, (uint64_t)device_info().num_sms * 16));
}

}  // namespace
}  // namespace gg

using namespace gg;

extern "C" {

gg_status gg_part_create(uint32_t n_global, uint32_t rank, uint32_t nranks, uint32_t n_local, const uint32_t* route,
                         const uint32_t* row_offsets, const uint32_t* cols, const uint32_t* weights,
                         cudaStream_t stream, gg_part_t* out) {
  NvtxRange nvtx_range("gg_part_create");
  if (!out) return fail(GG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!route || !row_offsets) return fail(GG_ERR_INVALID_ARG, "route/row_offsets is NULL");
  if (nranks == 0 || nranks > kPartMaxRanks || rank >= nranks) return fail(GG_ERR_INVALID_ARG, "rank/nranks out of range");
  if (n_global == 0 || n_local > n_global || n_local > kPartMaxLocal)
    return fail(GG_ERR_INVALID_ARG, "n_local must be <= n_global and <= 2^24");
  const uint64_t m = row_offsets[n_local];
  if (m >= 0xFFFFFFFFull) return fail(GG_ERR_INVALID_ARG, "a part must hold fewer than 2^32 - 1 edges");
  if (m && (!cols || !weights)) return fail(GG_ERR_INVALID_ARG, "cols/weights is NULL");
  // host checks: monotone offsets, columns < n_global, routes consistent with this rank's count
  if (row_offsets[0] != 0) return fail(GG_ERR_INVALID_ARG, "row_offsets[0] must be 0");
  for (uint32_t i = 0; i < n_local; ++i)
    if (row_offsets[i + 1] < row_offsets[i]) return fail(GG_ERR_INVALID_ARG, "row_offsets must be non-decreasing");
  for (uint64_t e = 0; e < m; ++e)
    if (cols[e] >= n_global) return fail(GG_ERR_INVALID_ARG, "a column is >= n_global");
  uint64_t mine = 0;
  for (uint32_t v = 0; v < n_global; ++v) {
    const uint32_t own = route[v] >> 24, li = route[v] & 0xFFFFFFu;
    if (own >= nranks) return fail(GG_ERR_INVALID_ARG, "a route names a rank >= nranks");
    if (own == rank) {
      if (li >= n_local) return fail(GG_ERR_INVALID_ARG, "a route's local index is >= n_local");
      ++mine;
    }
  }
  if (mine != n_local) return fail(GG_ERR_INVALID_ARG, "route assigns a different number of vertices to this rank");
  int device = -1;
  GG_CK(cudaGetDevice(&device));
  gg_part* p = new gg_part();
  p->device = device;
  p->n_global = n_global;
  p->rank = rank;
  p->nranks = nranks;
  p->n_local = n_local;
  p->m_local = m;
  auto r256 = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t nl = std::max<uint32_t>(n_local, 1), ml = std::max<uint64_t>(m, 1), nw = (nl + 31) / 32;
  const size_t total = r256(4ull * n_global) + r256(4 * (nl + 1)) + 2 * r256(4 * ml) + r256(4 * nl) +
                       2 * r256(4 * nl) + 2 * r256(4 * nw) + 2 * r256(4 * ml) + r256(4 * (4 + kPartMaxRanks));
  char* b = nullptr;
  cudaError_t e = cudaMalloc(&b, total);
  if (e != cudaSuccess) { delete p; return cuda_fail(e, "cudaMalloc(part)"); }
  p->block = b;
  size_t off = 0;
  auto take = [&](size_t bytes) { char* q = b + off; off += r256(bytes); return reinterpret_cast<uint32_t*>(q); };
  p->route = take(4ull * n_global);
  p->ro = take(4 * (nl + 1));
  p->col = take(4 * ml);
  p->w = take(4 * ml);
  p->dist = take(4 * nl);
  p->fv[0] = take(4 * nl);
  p->fv[1] = take(4 * nl);
  p->bm[0] = take(4 * nw);
  p->bm[1] = take(4 * nw);
  p->skey = take(4 * ml);
  p->sval = take(4 * ml);
  p->ctl = take(4 * (4 + kPartMaxRanks));
  e = cudaMemcpyAsync(p->route, route, 4ull * n_global, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->ro, row_offsets, 4ull * (n_local + 1), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess && m) e = cudaMemcpyAsync(p->col, cols, 4 * m, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess && m) e = cudaMemcpyAsync(p->w, weights, 4 * m, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMallocHost(&p->h_ctl, 4 * (4 + kPartMaxRanks));
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    if (p->h_ctl) cudaFreeHost(p->h_ctl);
    cudaFree(p->block);
    delete p;
    return cuda_fail(e, "gg_part_create upload");
  }
  *out = p;
  return GG_OK;
}

gg_status gg_part_destroy(gg_part_t p) {
  if (!p) return fail(GG_ERR_INVALID_ARG, "part is NULL");
  cudaDeviceSynchronize();
  if (p->h_ctl) cudaFreeHost(p->h_ctl);
  cudaFree(p->block);
  delete p;
  return GG_OK;
}

gg_status gg_part_info(gg_part_t p, uint32_t* n_local, uint64_t* m_local) {
  if (!p) return fail(GG_ERR_INVALID_ARG, "part is NULL");
  if (n_local) *n_local = p->n_local;
  if (m_local) *m_local = p->m_local;
  return GG_OK;
}

gg_status gg_part_begin(gg_part_t p, uint32_t src_global, cudaStream_t s) {
  NvtxRange nvtx_range("gg_part_begin");
  if (!p) return fail(GG_ERR_INVALID_ARG, "part is NULL");
  if (src_global >= p->n_global) return fail(GG_ERR_INVALID_ARG, "src >= n_global");
  GG_CK(cudaMemcpyAsync(p->h_ctl, p->route + src_global, 4, cudaMemcpyDeviceToHost, s));
  GG_CK(cudaStreamSynchronize(s));
  const uint32_t r = p->h_ctl[0];
  p->parity = 0;
  k_part_init<<<grid_of(std::max<uint64_t>(p->n_local, 1), kPB), kPB, 0, s>>>(p->n_local, p->dist, p->bm[0], p->bm[1],
                                                                                p->ctl, 4 + kPartMaxRanks);
  if ((r >> 24) == p->rank) k_part_seed<<<1, 1, 0, s>>>(r & 0xFFFFFFu, p->dist, p->fv[0], p->bm[0], p->ctl);
  GG_CK(cudaGetLastError());
  return GG_OK;
}

gg_status gg_part_advance(gg_part_t p, cudaStream_t s, uint32_t* send_pairs, uint64_t cap, uint64_t* send_counts) {
  NvtxRange nvtx_range("gg_part_advance");
  if (!p || !send_counts) return fail(GG_ERR_INVALID_ARG, "part/send_counts is NULL");
  if (cap && !send_pairs) return fail(GG_ERR_INVALID_ARG, "cap > 0 with send_pairs NULL");
  const uint32_t par = p->parity;
  // clear this superstep's send count and the per-rank counters
  GG_CK(cudaMemsetAsync(p->ctl + 2, 0, 4, s));
  GG_CK(cudaMemsetAsync(p->ctl + 4, 0, 4ull * p->nranks, s));
  GG_CK(cudaMemcpyAsync(p->h_ctl, p->ctl, 8, cudaMemcpyDeviceToHost, s));
  GG_CK(cudaStreamSynchronize(s));
  const uint32_t F = p->h_ctl[par];
  if (F) k_part_advance<<<grid_of(F, kPB / 32), kPB, 0, s>>>(*p, par);
  GG_CK(cudaGetLastError());
  k_part_count<<<grid_of(std::max<uint64_t>(p->m_local, 1) / 8 + 1, kPB), kPB, 0, s>>>(*p);
  GG_CK(cudaGetLastError());
  GG_CK(cudaMemcpyAsync(p->h_ctl, p->ctl, 4ull * (4 + p->nranks), cudaMemcpyDeviceToHost, s));
  GG_CK(cudaStreamSynchronize(s));
  std::vector<unsigned long long> offs(p->nranks);
  unsigned long long tot = 0;
  for (uint32_t d = 0; d < p->nranks; ++d) {
    send_counts[d] = p->h_ctl[4 + d];
    offs[d] = tot;
    tot += p->h_ctl[4 + d];
  }
  if (tot > cap) return fail(GG_ERR_INVALID_ARG, "send buffer smaller than this superstep's remote updates");
  if (tot) {
    unsigned long long* d_offs = nullptr;
    GG_CK(dev_malloc(&d_offs, 8ull * p->nranks, s));
    GG_CK(cudaMemcpyAsync(d_offs, offs.data(), 8ull * p->nranks, cudaMemcpyHostToDevice, s));
    GG_CK(cudaMemsetAsync(p->ctl + 4, 0, 4ull * p->nranks, s));
    k_part_scatter<<<grid_of(tot, kPB), kPB, 0, s>>>(*p, d_offs, send_pairs);
    GG_CK(cudaGetLastError());
    dev_free(d_offs, s);
    GG_CK(cudaStreamSynchronize(s));
  }
  return GG_OK;
}

gg_status gg_part_apply(gg_part_t p, const uint32_t* recv_pairs, uint64_t count, cudaStream_t s, uint32_t* next_size) {
  NvtxRange nvtx_range("gg_part_apply");
  if (!p || !next_size) return fail(GG_ERR_INVALID_ARG, "part/next_size is NULL");
  if (count && !recv_pairs) return fail(GG_ERR_INVALID_ARG, "count > 0 with recv_pairs NULL");
  const uint32_t par = p->parity;
  if (count) {
    k_part_apply<<<grid_of(count, kPB), kPB, 0, s>>>(*p, par, recv_pairs, count);
    GG_CK(cudaGetLastError());
  }
  // close the superstep: the consumed frontier's count is cleared, parity flips
  GG_CK(cudaMemsetAsync(p->ctl + par, 0, 4, s));
  GG_CK(cudaMemcpyAsync(p->h_ctl, p->ctl, 16, cudaMemcpyDeviceToHost, s));
  GG_CK(cudaStreamSynchronize(s));
  p->parity = par ^ 1u;
  *next_size = p->h_ctl[par ^ 1u];
  if (p->h_ctl[3] & DS_OVERFLOW) return fail(GG_ERR_OVERFLOW, "a finite distance did not fit below 0xFFFFFFFF");
  return GG_OK;
}

gg_status gg_part_distances(gg_part_t p, uint32_t* dist_out, cudaStream_t s) {
  if (!p || !dist_out) return fail(GG_ERR_INVALID_ARG, "part/dist_out is NULL");
  if (p->n_local) GG_CK(cudaMemcpyAsync(dist_out, p->dist, 4ull * p->n_local, cudaMemcpyDeviceToDevice, s));
  return GG_OK;
}

}  // extern "C"
