// gg_noalloc.cu -- gg_sssp_noalloc: single-source shortest paths that
// allocate no device memory at all.
//
// Who needs it: a caller whose device memory already belongs to someone
// else's allocator (for example a framework whose caching allocator has
// reserved nearly all of the GPU, so a fresh cudaMalloc fails or fragments
// the pool), or a caller that cannot afford the implicit device-wide
// synchronisation cudaFree performs (a latency-sensitive loop sharing the GPU
// with other streams).  gg_sssp needs a graph handle, and building one copies
// the CSR and allocates per-graph frontier buffers; this entry point instead
// reads the caller's device CSR in place and keeps its frontier in one
// fixed-size array compiled into the library.
//
// The scratch array: g_noalloc_scratch, a file-scope __device__ array of
// kNoallocScratchBytes (about 24.3 MiB: sparse frontier ping-pong buffers,
// two dedup bitmaps and a control block for up to GG_NOALLOC_MAX_VERTICES
// vertices).  Every GPU on which the library's module is loaded holds it until
// the process exits.  All calls share it and it keeps the previous call's
// contents, so every call clears the parts that must start at zero, and two
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race on it: the caller must order them.
//
// Its host-side name is only a stand-in for the device array, so host code
// never passes it to a kernel directly: on the first call on each device,
// with that device current, cudaGetSymbolAddress resolves the device address
// once and it is cached per device.  Make that first call outside any stream
// capture.
//
// The kernel is a variant of the merge-path push superstep of gg_bsp.cu
// (advance relaxing every frontier out-edge with atomicMin, fused with the
// bitmap-dedup filter that appends improved vertices with their edge-prefix
// coordinates) that reads the caller's separate col_indices / weights arrays
// and runs push-only, launched superstep by superstep from the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "gg_host.h"
#include "gg_nvtx.h"

namespace gg {
namespace {

constexpr uint32_t kNaMaxN = GG_NOALLOC_MAX_VERTICES;
constexpr uint32_t kNaWords = (kNaMaxN + 31) / 32;
constexpr int kNaBlock = 256;
constexpr int kNaEpt = 4;
constexpr int kNaTile = kNaBlock * kNaEpt;
constexpr int kNaCap = kNaTile + 1;

struct NaCtl {
  unsigned long long cnt[2];   // (count << 32) | edge total of the frontier being built, by parity
  uint32_t iter;
  uint32_t done_ctas;
  uint32_t status;             // DS_* bits
  uint32_t running;
  uint32_t bad_csr;            // structural check result
};

constexpr size_t kCtlBytes = 256;
constexpr size_t kArrBytes = sizeof(uint32_t) * (size_t)kNaMaxN;
constexpr size_t kBmBytes = sizeof(uint32_t) * (size_t)kNaWords;
constexpr size_t kNoallocScratchBytes = kCtlBytes + 6 * kArrBytes + 2 * kBmBytes;
static_assert(sizeof(NaCtl) <= kCtlBytes, "control block");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

struct NaArgs {
  uint32_t n, m;
  const uint32_t* ro;
  const uint32_t* col;
  const uint32_t* w;
  uint32_t* dist;
  NaCtl* ctl;
  uint32_t* fv[2];
  uint32_t* fr[2];
  uint32_t* fs[2];
  uint32_t* bm[2];
};

NaArgs make_args(unsigned char* base, uint32_t n, uint32_t m, const uint32_t* ro, const uint32_t* col,
                 const uint32_t* w, uint32_t* dist) {
  NaArgs a;
  a.n = n;
  a.m = m;
  a.ro = ro;
  a.col = col;
  a.w = w;
  a.dist = dist;
  a.ctl = reinterpret_cast<NaCtl*>(base);
  unsigned char* p = base + kCtlBytes;
  for (int i = 0; i < 2; ++i) {
    a.fv[i] = reinterpret_cast<uint32_t*>(p); p += kArrBytes;
    a.fr[i] = reinterpret_cast<uint32_t*>(p); p += kArrBytes;
    a.fs[i] = reinterpret_cast<uint32_t*>(p); p += kArrBytes;
  }
  for (int i = 0; i < 2; ++i) {
    a.bm[i] = reinterpret_cast<uint32_t*>(p); p += kBmBytes;
  }
  return a;
}

// Structural check of the caller's CSR (offsets monotone from 0 to m, columns < n).
__global__ void k_na_validate(NaArgs a) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (uint64_t i = t; i < a.n; i += stride)
    if (a.ro[i + 1] < a.ro[i]) atomicOr(&a.ctl->bad_csr, 1u);
  for (uint64_t e = t; e < a.m; e += stride)
    if (a.col[e] >= a.n) atomicOr(&a.ctl->bad_csr, 2u);
  if (t == 0 && (a.ro[0] != 0 || a.ro[a.n] != a.m)) atomicOr(&a.ctl->bad_csr, 4u);
}

__global__ void k_na_clear_flag(NaArgs a) { a.ctl->bad_csr = 0u; }

// dist := INF; both bitmaps := 0 (the scratch keeps the last call's bits).
__global__ void k_na_init(NaArgs a) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (uint64_t i = t; i < a.n; i += stride) a.dist[i] = kInf;
  const uint32_t nw = (a.n + 31) / 32;
  for (uint64_t i = t; i < nw; i += stride) {
    a.bm[0][i] = 0u;
    a.bm[1][i] = 0u;
  }
}

__global__ void k_na_seed(NaArgs a, uint32_t src) {
  NaCtl* c = a.ctl;
  a.dist[src] = 0u;
  const uint32_t rs = a.ro[src], re = a.ro[src + 1];
  c->cnt[1] = 0ull;
  c->iter = 0;
  c->done_ctas = 0;
  c->status = 0;
  if (re > rs) {
    a.fv[0][0] = src;
    a.fr[0][0] = rs;
    a.fs[0][0] = 0u;
    a.bm[0][src >> 5] = 1u << (src & 31);
    c->cnt[0] = (1ull << 32) | (re - rs);
    c->running = 1u;
  } else {
    c->cnt[0] = 0ull;
    c->running = 0u;
  }
}

struct NaSmem {
  uint32_t es[kNaCap], eb[kNaCap], ec[kNaCap];
  uint32_t qv[kNaCap], qr[kNaCap], qd[kNaCap];
  uint32_t wsum[kNaBlock / 32];
  uint32_t qn, j, last, ovf;
  unsigned long long base;
};

__device__ __forceinline__ void na_candidate(NaSmem& sm, const NaArgs& a, uint32_t* bm_next, uint32_t v) {
  const uint32_t rs = __ldg(a.ro + v), re = __ldg(a.ro + v + 1);
  if (re > rs) {
    const uint32_t bit = 1u << (v & 31);
    if (!(atomicOr(bm_next + (v >> 5), bit) & bit)) {
      const uint32_t q = atomicAdd(&sm.qn, 1u);
      sm.qv[q] = v;
      sm.qr[q] = rs;
      sm.qd[q] = re - rs;
    }
  }
}

__device__ __forceinline__ void na_flush(NaSmem& sm, unsigned long long* cnt_next, uint32_t* fv, uint32_t* fr,
                                         uint32_t* fs) {
  __syncthreads();
  const uint32_t qn = sm.qn;
  if (qn == 0) return;
  const uint32_t tot = block_scan_excl<kNaBlock>(sm.qd, qn, sm.wsum);
  if (threadIdx.x == 0) sm.base = atomicAdd(cnt_next, ((unsigned long long)qn << 32) | tot);
  __syncthreads();
  const uint32_t pos0 = (uint32_t)(sm.base >> 32), eb0 = (uint32_t)sm.base;
  for (uint32_t i = threadIdx.x; i < qn; i += kNaBlock) {
    fv[pos0 + i] = sm.qv[i];
    fr[pos0 + i] = sm.qr[i];
    fs[pos0 + i] = eb0 + sm.qd[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) sm.qn = 0;
  __syncthreads();
}

// One push superstep over the caller's CSR (merge-path equal edge ranges per
// CTA, fused dedup filter); the last CTA closes the superstep.
__global__ void __launch_bounds__(kNaBlock) k_na_superstep(NaArgs a) {
  __shared__ NaSmem sm;
  NaCtl* ctl = a.ctl;
  const uint32_t it = ctl->iter, p = it & 1u;
  const unsigned long long c = ctl->cnt[p];
  const uint32_t F = (uint32_t)(c >> 32), E = (uint32_t)c;
  uint32_t* bm_cur = a.bm[p];
  uint32_t* bm_next = a.bm[p ^ 1u];
  const uint32_t* S = a.fs[p];
  const uint32_t tid = threadIdx.x;
  if (tid == 0) { sm.qn = 0; sm.ovf = 0; }
  __syncthreads();
  bool ovf = false;
  const uint32_t e0 = (uint32_t)(((unsigned long long)blockIdx.x * E) / gridDim.x);
  const uint32_t e1 = (uint32_t)(((unsigned long long)(blockIdx.x + 1) * E) / gridDim.x);
  if (F > 0 && e0 < e1) {
    if (tid < 32) {
      const uint32_t j = warp_search_le(S, F, e0);
      if (tid == 0) sm.j = j;
    }
    __syncthreads();
    uint32_t j = sm.j;
    for (uint32_t t0 = e0; t0 < e1; t0 += kNaTile) {
      const uint32_t t1 = min(t0 + (uint32_t)kNaTile, e1);
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
          const uint32_t v = a.fv[p][idx];
          sm.es[nent + tid] = s;
          sm.eb[nent + tid] = a.fr[p][idx];
          sm.ec[nent + tid] = ld_cg(a.dist + v);
          bm_cur[v >> 5] = 0u;
        }
        const int cnt = __syncthreads_count(valid);
        nent += (uint32_t)cnt;
        if (cnt < kNaBlock) break;
      }
      uint32_t dst[kNaEpt], nd[kNaEpt];
      bool ok[kNaEpt];
#pragma unroll
      for (int k = 0; k < kNaEpt; ++k) {
        const uint32_t g = t0 + k * kNaBlock + tid;
        ok[k] = g < t1;
        if (ok[k]) {
          const uint32_t jj = smem_upper_bound_minus1(sm.es, nent, g);
          const uint32_t e = sm.eb[jj] + (g - sm.es[jj]);
          dst[k] = __ldg(a.col + e);
          nd[k] = add_sat(sm.ec[jj], __ldg(a.w + e), ovf);
        }
      }
#pragma unroll
      for (int k = 0; k < kNaEpt; ++k) {
        if (ok[k] && nd[k] < ld_cg(a.dist + dst[k])) {
          const uint32_t old = atomicMin(a.dist + dst[k], nd[k]);
          if (nd[k] < old) na_candidate(sm, a, bm_next, dst[k]);
        }
      }
      na_flush(sm, &ctl->cnt[p ^ 1u], a.fv[p ^ 1u], a.fr[p ^ 1u], a.fs[p ^ 1u]);
      j = j + nent - 1;
    }
  }
  if (ovf) sm.ovf = 1u;
  __syncthreads();
  if (tid == 0) {
    if (sm.ovf) atomicOr(&ctl->status, DS_OVERFLOW);
    sm.last = arrive_last(&ctl->done_ctas, gridDim.x) ? 1u : 0u;
  }
  __syncthreads();
  if (sm.last && tid == 0) {
    const unsigned long long cn = atomicAdd(&ctl->cnt[p ^ 1u], 0ull);
    ctl->cnt[p] = 0ull;
    ctl->done_ctas = 0u;
    ctl->iter = it + 1;
    ctl->running = (cn >> 32) != 0 ? 1u : 0u;
  }
}

std::mutex g_na_mu;
unsigned char* g_na_ptr[64] = {};
int g_na_grid[64] = {};

// Once per device, with that device current: resolve the array's device
// address and the persistent grid size.
gg_status na_setup(int dev, unsigned char** base, int* grid) {
  if (dev < 0 || dev >= 64) return fail(GG_ERR_NOT_SUPPORTED, "device index out of range for gg_sssp_noalloc");
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_na_superstep, kNaBlock, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    g_na_grid[dev] = std::max(1, per_sm) * sms;
    g_na_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *base = g_na_ptr[dev];
  *grid = g_na_grid[dev];
  return GG_OK;
}

}  // namespace
}  // namespace gg

using namespace gg;

extern "C" gg_status gg_sssp_noalloc(uint32_t n, uint64_t m, const uint32_t* row_offsets,
                                     const uint32_t* col_indices, const uint32_t* weights, uint32_t src,
                                     uint32_t* dist_out, cudaStream_t stream) {
  NvtxRange nvtx_range("gg_sssp_noalloc");
  if (n == 0) return fail(GG_ERR_INVALID_ARG, "n must be >= 1");
  if (n > kNaMaxN)
    return fail(GG_ERR_INVALID_ARG, "gg_sssp_noalloc: n exceeds GG_NOALLOC_MAX_VERTICES (1048576); "
                                    "use gg_graph_create_csr + gg_sssp for larger graphs");
  if (m >= 0xFFFFFFFFull) return fail(GG_ERR_INVALID_ARG, "m must be < 2^32 - 1");
  if (!row_offsets || !dist_out) return fail(GG_ERR_INVALID_ARG, "row_offsets/dist_out is NULL");
  if (m > 0 && (!col_indices || !weights)) return fail(GG_ERR_INVALID_ARG, "col_indices/weights is NULL");
  if (src >= n) return fail(GG_ERR_INVALID_ARG, "src >= n");
  int dev = 0;
  GG_CK(cudaGetDevice(&dev));
  unsigned char* base = nullptr;
  int grid = 0;
  gg_status st = na_setup(dev, &base, &grid);
  if (st != GG_OK) return st;
  NaArgs a = make_args(base, n, (uint32_t)m, row_offsets, col_indices, weights, dist_out);
  const unsigned ib = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(((uint64_t)std::max<uint64_t>(n, m) + 255) / 256,
                                                                        (uint64_t)grid));
  // structural check of the caller's CSR
  k_na_clear_flag<<<1, 1, 0, stream>>>(a);
  k_na_validate<<<ib, 256, 0, stream>>>(a);
  GG_CK(cudaGetLastError());
  uint32_t bad = 0;
  GG_CK(cudaMemcpyAsync(&bad, &a.ctl->bad_csr, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
  GG_CK(cudaStreamSynchronize(stream));
  if (bad & 4u) return fail(GG_ERR_INVALID_ARG, "row_offsets must start at 0 and end at m");
  if (bad & 1u) return fail(GG_ERR_INVALID_ARG, "row_offsets must be non-decreasing");
  if (bad & 2u) return fail(GG_ERR_INVALID_ARG, "col_indices must be < n");
  k_na_init<<<ib, 256, 0, stream>>>(a);
  k_na_seed<<<1, 1, 0, stream>>>(a, src);
  GG_CK(cudaGetLastError());
  // supersteps, launched in growing batches between checks of the frontier size
  uint32_t running = 1, launched = 0, batch = 1;
  const uint64_t cap = (uint64_t)n + 2;
  while (running) {
    for (uint32_t k = 0; k < batch; ++k) k_na_superstep<<<grid, kNaBlock, 0, stream>>>(a);
    GG_CK(cudaGetLastError());
    launched += batch;
    GG_CK(cudaMemcpyAsync(&running, &a.ctl->running, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
    GG_CK(cudaStreamSynchronize(stream));
    if (running && launched > cap) return fail(GG_ERR_INTERNAL, "superstep cap reached before the frontier emptied");
    batch = std::min<uint32_t>(batch * 2, 64);
  }
  uint32_t status = 0;
  GG_CK(cudaMemcpyAsync(&status, &a.ctl->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
  GG_CK(cudaStreamSynchronize(stream));
  if (status & DS_OVERFLOW) return fail(GG_ERR_OVERFLOW, "a finite distance did not fit below 0xFFFFFFFF");
  return GG_OK;
}
