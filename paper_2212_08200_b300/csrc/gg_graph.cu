// gg_graph.cu -- graph handle construction (Sec. IV-A, Listing 1 of the paper:
// a CSR queried through a graph API; the "Push vs. Pull" box: keep the
// transposed representation beside it for pull traversals).
//
// Device preprocessing, run once per handle (not part of an SSSP run):
//   check      one pass: offsets start at 0, never decrease, end at m; every
//              column < n; the largest weight (decides the edge encoding)
//   encode     col/weight arrays -> packed (col << wbits) | weight words, or
//              interleaved uint2 {col, weight} when they do not fit
//   transpose  CSC by counting sort (only for graphs not declared symmetric)
//   pull list  vertices with a non-empty CSC row, with the row start
#include <cuda_runtime.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "gg_host.h"

#ifndef GG_LH_K
#define GG_LH_K 2.7   // light edges per vertex aimed at by the default light/heavy bucket width
#endif

namespace gg {

namespace {

constexpr int SCAN_BLOCK = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

// One pass over the uploaded CSR: structural checks (offsets start at 0,
// never decrease, end at m; every column < n) when validate is set, and the
// largest weight.  out[0]: error bits, out[1]: largest weight (bit pattern).
__global__ void k_check(uint32_t n, uint32_t m, const uint32_t* __restrict__ ro, const uint32_t* __restrict__ col,
                        const uint32_t* __restrict__ w, uint32_t validate, uint32_t* __restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t err = 0, mx = 0;
  if (validate) {
    for (uint64_t i = t; i < n; i += stride)
      if (ro[i + 1] < ro[i]) err |= 1u;
    if (t == 0 && (ro[0] != 0 || ro[n] != m)) err |= 4u;
  }
  for (uint64_t e = t; e < m; e += stride) {
    if (validate && col[e] >= n) err |= 2u;
    mx = max(mx, w[e]);
  }
  for (int o = 16; o; o >>= 1) {
    mx = max(mx, __shfl_down_sync(0xFFFFFFFFu, mx, o));
    err |= __shfl_down_sync(0xFFFFFFFFu, err, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (err) atomicOr(out, err);
    atomicMax(out + 1, mx);
  }
}

// {col, w} arrays -> the handle's edge encoding: (col << wbits) | w when PK,
// else interleaved uint2 {col, w}
template <bool PK>
__global__ void k_encode(uint32_t m, const uint32_t* __restrict__ col, const uint32_t* __restrict__ w,
                         uint32_t wbits, void* __restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    if (PK) static_cast<uint32_t*>(out)[e] = (col[e] << wbits) | w[e];
    else static_cast<uint2*>(out)[e] = make_uint2(col[e], w[e]);
  }
}

__global__ void k_count_cols(uint32_t m, const uint32_t* __restrict__ col, uint32_t* __restrict__ cnt) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) atomicAdd(&cnt[col[e]], 1u);
}

// warp per source row: every edge u->v into v's CSC row as u (with its
// weight), in the handle's edge encoding
template <bool PK>
__global__ void k_transpose(uint32_t n, const uint32_t* __restrict__ ro, const uint32_t* __restrict__ col,
                            const uint32_t* __restrict__ w, uint32_t wbits, uint32_t* __restrict__ cursor,
                            void* __restrict__ out) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t u = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
    for (uint32_t e = ro[u] + lane; e < ro[u + 1]; e += 32) {
      const uint32_t pos = atomicAdd(&cursor[col[e]], 1u);
      if (PK) static_cast<uint32_t*>(out)[pos] = ((uint32_t)u << wbits) | w[e];
      else static_cast<uint2*>(out)[pos] = make_uint2((uint32_t)u, w[e]);
    }
  }
}

// per-tile sums of a u32 array
__global__ void k_scan_reduce(const uint32_t* __restrict__ in, uint64_t count, uint32_t* __restrict__ sums) {
  __shared__ uint32_t ws[SCAN_BLOCK / 32];
  const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
  uint32_t s = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const uint64_t i = base + (uint64_t)k * SCAN_BLOCK + threadIdx.x;
    if (i < count) s += in[i];
  }
  for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int i = 0; i < SCAN_BLOCK / 32; ++i) t += ws[i];
    sums[blockIdx.x] = t;
  }
}

// exclusive scan of one tile (in place), plus the tile offset
__global__ void k_scan_tile(uint32_t* __restrict__ data, uint64_t count, const uint32_t* __restrict__ offs) {
  __shared__ uint32_t buf[SCAN_TILE];
  __shared__ uint32_t ws[SCAN_BLOCK / 32];
  const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
  const uint64_t rem = count - base;
  const uint32_t valid = rem < (uint64_t)SCAN_TILE ? (uint32_t)rem : (uint32_t)SCAN_TILE;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const uint32_t i = k * SCAN_BLOCK + threadIdx.x;
    buf[i] = i < valid ? data[base + i] : 0u;
  }
  __syncthreads();
  block_scan_excl<SCAN_BLOCK>(buf, valid, ws);
  const uint32_t off = offs ? offs[blockIdx.x] : 0u;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const uint32_t i = k * SCAN_BLOCK + threadIdx.x;
    if (i < valid) data[base + i] = buf[i] + off;
  }
}

// exclusive scan in place (recursive over tile sums)
gg_status scan_excl(uint32_t* data, uint64_t count, cudaStream_t s) {
  if (count == 0) return GG_OK;
  const uint64_t tiles = (count + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles == 1) {
    k_scan_tile<<<1, SCAN_BLOCK, 0, s>>>(data, count, nullptr);
    GG_CK(cudaGetLastError());
    return GG_OK;
  }
  uint32_t* sums = nullptr;
  GG_CK(dev_malloc(&sums, tiles * sizeof(uint32_t), s));
  k_scan_reduce<<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(data, count, sums);
  GG_CK(cudaGetLastError());
  gg_status st = scan_excl(sums, tiles, s);
  if (st != GG_OK) { dev_free(sums, s); return st; }
  k_scan_tile<<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(data, count, sums);
  GG_CK(cudaGetLastError());
  dev_free(sums, s);
  return GG_OK;
}

__global__ void k_nonempty_flags(uint32_t n, const uint32_t* __restrict__ t_ro, uint32_t* __restrict__ flag) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    flag[v] = t_ro[v + 1] > t_ro[v] ? 1u : 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) flag[n] = 0;
}

// sinks: reachable vertices (non-empty CSC row) without out-edges
__global__ void k_find_sinks(uint32_t n, const uint32_t* __restrict__ ro, const uint32_t* __restrict__ t_ro,
                             uint32_t* __restrict__ flag) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    if (t_ro[v + 1] > t_ro[v] && ro[v + 1] == ro[v]) *flag = 1u;
}

__global__ void k_pull_list(uint32_t n, const uint32_t* __restrict__ t_ro, const uint32_t* __restrict__ pos,
                            uint32_t* __restrict__ pv, uint32_t* __restrict__ ps) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    if (t_ro[v + 1] > t_ro[v]) {
      pv[pos[v]] = (uint32_t)v;
      ps[pos[v]] = t_ro[v];
    }
  }
}

// Light/heavy partition of every row (bucket width delta): flag[e] = 1 when
// edge e is light (weight < delta); flag[m] = 0 closes the scan.
template <bool PK>
__global__ void k_lh_flags(uint32_t m, const void* __restrict__ edges, uint32_t wbits, uint32_t delta,
                           uint32_t* __restrict__ flag) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    const uint32_t w = PK ? (static_cast<const uint32_t*>(edges)[e] & ((1u << wbits) - 1u))
                          : static_cast<const uint2*>(edges)[e].y;
    flag[e] = w < delta ? 1u : 0u;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) flag[m] = 0u;
}

// lend[v] = ro[v] + (light edges of row v), from the exclusive scan L of the flags
__global__ void k_lh_lend(uint32_t n, const uint32_t* __restrict__ ro, const uint32_t* __restrict__ L,
                          uint32_t* __restrict__ lend) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    lend[v] = ro[v] + (L[ro[v + 1]] - L[ro[v]]);
}

// cnt[ro[v]] += 1 for every vertex whose row starts before m: after an
// exclusive scan X of cnt (m + 1 entries), edge e lies in row X[e + 1] - 1
// (the last vertex whose row starts at or before e)
__global__ void k_row_starts(uint32_t n, uint32_t m, const uint32_t* __restrict__ ro, uint32_t* __restrict__ cnt) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    if (ro[v] < m) atomicAdd(&cnt[ro[v]], 1u);
}

// thread per edge: light edges to the front of their row in their original
// order, heavy edges after them in theirs
template <bool PK>
__global__ void k_lh_scatter(uint32_t m, const uint32_t* __restrict__ ro, const uint32_t* __restrict__ X,
                             const void* __restrict__ edges, const uint32_t* __restrict__ L,
                             const uint32_t* __restrict__ lend, uint32_t wbits, uint32_t delta,
                             void* __restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    const uint32_t u = X[e + 1] - 1u;
    const uint32_t r0 = __ldg(ro + u);
    const uint32_t before = L[e] - __ldg(L + r0);   // light edges of the row before e
    const uint32_t le = __ldg(lend + u);
    if (PK) {
      const uint32_t x = static_cast<const uint32_t*>(edges)[e];
      const uint32_t d = (x & ((1u << wbits) - 1u)) < delta ? r0 + before : le + ((uint32_t)e - r0 - before);
      static_cast<uint32_t*>(out)[d] = x;
    } else {
      const uint2 x = static_cast<const uint2*>(edges)[e];
      const uint32_t d = x.y < delta ? r0 + before : le + ((uint32_t)e - r0 - before);
      static_cast<uint2*>(out)[d] = x;
    }
  }
}

unsigned grid_for(uint64_t work) {
  const DeviceInfo di = device_info();
  uint64_t b = (work + 255) / 256;
  const uint64_t cap = (uint64_t)di.num_sms * 8;
  if (b > cap) b = cap;
  if (b == 0) b = 1;
  return (unsigned)b;
}

}  // namespace

gg_status graph_build(gg_graph* g, uint32_t n, uint64_t m64, const uint32_t* ro_in, const uint32_t* col_in,
                      const uint32_t* w_in, uint32_t flags, cudaStream_t s) {
  const bool dev = (flags & GG_DEVICE_PTRS) != 0;
  const bool validate = (flags & GG_NO_VALIDATE) == 0;
  const uint32_t m = (uint32_t)m64;
  g->n = n;
  g->m = m;
  g->symmetric = (flags & GG_SYMMETRIC) != 0;
  g->float_weights = (flags & GG_FLOAT_WEIGHTS) != 0;
  // cheap host-side check first; monotonicity and column range are checked on
  // the device after the upload (k_check)
  if (!dev && validate && (ro_in[0] != 0 || ro_in[n] != m))
    return fail(GG_ERR_INVALID_ARG, "row_offsets must start at 0 and end at m");
  GG_CK(cudaGetDevice(&g->device));

  GG_CK(dev_malloc(&g->ro, sizeof(uint32_t) * ((size_t)n + 1), s));
  g->bytes = sizeof(uint32_t) * ((size_t)n + 1);
  GG_CK(cudaMemcpyAsync(g->ro, ro_in, sizeof(uint32_t) * ((size_t)n + 1),
                        dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  // packed 4-byte edges when the column bits of n - 1 and the bits of the
  // largest weight fit in one word
  uint32_t colbits = 1;
  while (colbits < 32 && ((uint64_t)(n - 1) >> colbits) != 0) ++colbits;
  const uint32_t wbits = 32 - colbits;
  bool pack = false;
  uint32_t wmax = 0;
  if (m > 0) {
    const uint32_t* dcol = col_in;
    const uint32_t* dw = w_in;
    uint32_t* tmp = nullptr;
    if (!dev) {
      GG_CK(dev_malloc(&tmp, sizeof(uint32_t) * 2 * (size_t)m, s));
      GG_CK(cudaMemcpyAsync(tmp, col_in, sizeof(uint32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
      GG_CK(cudaMemcpyAsync(tmp + m, w_in, sizeof(uint32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
      dcol = tmp;
      dw = tmp + m;
    }
    // checks and the largest weight in one pass, one read-back
    uint32_t* chk = nullptr;
    GG_CK(dev_malloc(&chk, 2 * sizeof(uint32_t), s));
    GG_CK(cudaMemsetAsync(chk, 0, 2 * sizeof(uint32_t), s));
    k_check<<<grid_for(std::max<uint64_t>(n, m)), 256, 0, s>>>(n, m, g->ro, dcol, dw, validate ? 1u : 0u, chk);
    GG_CK(cudaGetLastError());
    uint32_t h[2] = {0, 0};
    GG_CK(cudaMemcpyAsync(h, chk, sizeof(h), cudaMemcpyDeviceToHost, s));
    dev_free(chk, s);
    GG_CK(cudaStreamSynchronize(s));
    wmax = h[1];
    const char* bad = (h[0] & 4u)   ? "row_offsets must start at 0 and end at m"
                      : (h[0] & 1u) ? "row_offsets must be non-decreasing"
                      : (h[0] & 2u) ? "col_indices must be < n"
                      // binary32 weights must be finite and >= +0: as bit patterns, every
                      // such value is below +inf's 0x7F800000 and every other one (negative,
                      // -0, inf, NaN) is not, so the largest pattern decides
                      : (validate && (flags & GG_FLOAT_WEIGHTS) && wmax >= 0x7F800000u)
                          ? "binary32 weights must be finite and >= +0.0"
                          : nullptr;
    if (bad) {
      if (tmp) dev_free(tmp, s);
      return fail(GG_ERR_INVALID_ARG, bad);
    }
    pack = !(flags & GG_NO_PACK) && colbits < 32 && (uint64_t)wmax < (1ull << wbits);
    const size_t esz = pack ? sizeof(uint32_t) : sizeof(uint2);
    void* enc = nullptr;
    GG_CK(dev_malloc(&enc, esz * (size_t)m, s));
    g->bytes += esz * (size_t)m;
    if (pack) {
      g->edges4 = static_cast<uint32_t*>(enc);
      k_encode<true><<<grid_for(m), 256, 0, s>>>(m, dcol, dw, wbits, enc);
    } else {
      g->edges = static_cast<uint2*>(enc);
      k_encode<false><<<grid_for(m), 256, 0, s>>>(m, dcol, dw, wbits, enc);
    }
    GG_CK(cudaGetLastError());
    // transpose (CSC) for pull, built from the uploaded arrays
    if (!g->symmetric) {
      GG_CK(dev_malloc(&g->t_ro, sizeof(uint32_t) * ((size_t)n + 1), s));
      void* tenc = nullptr;
      GG_CK(dev_malloc(&tenc, esz * (size_t)m, s));
      g->bytes += sizeof(uint32_t) * ((size_t)n + 1) + esz * (size_t)m;
      if (pack) g->t_edges4 = static_cast<uint32_t*>(tenc);
      else g->t_edges = static_cast<uint2*>(tenc);
      GG_CK(cudaMemsetAsync(g->t_ro, 0, sizeof(uint32_t) * ((size_t)n + 1), s));
      k_count_cols<<<grid_for(m), 256, 0, s>>>(m, dcol, g->t_ro);
      GG_CK(cudaGetLastError());
      gg_status st = scan_excl(g->t_ro, (uint64_t)n + 1, s);
      if (st != GG_OK) { if (tmp) dev_free(tmp, s); return st; }
      uint32_t* cursor = nullptr;
      GG_CK(dev_malloc(&cursor, sizeof(uint32_t) * ((size_t)n + 1), s));
      GG_CK(cudaMemcpyAsync(cursor, g->t_ro, sizeof(uint32_t) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, s));
      if (pack) k_transpose<true><<<grid_for((uint64_t)n * 32), 256, 0, s>>>(n, g->ro, dcol, dw, wbits, cursor, tenc);
      else k_transpose<false><<<grid_for((uint64_t)n * 32), 256, 0, s>>>(n, g->ro, dcol, dw, wbits, cursor, tenc);
      GG_CK(cudaGetLastError());
      dev_free(cursor, s);
    } else {
      g->t_ro = g->ro;
      g->t_edges = g->edges;
      g->t_edges4 = g->edges4;
    }
    if (tmp) dev_free(tmp, s);
  } else {
    if (dev && validate) {
      uint32_t h[2] = {0, 0};
      GG_CK(cudaMemcpyAsync(h, g->ro, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
      GG_CK(cudaMemcpyAsync(h + 1, g->ro + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
      GG_CK(cudaStreamSynchronize(s));
      if (h[0] != 0 || h[1] != 0) return fail(GG_ERR_INVALID_ARG, "row_offsets must start at 0 and end at m");
    }
    GG_CK(dev_malloc(&g->edges, sizeof(uint2), s));   // a placeholder: no edge is ever read
    g->bytes += sizeof(uint2);
    if (g->symmetric) {
      g->t_ro = g->ro;
      g->t_edges = g->edges;
    } else {
      GG_CK(dev_malloc(&g->t_ro, sizeof(uint32_t) * ((size_t)n + 1), s));
      GG_CK(cudaMemsetAsync(g->t_ro, 0, sizeof(uint32_t) * ((size_t)n + 1), s));
      g->t_edges = g->edges;
      g->bytes += sizeof(uint32_t) * ((size_t)n + 1);
    }
  }

  // pull entry list: vertices with a non-empty CSC row
  {
    uint32_t* pos = nullptr;
    GG_CK(dev_malloc(&pos, sizeof(uint32_t) * ((size_t)n + 1), s));
    k_nonempty_flags<<<grid_for(n), 256, 0, s>>>(n, g->t_ro, pos);
    GG_CK(cudaGetLastError());
    gg_status st = scan_excl(pos, (uint64_t)n + 1, s);
    if (st != GG_OK) return st;
    // sized for every vertex, so that no read-back of the count has to come first
    GG_CK(dev_malloc(&g->pv, sizeof(uint32_t) * std::max<size_t>(n, 1), s));
    GG_CK(dev_malloc(&g->ps, sizeof(uint32_t) * std::max<size_t>(n, 1), s));
    g->bytes += 2 * sizeof(uint32_t) * std::max<size_t>(n, 1);
    k_pull_list<<<grid_for(n), 256, 0, s>>>(n, g->t_ro, pos, g->pv, g->ps);
    GG_CK(cudaGetLastError());
    uint32_t h[2] = {0, 0};   // vertices with in-edges; sinks
    GG_CK(cudaMemcpyAsync(&h[0], pos + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    if (!g->symmetric) {   // a symmetric graph's reachable vertices all have out-edges
      GG_CK(cudaMemsetAsync(pos + n, 0, sizeof(uint32_t), s));
      k_find_sinks<<<grid_for(n), 256, 0, s>>>(n, g->ro, g->t_ro, pos + n);
      GG_CK(cudaGetLastError());
      GG_CK(cudaMemcpyAsync(&h[1], pos + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    }
    dev_free(pos, s);
    GG_CK(cudaStreamSynchronize(s));
    g->dg.np = h[0];
    g->dg.sinks = h[1];
  }

  g->dg.packed = pack ? 1u : 0u;
  g->dg.wbits = wbits;
  // default near-far bucket width (measured on B300, see the autotuner for
  // per-graph choices): low-degree, high-diameter graphs (grids) use buckets
  // of 16 maximum edge weights, which cut Bellman-Ford re-relaxation from
  // ~200x to ~4x the edge count; on skewed, low-diameter graphs (mean degree
  // >= 8, e.g. RMAT) the extra supersteps cost more than the saved edges, so
  // they run the plain frontier loop
  g->wmax = wmax;
  {
    const double davg = g->dg.np ? (double)m / (double)g->dg.np : 1.0;
    const double d = (double)std::max<uint32_t>(wmax, 1) * 16.0;
    g->default_delta = (davg >= 8.0 || !m) ? GG_DELTA_NONE : (uint32_t)std::min(d, 4.0e9);
    g->low_degree = davg < 8.0;
    // light/heavy buckets (single-source bulk-synchronous loop only) on the
    // same skewed graphs: width ~ GG_LH_K * wmax / mean degree, so that a
    // vertex has about GG_LH_K light edges
    g->default_delta_lh = GG_DELTA_NONE;
    if (davg >= 8.0 && m && !g->float_weights && wmax >= 2) {
      const double dl = std::max(1.0, std::floor((double)wmax * GG_LH_K / davg));
      g->default_delta_lh = (uint32_t)std::min<double>(dl, (double)wmax);
    }
  }
  g->dg.n = n;
  g->dg.m = m;
  g->dg.nwords = (n + 31) / 32;
  g->dg.ro = g->ro;
  g->dg.edges = pack ? static_cast<const void*>(g->edges4) : static_cast<const void*>(g->edges);
  g->dg.t_ro = g->t_ro;
  g->dg.t_edges = pack ? static_cast<const void*>(g->t_edges4) : static_cast<const void*>(g->t_edges);
  g->dg.pv = g->pv;
  g->dg.ps = g->ps;
  return GG_OK;
}

gg_status lh_prepare(gg_graph* g, uint32_t delta, cudaStream_t s) {
  if (g->lh_block && g->lh_delta == delta) return GG_OK;
  const size_t n = g->n, m = g->m;
  const bool pk = g->dg.packed != 0;
  const size_t esz = pk ? sizeof(uint32_t) : sizeof(uint2);
  auto r256 = [](size_t b) { return (b + 255) & ~size_t(255); };
  if (!g->lh_block) {
    const size_t nw = (n + 31) / 32;
    const size_t vb = sizeof(uint32_t) * std::max<size_t>(n, 1);
    const size_t total = r256(esz * std::max<size_t>(m, 1)) + 7 * r256(vb) + 2 * r256(sizeof(uint32_t) * nw);
    char* p = nullptr;
    GG_CK(dev_malloc(&p, total, s));
    size_t off = 0;
    auto take = [&](size_t b) { char* q = p + off; off += r256(b); return q; };
    g->lhb.edges = take(esz * std::max<size_t>(m, 1));
    g->lhb.lend = reinterpret_cast<const uint32_t*>(take(vb));
    for (int i = 0; i < 2; ++i) {
      g->lhb.rv[i] = reinterpret_cast<uint32_t*>(take(vb));
      g->lhb.rr[i] = reinterpret_cast<uint32_t*>(take(vb));
      g->lhb.rs[i] = reinterpret_cast<uint32_t*>(take(vb));
    }
    for (int i = 0; i < 2; ++i) g->lhb.bm_r[i] = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * nw));
    if (off != total) {
      dev_free(p, s);
      return fail(GG_ERR_INTERNAL, "light/heavy buffer layout");
    }
    g->lh_block = p;
    g->lh_bytes = total;
  }
  g->lh_delta = 0;   // invalid until the partition below is complete
  uint32_t* L = nullptr;
  GG_CK(dev_malloc(&L, sizeof(uint32_t) * (m + 1), s));
  if (pk) k_lh_flags<true><<<grid_for(m), 256, 0, s>>>((uint32_t)m, g->dg.edges, g->dg.wbits, delta, L);
  else k_lh_flags<false><<<grid_for(m), 256, 0, s>>>((uint32_t)m, g->dg.edges, g->dg.wbits, delta, L);
  GG_CK(cudaGetLastError());
  gg_status st = scan_excl(L, (uint64_t)m + 1, s);
  if (st != GG_OK) { dev_free(L, s); return st; }
  uint32_t nlight = 0;
  GG_CK(cudaMemcpyAsync(&nlight, L + m, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  uint32_t* lend = const_cast<uint32_t*>(g->lhb.lend);
  k_lh_lend<<<grid_for(n), 256, 0, s>>>((uint32_t)n, g->ro, L, lend);
  GG_CK(cudaGetLastError());
  if (m) {
    uint32_t* X = nullptr;
    GG_CK(dev_malloc(&X, sizeof(uint32_t) * (m + 1), s));
    GG_CK(cudaMemsetAsync(X, 0, sizeof(uint32_t) * (m + 1), s));
    k_row_starts<<<grid_for(n), 256, 0, s>>>((uint32_t)n, (uint32_t)m, g->ro, X);
    GG_CK(cudaGetLastError());
    st = scan_excl(X, (uint64_t)m + 1, s);
    if (st != GG_OK) { dev_free(X, s); dev_free(L, s); return st; }
    void* out = const_cast<void*>(g->lhb.edges);
    if (pk) k_lh_scatter<true><<<grid_for(m), 256, 0, s>>>((uint32_t)m, g->ro, X, g->dg.edges, L, lend,
                                                            g->dg.wbits, delta, out);
    else k_lh_scatter<false><<<grid_for(m), 256, 0, s>>>((uint32_t)m, g->ro, X, g->dg.edges, L, lend,
                                                          g->dg.wbits, delta, out);
    GG_CK(cudaGetLastError());
    dev_free(X, s);
  }
  dev_free(L, s);
  GG_CK(cudaStreamSynchronize(s));
  g->lh_heavy_total = m - nlight;
  g->lh_delta = delta;
  return GG_OK;
}

// Callers have synchronised the handle's work: the frees go on the legacy stream.
void graph_free(gg_graph* g) {
  dev_free(g->lh_block, 0);
  g->lh_block = nullptr;
  g->lh_delta = 0;
  if (g->t_ro && g->t_ro != g->ro) dev_free(g->t_ro, 0);
  if (g->t_edges && g->t_edges != g->edges) dev_free(g->t_edges, 0);
  if (g->t_edges4 && g->t_edges4 != g->edges4) dev_free(g->t_edges4, 0);
  dev_free(g->edges4, 0);
  g->edges4 = g->t_edges4 = nullptr;
  dev_free(g->ro, 0);
  dev_free(g->edges, 0);
  dev_free(g->pv, 0);
  dev_free(g->ps, 0);
  g->ro = g->t_ro = g->pv = g->ps = nullptr;
  g->edges = g->t_edges = nullptr;
}

}  // namespace gg
