"""Seeded synthetic graph inputs for the frontier SSSP path.

This package builds inputs only (CSR arrays, uint32 weights, source choices).
It contains no shortest-path arithmetic, so the CPU oracle and the CUDA
library can both be fed from it while sharing no method code.

Graphs are returned as ``(row_offsets, col_indices, weights)`` numpy uint32
arrays (CSR, rows sorted by destination id).

Workload recipes (the graph shapes the SSSP hot path is measured on):

* ``grid(side, W, seed)``: 2D 4-neighbour undirected grid, vertex id
  ``y*side + x``, one weight per unordered pair, uniform in ``[1, W]``.
* ``rmat(scale, ef, a, b, c, seed, W)``: RMAT graph with ``ef * 2**scale``
  edge draws, seeded vertex relabelling, symmetrised, self-loops and
  duplicates removed, pair weights uniform in ``[1, W]``.
* ``serving_pool()``: the 32-graph pool (RMAT scales 12-20 and grids
  64^2-2048^2) used for the query-serving workload.

All random numbers come from counter-based splitmix64 (Steele, Lea and
Flood, 2014), so every output is a pure function of its arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "libgraphgen.so")
_lib = None
_lock = threading.Lock()

U32 = np.uint32
INF = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile graphgen.c into libgraphgen.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-march=x86-64-v2", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER(ctypes.c_uint32)
            lib.ggen_splitmix64.restype = ctypes.c_uint64
            lib.ggen_splitmix64.argtypes = [ctypes.c_uint64]
            lib.ggen_pair_weight.restype = ctypes.c_uint32
            lib.ggen_pair_weight.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
            lib.ggen_grid_num_edges.restype = ctypes.c_uint64
            lib.ggen_grid_num_edges.argtypes = [ctypes.c_uint32]
            lib.ggen_grid.restype = ctypes.c_int
            lib.ggen_grid.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, P, P, P]
            lib.ggen_rmat.restype = ctypes.c_void_p
            lib.ggen_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64]
            lib.ggen_csr_n.restype = ctypes.c_uint32
            lib.ggen_csr_n.argtypes = [ctypes.c_void_p]
            lib.ggen_csr_m.restype = ctypes.c_uint64
            lib.ggen_csr_m.argtypes = [ctypes.c_void_p]
            lib.ggen_csr_export.restype = None
            lib.ggen_csr_export.argtypes = [ctypes.c_void_p, P, P, P]
            lib.ggen_csr_free.restype = None
            lib.ggen_csr_free.argtypes = [ctypes.c_void_p]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.uint32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def splitmix64(x: int) -> int:
    return int(_load().ggen_splitmix64(ctypes.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def pair_weight(seed: int, u: int, v: int, W: int) -> int:
    return int(_load().ggen_pair_weight(seed, u, v, W))


def grid(side: int, W: int = 64, seed: int = 1, const_w: int = 0):
    """side x side 4-neighbour grid.  W == 0 gives unit weights; const_w > 0
    gives every edge that weight; otherwise pair weights uniform in [1, W]."""
    lib = _load()
    n = side * side
    m = int(lib.ggen_grid_num_edges(side))
    ro = np.empty(n + 1, U32)
    col = np.empty(max(m, 1), U32)
    w = np.empty(max(m, 1), U32)
    rc = lib.ggen_grid(side, W, const_w, seed, _p(ro), _p(col), _p(w))
    if rc != 0:
        raise ValueError("grid side must be >= 1")
    return ro, col[:m], w[:m]


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, W: int = 255, wseed: int | None = None):
    """Symmetrised, deduplicated RMAT graph without self-loops."""
    lib = _load()
    h = lib.ggen_rmat(scale, edge_factor, a, b, c, seed, W, seed if wseed is None else wseed)
    if not h:
        raise MemoryError("rmat generation failed")
    try:
        n = int(lib.ggen_csr_n(h))
        m = int(lib.ggen_csr_m(h))
        ro = np.empty(n + 1, U32)
        col = np.empty(max(m, 1), U32)
        w = np.empty(max(m, 1), U32)
        lib.ggen_csr_export(h, _p(ro), _p(col), _p(w))
    finally:
        lib.ggen_csr_free(h)
    return ro, col[:m], w[:m]


def from_edges(n: int, src, dst, w):
    """CSR from an edge list (kept in order within each row after a stable
    sort by source).  Multi-edges and self-loops are kept."""
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    w = np.asarray(w, np.int64)
    order = np.argsort(src, kind="stable")
    ro = np.zeros(n + 1, np.int64)
    np.add.at(ro, src + 1, 1)
    ro = np.cumsum(ro)
    return ro.astype(U32), dst[order].astype(U32), w[order].astype(U32)


def random_graph(n: int, m: int, W: int, seed: int, symmetric: bool = False, wmin: int = 1):
    """Small random graph: m edge draws, endpoints uniform (self-loops and
    multi-edges possible), weights uniform in [wmin, W].  For tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = rng.integers(0, n, m)
    d = rng.integers(0, n, m)
    w = rng.integers(wmin, W + 1, m)
    if symmetric:
        s, d, w = np.concatenate([s, d]), np.concatenate([d, s]), np.concatenate([w, w])
    return from_edges(n, s, d, w)


def path_graph(n: int, weights):
    """Directed path 0 -> 1 -> ... -> n-1 with the given n-1 weights."""
    weights = np.asarray(weights, np.int64)
    return from_edges(n, np.arange(n - 1), np.arange(1, n), weights)


def star_graph(n: int, weights):
    """Hub 0 with edges to and from every leaf 1..n-1 (leaf i weight w[i-1])."""
    weights = np.asarray(weights, np.int64)
    leaves = np.arange(1, n)
    return from_edges(n, np.concatenate([np.zeros(n - 1, np.int64), leaves]),
                      np.concatenate([leaves, np.zeros(n - 1, np.int64)]),
                      np.concatenate([weights, weights]))


def degrees(ro: np.ndarray) -> np.ndarray:
    return np.diff(ro.astype(np.int64))


def max_degree_vertex(ro: np.ndarray) -> int:
    """Vertex of maximum out-degree; ties go to the lowest id."""
    return int(np.argmax(degrees(ro)))


def sample_sources(ro: np.ndarray, k: int, seed: int = 1) -> np.ndarray:
    """k distinct vertices of out-degree >= 1, drawn by splitmix64(seed, i)."""
    deg = degrees(ro)
    n = deg.shape[0]
    if int((deg > 0).sum()) < k:
        raise ValueError("not enough vertices with out-degree >= 1")
    out, seen, i = [], set(), 0
    base = splitmix64(seed ^ 0x50C0FFEE)
    while len(out) < k:
        v = splitmix64((base + i) & 0xFFFFFFFFFFFFFFFF) % n
        i += 1
        if deg[v] > 0 and v not in seen:
            seen.add(v)
            out.append(v)
    return np.asarray(out, U32)


def serving_pool_spec():
    """The 32-graph pool of the serving workload.

    Graphs 0..15: RMAT scale 12 + (i mod 9), edge factor 8 for even i, 16 for
    odd i.  Graphs 16..31: grids of side 64 * 2**((i-16) mod 6).  Seeds
    1000 + i, weights uniform in [1, 255]."""
    spec = []
    for i in range(32):
        if i < 16:
            spec.append(("rmat", 12 + (i % 9), 8 if i % 2 == 0 else 16, 1000 + i))
        else:
            spec.append(("grid", 64 * 2 ** ((i - 16) % 6), 0, 1000 + i))
    return spec


def build_pool_graph(entry):
    kind, a, b, seed = entry
    if kind == "rmat":
        return rmat(a, b, seed=seed, W=255)
    return grid(a, W=255, seed=seed)


def poisson_queries(pool_degrees, count: int = 2000, seed: int = 1, rate_qps: float | None = None):
    """(graph index, source, arrival time in s) for `count` queries: graph
    uniform over the pool, source uniform among that graph's vertices of
    out-degree >= 1, exponential inter-arrival times (all at t=0 when
    rate_qps is None, i.e. the saturation workload)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    G = len(pool_degrees)
    gids = rng.integers(0, G, count)
    srcs = np.empty(count, np.uint32)
    cand = [np.flatnonzero(d > 0) for d in pool_degrees]
    for q in range(count):
        c = cand[gids[q]]
        srcs[q] = c[rng.integers(0, c.shape[0])]
    if rate_qps is None:
        t = np.zeros(count)
    else:
        t = np.cumsum(rng.exponential(1.0 / rate_qps, count))
    return gids.astype(np.int64), srcs, t


def grid_source(side: int, x: int = 0, y: int = 0) -> int:
    return y * side + x


WORKLOADS = {
    # name: (description, builder, source chooser)
    "grid64": "64x64 grid, weights U[1,64] seed 1, source 0",
    "rmat20": "RMAT scale 20 EF16 (0.57,0.19,0.19,0.05) symmetrised, U[1,255], source = max-degree vertex",
    "grid4096": "4096x4096 grid, weights U[1,1000] seed 1, source (0,0)",
    "rmat22": "RMAT scale 22 EF16 same params, U[1,255]; 64 seeded sources / max-degree single source",
}


def workload(name: str):
    """(row_offsets, cols, weights, source) for a named workload."""
    if name == "grid64":
        ro, col, w = grid(64, 64, 1)
        return ro, col, w, 0
    if name == "rmat20":
        ro, col, w = rmat(20, 16, seed=1, W=255)
        return ro, col, w, max_degree_vertex(ro)
    if name == "grid4096":
        ro, col, w = grid(4096, 1000, 1)
        return ro, col, w, 0
    if name == "rmat22":
        ro, col, w = rmat(22, 16, seed=1, W=255)
        return ro, col, w, max_degree_vertex(ro)
    if name.startswith("rmat") and name[4:].isdigit():
        s = int(name[4:])
        ro, col, w = rmat(s, 16, seed=1, W=255)
        return ro, col, w, max_degree_vertex(ro)
    if name.startswith("grid") and name[4:].isdigit():
        side = int(name[4:])
        ro, col, w = grid(side, 1000 if side >= 1024 else 64, 1)
        return ro, col, w, 0
    raise KeyError(name)
