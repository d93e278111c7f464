"""CPU oracle for single-source shortest paths -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this package.  The CUDA
library never calls it, and it shares no code with that library.

What it computes (the paper's parallel SSSP, Listing 4, driven by the
``neighbors_expand`` operator of Listing 3): the least fixed point of the
relaxation ``d[v] = min(d[v], d[u] + w(u, v))`` from ``d[source] = 0``,
which for non-negative weights is the shortest-path distance

    dist[v] = min over directed paths source ~> v of sum of weights,

with 0xFFFFFFFF for unreachable vertices.  It is computed by binary-heap
Dijkstra (``dijkstra``), and pinned against independent algorithms and
closed forms in ``tests/test_oracle_pins.py``: Floyd-Warshall brute force
(``floyd_warshall``), BFS hop counts for unit weights (``bfs_hops``),
Bellman-Ford rounds (``bellman_ford``), grid/path/star closed forms and the
shortest-path invariants (``check``).  ``sp_tree`` is the edge-frontier
program on a distance vector: the tight edges and the smallest tight
predecessor of each vertex.

The paper's own float variant is ``dijkstra_f32`` (and ``bellman_ford_f32``):
binary32 weights, one rounded single-precision addition per relaxation,
unreached = FLT_MAX as in the paper's initialisation; results are the
distances' bit patterns.

Readings of the paper used by the uint32 functions:

* distances are uint32, accumulated in uint64 inside the oracle, and
  0xFFFFFFFF means unreachable; a finite distance that does not fit is an
  error (``RangeError``);
* self-loops, zero weights and multi-edges are allowed (the minimum wins).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

INF = 0xFFFFFFFF
INF64 = 0xFFFFFFFFFFFFFFFF


class RangeError(ArithmeticError):
    """A finite shortest distance does not fit in uint32 below 0xFFFFFFFF."""


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc -O2, pthreads)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER(ctypes.c_uint32)
            P64 = ctypes.POINTER(ctypes.c_uint64)
            u32 = ctypes.c_uint32
            lib.oracle_dijkstra.restype = ctypes.c_int
            lib.oracle_dijkstra.argtypes = [u32, P, P, P, u32, P, P64]
            lib.oracle_floyd_warshall.restype = ctypes.c_int
            lib.oracle_floyd_warshall.argtypes = [u32, P, P, P, P64]
            lib.oracle_bellman_ford.restype = ctypes.c_int
            lib.oracle_bellman_ford.argtypes = [u32, P, P, P, u32, P, P]
            lib.oracle_bfs_hops.restype = ctypes.c_int
            lib.oracle_bfs_hops.argtypes = [u32, P, P, u32, P]
            lib.oracle_check.restype = ctypes.c_int
            lib.oracle_check.argtypes = [u32, P, P, P, u32, P, P]
            lib.oracle_dijkstra_f32.restype = ctypes.c_int
            lib.oracle_dijkstra_f32.argtypes = [u32, P, P, P, u32, P]
            lib.oracle_bellman_ford_f32.restype = ctypes.c_int
            lib.oracle_bellman_ford_f32.argtypes = [u32, P, P, P, u32, P, P]
            lib.oracle_sp_tree.restype = ctypes.c_int
            lib.oracle_sp_tree.argtypes = [u32, P, P, P, u32, P, P, ctypes.POINTER(ctypes.c_ubyte)]
            lib.oracle_dijkstra_many.restype = ctypes.c_int
            lib.oracle_dijkstra_many.argtypes = [u32, P, P, P, P, u32, P, u32]
            _lib = lib
    return _lib


def _u32(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return a


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _graph(ro, col, w):
    ro, col, w = _u32(ro), _u32(col), _u32(w)
    n = ro.shape[0] - 1
    if col.shape[0] == 0:           # keep a valid pointer for empty graphs
        col = np.zeros(1, np.uint32)
        w = np.zeros(1, np.uint32)
    return n, ro, col, w


def _rc(rc: int):
    if rc == 1:
        raise ValueError("invalid argument")
    if rc == 2:
        raise RangeError("a finite distance does not fit in uint32")
    if rc == 3:
        raise MemoryError("oracle allocation failed")


def dijkstra(ro, col, w, src: int, return_scanned: bool = False):
    """Shortest-path distances from src (uint32, INF = unreachable)."""
    n, ro, col, w = _graph(ro, col, w)
    dist = np.empty(n, np.uint32)
    scanned = ctypes.c_uint64(0)
    _rc(_load().oracle_dijkstra(n, _p(ro), _p(col), _p(w), src, _p(dist), ctypes.byref(scanned)))
    return (dist, int(scanned.value)) if return_scanned else dist


def dijkstra_many(ro, col, w, srcs, threads: int = 1) -> np.ndarray:
    """Distances from each source, shape (k, n); one Dijkstra per source,
    spread over `threads` host threads."""
    n, ro, col, w = _graph(ro, col, w)
    srcs = _u32(srcs)
    k = srcs.shape[0]
    out = np.empty((k, n), np.uint32)
    _rc(_load().oracle_dijkstra_many(n, _p(ro), _p(col), _p(w), _p(srcs), k, _p(out), threads))
    return out


def floyd_warshall(ro, col, w) -> np.ndarray:
    """All-pairs distances (uint64 n x n, INF64 = unreachable)."""
    n, ro, col, w = _graph(ro, col, w)
    D = np.empty((n, n), np.uint64)
    _rc(_load().oracle_floyd_warshall(n, _p(ro), _p(col), _p(w),
                                      D.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
    return D


def bellman_ford(ro, col, w, src: int):
    """(distances, number of productive rounds) by Bellman-Ford rounds."""
    n, ro, col, w = _graph(ro, col, w)
    dist = np.empty(n, np.uint32)
    rounds = ctypes.c_uint32(0)
    _rc(_load().oracle_bellman_ford(n, _p(ro), _p(col), _p(w), src, _p(dist), ctypes.byref(rounds)))
    return dist, int(rounds.value)


FLT_MAX_BITS = 0x7F7FFFFF   # "unreached" for binary32 distances (the paper's initial FLT_MAX)


def _f32_bits(w) -> np.ndarray:
    w = np.asarray(w)
    return np.ascontiguousarray(w.view(np.uint32) if w.dtype == np.float32 else w, dtype=np.uint32)


def dijkstra_f32(ro, col, w, src: int) -> np.ndarray:
    """The paper's float variant: binary32 weights (float32 array or its
    uint32 bit patterns), one rounded float addition per relaxation; returns
    the distances' bit patterns (uint32; FLT_MAX_BITS = unreached)."""
    n, ro, col, wb = _graph(ro, col, _f32_bits(w))
    dist = np.empty(n, np.uint32)
    _rc(_load().oracle_dijkstra_f32(n, _p(ro), _p(col), _p(wb), src, _p(dist)))
    return dist


def bellman_ford_f32(ro, col, w, src: int):
    """(distance bit patterns, productive rounds) by Bellman-Ford rounds over binary32."""
    n, ro, col, wb = _graph(ro, col, _f32_bits(w))
    dist = np.empty(n, np.uint32)
    rounds = ctypes.c_uint32(0)
    _rc(_load().oracle_bellman_ford_f32(n, _p(ro), _p(col), _p(wb), src, _p(dist), ctypes.byref(rounds)))
    return dist, int(rounds.value)


def bfs_hops(ro, col, src: int) -> np.ndarray:
    n, ro, col, _ = _graph(ro, col, np.zeros_like(np.asarray(col, np.uint32)))
    hops = np.empty(n, np.uint32)
    _rc(_load().oracle_bfs_hops(n, _p(ro), _p(col), src, _p(hops)))
    return hops


CHECK_CODES = {
    0: "ok",
    1: "dist[src] != 0",
    2: "an edge violates dist[v] <= dist[u] + w",
    3: "a reachable vertex has no tight in-edge",
    4: "finite/infinite pattern differs from reachability",
}


def check(ro, col, w, src: int, dist):
    """(code, bad_vertex) of the shortest-path invariants; code 0 = ok."""
    n, ro, col, w = _graph(ro, col, w)
    dist = _u32(dist)
    bad = ctypes.c_uint32(0)
    rc = _load().oracle_check(n, _p(ro), _p(col), _p(w), src, _p(dist), ctypes.byref(bad))
    return int(rc), int(bad.value)


def sp_tree(ro, col, w, src: int, dist):
    """The edge-frontier program on a distance vector: (parent, tight) with
    tight a bool per edge (dist[u] + w == dist[v], dist[u] finite) and
    parent[v] the smallest u over v's tight in-edges (parent[src] = src,
    INF when there is none)."""
    n, ro, col, w = _graph(ro, col, w)
    dist = _u32(dist)
    parent = np.empty(n, np.uint32)
    tight = np.zeros(max(col.shape[0], 1), np.uint8)
    _rc(_load().oracle_sp_tree(n, _p(ro), _p(col), _p(w), src, _p(dist), _p(parent),
                               tight.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))))
    m = int(ro[-1])
    return parent, tight[:m].astype(bool)


def traversed_edges(ro, dist) -> int:
    """m_trav: sum of out-degrees over vertices with finite distance (each
    edge of the reached component counted once)."""
    ro = np.asarray(ro, np.int64)
    reach = np.asarray(dist) != INF
    return int((ro[1:] - ro[:-1])[reach].sum())
