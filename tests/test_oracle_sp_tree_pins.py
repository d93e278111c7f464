"""Pins the oracle's edge-frontier program (oracle.sp_tree) to facts other
than itself (no GPU needed).

The program (Sec. III-C: an operator over a frontier of edges) takes a
distance vector from src and returns the tight edges, those (u, v, w) with
dist[u] finite and dist[u] + w == dist[v], and for each vertex the smallest
u among its tight in-edges (the source is its own parent).

* brute force: on tiny graphs with positive weights, the tight edges are
  exactly the edges that appear on some minimum-weight simple path from the
  source, found by enumerating every simple path;
* a hand-worked fixture (tests/golden/hand_directed7.txt, worked below) and
  hand cases for zero weights around the source and between unreached
  vertices;
* planted mistakes: mutated copies of oracle.c must fail these pins.
"""
import os
import re
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import graphgen
import oracle
from golden_io import load

INF = oracle.INF


def enumerate_tight(ro, col, w, src):
    """(parent, tight) from every simple path out of src (positive weights)."""
    n = ro.shape[0] - 1
    best = [None] * n
    paths = []   # (length, edge ids) of every simple path from src

    def dfs(u, length, edges, seen):
        paths.append((length, list(edges)))
        for e in range(int(ro[u]), int(ro[u + 1])):
            v = int(col[e])
            if v in seen:
                continue
            seen.add(v)
            edges.append(e)
            dfs(v, length + int(w[e]), edges, seen)
            edges.pop()
            seen.remove(v)

    dfs(src, 0, [], {src})
    end = {}
    for length, edges in paths:
        v = int(col[edges[-1]]) if edges else src
        end.setdefault(v, []).append((length, edges))
        best[v] = length if best[v] is None else min(best[v], length)
    tight = np.zeros(int(ro[-1]), bool)
    for v, lst in end.items():
        for length, edges in lst:
            if length == best[v]:
                tight[edges] = True
    rows = np.repeat(np.arange(n), np.diff(ro.astype(np.int64)))
    parent = np.full(n, INF, np.uint32)
    parent[src] = src
    for e in np.flatnonzero(tight):
        v = int(col[e])
        if v != src:
            parent[v] = min(parent[v], rows[e])
    return parent, tight


@pytest.mark.parametrize("seed", range(25))
def test_tight_edges_equal_simple_path_enumeration(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(rng.integers(2, 8))
    ro, col, w = graphgen.random_graph(n, int(rng.integers(1, 16)), 6, seed, wmin=1)
    src = int(rng.integers(0, n))
    dist = oracle.dijkstra(ro, col, w, src)
    parent, tight = oracle.sp_tree(ro, col, w, src, dist)
    ep, et = enumerate_tight(ro, col, w, src)
    np.testing.assert_array_equal(tight, et)
    np.testing.assert_array_equal(parent, ep)


def test_hand_worked_fixture():
    """hand_directed7: d = 0 2 1 3 6 6 INF.  Worked by hand, edge by edge in
    CSR order (rows sorted by source, stable): 0->1 w4 (0+4 != 2), 0->2 w1
    (tight), 0->1 w2 (tight), 1->3 w1 (tight), 1->1 w3 (self-loop, no),
    2->1 w2 (1+2 != 2), 2->3 w5 (no), 3->4 w3 (tight), 4->5 w0 (tight),
    5->3 w1 (7 != 3), 6->0 w1 (6 unreached).  Parents: 1 <- 0, 2 <- 0,
    3 <- 1, 4 <- 3, 5 <- 4, 6 none."""
    g = load("hand_directed7.txt")
    ro, col, w = g["ro"], g["col"], g["w"]
    dist = oracle.dijkstra(ro, col, w, g["src"])
    parent, tight = oracle.sp_tree(ro, col, w, g["src"], dist)
    rows = np.repeat(np.arange(g["n"]), np.diff(ro.astype(np.int64)))
    got = sorted((int(rows[e]), int(col[e]), int(w[e])) for e in np.flatnonzero(tight))
    assert got == sorted([(0, 2, 1), (0, 1, 2), (1, 3, 1), (3, 4, 3), (4, 5, 0)])
    assert parent.tolist() == [0, 0, 0, 1, 3, 4, INF]


def test_zero_weights_at_the_source_and_between_unreached_vertices():
    """Source 2; 2 -> 0 (0), 0 -> 2 (0), 0 -> 1 (3); 3 -> 4 (0) is unreached.
    CSR order: 0->2, 0->1, 2->0, 3->4.  The edge 0 -> 2 is tight (0 + 0 == 0)
    but the source keeps itself as parent (vertex 0 has the smaller id); the
    unreached zero-weight edge is not tight (dist[3] is not finite)."""
    ro, col, w = graphgen.from_edges(5, [2, 0, 0, 3], [0, 2, 1, 4], [0, 0, 3, 0])
    dist = oracle.dijkstra(ro, col, w, 2)
    assert dist.tolist() == [0, 3, 0, INF, INF]
    parent, tight = oracle.sp_tree(ro, col, w, 2, dist)
    assert tight.tolist() == [True, True, True, False]
    assert parent.tolist() == [2, 0, 2, INF, INF]


# --- planted mistakes: each mutated copy of oracle.c must fail a pin ---------
MUTATIONS = {
    "weight dropped": ("(uint64_t)dist[u] + weights[e] == (uint64_t)dist[v];", "(uint64_t)dist[u] == (uint64_t)dist[v];"),
    "largest parent": ("if (t && v != src && u < parent[v]) parent[v] = u;",
                       "if (t && v != src && (parent[v] == OR_INF32 || u > parent[v])) parent[v] = u;"),
    "source takes a parent": ("if (t && v != src && u < parent[v])", "if (t && u < parent[v])"),
    "unreached edges": ("const int t = dist[u] != OR_INF32 && ", "const int t = "),
    "transposed test": ("(uint64_t)dist[u] + weights[e] == (uint64_t)dist[v];",
                        "(uint64_t)dist[v] + weights[e] == (uint64_t)dist[u];"),
}


def _tree_pins_pass(lib_path):
    import ctypes
    lib = ctypes.CDLL(lib_path)
    P = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_sp_tree.restype = ctypes.c_int
    lib.oracle_sp_tree.argtypes = [ctypes.c_uint32, P, P, P, ctypes.c_uint32, P, P, ctypes.POINTER(ctypes.c_ubyte)]

    def tree(ro, col, w, src, dist):
        n = ro.shape[0] - 1
        parent = np.empty(n, np.uint32)
        tight = np.zeros(max(col.shape[0], 1), np.uint8)
        c2 = col if col.shape[0] else np.zeros(1, np.uint32)
        w2 = w if w.shape[0] else np.zeros(1, np.uint32)
        lib.oracle_sp_tree(n, ro.ctypes.data_as(P), c2.ctypes.data_as(P), w2.ctypes.data_as(P), src,
                           dist.ctypes.data_as(P), parent.ctypes.data_as(P),
                           tight.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
        return parent, tight[:col.shape[0]].astype(bool)

    for seed in range(25):
        rng = np.random.Generator(np.random.PCG64(seed))
        n = int(rng.integers(2, 8))
        ro, col, w = graphgen.random_graph(n, int(rng.integers(1, 16)), 6, seed, wmin=1)
        src = int(rng.integers(0, n))
        p, t = tree(ro, col, w, src, oracle.dijkstra(ro, col, w, src))
        ep, et = enumerate_tight(ro, col, w, src)
        if not (np.array_equal(p, ep) and np.array_equal(t, et)):
            return False
    ro, col, w = graphgen.from_edges(5, [2, 0, 0, 3], [0, 2, 1, 4], [0, 0, 3, 0])
    p, t = tree(ro, col, w, 2, oracle.dijkstra(ro, col, w, 2))
    if t.tolist() != [True, True, True, False] or p.tolist() != [2, 0, 2, INF, INF]:
        return False
    g = load("hand_directed7.txt")
    p, _ = tree(g["ro"], g["col"], g["w"], g["src"], oracle.dijkstra(g["ro"], g["col"], g["w"], g["src"]))
    return p.tolist() == [0, 0, 0, 1, 3, 4, INF]


def test_planted_mistakes_are_caught():
    src = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")
    text = open(src).read()
    tmp = tempfile.mkdtemp(prefix="oracle_tree_mut_")
    try:
        clean = os.path.join(tmp, "clean.so")
        subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-pthread", "-o", clean, src])
        assert _tree_pins_pass(clean)
        for label, (old, new) in MUTATIONS.items():
            assert text.count(old) == 1, f"mutation anchor missing: {label}"
            cpath = os.path.join(tmp, re.sub(r"\W", "_", label) + ".c")
            with open(cpath, "w") as f:
                f.write(text.replace(old, new, 1))
            so = cpath[:-2] + ".so"
            subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-pthread", "-o", so, cpath])
            assert not _tree_pins_pass(so), f"planted mistake not caught: {label}"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
