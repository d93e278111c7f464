"""Pins the CPU oracle to facts other than itself (no GPU needed).

The oracle computes shortest-path distances, the fixed point reached by the
paper's frontier loop (Listing 4 with the expand operator of Listing 3).
Each test checks it against something independent:

* brute force: Floyd-Warshall min-plus closure on graphs of <= 64 vertices;
* the unit-weight special case: BFS hop counts;
* closed forms: uniform-weight grids (c * Manhattan distance), paths
  (prefix sums), stars;
* a different algorithm: Bellman-Ford rounds;
* hand-worked fixtures in tests/golden/;
* the shortest-path invariants (and that corrupted vectors violate them);
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
from golden_io import hand_fixtures, load

INF = oracle.INF


def fw_row(ro, col, w, src):
    D = oracle.floyd_warshall(ro, col, w)
    row = D[src]
    return np.where(row == oracle.INF64, INF, row).astype(np.uint32)


CASES = [
    # (n, m, W, symmetric, wmin)
    (1, 0, 5, False, 1),
    (2, 1, 5, False, 1),
    (8, 12, 9, False, 0),
    (16, 40, 20, False, 1),
    (33, 64, 100, True, 1),
    (64, 150, 255, False, 0),
    (64, 400, 3, True, 0),
    (64, 80, 1000, False, 1),
]


@pytest.mark.parametrize("case", CASES)
def test_dijkstra_matches_floyd_warshall(case):
    n, m, W, sym, wmin = case
    for seed in range(60):
        ro, col, w = graphgen.random_graph(n, m, W, seed, symmetric=sym, wmin=wmin)
        D = oracle.floyd_warshall(ro, col, w)
        for src in {0, n // 2, n - 1}:
            d = oracle.dijkstra(ro, col, w, src)
            expect = np.where(D[src] == oracle.INF64, INF, D[src]).astype(np.uint32)
            np.testing.assert_array_equal(d, expect, err_msg=f"seed={seed} src={src} case={case}")


def test_floyd_warshall_itself_small_closed_form():
    # Floyd-Warshall is the brute-force pin; check it on a 3-vertex case by hand:
    # 0->1 (5), 1->2 (2), 0->2 (9): d(0,2) = 7; nothing reaches 0 from 1 or 2.
    ro, col, w = graphgen.from_edges(3, [0, 1, 0], [1, 2, 2], [5, 2, 9])
    D = oracle.floyd_warshall(ro, col, w)
    assert D[0].tolist() == [0, 5, 7]
    assert D[1].tolist() == [oracle.INF64, 0, 2]
    assert D[2].tolist() == [oracle.INF64, oracle.INF64, 0]


@pytest.mark.parametrize("seed", range(5))
def test_unit_weights_equal_bfs_hops(seed):
    ro, col, _ = graphgen.random_graph(500, 1500, 1, seed)
    w = np.ones_like(col)
    for src in (0, 17, 499):
        np.testing.assert_array_equal(oracle.dijkstra(ro, col, w, src), oracle.bfs_hops(ro, col, src))
    ro, col, _ = graphgen.rmat(12, 8, seed=seed + 7, W=1)
    w = np.ones_like(col)
    src = graphgen.max_degree_vertex(ro)
    np.testing.assert_array_equal(oracle.dijkstra(ro, col, w, src), oracle.bfs_hops(ro, col, src))


@pytest.mark.parametrize("side,c", [(1, 3), (2, 1), (7, 5), (40, 3), (64, 1)])
def test_uniform_grid_manhattan_closed_form(side, c):
    ro, col, w = graphgen.grid(side, const_w=c)
    assert np.all(w == c)
    ys, xs = np.divmod(np.arange(side * side), side)
    for (x0, y0) in {(0, 0), (side - 1, side // 2), (side // 3, side - 1)}:
        src = y0 * side + x0
        expect = (c * (np.abs(xs - x0) + np.abs(ys - y0))).astype(np.uint32)
        np.testing.assert_array_equal(oracle.dijkstra(ro, col, w, src), expect)


def test_path_prefix_sums_and_star():
    rng = np.random.Generator(np.random.PCG64(3))
    wts = rng.integers(0, 1000, 99)
    ro, col, w = graphgen.path_graph(100, wts)
    d = oracle.dijkstra(ro, col, w, 0)
    np.testing.assert_array_equal(d, np.concatenate([[0], np.cumsum(wts)]).astype(np.uint32))
    d = oracle.dijkstra(ro, col, w, 50)             # directed path: nothing behind 50
    assert np.all(d[:50] == INF) and d[50] == 0
    np.testing.assert_array_equal(d[51:], np.cumsum(wts[50:]).astype(np.uint32))
    sw = rng.integers(1, 50, 63)
    ro, col, w = graphgen.star_graph(64, sw)
    np.testing.assert_array_equal(oracle.dijkstra(ro, col, w, 0), np.concatenate([[0], sw]).astype(np.uint32))
    d = oracle.dijkstra(ro, col, w, 5)               # leaf 5 -> hub -> leaf j
    expect = np.concatenate([[sw[4]], sw[4] + sw]).astype(np.uint32)
    expect[5] = 0
    np.testing.assert_array_equal(d, expect)


@pytest.mark.parametrize("name", hand_fixtures())
def test_hand_worked_fixtures(name):
    g = load(name)
    if isinstance(g["expect"], str):
        with pytest.raises(oracle.RangeError):
            oracle.dijkstra(g["ro"], g["col"], g["w"], g["src"])
        with pytest.raises(oracle.RangeError):
            oracle.bellman_ford(g["ro"], g["col"], g["w"], g["src"])
        return
    np.testing.assert_array_equal(oracle.dijkstra(g["ro"], g["col"], g["w"], g["src"]), g["expect"])
    np.testing.assert_array_equal(oracle.bellman_ford(g["ro"], g["col"], g["w"], g["src"])[0], g["expect"])


@pytest.mark.parametrize("maker", ["rmat12", "rmat14", "grid64", "grid100"])
def test_dijkstra_equals_bellman_ford(maker):
    if maker.startswith("rmat"):
        ro, col, w = graphgen.rmat(int(maker[4:]), 16, seed=11, W=255)
        src = graphgen.max_degree_vertex(ro)
    else:
        ro, col, w = graphgen.grid(int(maker[4:]), 64, seed=5)
        src = 0
    d = oracle.dijkstra(ro, col, w, src)
    bf, rounds = oracle.bellman_ford(ro, col, w, src)
    np.testing.assert_array_equal(d, bf)
    assert rounds >= 1


@pytest.mark.parametrize("maker", ["rmat12", "rmat16", "grid64"])
def test_invariants_hold_and_catch_corruption(maker):
    if maker.startswith("rmat"):
        ro, col, w = graphgen.rmat(int(maker[4:]), 16, seed=2, W=255)
        src = graphgen.max_degree_vertex(ro)
    else:
        ro, col, w = graphgen.grid(64, 64, seed=1)
        src = 0
    d = oracle.dijkstra(ro, col, w, src)
    assert oracle.check(ro, col, w, src, d) == (0, 0)
    reach = np.flatnonzero((d != INF) & (np.arange(d.shape[0]) != src))
    v = int(reach[len(reach) // 2])
    bad = d.copy(); bad[src] = 1
    assert oracle.check(ro, col, w, src, bad)[0] == 1
    bad = d.copy(); bad[v] += 1000          # too long: some in-edge now violates
    assert oracle.check(ro, col, w, src, bad)[0] == 2
    bad = d.copy(); bad[v] -= 1             # too short: no tight in-edge
    assert oracle.check(ro, col, w, src, bad)[0] in (2, 3)
    if np.any(d == INF):
        bad = d.copy(); u = int(np.flatnonzero(d == INF)[0]); bad[u] = 10 ** 9
        assert oracle.check(ro, col, w, src, bad)[0] in (3, 4)
    bad = d.copy(); bad[v] = INF
    assert oracle.check(ro, col, w, src, bad)[0] in (2, 4)


def test_dijkstra_many_matches_single():
    ro, col, w = graphgen.rmat(12, 16, seed=4, W=255)
    srcs = graphgen.sample_sources(ro, 8, seed=1)
    out = oracle.dijkstra_many(ro, col, w, srcs, threads=4)
    for i, s in enumerate(srcs):
        np.testing.assert_array_equal(out[i], oracle.dijkstra(ro, col, w, int(s)))


def test_range_error_on_unrepresentable_distance():
    ro, col, w = graphgen.path_graph(3, [2 ** 31, 2 ** 31 - 1])
    with pytest.raises(oracle.RangeError):
        oracle.dijkstra(ro, col, w, 0)


def test_traversed_edges_counts_reached_rows_once():
    ro, col, w = graphgen.from_edges(4, [0, 0, 1, 3, 3], [1, 2, 0, 0, 1], [1, 1, 1, 1, 1])
    d = oracle.dijkstra(ro, col, w, 0)
    assert d.tolist() == [0, 1, 1, INF]
    assert oracle.traversed_edges(ro, d) == 3       # rows 0 (2 edges) and 1 (1 edge); row 2 empty


# --- planted mistakes: each mutated copy of oracle.c must fail a pin ---------
MUTATIONS = {
    "dropped weight": ("uint64_t nd = d[u] + (uint64_t)weights[e];", "uint64_t nd = d[u] + 1;"),
    "wrong comparison": ("if (nd < d[v]) {", "if (nd > d[v] || d[v] == OR_INF64) {"),
    "dropped last edge": ("for (uint32_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {\n            uint32_t v = cols[e];\n            uint64_t nd",
                          "for (uint32_t e = row_offsets[u]; e + 1 < row_offsets[u + 1]; ++e) {\n            uint32_t v = cols[e];\n            uint64_t nd"),
    "transposed edge": ("            uint32_t v = cols[e];\n            uint64_t nd", "            uint32_t v = cols[e] ^ 1u;\n            if (v >= n) v = cols[e];\n            uint64_t nd"),
    "source not zero": ("    d[src] = 0;\n    if (heap_push(&h, 0, src))", "    d[src] = 1;\n    if (heap_push(&h, 1, src))"),
    "max-heap order": [("if (h->a[p].d <= d) break;", "if (h->a[p].d >= d) break;"),
                       ("if (l < h->size && h->a[l].d < sd)", "if (l < h->size && h->a[l].d > sd)"),
                       ("if (r < h->size && h->a[r].d < sd)", "if (r < h->size && h->a[r].d > sd)")],
}


def _pins_pass(lib_path):
    """Runs the brute-force and closed-form pins against a compiled oracle."""
    import ctypes
    lib = ctypes.CDLL(lib_path)
    P = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_dijkstra.restype = ctypes.c_int
    lib.oracle_dijkstra.argtypes = [ctypes.c_uint32, P, P, P, ctypes.c_uint32, P, ctypes.c_void_p]

    def dij(ro, col, w, src):
        n = ro.shape[0] - 1
        col = col if col.shape[0] else np.zeros(1, np.uint32)
        w = w if w.shape[0] else np.zeros(1, np.uint32)
        d = np.empty(n, np.uint32)
        lib.oracle_dijkstra(n, ro.ctypes.data_as(P), col.ctypes.data_as(P), w.ctypes.data_as(P), src,
                            d.ctypes.data_as(P), None)
        return d

    for seed in range(40):
        ro, col, w = graphgen.random_graph(24, 70, 30, seed)
        if not np.array_equal(dij(ro, col, w, 0), fw_row(ro, col, w, 0)):
            return False
    ro, col, w = graphgen.grid(9, const_w=2)
    ys, xs = np.divmod(np.arange(81), 9)
    if not np.array_equal(dij(ro, col, w, 0), (2 * (xs + ys)).astype(np.uint32)):
        return False
    for name in hand_fixtures():
        g = load(name)
        if not isinstance(g["expect"], str) and not np.array_equal(dij(g["ro"], g["col"], g["w"], g["src"]), g["expect"]):
            return False
    return True


def test_planted_mistakes_are_caught():
    src = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")
    text = open(src).read()
    tmp = tempfile.mkdtemp(prefix="oracle_mut_")
    try:
        clean = os.path.join(tmp, "clean.so")
        subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-pthread", "-o", clean, src])
        assert _pins_pass(clean)
        for label, edits in MUTATIONS.items():
            mutated = text
            for old, new in (edits if isinstance(edits, list) else [edits]):
                assert mutated.count(old) >= 1, f"mutation anchor missing: {label}"
                mutated = mutated.replace(old, new, 1)
            cpath = os.path.join(tmp, re.sub(r"\W", "_", label) + ".c")
            with open(cpath, "w") as f:
                f.write(mutated)
            so = cpath[:-2] + ".so"
            subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-pthread", "-o", so, cpath])
            assert not _pins_pass(so), f"planted mistake not caught: {label}"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
