"""Pins the oracle's binary32 variant (the paper's float weights and
distances, Listings 1 and 4) to facts other than itself (no GPU needed).

The definition: from d[src] = +0 and FLT_MAX elsewhere, the least fixed
point of d[v] = min(d[v], fl(d[u] + w)), one round-to-nearest float32
addition per relaxation.  Since fl(x + w) is non-decreasing in x and never
below x for w >= 0, that is min(FLT_MAX, the smallest left-to-right rounded
sum over the simple paths src ~> v).  The pins:

* brute force: that path minimum, enumerated in numpy float32, on tiny graphs
  whose weights span many magnitudes (so rounding decides the result);
* exact special case: small integer weights make every sum exact, so the
  float result is the uint32 oracle's distance converted to float;
* a hand-worked chain where rounding after every step differs from rounding
  the exact sum once;
* a different algorithm: Bellman-Ford rounds in float32;
* planted mistakes: mutated copies of the float Dijkstra fail these pins.
"""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import graphgen
import oracle

FMAX = oracle.FLT_MAX_BITS


def rand_f32_weights(m, seed, spread=True):
    rng = np.random.Generator(np.random.PCG64(seed))
    if spread:   # magnitudes from 1e-3 to 1e7, plus some exact zeros
        w = (10.0 ** rng.uniform(-3, 7, m)).astype(np.float32)
        w[rng.random(m) < 0.05] = np.float32(0.0)
    else:
        w = rng.uniform(0, 100, m).astype(np.float32)
    return w


def brute_force_f32(ro, col, w, src):
    """min over simple paths of the left-to-right float32 sum, capped at FLT_MAX (bit patterns)."""
    n = ro.shape[0] - 1
    best = np.full(n, np.float32(np.finfo(np.float32).max), np.float32)
    best[src] = np.float32(0.0)
    on_path = np.zeros(n, bool)

    def dfs(u, d):
        on_path[u] = True
        for e in range(int(ro[u]), int(ro[u + 1])):
            v = int(col[e])
            if on_path[v]:
                continue
            nd = np.float32(d + w[e])            # one rounded float32 addition
            if nd < best[v]:
                best[v] = nd
            dfs(v, nd)
        on_path[u] = False

    with np.errstate(over="ignore"):
        dfs(src, np.float32(0.0))
    return best.view(np.uint32)


@pytest.mark.parametrize("seed", range(30))
def test_dijkstra_f32_equals_brute_force_path_minimum(seed):
    n = 3 + seed % 5
    ro, col, _ = graphgen.random_graph(n, 2 * n + seed % 7, 10, seed, symmetric=(seed % 3 == 0), wmin=0)
    w = rand_f32_weights(col.shape[0], seed)
    for src in range(min(n, 3)):
        np.testing.assert_array_equal(oracle.dijkstra_f32(ro, col, w, src), brute_force_f32(ro, col, w, src),
                                      err_msg=f"seed={seed} src={src}")


@pytest.mark.parametrize("seed", range(6))
def test_small_integer_weights_are_exact(seed):
    ro, col, wi = graphgen.random_graph(200, 900, 1000, seed, symmetric=True, wmin=0)
    d_int = oracle.dijkstra(ro, col, wi, 0)
    expect = np.where(d_int == oracle.INF, np.float32(np.finfo(np.float32).max),
                      d_int.astype(np.float32)).astype(np.float32).view(np.uint32)
    np.testing.assert_array_equal(oracle.dijkstra_f32(ro, col, wi.astype(np.float32), 0), expect)


def test_rounding_after_every_step():
    # chain 0 -> 1 -> 2 -> 3 with weights 1, 2^-24, 2^-24: each addition of
    # 2^-24 to 1.0 is a tie that rounds to even (1.0), while the exact sum
    # 1 + 2^-23 is representable, so rounding once at the end would differ
    ro = np.array([0, 1, 2, 3, 3], np.uint32)
    col = np.array([1, 2, 3], np.uint32)
    w = np.array([1.0, 2.0 ** -24, 2.0 ** -24], np.float32)
    d = oracle.dijkstra_f32(ro, col, w, 0).view(np.float32)
    assert d.tolist() == [0.0, 1.0, 1.0, 1.0]
    assert np.float32(1.0) + np.float32(2.0 ** -23) != np.float32(1.0)   # the exact sum differs
    # a second path 0 -> 3 of weight 1 + 2^-22 loses to the rounded chain
    ro2 = np.array([0, 2, 3, 4, 4], np.uint32)
    col2 = np.array([1, 3, 2, 3], np.uint32)
    w2 = np.array([1.0, 1.0 + 2.0 ** -22, 2.0 ** -24, 2.0 ** -24], np.float32)
    assert oracle.dijkstra_f32(ro2, col2, w2, 0).view(np.float32)[3] == np.float32(1.0)


def test_unreached_is_flt_max_and_overflow_never_improves():
    # 0 -> 1 (3e38), 1 -> 2 (3e38): the second sum rounds to +inf, so 2 stays unreached
    ro = np.array([0, 1, 2, 2, 2], np.uint32)
    col = np.array([1, 2], np.uint32)
    w = np.array([3e38, 3e38], np.float32)
    d = oracle.dijkstra_f32(ro, col, w, 0)
    assert d.tolist() == [0, np.float32(3e38).view(np.uint32), FMAX, FMAX]


def test_rejects_negative_nan_inf_and_negative_zero():
    ro = np.array([0, 1, 1], np.uint32)
    col = np.array([1], np.uint32)
    for bad in (-1.0, float("nan"), float("inf"), -0.0):
        with pytest.raises(ValueError):
            oracle.dijkstra_f32(ro, col, np.array([bad], np.float32), 0)


@pytest.mark.parametrize("maker", ["rmat", "grid"])
def test_dijkstra_f32_equals_bellman_ford_f32(maker):
    if maker == "rmat":
        ro, col, _ = graphgen.rmat(11, 8, seed=4, W=255)
    else:
        ro, col, _ = graphgen.grid(30)
    w = rand_f32_weights(col.shape[0], 7, spread=(maker == "rmat"))
    for src in (0, int(ro.shape[0] // 3)):
        d = oracle.dijkstra_f32(ro, col, w, src)
        b, _ = oracle.bellman_ford_f32(ro, col, w, src)
        np.testing.assert_array_equal(d, b)


# --- planted mistakes in the float Dijkstra must fail the pins above ----------
F32_MUTATIONS = {
    "dropped weight": ("volatile float nd = d[u] + f32_of(weight_bits[e]);", "volatile float nd = d[u] + 1.0f;"),
    "unreached as +inf": ("    for (uint32_t v = 0; v < n; ++v) d[v] = FLT_MAX;\n    d[src] = 0.0f;\n    if (fheap_push",
                          "    for (uint32_t v = 0; v < n; ++v) d[v] = 1.0f / 0.0f;\n    d[src] = 0.0f;\n    if (fheap_push"),
    "rounding perturbed at 2^-30 relative": ("volatile float nd = d[u] + f32_of(weight_bits[e]);",
                            "volatile float nd = (float)((double)d[u] + (double)f32_of(weight_bits[e]) + (double)(e % 2) * 0x1p-30 * (double)d[u]);"),
    "dropped last edge": ("for (uint32_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {\n            uint32_t v = cols[e];\n            volatile float nd",
                          "for (uint32_t e = row_offsets[u]; e + 1 < row_offsets[u + 1]; ++e) {\n            uint32_t v = cols[e];\n            volatile float nd"),
    "max-heap order": [("if (h->a[p].d <= d) break;\n        h->a[i] = h->a[p];\n        i = p;\n    }\n    h->a[i].d = d; h->a[i].v = v;\n    return 0;\n}\n\nstatic fheap_item",
                        "if (h->a[p].d >= d) break;\n        h->a[i] = h->a[p];\n        i = p;\n    }\n    h->a[i].d = d; h->a[i].v = v;\n    return 0;\n}\n\nstatic fheap_item")],
}


def _f32_pins_pass(lib_path):
    lib = ctypes.CDLL(lib_path)
    P = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_dijkstra_f32.restype = ctypes.c_int
    lib.oracle_dijkstra_f32.argtypes = [ctypes.c_uint32, P, P, P, ctypes.c_uint32, P]

    def dij(ro, col, w, src):
        n = ro.shape[0] - 1
        wb = np.ascontiguousarray(w.view(np.uint32))
        d = np.empty(n, np.uint32)
        rc = lib.oracle_dijkstra_f32(n, ro.ctypes.data_as(P), col.ctypes.data_as(P), wb.ctypes.data_as(P), src,
                                     d.ctypes.data_as(P))
        return d if rc == 0 else None

    for seed in range(30):
        n = 3 + seed % 5
        ro, col, _ = graphgen.random_graph(n, 2 * n + seed % 7, 10, seed, symmetric=(seed % 3 == 0), wmin=0)
        w = rand_f32_weights(col.shape[0], seed)
        for src in range(min(n, 3)):
            got = dij(ro, col, w, src)
            if got is None or not np.array_equal(got, brute_force_f32(ro, col, w, src)):
                return False
    ro = np.array([0, 1, 2, 2, 2], np.uint32)
    col = np.array([1, 2], np.uint32)
    got = dij(ro, col, np.array([3e38, 3e38], np.float32), 0)
    if got is None or got[3] != FMAX or got[2] != FMAX:
        return False
    return True


def test_planted_float_mistakes_are_caught():
    src = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")
    text = open(src).read()
    tmp = tempfile.mkdtemp(prefix="oracle_f32_mut_")
    try:
        clean = os.path.join(tmp, "clean.so")
        subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-pthread", "-o", clean, src])
        assert _f32_pins_pass(clean)
        for label, edits in F32_MUTATIONS.items():
            mutated = text
            for old, new in (edits if isinstance(edits, list) else [edits]):
                assert mutated.count(old) >= 1, f"mutation anchor missing: {label}"
                mutated = mutated.replace(old, new, 1)
            cpath = os.path.join(tmp, "m_" + "".join(c if c.isalnum() else "_" for c in label) + ".c")
            with open(cpath, "w") as f:
                f.write(mutated)
            so = cpath[:-2] + ".so"
            subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-pthread", "-o", so, cpath])
            assert not _f32_pins_pass(so), f"planted mistake not caught: {label}"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
