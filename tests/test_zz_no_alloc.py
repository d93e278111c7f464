"""gg_sssp_noalloc: the entry point for callers that must not allocate device
memory (their GPU memory is owned by another allocator, or they cannot take
cudaFree's device-wide synchronisation).  It must return exactly the
distances gg_sssp returns, on consecutive calls that reuse its built-in
scratch array, and refuse graphs above its fixed vertex limit.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

import golden_io
import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda().view(torch.uint32)


@pytest.mark.parametrize("name", ["rmat16", "grid64", "rmat20"])
def test_noalloc_matches_gg_sssp_on_consecutive_calls(name):
    import paper_2212_08200_b300 as gg
    ro, col, w, src = graphgen.workload(name)
    n = ro.shape[0] - 1
    assert n <= gg.GG_NOALLOC_MAX_VERTICES
    g = gg.Graph(ro, col, w, symmetric=True)
    d_ro, d_col, d_w = _dev(ro), _dev(col), _dev(w)
    srcs = [src, int(graphgen.sample_sources(ro, 1, seed=11)[0])]
    out = torch.empty(n, dtype=torch.uint32, device="cuda")
    for s in srcs:                                   # two calls in a row share the scratch array
        ref = g.sssp(s)
        torch.cuda.synchronize()
        out.fill_(7)                                 # stale garbage must not leak into the result
        gg.gg_sssp_noalloc(d_ro, d_col, d_w, s, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_array_equal(got, ref.cpu().numpy(), err_msg=f"{name} src={s}")
        np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, s), err_msg=f"{name} src={s} vs oracle")
    g.close()


def test_noalloc_rejects_too_many_vertices_and_bad_csr():
    import paper_2212_08200_b300 as gg
    n = gg.GG_NOALLOC_MAX_VERTICES + 1
    ro = torch.zeros(n + 1, dtype=torch.uint32, device="cuda")
    empty = torch.zeros(1, dtype=torch.uint32, device="cuda")[:0]
    out = torch.empty(n, dtype=torch.uint32, device="cuda")
    with pytest.raises(gg.GGError) as ei:
        gg.gg_sssp_noalloc(ro, empty, empty, 0, out)
    assert ei.value.status_name == "GG_ERR_INVALID_ARG"
    assert "GG_NOALLOC_MAX_VERTICES" in str(ei.value)
    bad = _dev(np.array([0, 1, 2, 3], np.uint32))
    with pytest.raises(gg.GGError) as ei:            # column 5 >= n = 3
        gg.gg_sssp_noalloc(bad, _dev(np.array([1, 2, 5], np.uint32)), _dev(np.array([1, 1, 1], np.uint32)), 0,
                           torch.empty(3, dtype=torch.uint32, device="cuda"))
    assert ei.value.status_name == "GG_ERR_INVALID_ARG"
    one = _dev(np.array([1, 1, 1], np.uint32))
    cols = _dev(np.array([1, 2, 0], np.uint32))
    out3 = torch.empty(3, dtype=torch.uint32, device="cuda")
    for offsets in ([0, 2, 1, 3], [0, 1, 1, 2]):     # not monotone; does not end at m = 3
        with pytest.raises(gg.GGError) as ei:
            gg.gg_sssp_noalloc(_dev(np.array(offsets, np.uint32)), cols, one, 0, out3)
        assert ei.value.status_name == "GG_ERR_INVALID_ARG", offsets
    ok_ro = _dev(np.array([0, 1, 2, 3], np.uint32))
    with pytest.raises(ValueError):                  # weights shorter than col_indices
        gg.gg_sssp_noalloc(ok_ro, cols, one[:2], 0, out3)
    with pytest.raises(ValueError):                  # dist_out shorter than n
        gg.gg_sssp_noalloc(ok_ro, cols, one, 0, out3[:2])


def test_noalloc_overflow_and_sink_source():
    """A distance of 2^32 - 1 is a range error; a source without out-edges on
    a directed graph leaves every other vertex unreached."""
    import paper_2212_08200_b300 as gg
    fx = golden_io.load("hand_path_overflow.txt")
    assert fx["expect"] == "RANGE_ERROR"
    out = torch.empty(fx["n"], dtype=torch.uint32, device="cuda")
    with pytest.raises(gg.GGError) as ei:
        gg.gg_sssp_noalloc(_dev(fx["ro"]), _dev(fx["col"]), _dev(fx["w"]), fx["src"], out)
    assert ei.value.status_name == "GG_ERR_OVERFLOW"
    ro, col, w = graphgen.random_graph(300, 450, 50, seed=3)      # directed, with sinks
    n = ro.shape[0] - 1
    deg = np.diff(ro.astype(np.int64))
    sinks = np.flatnonzero(deg == 0)
    assert sinks.size
    for s in (int(np.argmax(deg)), int(sinks[0])):
        out = torch.full((n,), 5, dtype=torch.uint32, device="cuda")
        gg.gg_sssp_noalloc(_dev(ro), _dev(col), _dev(w), s, out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), oracle.dijkstra(ro, col, w, s), err_msg=f"src={s}")
