"""GPU parity of batched multi-source SSSP (gg_sssp_batch) against the CPU
oracle, one Dijkstra per source.  Bit-exact (tolerance 0)."""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def gg():
    import paper_2212_08200_b300 as m
    m.load()
    return m


def run_batch(g, srcs, **kw):
    m = gg()
    st = m.gg_stats()
    d = g.sssp_batch(srcs, stats=st, **kw)
    torch.cuda.synchronize()
    return d.cpu().numpy(), st.as_dict()


@pytest.mark.parametrize("k,pack,delta,policy", [(1, True, 0, 0), (5, False, 0, 0), (64, True, 0, 0),
                                                 (100, False, 0, 0), (64, True, 1, 0), (64, False, 25, 0),
                                                 (100, True, 0xFFFFFFFF, 0), (5, True, 300, 0), (64, True, 0, 2),
                                                 (70, False, 9, 2)])
def test_rmat16_batch_matches_oracle(k, pack, delta, policy):
    ro, col, w, _ = graphgen.workload("rmat16")
    srcs = graphgen.sample_sources(ro, k, seed=3)
    g = gg().Graph(ro, col, w, symmetric=True, pack=pack)
    got, st = run_batch(g, srcs, delta=delta, policy=policy)   # policy 2: host-launched supersteps
    ref = oracle.dijkstra_many(ro, col, w, srcs, threads=8)
    for s in range(k):
        np.testing.assert_array_equal(got[:, s], ref[s], err_msg=f"column {s}")
    assert st["iterations"] > 0 and st["device_status"] == 0
    g.close()


def test_duplicates_isolated_and_tiny_graphs():
    m = gg()
    for seed in range(6):
        ro, col, w = graphgen.random_graph(40, 120, 50, seed, wmin=0)
        g = m.Graph(ro, col, w)
        srcs = np.array([0, 3, 3, 39, 0, 17, 5], np.uint32)
        got, _ = run_batch(g, srcs)
        ref = oracle.dijkstra_many(ro, col, w, srcs)
        np.testing.assert_array_equal(got.T, ref)
        g.close()
    ro = np.zeros(5, np.uint32)                     # n = 4 vertices, no edges
    g = m.Graph(ro, np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    got, _ = run_batch(g, np.array([2, 0], np.uint32))
    assert got[:, 0].tolist() == [0xFFFFFFFF, 0xFFFFFFFF, 0, 0xFFFFFFFF]
    assert got[:, 1].tolist() == [0, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF]
    g.close()


@pytest.mark.parametrize("delta", [0, 1, 50, 0xFFFFFFFF])
def test_grid64_batch_and_reuse(delta):
    ro, col, w, _ = graphgen.workload("grid64")
    g = gg().Graph(ro, col, w, symmetric=True)
    for seed in (1, 2):                               # workspace reuse across calls
        srcs = graphgen.sample_sources(ro, 64, seed=seed)
        got, _ = run_batch(g, srcs, delta=delta)
        ref = oracle.dijkstra_many(ro, col, w, srcs, threads=8)
        np.testing.assert_array_equal(got.T, ref)
    g.close()


def test_batch_equals_single_source_calls():
    ro, col, w, _ = graphgen.workload("rmat16")
    srcs = graphgen.sample_sources(ro, 64, seed=9)
    g = gg().Graph(ro, col, w, symmetric=True)
    got, _ = run_batch(g, srcs)
    for s in (0, 31, 32, 63):
        d = g.sssp(int(srcs[s]))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got[:, s], d.cpu().numpy())
    g.close()


@pytest.mark.parametrize("k,offset", [(64, 0), (64, 1), (68, 0), (68, 3), (12, 0)])
def test_row_read_modes(k, offset):
    """k a multiple of 4 on a 16-byte aligned matrix reads rows as 16-byte
    vectors; an offset matrix or another k reads them word by word."""
    ro, col, w, _ = graphgen.workload("rmat16")
    srcs = graphgen.sample_sources(ro, k, seed=11)
    g = gg().Graph(ro, col, w, symmetric=True)
    buf = torch.empty(g.n * k + offset, dtype=torch.uint32, device="cuda")
    out = buf[offset:]
    g.sssp_batch(srcs, out)
    torch.cuda.synchronize()
    got = out.view(g.n, k).cpu().numpy()
    ref = oracle.dijkstra_many(ro, col, w, srcs, threads=8)
    np.testing.assert_array_equal(got.T, ref)
    g.close()


def test_rmat22_64_sources_config():
    """The batched workload itself: all 64 columns of the RMAT-22 distance
    matrix equal the oracle's (their sha256, stored by
    tests/golden/make_golden.py from oracle.dijkstra_many), and three columns
    are compared element by element with a live oracle run."""
    import hashlib
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "workloads.json")) as f:
        rec = json.load(f)["rmat22_batch64"]
    ro, col, w = graphgen.rmat(22, 16, seed=1, W=255)
    srcs = graphgen.sample_sources(ro, 64, seed=1)
    assert [int(x) for x in srcs] == rec["sources"]
    g = gg().Graph(ro, col, w, symmetric=True)
    got, st = run_batch(g, srcs)
    g.close()
    assert st["device_status"] == 0
    bad = [s for s in range(64)
           if hashlib.sha256(np.ascontiguousarray(got[:, s]).tobytes()).hexdigest() != rec["column_sha256"][s]]
    assert not bad, f"columns {bad} differ from the oracle's"
    assert hashlib.sha256(np.ascontiguousarray(got).tobytes()).hexdigest() == rec["matrix_sha256"]
    ref = oracle.dijkstra_many(ro, col, w, srcs[[0, 33, 63]], threads=3)
    for i, s in enumerate([0, 33, 63]):
        np.testing.assert_array_equal(got[:, s], ref[i], err_msg=f"column {s}")


def test_batch_argument_errors():
    m = gg()
    ro, col, w, _ = graphgen.workload("grid64")
    g = m.Graph(ro, col, w, symmetric=True)
    out = torch.empty(g.n * 2, dtype=torch.uint32, device="cuda")
    with pytest.raises(m.GGError):
        m.gg_sssp_batch(g.handle, np.array([0, g.n], np.uint32), out)
    with pytest.raises(m.GGError):
        m.gg_sssp_batch(g.handle, np.zeros(0, np.uint32), out)
    g.close()


@pytest.mark.parametrize("lh,delta", [(2, 0), (2, 20), (0, 20), (0, 255), (1, 0)])
def test_batch_schedules_and_widths(lh, delta):
    """The batched schedules side by side on a skewed graph: light-first
    rounds (GG_LH_ROUNDS), normalised buckets at an explicit light/heavy
    width, the largest width (every edge light) and no light/heavy split
    (GG_LH_OFF): the same distances as the oracle."""
    ro, col, w, _ = graphgen.workload("rmat16")
    srcs = graphgen.sample_sources(ro, 40, seed=13)
    g = gg().Graph(ro, col, w, symmetric=True)
    got, st = run_batch(g, srcs, light_heavy=lh, delta=delta)
    np.testing.assert_array_equal(got.T, oracle.dijkstra_many(ro, col, w, srcs, threads=8))
    assert st["device_status"] == 0
    g.close()


def test_batch_directed_graph_normalised_buckets():
    """A directed skewed graph (no pull: its heavy in-edges are not its
    out-edges) with sinks: normalised buckets with the heavy push."""
    rng = np.random.Generator(np.random.PCG64(8))
    n, m = 20000, 400000
    src = rng.integers(0, 15000, m)                  # vertices 15000.. have no out-edges
    ro, col, w = graphgen.from_edges(n, src, rng.integers(0, n, m), rng.integers(1, 256, m))
    srcs = graphgen.sample_sources(ro, 33, seed=2)
    g = gg().Graph(ro, col, w)
    got, _ = run_batch(g, srcs)
    np.testing.assert_array_equal(got.T, oracle.dijkstra_many(ro, col, w, srcs, threads=8))
    g.close()


@pytest.mark.parametrize("name,k,policy", [("rmat16", 64, 0), ("rmat16", 40, 2), ("rmat18", 64, 0)])
def test_batch_pull_that_ends_the_buckets(name, k, policy):
    """On a skewed symmetric graph the dense bucket's heavy superstep pulls,
    and the drain rule then holds: that pull (trace kind 5) starts the plain
    push itself, so only tail pushes (kind 16) follow, with no mask clear and
    no split; every column equals the oracle."""
    ro, col, w, _ = graphgen.workload(name)
    srcs = graphgen.sample_sources(ro, k, seed=29)
    g = gg().Graph(ro, col, w, symmetric=True)
    m = gg()
    trace = torch.zeros(4 * 4096, dtype=torch.uint32, device="cuda")
    st = m.gg_stats()
    d = g.sssp_batch(srcs, stats=st, policy=policy, trace=trace, trace_cap=4096)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d.cpu().numpy().T, oracle.dijkstra_many(ro, col, w, srcs, threads=8))
    assert st.device_status == 0
    tr = trace.cpu().numpy().reshape(-1, 4)[:st.iterations]
    kinds = tr[:, 0]
    k5 = np.flatnonzero(kinds == 5)
    assert k5.size == 1, kinds
    rest = kinds[k5[0] + 1:]
    assert rest.size > 0 and (rest == 16).all(), kinds
    assert tr[k5[0], 3] > 0 and tr[k5[0] + 1, 1] == tr[k5[0], 3]   # its frontier feeds the first tail push
    g.close()
