"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Shortest-path distances are unique integers, so every policy, direction and
load-balance mode must match the oracle bit for bit (tolerance 0).
"""
import hashlib
import json
import os

import numpy as np
import pytest

import graphgen
import oracle
from golden_io import hand_fixtures, load

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "workloads.json")))
INF = 0xFFFFFFFF


def gg():
    import paper_2212_08200_b300 as m
    m.load()
    return m


POLICIES = {"graph": 0, "async": 1, "host": 2, "persistent": 3}
DIRS = {"auto": 0, "push": 1, "pull": 2}
LB = {"mp": 1, "bins": 2, "warp": 3, "local": 4}
NONE = 0xFFFFFFFF
# (policy, direction, load balance, near-far delta; 0 = the graph's default)
MODES = [("graph", "auto"), ("graph", "push"), ("graph", "pull"), ("host", "auto"), ("host", "pull"),
         ("async", "auto"), ("graph", "push", "bins"), ("host", "auto", "bins"),
         ("graph", "push", "mp", NONE), ("graph", "auto", "mp", 1), ("graph", "push", "bins", 3),
         ("persistent", "push"), ("persistent", "auto", "mp", NONE), ("persistent", "pull"),
         ("persistent", "push", "bins", 5), ("graph", "push", "warp"), ("host", "auto", "warp", 4),
         ("persistent", "push", "warp", NONE), ("graph", "push", "warp", 2),
         ("graph", "push", "local"), ("host", "push", "local", 3), ("graph", "push", "local", NONE),
         ("graph", "auto", "local")]


def run(g, src, policy="graph", direction="auto", lb="mp", delta=0, **kw):
    m = gg()
    st = m.gg_stats()
    d = g.sssp(src, policy=POLICIES[policy], direction=DIRS[direction], lb_mode=LB[lb], delta=delta, stats=st,
               **kw)
    torch.cuda.synchronize()
    return d.cpu().numpy(), st.as_dict()


def sha(a):
    return hashlib.sha256(np.ascontiguousarray(a, np.uint32).tobytes()).hexdigest()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("case", [(8, 12, 9, False, 0), (33, 64, 100, True, 1), (64, 150, 255, False, 0),
                                  (64, 400, 3, True, 0), (50, 30, 20, False, 1)])
def test_tiny_random_graphs(mode, case):
    n, m, W, sym, wmin = case
    for seed in range(12):
        ro, col, w = graphgen.random_graph(n, m, W, seed, symmetric=sym, wmin=wmin)
        g = gg().Graph(ro, col, w, symmetric=False)
        for src in (0, n // 2, n - 1):
            got, _ = run(g, src, *mode)
            np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, src),
                                          err_msg=f"seed={seed} src={src} mode={mode}")
        g.close()


@pytest.mark.parametrize("name", hand_fixtures())
@pytest.mark.parametrize("mode", MODES)
def test_hand_worked_fixtures(name, mode):
    f = load(name)
    g = gg().Graph(f["ro"], f["col"], f["w"])
    got, st = run(g, f["src"], *mode) if not isinstance(f["expect"], str) else (None, None)
    if isinstance(f["expect"], str):
        m = gg()
        d = g.sssp(f["src"], policy=POLICIES[mode[0]], direction=DIRS[mode[1]],
                   lb_mode=LB[mode[2] if len(mode) > 2 else "mp"], delta=mode[3] if len(mode) > 3 else 0)
        with pytest.raises(m.GGError) as ei:
            g.check()
        assert ei.value.status_name == "GG_ERR_OVERFLOW"
        assert d.cpu().numpy()[2] == 0xFFFFFFFE              # saturated, not wrapped
    else:
        np.testing.assert_array_equal(got, f["expect"])
        g.check()
    g.close()


@pytest.mark.parametrize("mode", MODES)
def test_grid64_config(mode):
    ro, col, w, src = graphgen.workload("grid64")
    g = gg().Graph(ro, col, w, symmetric=True)
    got, st = run(g, src, *mode)
    assert sha(got) == GOLD["grid64"]["dist_sha256"]
    np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, src))
    g.close()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("sym,pack", [(True, True), (False, True), (True, False), (False, False)])
def test_rmat16_multi_tile(mode, sym, pack):
    ro, col, w, src = graphgen.workload("rmat16")
    g = gg().Graph(ro, col, w, symmetric=sym, pack=pack)
    ref = oracle.dijkstra(ro, col, w, src)
    for s in (src, int(graphgen.sample_sources(ro, 1, seed=5)[0])):
        got, st = run(g, s, *mode)
        np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, s) if s != src else ref)
    g.close()


@pytest.mark.parametrize("thr", [(2, 8), (32, 1024), (1, 1), (4096, 8192)])
def test_bins_thresholds(thr):
    ro, col, w, src = graphgen.workload("rmat16")
    g = gg().Graph(ro, col, w, symmetric=True)
    ref = oracle.dijkstra(ro, col, w, src)
    got, _ = run(g, src, "graph", "push", "bins", warp_threshold=thr[0], cta_threshold=thr[1])
    np.testing.assert_array_equal(got, ref)
    g.close()


@pytest.mark.parametrize("delta", [1, 2, 17, 200, 5000, NONE])
@pytest.mark.parametrize("workload", ["grid64", "rmat16"])
def test_near_far_deltas(delta, workload):
    ro, col, w, src = graphgen.workload(workload)
    g = gg().Graph(ro, col, w, symmetric=True)
    ref = oracle.dijkstra(ro, col, w, src)
    for mode in [("graph", "push"), ("graph", "auto"), ("host", "push", "bins"), ("persistent", "push"),
                 ("persistent", "auto"), ("async", "auto")]:
        got, st = run(g, src, *mode, delta=delta)
        np.testing.assert_array_equal(got, ref, err_msg=f"delta={delta} {mode}")
    g.close()


def test_near_far_high_diameter_grid_reduces_work():
    ro, col, w = graphgen.grid(256, 1000, 3)
    g = gg().Graph(ro, col, w, symmetric=True)
    ref = oracle.dijkstra(ro, col, w, 0)
    got, st_bf = run(g, 0, "graph", "push", delta=NONE)
    np.testing.assert_array_equal(got, ref)
    got, st_nf = run(g, 0, "graph", "push", delta=500)
    np.testing.assert_array_equal(got, ref)
    assert st_nf["edges_scanned"] < st_bf["edges_scanned"]
    got, st_abf = run(g, 0, "async", delta=NONE)
    np.testing.assert_array_equal(got, ref)
    got, st_anf = run(g, 0, "async", delta=500)
    np.testing.assert_array_equal(got, ref)
    assert st_anf["edges_scanned"] < st_abf["edges_scanned"]
    g.close()


def test_rmat20_config_push_pull():
    ro, col, w, src = graphgen.workload("rmat20")
    g = gg().Graph(ro, col, w, symmetric=True)
    ref = oracle.dijkstra(ro, col, w, src)
    assert sha(ref) == GOLD["rmat20"]["dist_sha256"]
    got, st = run(g, src, "graph", "auto", delta=NONE)
    np.testing.assert_array_equal(got, ref)
    assert st["pull_iterations"] > 0          # the switch really went to pull
    got, st = run(g, src, "graph", "push")
    np.testing.assert_array_equal(got, ref)
    assert st["pull_iterations"] == 0
    got, _ = run(g, src, "async")
    np.testing.assert_array_equal(got, ref)
    got, _ = run(g, src, "graph", "auto", "bins")
    np.testing.assert_array_equal(got, ref)
    got, _ = run(g, src, "graph", "push", "warp")
    np.testing.assert_array_equal(got, ref)
    g.close()


@pytest.mark.parametrize("name", ["grid4096", "rmat22"])
def test_full_size_configs_against_golden(name):
    ro, col, w, src = graphgen.workload(name)
    g = gg().Graph(ro, col, w, symmetric=True)
    modes = [("graph", "auto"), ("async", "auto"), ("persistent", "push"), ("graph", "push", "warp")]
    for mode in modes:
        got, st = run(g, src, *mode)
        assert sha(got) == GOLD[name]["dist_sha256"], f"{name} {mode}"
    # independent of the stored hash: the invariants of shortest-path distances
    assert oracle.check(ro, col, w, src, got) == (0, 0)
    g.close()


def test_rmat22_batch_of_sources_sampled():
    ro, col, w = graphgen.rmat(22, 16, seed=1, W=255)
    srcs = graphgen.sample_sources(ro, 3, seed=1)
    g = gg().Graph(ro, col, w, symmetric=True)
    for s in srcs:
        got, _ = run(g, int(s), "graph", "auto")
        np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, int(s)))
    g.close()


# ---- edge cases ------------------------------------------------------------

def test_graph_without_edges():
    m = gg()
    ro = np.zeros(6, np.uint32)
    g = m.Graph(ro, np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    for mode in MODES:
        got, st = run(g, 3, *mode)
        assert got.tolist() == [INF, INF, INF, 0, INF]
    g.close()
    g = m.Graph(np.zeros(2, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    got, _ = run(g, 0)
    assert got.tolist() == [0]
    g.close()


def test_isolated_source_in_rmat():
    ro, col, w, _ = graphgen.workload("rmat16")
    iso = int(np.flatnonzero(np.diff(ro.astype(np.int64)) == 0)[0])
    g = gg().Graph(ro, col, w, symmetric=True)
    for mode in MODES:
        got, st = run(g, iso, *mode)
        assert got[iso] == 0 and np.all(np.delete(got, iso) == INF)
    g.close()


def test_star_hub_forces_big_rows():
    n = 200_001
    rng = np.random.Generator(np.random.PCG64(9))
    wts = rng.integers(1, 1000, n - 1)
    ro, col, w = graphgen.star_graph(n, wts)
    g = gg().Graph(ro, col, w, symmetric=True)
    for src in (0, 77):
        ref = oracle.dijkstra(ro, col, w, src)
        for mode in MODES:
            got, _ = run(g, src, *mode)
            np.testing.assert_array_equal(got, ref, err_msg=f"{mode}")
    g.close()


def test_long_path_many_supersteps():
    n = 20_000
    wts = np.random.Generator(np.random.PCG64(2)).integers(0, 50, n - 1)
    ro, col, w = graphgen.path_graph(n, wts)
    g = gg().Graph(ro, col, w)
    ref = oracle.dijkstra(ro, col, w, 0)
    for mode in [("graph", "push"), ("async", "auto"), ("graph", "auto")]:
        got, st = run(g, 0, *mode, delta=NONE)
        np.testing.assert_array_equal(got, ref)
        if mode[0] == "graph":
            assert st["iterations"] == n - 1     # one hop per superstep on a directed path
    got, st = run(g, 0, "graph", "push", delta=7)
    np.testing.assert_array_equal(got, ref)
    g.close()


def test_ties_zero_and_large_weights():
    ro, col, _ = graphgen.grid(57)                                 # ragged n = 3249 (not a multiple of 32)
    # n = 3249 needs 12 column bits, leaving 20 weight bits: 2^20 - 1 is the
    # largest weight stored packed, 2^20 falls back to 8-byte edges
    for wval in (0, 7, 2 ** 20 - 1, 2 ** 20):
        w = np.full(col.shape[0], wval, np.uint32)
        g = gg().Graph(ro, col, w, symmetric=True)
        for mode in MODES:
            got, _ = run(g, 1000, *mode)
            np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, 1000), err_msg=f"w={wval} {mode}")
        g.close()


def test_directed_graph_needs_transpose_for_pull():
    ro, col, w = graphgen.random_graph(3000, 12000, 100, seed=4)
    g = gg().Graph(ro, col, w, symmetric=False)
    for src in (0, 1234):
        ref = oracle.dijkstra(ro, col, w, src)
        for mode in MODES:
            got, _ = run(g, src, *mode)
            np.testing.assert_array_equal(got, ref, err_msg=f"{mode}")
    g.close()


def test_device_pointer_inputs_and_reuse():
    m = gg()
    ro, col, w, src = graphgen.workload("rmat16")
    t = [torch.from_numpy(a.view(np.int32)).cuda() for a in (ro, col, w)]
    g = m.Graph(*[x.view(torch.uint32) for x in t], symmetric=True)
    ref = oracle.dijkstra(ro, col, w, src)
    out = torch.empty(g.n, dtype=torch.uint32, device="cuda")
    for _ in range(3):                                          # workspace reuse across calls
        g.sssp(src, out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref)
    g.close()


def test_two_streams_same_handle_are_ordered():
    ro, col, w, src = graphgen.workload("rmat16")
    g = gg().Graph(ro, col, w, symmetric=True)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    a = torch.empty(g.n, dtype=torch.uint32, device="cuda")
    b = torch.empty(g.n, dtype=torch.uint32, device="cuda")
    other = int(graphgen.sample_sources(ro, 1, seed=3)[0])
    g.sssp(src, a, stream=s1)
    g.sssp(other, b, stream=s2)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.cpu().numpy(), oracle.dijkstra(ro, col, w, src))
    np.testing.assert_array_equal(b.cpu().numpy(), oracle.dijkstra(ro, col, w, other))
    g.close()


def test_trace_and_stats():
    m = gg()
    ro, col, w, src = graphgen.workload("grid64")
    g = m.Graph(ro, col, w, symmetric=True)
    trace = torch.zeros(4 * 4096, dtype=torch.uint32, device="cuda")
    got, st = run(g, src, "graph", "push", trace=trace, delta=NONE)
    tr = trace.cpu().numpy().reshape(-1, 4)[: st["iterations"]]
    assert tr[0, 0] == 1 and tr[0, 1] == ro[src + 1] - ro[src]
    assert np.array_equal(tr[1:, 0], tr[:-1, 3])                # next frontier size feeds the next step
    assert tr[-1, 3] == 0
    assert st["edges_scanned"] == int(tr[:, 1].astype(np.int64).sum())
    assert st["max_frontier"] == int(tr[:, 0].max())
    g.close()


def test_device_side_validation_errors():
    m = gg()
    ro = np.array([0, 2, 1, 3], np.uint32)                          # decreasing offsets
    col = np.array([1, 2, 0], np.uint32)
    w = np.array([1, 1, 1], np.uint32)
    with pytest.raises(m.GGError) as ei:
        m.Graph(ro, col, w)
    assert ei.value.status_name == "GG_ERR_INVALID_ARG"
    ro = np.array([0, 1, 2, 3], np.uint32)
    col = np.array([1, 2, 3], np.uint32)                            # 3 >= n
    with pytest.raises(m.GGError):
        m.Graph(ro, col, w)
    g = m.Graph(ro, np.array([1, 2, 0], np.uint32), w)
    with pytest.raises(m.GGError):
        g.sssp(3)                                                   # src >= n
    g.close()


def test_async_watchdog_reports_timeout_and_recovers():
    m = gg()
    ro, col, w, src = graphgen.workload("grid64")
    g = m.Graph(ro, col, w, symmetric=True)
    g.sssp(src, policy=1, watchdog_ns=1)                            # every wait runs out at once
    with pytest.raises(m.GGError) as ei:
        g.check()
    assert ei.value.status_name == "GG_ERR_TIMEOUT"
    got, _ = run(g, src, "async")                                   # the next run is unaffected
    np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, src))
    g.check()
    g.close()


def test_async_repeated_runs_wrap_the_ring():
    """Each RMAT-20 run from the hub pushes more items than the ring has
    slots, so producers wrap onto slots of the previous lap while the warp
    expanding the hub still holds reservations: every run must drain, bit-exact."""
    ro, col, w, src = graphgen.workload("rmat20")
    g = gg().Graph(ro, col, w, symmetric=True)
    ref = oracle.dijkstra(ro, col, w, src)
    for rep in range(40):
        got, st = run(g, src, "async")
        assert st["device_status"] == 0, f"rep {rep}"
        np.testing.assert_array_equal(got, ref, err_msg=f"rep {rep}")
    g.close()


@pytest.mark.parametrize("policy", ["persistent", "graph"])
def test_bsp_watchdog_reports_timeout_and_recovers(policy):
    m = gg()
    ro, col, w, src = graphgen.workload("grid64")
    g = m.Graph(ro, col, w, symmetric=True)
    g.sssp(src, policy=POLICIES[policy], watchdog_ns=1)              # the deadline has passed at once
    with pytest.raises(m.GGError) as ei:
        g.check()
    assert ei.value.status_name == "GG_ERR_TIMEOUT"
    got, _ = run(g, src, policy)                                     # the next run is unaffected
    np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, src))
    g.check()
    g.close()


def test_iteration_cap_reports_internal():
    m = gg()
    ro, col, w, src = graphgen.workload("grid64")
    g = m.Graph(ro, col, w, symmetric=True)
    g.sssp(src, max_iterations=3)
    with pytest.raises(m.GGError) as ei:
        g.check()
    assert ei.value.status_name == "GG_ERR_INTERNAL"
    g.close()


@pytest.mark.parametrize("side,delta", [(512, 0), (300, 0), (256, NONE), (128, 40)])
def test_local_rounds_on_grids(side, delta):
    """Warp-local rounds (GG_LB_LOCAL) on high-diameter grids: the oracle's
    distances in fewer supersteps than plain warp streaming."""
    ro, col, w = graphgen.grid(side, 1000, 3)
    g = gg().Graph(ro, col, w, symmetric=True)
    ref = oracle.dijkstra(ro, col, w, 0)
    got, st = run(g, 0, "graph", "push", "local", delta)
    np.testing.assert_array_equal(got, ref)
    _, st_w = run(g, 0, "graph", "push", "warp", delta)
    assert st["iterations"] <= st_w["iterations"]
    if delta == 0:   # the graph's bucket width leaves room for several hops per superstep
        assert st["iterations"] < st_w["iterations"]
    g.close()


@pytest.mark.parametrize("name", ["rmat16", "grid64"])
def test_local_rounds_float_and_bfs(name):
    """The local rounds under the other weight modes: binary32 weights (the
    paper's float variant) and unit weights (BFS)."""
    m = gg()
    ro, col, w, src = graphgen.workload(name)
    wf = (w.astype(np.float32) * np.float32(0.37)).astype(np.float32)
    gf = m.Graph(ro, col, wf, symmetric=True, float_weights=True)
    d = gf.sssp(src, lb_mode=LB["local"], direction=DIRS["push"])
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d.cpu().numpy(), oracle.dijkstra_f32(ro, col, wf, src))
    gf.close()
    g = m.Graph(ro, col, w, symmetric=True)
    h = g.bfs(src, lb_mode=LB["local"], direction=DIRS["push"])
    torch.cuda.synchronize()
    np.testing.assert_array_equal(h.cpu().numpy(), oracle.bfs_hops(ro, col, src))
    g.close()
