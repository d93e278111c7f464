"""GPU parity of the paper's float variant (binary32 weights and distances,
GG_FLOAT_WEIGHTS) and of BFS (gg_bfs) against the CPU oracle, bit for bit."""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FMAX = oracle.FLT_MAX_BITS
POLICIES = {"graph": 0, "async": 1, "host": 2, "persistent": 3}
DIRS = {"auto": 0, "push": 1, "pull": 2}
LB = {"mp": 1, "bins": 2, "warp": 3, "local": 4}
MODES = [("graph", "push", "warp"), ("graph", "auto", "warp"), ("graph", "pull", "mp"), ("host", "push", "mp"),
         ("host", "auto", "bins"), ("persistent", "push", "warp"), ("persistent", "auto", "mp"),
         ("async", "push", "warp"), ("graph", "push", "local"), ("host", "auto", "local")]


def gg():
    import paper_2212_08200_b300 as m
    m.load()
    return m


def spread_weights(m, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    w = (10.0 ** rng.uniform(-3, 7, m)).astype(np.float32)
    w[rng.random(m) < 0.05] = np.float32(0.0)
    return w


def symmetric_spread_weights(ro, col, seed):
    """Weights of spread magnitudes that agree on (u, v) and (v, u), as a
    symmetric graph's CSR must (pull reads it as its own transpose)."""
    n = ro.shape[0] - 1
    u = np.repeat(np.arange(n, dtype=np.uint64), np.diff(ro.astype(np.int64)))
    v = col.astype(np.uint64)
    with np.errstate(over="ignore"):
        x = np.minimum(u, v) * np.uint64(n) + np.maximum(u, v) + np.uint64(seed) * np.uint64(0x9E3779B97F4A7C15)
        x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        x = x ^ (x >> np.uint64(31))
    unit = (x >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    return (10.0 ** (unit * 10.0 - 3.0)).astype(np.float32)


def run_f32(g, src, mode):
    d = g.sssp(src, policy=POLICIES[mode[0]], direction=DIRS[mode[1]], lb_mode=LB[mode[2]])
    torch.cuda.synchronize()
    g.check()
    return d.cpu().numpy()


@pytest.mark.parametrize("mode", MODES)
def test_float_random_graphs(mode):
    for seed in range(8):
        n = 20 + 13 * seed
        ro, col, _ = graphgen.random_graph(n, 4 * n, 10, seed, symmetric=(seed % 2 == 0), wmin=0)
        w = spread_weights(col.shape[0], seed)
        g = gg().Graph(ro, col, w, symmetric=False, float_weights=True)
        for src in (0, n // 2):
            np.testing.assert_array_equal(run_f32(g, src, mode), oracle.dijkstra_f32(ro, col, w, src),
                                          err_msg=f"seed={seed} src={src} mode={mode}")
        g.close()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("sym", [True, False])
def test_float_rmat16(mode, sym):
    ro, col, _, src = graphgen.workload("rmat16")
    w = symmetric_spread_weights(ro, col, 3) if sym else spread_weights(col.shape[0], 3)
    g = gg().Graph(ro, col, w, symmetric=sym, float_weights=True)
    np.testing.assert_array_equal(run_f32(g, src, mode), oracle.dijkstra_f32(ro, col, w, src))
    g.close()


def test_float_grid_with_integer_and_fractional_weights():
    ro, col, wi, src = graphgen.workload("grid64")
    for w in (wi.astype(np.float32), wi.astype(np.float32) * np.float32(0.1)):
        g = gg().Graph(ro, col, w, symmetric=True, float_weights=True)
        for mode in MODES:
            np.testing.assert_array_equal(run_f32(g, src, mode), oracle.dijkstra_f32(ro, col, w, src),
                                          err_msg=f"{mode}")
        g.close()


def test_float_unreached_and_overflow_and_rounding_chain():
    m = gg()
    # 0 -> 1 (3e38) -> 2 (3e38): the second sum rounds to +inf; 3 unreachable
    ro = np.array([0, 1, 2, 2, 2], np.uint32)
    col = np.array([1, 2], np.uint32)
    g = m.Graph(ro, col, np.array([3e38, 3e38], np.float32), float_weights=True)
    for mode in MODES:
        assert run_f32(g, 0, mode).tolist() == [0, int(np.float32(3e38).view(np.uint32)), FMAX, FMAX]
    g.close()
    # 0 -> 1 -> 2 -> 3 with 1, 2^-24, 2^-24: rounding after every addition keeps 1.0
    ro = np.array([0, 1, 2, 3, 3], np.uint32)
    col = np.array([1, 2, 3], np.uint32)
    g = m.Graph(ro, col, np.array([1.0, 2.0 ** -24, 2.0 ** -24], np.float32), float_weights=True)
    for mode in MODES:
        assert run_f32(g, 0, mode).view(np.float32).tolist() == [0.0, 1.0, 1.0, 1.0]
    g.close()


def test_float_weights_rejected_and_unsupported_calls():
    m = gg()
    ro = np.array([0, 1, 1], np.uint32)
    col = np.array([1], np.uint32)
    for bad in (-1.0, float("nan"), float("inf"), -0.0):
        with pytest.raises(m.GGError) as ei:
            m.Graph(ro, col, np.array([bad], np.float32), float_weights=True)
        assert ei.value.status_name == "GG_ERR_INVALID_ARG"
    g = m.Graph(ro, col, np.array([2.5], np.float32), float_weights=True)
    with pytest.raises(m.GGError) as ei:
        g.sssp_batch(np.array([0], np.uint32))
    assert ei.value.status_name == "GG_ERR_NOT_SUPPORTED"
    out = torch.empty(2, dtype=torch.uint32, device="cuda")
    with pytest.raises(m.GGError) as ei:
        m.gg_sssp_multi([g.handle], np.array([0], np.uint32), [out])
    assert ei.value.status_name == "GG_ERR_NOT_SUPPORTED"
    g.close()


BFS_MODES = [("graph", "push", "warp"), ("graph", "auto", "mp"), ("graph", "pull", "mp"), ("host", "push", "bins"),
             ("persistent", "push", "warp"), ("async", "push", "warp")]


def run_bfs(g, src, mode):
    d = g.bfs(src, policy=POLICIES[mode[0]], direction=DIRS[mode[1]], lb_mode=LB[mode[2]])
    torch.cuda.synchronize()
    g.check()
    return d.cpu().numpy()


@pytest.mark.parametrize("mode", BFS_MODES)
def test_bfs_matches_oracle_hops(mode):
    m = gg()
    for seed in range(6):
        n = 30 + 40 * seed
        ro, col, w = graphgen.random_graph(n, 3 * n, 255, seed, symmetric=(seed % 2 == 1), wmin=0)
        g = m.Graph(ro, col, w)
        for src in (0, n - 1):
            np.testing.assert_array_equal(run_bfs(g, src, mode), oracle.bfs_hops(ro, col, src),
                                          err_msg=f"seed={seed} src={src}")
        g.close()
    for name in ("rmat16", "grid64"):
        ro, col, w, src = graphgen.workload(name)
        g = m.Graph(ro, col, w, symmetric=True)
        np.testing.assert_array_equal(run_bfs(g, src, mode), oracle.bfs_hops(ro, col, src))
        g.close()


def test_bfs_on_a_float_graph_and_rmat20_hops():
    m = gg()
    ro, col, _, src = graphgen.workload("rmat16")
    g = m.Graph(ro, col, symmetric_spread_weights(ro, col, 1), symmetric=True, float_weights=True)
    np.testing.assert_array_equal(run_bfs(g, src, ("graph", "push", "warp")), oracle.bfs_hops(ro, col, src))
    g.close()
    ro, col, w, src = graphgen.workload("rmat20")
    g = m.Graph(ro, col, w, symmetric=True)
    np.testing.assert_array_equal(run_bfs(g, src, ("graph", "push", "warp")), oracle.bfs_hops(ro, col, src))
    g.close()
