"""GPU parity of the multi-graph launch (gg_sssp_multi) and of the
continuous-batching server: every query's distances equal the oracle's, and
each result is the same alone (gg_sssp) and in the mix (tolerance 0)."""
import time

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


def small_pool(pack=True):
    specs = [("rmat", 10, 8, 1), ("rmat", 12, 16, 2), ("grid", 16, 0, 3), ("grid", 64, 0, 4),
             ("rmat", 11, 8, 5), ("grid", 33, 0, 6)]
    graphs = []
    for kind, a, b, seed in specs:
        ro, col, w = graphgen.rmat(a, b, seed=seed, W=255) if kind == "rmat" else graphgen.grid(a, W=255, seed=seed)
        graphs.append((ro, col, w, gg().Graph(ro, col, w, symmetric=True, pack=pack)))
    ro, col, w = graphgen.random_graph(50, 90, 40, seed=7, wmin=0)          # directed, zero weights
    graphs.append((ro, col, w, gg().Graph(ro, col, w)))
    ro = np.zeros(6, np.uint32)                                             # edgeless
    graphs.append((ro, np.zeros(0, np.uint32), np.zeros(0, np.uint32),
                   gg().Graph(ro, np.zeros(0, np.uint32), np.zeros(0, np.uint32))))
    return graphs


@pytest.mark.parametrize("pack,delta", [(True, None), (False, None), (True, 0xFFFFFFFF), (True, 1), (False, 37)])
def test_multi_matches_oracle(pack, delta):
    m = gg()
    pool = small_pool(pack)
    rng = np.random.Generator(np.random.PCG64(1))
    qs = []
    for i in range(100):                                  # more queries than 64 slots; graphs repeat
        gi = int(rng.integers(0, len(pool)))
        ro = pool[gi][0]
        qs.append((gi, int(rng.integers(0, ro.shape[0] - 1))))
    outs = [torch.empty(pool[gi][3].n, dtype=torch.uint32, device="cuda") for gi, _ in qs]
    m.gg_sssp_multi([pool[gi][3].handle for gi, _ in qs], [s for _, s in qs], outs, delta=delta)
    torch.cuda.synchronize()
    for (gi, s), d in zip(qs, outs):
        ro, col, w, _ = pool[gi]
        np.testing.assert_array_equal(d.cpu().numpy(), oracle.dijkstra(ro, col, w, s), err_msg=f"graph {gi} src {s}")
    # a second, smaller call reuses the engine
    d2 = [torch.empty(pool[i][3].n, dtype=torch.uint32, device="cuda") for i in (0, 3)]
    m.gg_sssp_multi([pool[0][3].handle, pool[3][3].handle], [3, 100], d2)
    torch.cuda.synchronize()
    for i, s, d in ((0, 3, d2[0]), (3, 100, d2[1])):
        ro, col, w, _ = pool[i]
        np.testing.assert_array_equal(d.cpu().numpy(), oracle.dijkstra(ro, col, w, s))
    for _, _, _, g in pool:
        g.close()


@pytest.mark.parametrize("delta", [0, 0xFFFFFFFF, 20])
def test_server_mixed_equals_alone_and_oracle(delta):
    m = gg()
    pool = small_pool()
    srv = m.Server(max_graph_vertices=max(g.n for *_, g in pool), max_slots=16, supersteps_per_launch=4,
                   delta=delta)
    rng = np.random.Generator(np.random.PCG64(3))
    qs, tickets, outs = [], [], []
    for i in range(150):
        gi = int(rng.integers(0, len(pool)))
        s = int(rng.integers(0, pool[gi][3].n))
        d = torch.full((pool[gi][3].n,), 7, dtype=torch.uint32, device="cuda")
        tickets.append(srv.submit(pool[gi][3], s, d))
        qs.append((gi, s))
        outs.append(d)
        if i % 37 == 0:
            time.sleep(0.002)                              # arrivals while others are in flight
    statuses = [srv.wait(t, 60000) for t in tickets]
    assert all(st == 0 for st in statuses)
    torch.cuda.synchronize()
    st = srv.stats()
    assert st["completed"] == 150 and st["p99_us"] >= st["p50_us"] > 0
    assert st["max_running"] > 1                           # queries really overlapped on the device
    for (gi, s), d in zip(qs, outs):
        ro, col, w, g = pool[gi]
        alone = g.sssp(s)
        torch.cuda.synchronize()
        got = d.cpu().numpy()
        np.testing.assert_array_equal(got, alone.cpu().numpy(), err_msg=f"mixed vs alone, graph {gi} src {s}")
        np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, s))
    srv.close()
    for *_, g in pool:
        g.close()


def test_server_poll_errors_and_budget():
    m = gg()
    ro, col, w = graphgen.grid(64, W=255, seed=1)
    g = m.Graph(ro, col, w, symmetric=True)
    # a budget of one graph at a time: queries are admitted one after another
    srv = m.Server(max_graph_vertices=g.n, max_slots=8, max_vertices_in_flight=g.n)
    outs = [torch.empty(g.n, dtype=torch.uint32, device="cuda") for _ in range(5)]
    ts = [srv.submit(g, s, d) for s, d in zip([0, 5, 100, 4095, 2000], outs)]
    for t in ts:
        assert srv.wait(t) == 0
    assert srv.stats()["max_running"] == 1
    for s, d in zip([0, 5, 100, 4095, 2000], outs):
        np.testing.assert_array_equal(d.cpu().numpy(), oracle.dijkstra(ro, col, w, s))
    with pytest.raises(m.GGError):
        srv.submit(g, g.n, outs[0])                         # src >= n
    with pytest.raises(m.GGError):
        srv.poll(123456789)                                 # unknown ticket
    big = m.Graph(*graphgen.grid(65, W=3, seed=1), symmetric=True)
    with pytest.raises(m.GGError):
        srv.submit(big, 0, torch.empty(big.n, dtype=torch.uint32, device="cuda"))   # larger than allowed
    srv.close()
    big.close()
    g.close()


def test_server_admission_follows_free_hbm():
    """Admission re-reads the device's free HBM at every round: while another
    allocation leaves less than hbm_reserve_bytes free, queued queries wait
    (the budget in force drops to the vertices in flight); once the memory is
    released they are admitted, and their distances equal the oracle's."""
    m = gg()
    ro, col, w = graphgen.grid(64, W=255, seed=1)
    g = m.Graph(ro, col, w, symmetric=True)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    reserve = free - (512 << 20)                  # about 512 MiB above the reserve
    srv = m.Server(max_graph_vertices=g.n, max_slots=8, hbm_reserve_bytes=reserve)
    free2, _ = torch.cuda.mem_get_info()
    hog = torch.empty(free2 - reserve + (64 << 20), dtype=torch.uint8, device="cuda")   # 64 MiB below the reserve
    torch.cuda.synchronize()
    srcs = [0, 77, 4095]
    outs = [torch.empty(g.n, dtype=torch.uint32, device="cuda") for _ in srcs]
    ts = [srv.submit(g, s, d) for s, d in zip(srcs, outs)]
    time.sleep(0.3)
    st = srv.stats()
    assert st["running"] == 0 and st["queued"] == len(srcs) and st["completed"] == 0
    assert st["vertex_budget"] == 0
    assert all(srv.poll(t) is None for t in ts)
    del hog
    torch.cuda.empty_cache()                      # hand the memory back to the driver
    for t in ts:
        assert srv.wait(t, 60000) == 0
    for s, d in zip(srcs, outs):
        np.testing.assert_array_equal(d.cpu().numpy(), oracle.dijkstra(ro, col, w, s))
    assert srv.stats()["vertex_budget"] > 0
    srv.close()
    g.close()
