"""GPU parity of the light/heavy bucket variant (Meyer-Sanders delta-stepping
on top of the near-far frontier split) of the bulk-synchronous SSSP loop.

Near supersteps relax only light edges (weight < delta); each vertex that
settles into a bucket has its heavy edges relaxed once, by a heavy superstep.
Distances are unique, so every width, load balance and policy must equal the
oracle bit for bit, and the variant must scan fewer edges than the plain
near-far split of the same width.
"""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NONE = 0xFFFFFFFF
POL = {"graph": 0, "host": 2, "persistent": 3, "async": 1}
LB = {"mp": 1, "bins": 2, "warp": 3}
HEAVY = (3, 4, 5)   # trace kinds of a heavy-edge superstep (push, pull, pull that ends bucketing)


def gg():
    import paper_2212_08200_b300 as m
    m.load()
    return m


def run(g, src, delta=0, lb="warp", policy="graph", lh=0, direction=1, trace_cap=0):
    m = gg()
    st = m.gg_stats()
    kw = {}
    tr = None
    if trace_cap:
        tr = torch.zeros(4 * trace_cap, dtype=torch.uint32, device="cuda")
        kw = {"trace": tr, "trace_cap": trace_cap}
    d = g.sssp(src, policy=POL[policy], direction=direction, lb_mode=LB[lb], delta=delta, light_heavy=lh, stats=st,
               **kw)
    torch.cuda.synchronize()
    kinds = None
    if tr is not None:
        kinds = tr.cpu().numpy().reshape(-1, 4)[: st.iterations, 2]
    return d.cpu().numpy(), st.as_dict(), kinds


@pytest.mark.parametrize("lb", ["warp", "mp", "bins"])
@pytest.mark.parametrize("policy", ["graph", "host"])
@pytest.mark.parametrize("delta", [1, 2, 9, 32, 100, 255, 256, 0])
def test_widths_and_load_balances_match_oracle(delta, policy, lb):
    ro, col, w, src = graphgen.workload("rmat16")
    g = gg().Graph(ro, col, w, symmetric=True)
    for s in (src, int(graphgen.sample_sources(ro, 1, seed=11)[0])):
        ref = oracle.dijkstra(ro, col, w, s)
        got, st, kinds = run(g, s, delta, lb, policy, trace_cap=8192)
        np.testing.assert_array_equal(got, ref, err_msg=f"delta={delta} {policy} {lb} src={s}")
        assert st["device_status"] == 0
        # delta <= the largest weight leaves heavy edges: heavy supersteps run;
        # 256 > 255 makes every edge light, so the plain near-far loop runs
        if delta == 256:
            assert not np.isin(kinds, HEAVY).any()
        else:
            assert np.isin(kinds, HEAVY).any()
    g.close()


def test_scans_fewer_edges_than_near_far_and_bellman_ford():
    ro, col, w, src = graphgen.workload("rmat18")
    g = gg().Graph(ro, col, w, symmetric=True)
    ref = oracle.dijkstra(ro, col, w, src)
    got_lh, st_lh, _ = run(g, src, 32)
    got_nf, st_nf, _ = run(g, src, 32, lh=1)
    got_bf, st_bf, _ = run(g, src, NONE)
    for got in (got_lh, got_nf, got_bf):
        np.testing.assert_array_equal(got, ref)
    m_trav = oracle.traversed_edges(ro, ref)
    assert st_lh["edges_scanned"] < st_nf["edges_scanned"] < st_bf["edges_scanned"]
    assert st_lh["edges_scanned"] < 1.6 * m_trav
    g.close()


def test_push_and_pull_heavy_supersteps_agree():
    """A symmetric graph declared directed takes the push form of the heavy
    superstep (its transpose is separate), the symmetric one may pull."""
    ro, col, w, src = graphgen.workload("rmat18")
    ref = oracle.dijkstra(ro, col, w, src)
    kinds_seen = set()
    for sym in (True, False):
        g = gg().Graph(ro, col, w, symmetric=sym)
        for delta in (0, 8, 24):
            got, st, kinds = run(g, src, delta, trace_cap=4096)
            np.testing.assert_array_equal(got, ref, err_msg=f"sym={sym} delta={delta}")
            kinds_seen |= set(int(k) for k in kinds)
            if not sym:
                assert not {4, 5} & set(int(k) for k in kinds)
        g.close()
    assert 3 in kinds_seen and {4, 5} & kinds_seen


def test_width_changes_rebuild_the_partition():
    ro, col, w, src = graphgen.workload("rmat16")
    for pack in (True, False):
        g = gg().Graph(ro, col, w, symmetric=True, pack=pack)
        ref = oracle.dijkstra(ro, col, w, src)
        for delta in (16, 40, 16, 3, 0, 40):
            got, _, _ = run(g, src, delta)
            np.testing.assert_array_equal(got, ref, err_msg=f"pack={pack} delta={delta}")
        # the graph's own edge order is untouched: other paths still agree
        got, _, _ = run(g, src, NONE, policy="async", direction=0)
        np.testing.assert_array_equal(got, ref)
        D = g.sssp_batch(np.array([src, 5, 77], np.uint32))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(D.cpu().numpy().reshape(g.n, 3)[:, 0], ref)
        g.close()


def test_directed_graph_with_sinks_and_zero_weights():
    for seed in range(4):
        ro, col, w = graphgen.random_graph(3000, 15000, 60, seed=seed, wmin=0)
        g = gg().Graph(ro, col, w, symmetric=False)
        sinks = int(((np.diff(ro.astype(np.int64)) == 0)).sum())
        assert sinks > 0
        for delta in (1, 5, 30):
            for lb in ("warp", "mp"):
                for s in (0, 1999):
                    got, _, _ = run(g, s, delta, lb)
                    np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, s),
                                                  err_msg=f"seed={seed} delta={delta} {lb} src={s}")
        g.close()


def test_source_without_light_edges_starts_with_a_heavy_step():
    n = 5000
    wts = np.random.Generator(np.random.PCG64(4)).integers(50, 200, n - 1)
    ro, col, w = graphgen.star_graph(n, wts)
    g = gg().Graph(ro, col, w, symmetric=True)
    for src in (0, 17):
        got, st, kinds = run(g, src, 40, trace_cap=64)
        np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, src))
        if src == 0:
            assert kinds[0] == 3           # a star has no unsettled core: push
    g.close()


def test_long_path_and_grid_with_small_widths():
    wts = np.random.Generator(np.random.PCG64(8)).integers(0, 30, 3999)
    ro, col, w = graphgen.path_graph(4000, wts)
    g = gg().Graph(ro, col, w)
    for delta in (1, 7, 29):
        got, _, _ = run(g, 0, delta)
        np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, 0))
    g.close()
    ro, col, w = graphgen.grid(100, 64, 3)
    g = gg().Graph(ro, col, w, symmetric=True)
    ref = oracle.dijkstra(ro, col, w, 0)
    for delta in (4, 33, 64):
        got, _, _ = run(g, 0, delta)
        np.testing.assert_array_equal(got, ref)
    g.close()


def test_other_policies_and_directions_keep_plain_buckets():
    ro, col, w, src = graphgen.workload("rmat16")
    g = gg().Graph(ro, col, w, symmetric=True)
    ref = oracle.dijkstra(ro, col, w, src)
    for policy, direction in (("persistent", 1), ("graph", 0), ("host", 2)):
        got, _, kinds = run(g, src, 20, policy=policy, direction=direction, trace_cap=4096)
        np.testing.assert_array_equal(got, ref)
        assert not np.isin(kinds, HEAVY).any()
    g.close()


def test_rmat20_default_width_is_light_heavy():
    ro, col, w, src = graphgen.workload("rmat20")
    g = gg().Graph(ro, col, w, symmetric=True)
    ref = oracle.dijkstra(ro, col, w, src)
    got, st, kinds = run(g, src, 0, trace_cap=4096)
    np.testing.assert_array_equal(got, ref)
    assert np.isin(kinds, HEAVY).any()
    got2, st2, _ = run(g, src, NONE)
    np.testing.assert_array_equal(got2, ref)
    assert st["edges_scanned"] < st2["edges_scanned"]
    g.close()


def _sink_graph(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    n, m = 6000, 90000
    src = rng.integers(0, 5000, m)             # vertices 5000.. have no out-edges (sinks)
    dst = rng.integers(0, n, m)
    return graphgen.from_edges(n, src, dst, rng.integers(0, 120, m))


@pytest.mark.parametrize("lb", ["warp", "mp", "bins"])
@pytest.mark.parametrize("graph", ["rmat18", "sinks"])
def test_plain_push_once_bucketing_ends(graph, lb):
    # once the unsettled vertices hold few heavy edges the threshold becomes
    # infinite, and every superstep after that is a plain push (kind 0) over
    # all edges of each vertex
    if graph == "rmat18":
        ro, col, w, src = graphgen.workload("rmat18")
        g = gg().Graph(ro, col, w, symmetric=True)
        cases = [(src, 0), (int(graphgen.sample_sources(ro, 1, seed=5)[0]), 0)]
    else:
        ro, col, w = _sink_graph(13)
        g = gg().Graph(ro, col, w, symmetric=False)
        cases = [(0, 20), (4321, 40)]
    ended = 0
    for s, delta in cases:
        got, st, kinds = run(g, s, delta, lb, trace_cap=8192)
        np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, s), err_msg=f"{graph} {lb} src={s}")
        assert st["device_status"] == 0
        # the threshold becomes infinite at a split, or at a heavy pull that
        # writes the plain tail's frontier itself (kind 5, no split after it)
        ends = np.flatnonzero((kinds == 2) | (kinds == 5))
        if ends.size and not np.isin(kinds[ends[-1] + 1:], HEAVY).any():
            tail = kinds[ends[-1] + 1:]
            assert (tail == 0).all(), kinds
            ended += tail.size > 0
    assert ended > 0   # the plain tail ran in at least one case
    g.close()


def test_heavy_pull_that_ends_bucketing_writes_the_tail_frontier():
    """From an RMAT hub the dense core settles in the first bucket; once its
    heavy pull leaves fewer than m / 8 heavy edges unsettled, that pull ends
    bucketing itself (kind 5): its next frontier is every unsettled vertex
    with a finite distance, and only plain pushes follow (no split).  It runs
    as soon as the bucket's light frontier is small (at most n / 256
    vertices), taking that frontier along."""
    early = 0
    for name in ("rmat18", "rmat20"):
        ro, col, w, src = graphgen.workload(name)
        g = gg().Graph(ro, col, w, symmetric=True)
        for policy in ("graph", "host"):
            trace = torch.zeros(4 * 4096, dtype=torch.uint32, device="cuda")
            m = gg()
            st = m.gg_stats()
            d = g.sssp(src, policy=POL[policy], direction=1, lb_mode=LB["warp"], stats=st, trace=trace,
                       trace_cap=4096)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(d.cpu().numpy(), oracle.dijkstra(ro, col, w, src),
                                          err_msg=f"{name} {policy}")
            tr = trace.cpu().numpy().reshape(-1, 4)[: st.iterations]
            kinds = tr[:, 2]
            k5 = np.flatnonzero(kinds == 5)
            assert k5.size == 1, kinds
            rest = kinds[k5[0] + 1:]
            assert rest.size > 0 and (rest == 0).all(), kinds
            assert tr[k5[0], 3] > 0 and tr[k5[0] + 1, 0] == tr[k5[0], 3]
            assert st.device_status == 0
            early += int(k5[0] > 0 and tr[k5[0] - 1, 3] > 0)   # a light frontier was still left
        g.close()
    assert early > 0


def test_bad_light_heavy_value_is_rejected():
    m = gg()
    ro, col, w, src = graphgen.workload("grid64")
    g = m.Graph(ro, col, w, symmetric=True)
    with pytest.raises(m.GGError) as ei:
        g.sssp(src, light_heavy=3)
    assert ei.value.status_name == "GG_ERR_INVALID_ARG"
    with pytest.raises(m.GGError) as ei:
        g.sssp_batch(np.array([src], np.uint32), light_heavy=3)
    assert ei.value.status_name == "GG_ERR_INVALID_ARG"
    d = g.sssp(src, light_heavy=m.GG_LH_ROUNDS)        # the batch-only schedule: single source runs as AUTO
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d.cpu().numpy(), oracle.dijkstra(ro, col, w, src))
    g.close()


# ---- batched multi-source: light-first rounds ---------------------------------

def run_batch(g, srcs, **kw):
    m = gg()
    st = m.gg_stats()
    d = g.sssp_batch(srcs, stats=st, **kw)
    torch.cuda.synchronize()
    return d.cpu().numpy(), st.as_dict()


@pytest.mark.parametrize("k,pack,policy", [(3, True, 0), (64, True, 0), (70, False, 0), (64, False, 2)])
def test_batch_light_first_rounds_match_oracle(k, pack, policy):
    ro, col, w, _ = graphgen.workload("rmat16")
    srcs = graphgen.sample_sources(ro, k, seed=21)
    g = gg().Graph(ro, col, w, symmetric=True, pack=pack)
    ref = oracle.dijkstra_many(ro, col, w, srcs, threads=8)
    got, st = run_batch(g, srcs, policy=policy)
    got_off, st_off = run_batch(g, srcs, policy=policy, light_heavy=1)
    for s in range(k):
        np.testing.assert_array_equal(got[:, s], ref[s], err_msg=f"column {s}")
        np.testing.assert_array_equal(got_off[:, s], ref[s], err_msg=f"column {s} (light/heavy off)")
    assert st["device_status"] == 0
    assert st["edges_scanned"] < st_off["edges_scanned"]
    g.close()


def test_batch_directed_sinks_zero_weights_and_heavy_only_sources():
    rng = np.random.Generator(np.random.PCG64(31))
    n, m = 4000, 60000
    src = rng.integers(0, 3500, m)             # vertices 3500.. have no out-edges (sinks)
    dst = rng.integers(0, n, m)
    w = rng.integers(0, 80, m)
    ro, col, wt = graphgen.from_edges(n, src, dst, w)
    # a source whose every edge is heavy starts with a heavy superstep
    hv = 7
    wt[ro[hv]:ro[hv + 1]] = 79
    g = gg().Graph(ro, col, wt, symmetric=False)
    srcs = np.array([hv, 0, 3999, 1234, hv, 42], np.uint32)
    ref = oracle.dijkstra_many(ro, col, wt, srcs)
    got, st = run_batch(g, srcs)
    np.testing.assert_array_equal(got.T, ref)
    assert st["device_status"] == 0
    g.close()


def test_batch_after_single_source_runs_with_other_widths():
    """The light-first copy is shared: a single-source run with another width
    re-partitions it, and the next batch re-partitions it back."""
    ro, col, w, src = graphgen.workload("rmat16")
    g = gg().Graph(ro, col, w, symmetric=True)
    srcs = graphgen.sample_sources(ro, 8, seed=2)
    ref = oracle.dijkstra_many(ro, col, w, srcs)
    for delta in (40, 0, 3):
        got1, _, _ = run(g, int(srcs[0]), delta)
        np.testing.assert_array_equal(got1, ref[0])
        got, _ = run_batch(g, srcs)
        np.testing.assert_array_equal(got.T, ref)
    g.close()


def test_create_run_destroy_cycles_reuse_pooled_memory():
    """Handles allocate from a pool that keeps freed memory: repeated create /
    run / destroy cycles (host and device inputs, packed and 8-byte edges,
    directed and symmetric) stay exact and do not grow the device footprint."""
    m = gg()
    ro, col, w, src = graphgen.workload("rmat16")
    ref = oracle.dijkstra(ro, col, w, src)
    dev = [torch.from_numpy(a.view(np.int32)).cuda().view(torch.uint32) for a in (ro, col, w)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for cycle in range(12):
        args = dev if cycle % 3 == 1 else (ro, col, w)
        g = m.Graph(*args, symmetric=cycle % 2 == 0, pack=cycle % 4 != 3)
        got, st, _ = run(g, src, 0)
        np.testing.assert_array_equal(got, ref, err_msg=f"cycle {cycle}")
        D = g.sssp_batch(np.array([src, 3], np.uint32))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(D.cpu().numpy().reshape(g.n, 2)[:, 0], ref)
        g.close()
    torch.cuda.synchronize()
    # the pool keeps at most a bounded amount mapped: far below 12 handles' worth
    assert free0 - torch.cuda.mem_get_info()[0] < 2 << 30
