"""GPU parity of the edge-frontier program (gg_sssp_tree) against the
oracle's sp_tree: the same predecessor for every vertex (bit-exact) and the
same set of tight edges (compared as sets: the edge frontier has no order)."""
import numpy as np
import pytest

import graphgen
import oracle
from golden_io import hand_fixtures, load

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def gg():
    import paper_2212_08200_b300 as m
    m.load()
    return m


def run_tree(g, src, cap=None, dist=None):
    m = gg()
    if dist is None:
        dist = g.sssp(src)
    parent = torch.empty(g.n, dtype=torch.uint32, device="cuda")
    cap = g.m if cap is None else cap
    tight = torch.empty(max(cap, 1), dtype=torch.uint32, device="cuda") if cap else None
    cnt = m.gg_sssp_tree(g.handle, src, dist, parent, tight)
    kept = min(cnt, cap)
    return (parent.cpu().numpy(), np.sort(tight[:kept].cpu().numpy()) if cap else None, cnt,
            dist.cpu().numpy())


def check(ro, col, w, src, g, cap=None):
    parent, tight, cnt, dist = run_tree(g, src, cap)
    ref = oracle.dijkstra(ro, col, w, src)
    np.testing.assert_array_equal(dist, ref)
    rp, rt = oracle.sp_tree(ro, col, w, src, ref)
    np.testing.assert_array_equal(parent, rp)
    assert cnt == int(rt.sum())
    if tight is not None and (cap is None or cap >= cnt):
        np.testing.assert_array_equal(tight, np.flatnonzero(rt).astype(np.uint32))
    return cnt


@pytest.mark.parametrize("name", ["rmat16", "grid64"])
@pytest.mark.parametrize("pack", [True, False])
def test_workloads_match_oracle(name, pack):
    ro, col, w, src = graphgen.workload(name)
    g = gg().Graph(ro, col, w, symmetric=True, pack=pack)
    for s in (src, int(graphgen.sample_sources(ro, 1, seed=3)[0])):
        check(ro, col, w, s, g)
    g.close()


@pytest.mark.parametrize("seed", range(4))
def test_directed_zero_weights_sinks(seed):
    """Zero weights make ties (several tight in-edges, equal-distance cycles);
    sinks and unreached vertices get no parent."""
    ro, col, w = graphgen.random_graph(3000, 12000, 6, seed, wmin=0)
    g = gg().Graph(ro, col, w)
    deg = np.diff(ro.astype(np.int64))
    for s in (int(np.argmax(deg)), int(np.flatnonzero(deg == 0)[0]) if (deg == 0).any() else 0):
        check(ro, col, w, s, g)
    g.close()


@pytest.mark.parametrize("name", [f for f in hand_fixtures() if "overflow" not in f])
def test_hand_fixtures(name):
    fx = load(name)
    g = gg().Graph(fx["ro"], fx["col"], fx["w"])
    check(fx["ro"], fx["col"], fx["w"], fx["src"], g)
    g.close()


def test_truncated_and_absent_edge_list():
    """A tight_out smaller than the frontier keeps a prefix of valid tight
    edges and reports the full count; without tight_out only parents come
    back."""
    ro, col, w, src = graphgen.workload("grid64")
    g = gg().Graph(ro, col, w, symmetric=True)
    full = check(ro, col, w, src, g)
    parent, tight, cnt, _ = run_tree(g, src, cap=100)
    assert cnt == full and tight.shape[0] == 100
    _, rt = oracle.sp_tree(ro, col, w, src, oracle.dijkstra(ro, col, w, src))
    assert np.all(rt[tight])
    parent0, _, cnt0, _ = run_tree(g, src, cap=0)
    assert cnt0 == full
    np.testing.assert_array_equal(parent0, parent)
    g.close()


def test_rmat22_full_size():
    """The RMAT-22 workload from its hub: every parent and the tight-edge
    count equal the oracle's."""
    ro, col, w, src = graphgen.workload("rmat22")
    g = gg().Graph(ro, col, w, symmetric=True)
    check(ro, col, w, src, g)
    g.close()
