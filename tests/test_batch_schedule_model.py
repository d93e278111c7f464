"""CPU model of the batched light-first rounds, checked against the oracle.

k sources share one loop with no distance threshold: a (source, vertex) pair
that improves joins the next light frontier (its light edges) and the current
epoch's R mask (its heavy edges); when the light frontier is empty, one heavy
superstep relaxes the heavy edges of the R pairs, and its improvements start
the next epoch.  The model takes these steps in this order (synchronous
relaxation per superstep) and must reach the oracle's distances for every
source.  No GPU is involved.
"""
import numpy as np
import pytest

import graphgen
import oracle

BIG = np.int64(1) << 40
INF32 = 0xFFFFFFFF


def rounds(ro, col, w, srcs, delta):
    """(k, n) distances (uint32, INF32 = unreached), light and heavy superstep counts."""
    ro = np.asarray(ro, np.int64)
    n, k = ro.size - 1, len(srcs)
    deg = np.diff(ro)
    rowid = np.repeat(np.arange(n), deg)
    w = np.asarray(w, np.int64)
    order = np.lexsort((w >= delta, rowid))   # light edges first in each row
    c2 = np.asarray(col, np.int64)[order]
    w2 = w[order]
    nl = np.bincount(rowid, weights=(w < delta), minlength=n).astype(np.int64)
    lend = ro[:-1] + nl
    ldeg, hdeg = nl, deg - nl
    dist = np.full((k, n), BIG)
    F = np.zeros((k, n), bool)
    R = np.zeros((k, n), bool)
    for s, v in enumerate(srcs):
        dist[s, v] = 0
        F[s, v] = ldeg[v] > 0
        R[s, v] = hdeg[v] > 0

    def relax(S, lo, hi):
        imp = np.zeros((k, n), bool)
        for s in range(k):
            us = np.flatnonzero(S[s])
            cnt = hi[us] - lo[us]
            tot = int(cnt.sum())
            if tot == 0:
                continue
            own = np.repeat(us, cnt)
            e = np.repeat(lo[us] - np.concatenate(([0], np.cumsum(cnt)[:-1])), cnt) + np.arange(tot)
            best = np.full(n, BIG)
            np.minimum.at(best, c2[e], dist[s, own] + w2[e])
            better = best < dist[s]
            dist[s, better] = best[better]
            imp[s] = better
        return imp

    light = heavy = 0
    while True:
        if F.any():
            light += 1
            imp = relax(F, ro[:-1], lend)
            F = imp & (ldeg > 0)
            R |= imp & (hdeg > 0)
        elif R.any():
            heavy += 1
            imp = relax(R, lend, ro[1:])
            F = imp & (ldeg > 0)
            R = imp & (hdeg > 0)   # the next epoch's R mask
        else:
            break
    return np.where(dist >= BIG, INF32, dist).astype(np.uint32), light, heavy


@pytest.mark.parametrize("scale,delta,k", [(10, 12, 16), (11, 14, 9), (11, 60, 5)])
def test_rmat_rounds_match_oracle(scale, delta, k):
    ro, col, w = graphgen.rmat(scale, 16, seed=scale, W=255)
    srcs = graphgen.sample_sources(ro, k, seed=3)
    got, light, heavy = rounds(ro, col, w, srcs, delta)
    np.testing.assert_array_equal(got, oracle.dijkstra_many(ro, col, w, srcs))
    assert heavy >= 1 and light >= 1


@pytest.mark.parametrize("seed", [0, 1])
def test_directed_sinks_zero_weights_and_heavy_only_sources(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    n, m = 2500, 30000
    src = rng.integers(0, 2000, m)   # vertices 2000.. have no out-edges
    ro, col, w = graphgen.from_edges(n, src, rng.integers(0, n, m), rng.integers(0, 80, m))
    hv = 11
    w = w.copy()
    w[ro[hv]:ro[hv + 1]] = 79        # a source whose every edge is heavy
    srcs = np.array([hv, 0, 2499, 1234, hv], np.uint32)   # a sink and a repeated source
    for delta in (1, 20, 79):
        got, _, _ = rounds(ro, col, w, srcs, delta)
        np.testing.assert_array_equal(got, oracle.dijkstra_many(ro, col, w, srcs), err_msg=f"delta={delta}")
