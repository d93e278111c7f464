"""CPU models of the batched schedules, checked against the oracle.

Light-first rounds (``rounds``): k sources share one loop with no distance
threshold: a (source, vertex) pair that improves joins the next light
frontier (its light edges) and the current epoch's R mask (its heavy edges);
when the light frontier is empty, one heavy superstep relaxes the heavy edges
of the R pairs, and its improvements start the next epoch.

Normalised buckets (``normalised_buckets``, the default batched schedule on
skewed graphs): the same light/heavy rounds inside one shared bucket
threshold T over shifted distances dist[s][v] + sh[s], sh[s] = max o - o_s
with o_s the source's distance from the hub.  Pairs at or above T are parked;
when no near pair and no R pair is left, T rises to max(T + width, smallest
parked shifted distance + 1) and a split moves the parked pairs below it into
the frontier; once the pairs not yet settled hold fewer than 1/drain of the
heavy edges (counted per pair when it first joins an R mask), T becomes
infinite and the rest is plain push over all edges.  When the heavy
superstep before that split is a pull, the pull itself starts the plain
push (the kernel's default): every pair not settled with a finite distance
forms the tail's first frontier, and no split follows.

The models take these steps in this order (synchronous relaxation per
superstep) and must reach the oracle's distances for every source, whatever
the offsets.  No GPU is involved.
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


def normalised_buckets(ro, col, w, srcs, delta, offs, width=None, drain=8, mistake=None, pull=False,
                       pull_tail=False):
    """(k, n) distances, supersteps and splits of the normalised-bucket
    schedule.  mistake (for the pin-strength test only) plants one error:
    "split_floor" drops the pairs at exactly the previous threshold,
    "split_no_r" leaves the pairs a split releases out of the R mask,
    "tail_light" gives the tail light rows only, "pull_tail_parked" gives the
    tail only the pairs the ending pull improved.  pull: heavy supersteps
    update only the pairs not yet settled (as the kernel's pull does).
    pull_tail: a pull after which the drain rule holds ends the buckets
    itself (no split): every pair not settled with a finite distance starts
    the tail."""
    ro = np.asarray(ro, np.int64)
    n, k = ro.size - 1, len(srcs)
    width = delta if width is None else width
    deg = np.diff(ro)
    rowid = np.repeat(np.arange(n), deg)
    w = np.asarray(w, np.int64)
    order = np.lexsort((w >= delta, rowid))
    c2 = np.asarray(col, np.int64)[order]
    w2 = w[order]
    nl = np.bincount(rowid, weights=(w < delta), minlength=n).astype(np.int64)
    lend = ro[:-1] + nl
    ldeg, hdeg = nl, deg - nl
    offs = np.where(np.asarray(offs, np.int64) >= INF32, 0, np.asarray(offs, np.int64))
    sh = offs.max() - offs
    heavy_k = int(hdeg.sum()) * k
    dist = np.full((k, n), BIG)
    F = np.zeros((k, n), bool)
    R = np.zeros((k, n), bool)
    far = np.zeros((k, n), bool)
    T, tprev, tail, settled, steps, splits = width, 0, False, 0, 0, 0
    for s, v in enumerate(srcs):
        dist[s, v] = 0
        if deg[v] == 0:
            continue
        if sh[s] >= T:
            far[s, v] = True
        else:
            F[s, v] |= ldeg[v] > 0
            if hdeg[v] > 0:
                settled += int(hdeg[v])
                R[s, v] = True

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

    def place(imp):
        nonlocal settled
        if tail:
            return imp & (deg > 0), np.zeros_like(imp)
        near = imp & (dist + sh[:, None] < T)
        newr = near & (hdeg > 0) & ~R
        settled += int((newr * hdeg[None, :]).sum())
        far_new = imp & ~near & (deg > 0)
        return near, far_new

    if not F.any() and not R.any() and far.any():          # every source parked
        T = int((dist + sh[:, None])[far].min()) + 1
        F = np.zeros((k, n), bool)
        split_due = True
    else:
        split_due = False
    while True:
        if split_due:
            splits += 1
            steps += 1
            shifted = dist + sh[:, None]
            mv = far & ((shifted > tprev) if mistake == "split_floor" else (shifted >= tprev)) & (shifted < T)
            keep = far & (shifted >= T)
            far = keep
            if tail:
                F = mv & (deg > 0)
            else:
                F = mv & (ldeg > 0)
                newr = mv & (hdeg > 0) & ~R
                settled += int((newr * hdeg[None, :]).sum())
                if mistake != "split_no_r":
                    R |= mv & (hdeg > 0)
            split_due = False
        elif F.any():
            steps += 1
            imp = relax(F, ro[:-1], ro[1:] if (tail and mistake != "tail_light") else lend)
            near, fnew = place(imp)
            far |= fnew
            F = near & ((deg > 0) if tail else (ldeg > 0))
            if not tail:
                R |= near & (hdeg > 0)
        elif R.any():
            steps += 1
            if pull:
                # the heavy superstep by pull writes only the pairs not yet
                # settled (shifted distance at or above the threshold)
                keep = dist.copy()
                open_ = dist + sh[:, None] >= T
                imp = relax(R, lend, ro[1:])
                dist[:] = np.where(open_, dist, keep)
                imp &= open_
                # a pull settles no pair: the drain rule after it is decided now
                if pull_tail and not tail and heavy_k - settled < heavy_k // drain:
                    if mistake == "pull_tail_parked":
                        F = imp & (deg > 0)
                    else:
                        F = open_ & (dist < BIG) & (deg > 0)
                    R = np.zeros((k, n), bool)
                    far = np.zeros((k, n), bool)
                    tail, tprev, T = True, T, BIG
                    continue
            else:
                imp = relax(R, lend, ro[1:])
            R = np.zeros((k, n), bool)
            near, fnew = place(imp)
            far |= fnew
            F = near & (ldeg > 0)
            R = near & (hdeg > 0)
        elif far.any():
            shifted = dist + sh[:, None]
            tn = max(T + width, int(shifted[far].min()) + 1)
            if tail or heavy_k - settled < heavy_k // drain:
                tail, tn = True, None
            tprev, T = T, (BIG if tn is None else tn)
            split_due = True
        else:
            break
    return np.where(dist >= BIG, INF32, dist).astype(np.uint32), steps, splits


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


@pytest.mark.parametrize("scale,delta,k,width,drain,pull", [(10, 12, 16, None, 8, False), (11, 14, 9, None, 2, False),
                                                            (11, 20, 64, 40, 8, False), (12, 12, 33, None, 1000, False),
                                                            (10, 12, 16, None, 8, True), (12, 12, 33, None, 1000, True)])
def test_normalised_buckets_match_oracle(scale, delta, k, width, drain, pull):
    """Hub offsets from the oracle's own Dijkstra (the kernel takes them from
    its single-source run): every source's distances equal the oracle's."""
    ro, col, w = graphgen.rmat(scale, 16, seed=scale + 1, W=255)
    srcs = graphgen.sample_sources(ro, k, seed=5)
    hub = int(np.argmax(np.diff(ro.astype(np.int64))))
    offs = oracle.dijkstra(ro, col, w, hub)[srcs]
    got, steps, splits = normalised_buckets(ro, col, w, srcs, delta, offs, width, drain, pull=pull)
    np.testing.assert_array_equal(got, oracle.dijkstra_many(ro, col, w, srcs))
    assert splits >= 1


def test_normalised_buckets_any_offsets_directed_sinks_zero_weights():
    """Offsets change only the order of the relaxations: random offsets, a
    directed graph with sinks and zero weights, a sink source, a heavy-only
    source and a repeated one still give the oracle's distances."""
    rng = np.random.Generator(np.random.PCG64(4))
    n, m = 2500, 30000
    src = rng.integers(0, 2000, m)
    ro, col, w = graphgen.from_edges(n, src, rng.integers(0, n, m), rng.integers(0, 80, m))
    hv = 11
    w = w.copy()
    w[ro[hv]:ro[hv + 1]] = 79
    srcs = np.array([hv, 0, 2499, 1234, hv, 77], np.uint32)
    for trial, delta in enumerate((1, 20, 79)):
        offs = rng.integers(0, 300, srcs.size)
        offs[trial] = INF32                      # a source the hub does not reach: offset 0
        got, _, _ = normalised_buckets(ro, col, w, srcs, delta, offs)
        np.testing.assert_array_equal(got, oracle.dijkstra_many(ro, col, w, srcs), err_msg=f"delta={delta}")


@pytest.mark.parametrize("mistake", ["split_floor", "split_no_r", "tail_light"])
def test_normalised_buckets_planted_mistakes_fail(mistake):
    """Each planted mistake in the split or the tail makes the model miss
    distances on the same inputs where the correct model matches."""
    ro, col, w = graphgen.rmat(11, 16, seed=11, W=255)
    srcs = graphgen.sample_sources(ro, 24, seed=5)
    hub = int(np.argmax(np.diff(ro.astype(np.int64))))
    offs = oracle.dijkstra(ro, col, w, hub)[srcs]
    ref = oracle.dijkstra_many(ro, col, w, srcs)
    got, _, _ = normalised_buckets(ro, col, w, srcs, 12, offs)
    np.testing.assert_array_equal(got, ref)
    bad, _, _ = normalised_buckets(ro, col, w, srcs, 12, offs, mistake=mistake)
    assert not np.array_equal(bad, ref)


@pytest.mark.parametrize("scale,delta,k", [(10, 12, 16), (11, 14, 9), (12, 12, 24)])
def test_pull_that_ends_the_buckets_replaces_mask_clear_and_split(scale, delta, k):
    # the pull after which the drain rule holds starts the tail itself: the same
    # distances as the split after the pull, in fewer supersteps and one split fewer
    ro, col, w = graphgen.rmat(scale, 16, seed=scale, W=255)
    hub = graphgen.max_degree_vertex(ro)
    srcs = graphgen.sample_sources(ro, k, seed=3)
    offs = oracle.dijkstra(ro, col, w, hub)[srcs]
    ref = oracle.dijkstra_many(ro, col, w, srcs)
    got_t, steps_t, splits_t = normalised_buckets(ro, col, w, srcs, delta, offs, pull=True, pull_tail=True)
    got_s, steps_s, splits_s = normalised_buckets(ro, col, w, srcs, delta, offs, pull=True)
    np.testing.assert_array_equal(got_t, ref)
    np.testing.assert_array_equal(got_s, ref)
    assert splits_t < splits_s and steps_t < steps_s


def test_pull_that_ends_the_buckets_planted_mistake_fails():
    # starting the tail from only the pairs the pull improved (dropping the
    # pairs parked earlier) must be caught by the oracle comparison
    caught = False
    for scale, delta, k in ((10, 12, 16), (11, 14, 9), (12, 12, 24)):
        ro, col, w = graphgen.rmat(scale, 16, seed=scale, W=255)
        hub = graphgen.max_degree_vertex(ro)
        srcs = graphgen.sample_sources(ro, k, seed=3)
        offs = oracle.dijkstra(ro, col, w, hub)[srcs]
        got, _, _ = normalised_buckets(ro, col, w, srcs, delta, offs, pull=True, pull_tail=True,
                                       mistake="pull_tail_parked")
        caught |= not np.array_equal(got, oracle.dijkstra_many(ro, col, w, srcs))
    assert caught
