"""CPU model of the single-source light/heavy superstep schedule, checked
against the oracle.

The GPU loop orders the paper's relaxations (Listing 4) with Meyer-Sanders
buckets:
- light supersteps relax the light edges (weight < delta) of the near frontier;
- each vertex that settles into a bucket joins an R list once per epoch;
- a heavy superstep relaxes R's heavy edges, by push, or on symmetric graphs by
  pull into the unsettled vertices;
- a split raises the threshold past the smallest parked distance;
- once the unsettled vertices hold fewer than m / 8 heavy edges, the threshold
  becomes infinite, and the rest of the run is plain push over all edges;
- when a heavy pull is what brings them below that share, the pull itself
  ends bucketing: every unsettled vertex with a finite distance forms the
  plain push's first frontier, and no split follows;
- that pull may run before the bucket's light frontier empties, once the
  frontier holds at most n / 256 vertices: the frontier joins the plain push's
  first frontier with whole rows.

This model takes the same decisions superstep by superstep (synchronous
relaxation within a superstep, which reaches the same fixed point as the
kernel's atomics). It checks that the schedule itself, including the switch
to plain push, yields the shortest distances on graphs of every shape. It
also checks that the switch removes supersteps without changing any
distance. No GPU is involved.
"""
import numpy as np
import pytest

import graphgen
import oracle

BIG = np.int64(1) << 40
INF32 = 0xFFFFFFFF
LIGHT, SPLIT, HEAVY_PUSH, HEAVY_PULL, HEAVY_PULL_TAIL = 0, 2, 3, 4, 5


def schedule(ro, col, w, src, delta, symmetric, drain_div=8, tail=True, lh=True, pull_tail=True, early_div=256):
    """Distances (uint32, INF32 = unreached) and the kind of every superstep.
    lh=False is the plain near-far loop (every edge light, no drain rule);
    pull_tail=False keeps the split after a heavy pull that ends bucketing;
    early_div: a light frontier of at most n / early_div vertices lets that
    pull run at once (0: never), taking the light frontier into the plain
    push's first frontier."""
    ro = np.asarray(ro, np.int64)
    n, m = ro.size - 1, len(col)
    deg = np.diff(ro)
    rowid = np.repeat(np.arange(n), deg)
    w = np.asarray(w, np.int64)
    is_light = (w < delta) if lh else np.ones(w.size, bool)
    order = np.lexsort((~is_light, rowid))   # light edges first in each row (stable)
    c2 = np.asarray(col, np.int64)[order]
    w2 = w[order]
    nl = np.bincount(rowid, weights=is_light, minlength=n).astype(np.int64)
    lend = ro[:-1] + nl
    ldeg, hdeg = nl, deg - nl
    heavy_total = int(hdeg.sum())

    dist = np.full(n, BIG)
    dist[src] = 0
    t_cur, t_prev = np.int64(delta), np.int64(0)
    far = np.zeros(n, bool)
    R = np.zeros(n, bool)
    F = np.array([src]) if ldeg[src] > 0 else np.zeros(0, np.int64)
    R[src] = hdeg[src] > 0
    heavy_done = 0
    bucketed = True
    kinds = []

    def push(us, lo, hi):
        cnt = hi[us] - lo[us]
        tot = int(cnt.sum())
        if tot == 0:
            return np.zeros(0, np.int64)
        own = np.repeat(us, cnt)
        e = np.repeat(lo[us] - np.concatenate(([0], np.cumsum(cnt)[:-1])), cnt) + np.arange(tot)
        best = np.full(n, BIG)
        np.minimum.at(best, c2[e], dist[own] + w2[e])
        imp = np.flatnonzero(best < dist)
        dist[imp] = best[imp]
        return imp

    def near_far(imp, r_into):
        """Improved vertices below the threshold join the light frontier (and
        the R list); the others are parked in the far pile."""
        near = imp[dist[imp] < t_cur]
        far[imp[dist[imp] >= t_cur]] = True
        if not bucketed:
            return near[deg[near] > 0]
        r_into[near[hdeg[near] > 0]] = True
        return near[ldeg[near] > 0]

    while True:
        early = bool(bucketed and early_div and F.size and F.size * early_div <= n and R.any())
        if early:   # the pull that ends the buckets, due now on the current R list
            rE = int(hdeg[np.flatnonzero(R)].sum())
            left = max(heavy_total - heavy_done - rE, 0)
            early = (symmetric and t_cur < BIG and rE > left + n // 8 and pull_tail and tail
                     and left * drain_div < m)
        if F.size and bucketed and not early:
            kinds.append(LIGHT)
            F = near_far(push(F, ro[:-1], lend), R)
        elif bucketed and R.any():
            Rv = np.flatnonzero(R)
            rE = int(hdeg[Rv].sum())
            left = max(heavy_total - heavy_done - rE, 0)
            R_next = np.zeros(n, bool)
            if symmetric and t_cur < BIG and rE > left + n // 8:
                ends = pull_tail and tail and left * drain_div < m
                kinds.append(HEAVY_PULL_TAIL if ends else HEAVY_PULL)
                F_light = F   # non-empty only when the buckets end early
                # every unsettled vertex takes the minimum over its heavy edges
                # from settled vertices (symmetric: in-edges = out-edges)
                un = np.flatnonzero(dist >= t_cur)
                cnt = hdeg[un]
                tot = int(cnt.sum())
                imp = np.zeros(0, np.int64)
                if tot:
                    own = np.repeat(un, cnt)
                    e = np.repeat(lend[un] - np.concatenate(([0], np.cumsum(cnt)[:-1])), cnt) + np.arange(tot)
                    du = dist[c2[e]]
                    ok = du < t_cur
                    best = np.full(n, BIG)
                    np.minimum.at(best, own[ok], du[ok] + w2[e][ok])
                    imp = np.flatnonzero(best < dist)
                    dist[imp] = best[imp]
                far[imp] = True   # every improvement is >= t_cur
                F = np.zeros(0, np.int64)
                if ends:
                    # the kernel takes every unsettled vertex with a finite
                    # distance: the vertices the split would move from the pile
                    fv = np.flatnonzero((dist >= t_cur) & (dist < BIG))
                    assert np.array_equal(fv, np.flatnonzero(far & (dist >= t_cur)))
                    far[:] = False
                    t_prev, t_cur = t_cur, BIG
                    bucketed = False
                    # and the light frontier of an early end, with whole rows
                    F = np.union1d(fv[deg[fv] > 0], F_light[deg[F_light] > 0])
            else:
                kinds.append(HEAVY_PUSH)
                F = near_far(push(Rv, lend, ro[1:]), R_next)
            heavy_done += rE
            R = R_next
        elif F.size:   # plain push once bucketing has ended
            kinds.append(LIGHT)
            F = near_far(push(F, ro[:-1], ro[1:]), R)
        elif far.any():
            # reached only with the light frontier and (while bucketed) the R
            # list empty, so a split that ends bucketing leaves no heavy edges
            # pending: every vertex's edges after it are relaxed by plain push
            kinds.append(SPLIT)
            fv = np.flatnonzero(far)
            tn = max(t_cur + delta, int(dist[fv].min()) + 1)
            if lh and bucketed and (heavy_total - min(heavy_done, heavy_total)) * drain_div < m:
                tn = BIG
                bucketed = not tail
            t_prev, t_cur = t_cur, np.int64(tn)
            moved = fv[dist[fv] < t_cur]
            far[moved] = False
            near = moved[dist[moved] >= t_prev]   # below t_prev: expanded already
            if bucketed:
                R[near[hdeg[near] > 0]] = True
                F = near[ldeg[near] > 0]
            else:
                F = near[deg[near] > 0]
        else:
            break
    out = np.where(dist >= BIG, INF32, dist).astype(np.uint32)
    return out, np.array(kinds)


def _after_drain(kinds):
    """Kinds after the step that ended bucketing (the last split, or a heavy
    pull that ended it), when nothing heavy follows it, else None."""
    s = np.flatnonzero((kinds == SPLIT) | (kinds == HEAVY_PULL_TAIL))
    if not s.size:
        return None
    rest = kinds[s[-1] + 1:]
    return None if np.isin(rest, (HEAVY_PUSH, HEAVY_PULL, HEAVY_PULL_TAIL)).any() else rest


def _sink_graph(seed, n=3000, m=40000, W=90):
    rng = np.random.Generator(np.random.PCG64(seed))
    src = rng.integers(0, n * 5 // 6, m)   # the last sixth of the vertices have no out-edges
    return graphgen.from_edges(n, src, rng.integers(0, n, m), rng.integers(0, W, m))


@pytest.mark.parametrize("scale,delta", [(10, 12), (11, 5), (12, 12), (12, 40)])
def test_rmat_schedule_matches_oracle(scale, delta):
    ro, col, w = graphgen.rmat(scale, 16, seed=scale, W=255)
    for s in (graphgen.max_degree_vertex(ro), int(graphgen.sample_sources(ro, 1, seed=7)[0])):
        got, kinds = schedule(ro, col, w, s, delta, symmetric=True)
        np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, s), err_msg=f"src={s}")
        assert np.isin(kinds, (HEAVY_PUSH, HEAVY_PULL, HEAVY_PULL_TAIL)).any()
        rest = _after_drain(kinds)
        if rest is not None:
            assert (rest == LIGHT).all()


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("delta", [1, 7, 30])
def test_directed_sinks_and_zero_weights_schedule_matches_oracle(seed, delta):
    ro, col, w = _sink_graph(seed)
    for s in (0, 1111, 2999):
        got, _ = schedule(ro, col, w, s, delta, symmetric=False)
        np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, s), err_msg=f"seed={seed} src={s}")


def test_path_and_grid_schedule_matches_oracle():
    wts = np.random.Generator(np.random.PCG64(3)).integers(0, 30, 1999)
    ro, col, w = graphgen.path_graph(2000, wts)
    for delta in (1, 9, 29):
        got, _ = schedule(ro, col, w, 0, delta, symmetric=False)
        np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, 0))
    ro, col, w = graphgen.grid(48, 64, 5)
    for delta in (3, 40, 64):
        got, _ = schedule(ro, col, w, 0, delta, symmetric=True)
        np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, 0))


def test_plain_tail_removes_supersteps_not_distances():
    # after the drain the remaining distances form one unbounded bucket: the
    # light/heavy alternation there relaxes the same edges in more supersteps
    ro, col, w = graphgen.rmat(12, 16, seed=1, W=255)
    hub = graphgen.max_degree_vertex(ro)
    got_t, kinds_t = schedule(ro, col, w, hub, 12, symmetric=True, tail=True)
    got_b, kinds_b = schedule(ro, col, w, hub, 12, symmetric=True, tail=False)
    np.testing.assert_array_equal(got_t, got_b)
    np.testing.assert_array_equal(got_t, oracle.dijkstra(ro, col, w, hub))
    assert _after_drain(kinds_t) is not None   # bucketing ended in this run
    assert {HEAVY_PULL, HEAVY_PULL_TAIL} & set(kinds_t.tolist())   # the first bucket's heavy superstep pulled
    assert len(kinds_t) < len(kinds_b)


@pytest.mark.parametrize("scale,seed,delta", [(12, 1, 20), (13, 3, 20), (14, 5, 12)])
def test_pull_that_ends_bucketing_replaces_the_split(scale, seed, delta):
    # (early_div=0: the pull comes where the bucket's light frontier empties)
    # the pull after which the drain rule holds writes the plain frontier
    # itself: the same distances, one superstep (the split) fewer, and the
    # first plain push works on the vertices the split would have moved
    ro, col, w = graphgen.rmat(scale, 16, seed=seed, W=255)
    hub = graphgen.max_degree_vertex(ro)
    got_p, kinds_p = schedule(ro, col, w, hub, delta, symmetric=True, early_div=0)
    got_s, kinds_s = schedule(ro, col, w, hub, delta, symmetric=True, pull_tail=False, early_div=0)
    np.testing.assert_array_equal(got_p, oracle.dijkstra(ro, col, w, hub))
    np.testing.assert_array_equal(got_s, got_p)
    k = np.flatnonzero(kinds_p == HEAVY_PULL_TAIL)
    assert k.size == 1
    # without it: a pull, then the split that ends bucketing
    assert kinds_s[k[0]] == HEAVY_PULL and kinds_s[k[0] + 1] == SPLIT
    np.testing.assert_array_equal(kinds_p[k[0] + 1:], kinds_s[k[0] + 2:])
    assert (kinds_p[k[0] + 1:] == LIGHT).all()


@pytest.mark.parametrize("graph", ["grid", "path", "sinks", "rmat"])
def test_plain_near_far_schedule_matches_oracle(graph):
    # without the light/heavy split every edge is light: near supersteps relax
    # all edges below the threshold, the rest wait in the far pile for a split
    if graph == "grid":
        ro, col, w = graphgen.grid(48, 64, 5)
        cases, sym = [(0, 16 * 64), (0, 50), (1175, 7)], True
    elif graph == "path":
        ro, col, w = graphgen.path_graph(1500, np.random.Generator(np.random.PCG64(9)).integers(0, 40, 1499))
        cases, sym = [(0, 1), (0, 100)], False
    elif graph == "sinks":
        ro, col, w = _sink_graph(5)
        cases, sym = [(0, 4), (777, 60)], False
    else:
        ro, col, w = graphgen.rmat(11, 16, seed=2, W=255)
        cases, sym = [(graphgen.max_degree_vertex(ro), 30)], True
    for s, delta in cases:
        got, kinds = schedule(ro, col, w, s, delta, symmetric=sym, lh=False)
        np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, s), err_msg=f"{graph} src={s} delta={delta}")
        assert not np.isin(kinds, (HEAVY_PUSH, HEAVY_PULL, HEAVY_PULL_TAIL)).any()
    assert SPLIT in kinds   # the far pile was used


@pytest.mark.parametrize("scale,seed,delta", [(12, 1, 20), (13, 3, 20), (14, 5, 12), (14, 7, 16)])
@pytest.mark.parametrize("early_div", [4, 16, 64])
def test_early_end_of_the_buckets_keeps_the_distances(scale, seed, delta, early_div):
    # a small light frontier lets the pull that ends the buckets run at once:
    # the frontier's vertices (distances not final yet) go into the plain
    # push's first frontier with their whole rows, and plain pushes finish
    # what the bucket's last light supersteps would have done
    ro, col, w = graphgen.rmat(scale, 16, seed=seed, W=255)
    hub = graphgen.max_degree_vertex(ro)
    ref = oracle.dijkstra(ro, col, w, hub)
    got_e, kinds_e = schedule(ro, col, w, hub, delta, symmetric=True, early_div=early_div)
    got_l, kinds_l = schedule(ro, col, w, hub, delta, symmetric=True, early_div=0)
    np.testing.assert_array_equal(got_e, ref)
    np.testing.assert_array_equal(got_l, ref)
    k_e, k_l = np.flatnonzero(kinds_e == HEAVY_PULL_TAIL), np.flatnonzero(kinds_l == HEAVY_PULL_TAIL)
    assert k_e.size == 1 and k_l.size == 1
    assert (kinds_e[k_e[0] + 1:] == LIGHT).all()
    assert k_e[0] < k_l[0]            # the buckets ended before their light frontier emptied
    assert len(kinds_e) < len(kinds_l)


def test_early_end_planted_mistake_is_caught():
    # dropping the light frontier at an early end (instead of carrying it into
    # the plain push) leaves distances too large: the oracle comparison sees it
    ro, col, w = graphgen.rmat(14, 16, seed=5, W=255)
    hub = graphgen.max_degree_vertex(ro)
    src = open(__file__).read()
    assert "F_light[deg[F_light] > 0]" in src
    ns = {}
    bad = src.replace("np.union1d(fv[deg[fv] > 0], F_light[deg[F_light] > 0])", "fv[deg[fv] > 0]")
    exec(compile(bad, __file__, "exec"), ns)
    ref = oracle.dijkstra(ro, col, w, hub)
    found = False
    for early_div in (4, 16, 64):
        got, kinds = ns["schedule"](ro, col, w, hub, 12, symmetric=True, early_div=early_div)
        early = HEAVY_PULL_TAIL in kinds.tolist()
        if early and not np.array_equal(got, ref):
            found = True
    assert found
