"""CPU model of the warp-local rounds (load balance GG_LB_LOCAL), checked
against the oracle.

In a superstep each "warp" takes an equal share of the frontier and relaxes
its rows; every strict decrease below the bucket threshold queues the vertex
in that warp's local queue together with the distance it was queued with
(no bitmap).  For up to L rounds the warp expands its queue: an entry whose
vertex has since dropped below its queued distance is skipped (a later
decrease queued it again), every other entry relaxes the vertex's row with its
current distance.  What the rounds leave, and what overflows a queue, joins
the next frontier once (bitmap).  Decreases at or above the threshold park the
vertex (near-far split as in the plain loop).  Relaxations inside a warp's
round are taken one edge at a time, in queue order, and the warps of a
superstep one after another, which is one of the orders the kernel's atomics
allow.  No GPU is involved.
"""
import numpy as np
import pytest

import graphgen
import oracle

BIG = np.int64(1) << 40
INF32 = 0xFFFFFFFF


def local_rounds(ro, col, w, src, delta, warps=7, rounds=4, qcap=6, mistake=None):
    """Distances (uint32) and the superstep count.  mistake (pin strength only):
    "skip_equal" also skips entries whose distance equals the queued one,
    "drop_leftover" drops what the rounds leave instead of passing it on."""
    ro = np.asarray(ro, np.int64)
    col = np.asarray(col, np.int64)
    w = np.asarray(w, np.int64)
    n = ro.size - 1
    dist = np.full(n, BIG)
    dist[src] = 0
    t_cur, t_prev = np.int64(delta), np.int64(0)
    frontier = [src] if ro[src + 1] > ro[src] else []
    far = set()
    steps = 0
    while True:
        if not frontier:
            if not far:
                break
            fm = min(int(dist[v]) for v in far)
            t_prev, t_cur = t_cur, max(t_cur + delta, fm + 1)
            nxt = sorted(v for v in far if t_prev <= dist[v] < t_cur)
            far = {v for v in far if dist[v] >= t_cur}
            frontier = [v for v in nxt if ro[v + 1] > ro[v]]
            steps += 1
            continue
        steps += 1
        nxt, in_next = [], set()

        def to_next(v):
            if v not in in_next:
                in_next.add(v)
                nxt.append(v)

        shares = np.array_split(np.asarray(frontier, np.int64), warps)
        for share in shares:
            queue = []                         # (vertex, queued distance)

            def relax(u):
                du = dist[u]
                for e in range(ro[u], ro[u + 1]):
                    v, nd = int(col[e]), du + int(w[e])
                    if nd < dist[v]:
                        dist[v] = nd
                        if ro[v + 1] == ro[v]:
                            continue
                        if nd < t_cur:
                            if len(queue) < qcap:
                                queue.append((v, nd))
                            else:
                                to_next(v)        # the queue is full: the next frontier
                        else:
                            far.add(v)

            for u in share:
                relax(int(u))
            for _ in range(rounds):
                if not queue:
                    break
                cur, queue = queue, []
                for v, q in cur:
                    stale = dist[v] <= q if mistake == "skip_equal" else dist[v] < q
                    if not stale:
                        relax(v)
            if mistake != "drop_leftover":
                for v, _ in queue:
                    to_next(v)
        frontier = nxt
    return np.where(dist >= BIG, INF32, dist).astype(np.uint32), steps


GRAPHS = {
    "grid40": lambda: graphgen.grid(40, 1000, 3),
    "grid17c": lambda: graphgen.grid(17, 0, 1, const_w=5),
    "rmat10": lambda: graphgen.rmat(10, 8, seed=2, W=255),
    "directed_zero": lambda: graphgen.random_graph(600, 2400, 9, seed=4, wmin=0),
    "path": lambda: graphgen.path_graph(300, np.arange(1, 300) % 7),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("delta,rounds,qcap", [(10 ** 9, 4, 6), (500, 4, 6), (60, 16, 64), (10 ** 9, 1, 2)])
def test_local_rounds_reach_the_oracle(name, delta, rounds, qcap):
    ro, col, w = GRAPHS[name]()
    for src in (0, (ro.shape[0] - 1) // 2):
        got, _ = local_rounds(ro, col, w, src, delta, rounds=rounds, qcap=qcap)
        np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, src), err_msg=f"{name} src={src}")


def test_local_rounds_cut_supersteps_on_a_grid():
    ro, col, w = graphgen.grid(40, 1000, 3)
    _, one = local_rounds(ro, col, w, 0, 10 ** 9, rounds=0)
    _, many = local_rounds(ro, col, w, 0, 10 ** 9, rounds=8, qcap=64)
    assert many < one / 3


@pytest.mark.parametrize("mistake", ["skip_equal", "drop_leftover"])
def test_planted_mistakes_fail(mistake):
    ro, col, w = graphgen.grid(40, 1000, 3)
    ref = oracle.dijkstra(ro, col, w, 0)
    got, _ = local_rounds(ro, col, w, 0, 10 ** 9, rounds=4, qcap=6)
    np.testing.assert_array_equal(got, ref)
    bad, _ = local_rounds(ro, col, w, 0, 10 ** 9, rounds=4, qcap=6, mistake=mistake)
    assert not np.array_equal(bad, ref)
