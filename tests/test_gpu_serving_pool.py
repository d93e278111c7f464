"""Parity of the serving workload itself: the 32-graph pool (RMAT scales
12-20 with edge factor 8 or 16, grids 64^2-2048^2, weights U[1,255]) and its
2,000-query Poisson stream (seed 1), pushed through the continuous-batching
server.

* A sample with at least one query on every pool graph (the 2048^2 grids and
  RMAT-20 included) is compared element by element with a live run of the
  CPU oracle.
* Every one of the 2,000 queries is compared with the hash of the oracle's
  distances that tests/golden/make_golden.py stored (it calls only the
  generators and the oracle).

Bit-exact (tolerance 0): every distance is an exact integer."""
import hashlib
import json
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    import paper_2212_08200_b300 as gg
    gg.load()
    data = [graphgen.build_pool_graph(e) for e in graphgen.serving_pool_spec()]
    graphs = [gg.Graph(ro, col, w, symmetric=True) for ro, col, w in data]
    yield data, graphs
    for g in graphs:
        g.close()


def _stream(data, nq=2000, seed=1):
    degs = [np.diff(ro.astype(np.int64)) for ro, _, _ in data]
    gids, srcs, _ = graphgen.poisson_queries(degs, nq, seed=seed)
    return gids, srcs


def _serve(graphs, queries, max_slots=64):
    import paper_2212_08200_b300 as gg
    outs = [torch.full((graphs[gi].n,), 0x5A5A5A5A, dtype=torch.int32, device="cuda").view(torch.uint32)
            for gi, _ in queries]
    srv = gg.Server(max_graph_vertices=max(g.n for g in graphs), max_slots=max_slots, supersteps_per_launch=8)
    tickets = [srv.submit(graphs[gi], int(s), o) for (gi, s), o in zip(queries, outs)]
    status = [srv.wait(t, 600000) for t in tickets]
    st = srv.stats()
    srv.close()
    assert status == [0] * len(queries)
    return outs, st


def test_pool_sample_matches_oracle(pool):
    """One query of the stream on every pool graph, plus the first 32 of the
    stream, served together; each compared with oracle.dijkstra."""
    data, graphs = pool
    gids, srcs = _stream(data)
    pick = []
    for gi in range(len(data)):
        pick.append(int(np.flatnonzero(gids == gi)[0]))
    pick += [i for i in range(32) if i not in pick]
    queries = [(int(gids[i]), int(srcs[i])) for i in pick]
    assert {gi for gi, _ in queries} == set(range(32))
    sides = {graphgen.serving_pool_spec()[gi][1] for gi, _ in queries if graphgen.serving_pool_spec()[gi][0] == "grid"}
    assert 2048 in sides
    outs, st = _serve(graphs, queries)
    assert st["max_running"] > 1                      # the queries really ran together

    def ref(q):
        gi, s = q
        ro, col, w = data[gi]
        return oracle.dijkstra(ro, col, w, s)

    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        refs = list(ex.map(ref, queries))
    for (gi, s), o, r in zip(queries, outs, refs):
        np.testing.assert_array_equal(o.cpu().numpy(), r, err_msg=f"pool graph {gi} source {s}")


def test_whole_stream_matches_stored_oracle_hashes(pool):
    """All 2,000 queries of the serving stream through the server; each
    distance vector hashes to the oracle's stored hash."""
    data, graphs = pool
    with open(os.path.join(os.path.dirname(__file__), "golden", "workloads.json")) as f:
        rec = json.load(f)["serving_pool"]
    gph = [hashlib.sha256(b"".join(np.ascontiguousarray(a, np.uint32).tobytes() for a in g)).hexdigest() for g in data]
    assert gph == rec["graph_sha256"]
    gids, srcs = _stream(data, rec["queries"], rec["seed"])
    assert [int(x) for x in gids] == rec["graph"] and [int(x) for x in srcs] == rec["source"]
    queries = [(int(g), int(s)) for g, s in zip(gids, srcs)]
    outs, _ = _serve(graphs, queries)
    bad = [i for i, o in enumerate(outs)
           if hashlib.sha256(o.cpu().numpy().tobytes()).hexdigest()[:16] != rec["dist_sha256_16"][i]]
    assert not bad, f"{len(bad)} queries differ from the oracle, first {bad[:8]}"
