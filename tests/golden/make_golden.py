"""Writes tests/golden/workloads.json: for each named workload, the hash of
the generated graph and of the oracle's distance vector, plus summary
numbers.  Calls only graphgen (inputs) and oracle (expected values).

Two multi-query records sit beside the single-source workloads:

* ``rmat22_batch64``: the 64 seeded sources of the batched workload (RMAT
  scale 22, splitmix64 seed 1): the sha256 of the vertex-major distance
  matrix (n x 64, dist[v * 64 + s]) and of each column;
* ``serving_pool``: the 2,000-query Poisson stream (seed 1) over the 32-graph
  pool: per query its graph, source and the first 16 hex digits of the
  sha256 of its distance vector.

Usage: python tests/golden/make_golden.py [workload ...]
       (names: the single-source workloads, rmat22_batch64, serving_pool)
"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import graphgen  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workloads.json")
DEFAULT = ["grid64", "rmat16", "rmat20", "grid4096", "rmat22"]


def sha(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a, np.uint32).tobytes())
    return h.hexdigest()


def record(name):
    ro, col, w, src = graphgen.workload(name)
    dist = oracle.dijkstra(ro, col, w, src)
    fin = dist[dist != oracle.INF].astype(np.int64)
    return dict(n=int(ro.shape[0] - 1), m=int(col.shape[0]), source=int(src),
                graph_sha256=sha(ro, col, w), dist_sha256=sha(dist),
                reached=int(fin.shape[0]), dist_sum=int(fin.sum()), dist_max=int(fin.max()),
                m_trav=oracle.traversed_edges(ro, dist))


def record_batch(scale=22, k=64, seed=1):
    ro, col, w = graphgen.rmat(scale, 16, seed=1, W=255)
    srcs = graphgen.sample_sources(ro, k, seed=seed)
    D = oracle.dijkstra_many(ro, col, w, srcs, threads=os.cpu_count() or 1)     # (k, n)
    vm = np.ascontiguousarray(D.T)                                               # vertex-major (n, k)
    return dict(n=int(ro.shape[0] - 1), k=k, sources=[int(x) for x in srcs], graph_sha256=sha(ro, col, w),
                matrix_sha256=sha(vm), column_sha256=[sha(D[s]) for s in range(k)],
                m_trav=[oracle.traversed_edges(ro, D[s]) for s in range(k)])


def record_serving(nq=2000, seed=1):
    from concurrent.futures import ThreadPoolExecutor
    spec = graphgen.serving_pool_spec()
    pool = [graphgen.build_pool_graph(e) for e in spec]
    degs = [np.diff(ro.astype(np.int64)) for ro, _, _ in pool]
    gids, srcs, _ = graphgen.poisson_queries(degs, nq, seed=seed)

    def one(i):
        ro, col, w = pool[gids[i]]
        return sha(oracle.dijkstra(ro, col, w, int(srcs[i])))[:16]

    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:      # the ctypes call releases the GIL
        hashes = list(ex.map(one, range(nq)))
    return dict(queries=nq, seed=seed, graph_sha256=[sha(*g) for g in pool], graph=[int(x) for x in gids],
                source=[int(x) for x in srcs], dist_sha256_16=hashes)


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    data["_about"] = ("Written by tests/golden/make_golden.py from graphgen inputs and the CPU "
                      "oracle (binary-heap Dijkstra); distances are uint32 little-endian, "
                      "0xFFFFFFFF = unreachable.")
    for nm in names:
        if nm == "rmat22_batch64":
            data[nm] = record_batch()
        elif nm == "serving_pool":
            data[nm] = record_serving()
        else:
            data[nm] = record(nm)
        print(nm, str(data[nm])[:300])
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or DEFAULT)
