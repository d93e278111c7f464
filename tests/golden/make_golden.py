"""Writes tests/golden/workloads.json: for each named workload, the hash of
the generated graph and of the oracle's distance vector, plus summary
numbers.  Calls only graphgen (inputs) and oracle (expected values).

Usage: python tests/golden/make_golden.py [workload ...]
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


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    data["_about"] = ("Written by tests/golden/make_golden.py from graphgen inputs and the CPU "
                      "oracle (binary-heap Dijkstra); distances are uint32 little-endian, "
                      "0xFFFFFFFF = unreachable.")
    for nm in names:
        data[nm] = record(nm)
        print(nm, data[nm])
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or DEFAULT)
