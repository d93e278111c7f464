"""Reader for the hand-worked SSSP fixtures in tests/golden/*.txt."""
import os

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
INF = 0xFFFFFFFF


def load(name):
    """Returns dict(n, src, ro, col, w, expect) where expect is a uint32 array
    or the string 'RANGE_ERROR'."""
    n = src = None
    undirected = False
    edges, expect = [], None
    mode = None
    with open(os.path.join(GOLDEN_DIR, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "n":
                n = int(tok[1])
            elif tok[0] == "src":
                src = int(tok[1])
            elif tok[0] == "undirected":
                undirected = True
            elif tok[0] in ("edges", "expect"):
                mode = tok[0]
            elif mode == "edges":
                u, v, w = map(int, tok)
                edges.append((u, v, w))
                if undirected:
                    edges.append((v, u, w))
            elif mode == "expect":
                if tok[0] == "RANGE_ERROR":
                    expect = "RANGE_ERROR"
                else:
                    expect = np.array([INF if t == "INF" else int(t) for t in tok], np.uint32)
    s = np.array([e[0] for e in edges], np.int64)
    d = np.array([e[1] for e in edges], np.int64)
    w = np.array([e[2] for e in edges], np.int64)
    order = np.argsort(s, kind="stable")
    ro = np.zeros(n + 1, np.int64)
    np.add.at(ro, s + 1, 1)
    ro = np.cumsum(ro).astype(np.uint32)
    return dict(n=n, src=src, ro=ro, col=d[order].astype(np.uint32), w=w[order].astype(np.uint32),
                expect=expect)


def hand_fixtures():
    return sorted(f for f in os.listdir(GOLDEN_DIR) if f.startswith("hand_") and f.endswith(".txt"))
