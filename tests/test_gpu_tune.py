"""The autotuner: returns valid options that reproduce the oracle's
distances, and caches them per graph class."""
import json

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_autotune_rmat_and_grid(tmp_path):
    import paper_2212_08200_b300 as gg
    from paper_2212_08200_b300 import tune
    cache = str(tmp_path / "tune.json")
    for name in ("rmat14", "grid128"):
        ro, col, w, src = graphgen.workload(name)
        g = gg.Graph(ro, col, w, symmetric=True)
        srcs = graphgen.sample_sources(ro, 2, seed=4)
        opts = tune.autotune(g, ro, srcs, cache_path=cache)
        assert set(opts) == set(tune.FIELDS)
        d = g.sssp(src, **opts)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(d.cpu().numpy(), oracle.dijkstra(ro, col, w, src))
        again = tune.autotune(g, ro, srcs, cache_path=cache)       # served from the cache
        assert again == opts
        g.close()
    data = json.load(open(cache))
    assert len(data) == 2 and all(v["ms_per_source"] > 0 for v in data.values())
