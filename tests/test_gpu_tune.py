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


def test_autotune_searches_light_heavy_widths():
    """On a skewed graph the single-source tuner's bucket-width step tries
    light/heavy widths around the graph's default (not only near-far ones):
    the result is a width up to the largest weight, or no buckets."""
    import paper_2212_08200_b300 as gg
    from paper_2212_08200_b300 import tune
    ro, col, w, src = graphgen.workload("rmat16")
    g = gg.Graph(ro, col, w, symmetric=True)
    opts = tune.autotune(g, ro, graphgen.sample_sources(ro, 2, seed=4), cache_path=None)
    assert opts["delta"] in (0, gg.GG_DELTA_NONE) or 1 <= opts["delta"] <= int(w.max())
    d = g.sssp(src, **opts)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d.cpu().numpy(), oracle.dijkstra(ro, col, w, src))
    g.close()


def test_autotune_batch(tmp_path):
    """The batched tuner picks a schedule and width; the batch run with them
    reproduces the oracle, and the choice is cached per graph class and k."""
    import paper_2212_08200_b300 as gg
    from paper_2212_08200_b300 import tune
    cache = str(tmp_path / "tune.json")
    ro, col, w, _ = graphgen.workload("rmat14")
    srcs = graphgen.sample_sources(ro, 64, seed=6)
    g = gg.Graph(ro, col, w, symmetric=True)
    opts = tune.autotune_batch(g, ro, srcs, cache_path=cache)
    assert set(opts) == set(tune.BATCH_FIELDS)
    assert opts["light_heavy"] in (gg.GG_LH_AUTO, gg.GG_LH_ROUNDS)
    got = g.sssp_batch(srcs, **opts)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy().T, oracle.dijkstra_many(ro, col, w, srcs, threads=8))
    assert tune.autotune_batch(g, ro, srcs, cache_path=cache) == opts
    data = json.load(open(cache))
    assert any(k.startswith("batch:") and v["ms_per_call"] > 0 for k, v in data.items())
    g.close()
