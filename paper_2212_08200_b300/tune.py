"""Autotuner front end: runs gg_autotune / gg_autotune_batch (the native
tuners in libgg.so) on a graph and caches the winning options per graph
class, so graphs of the same shape reuse them without re-tuning.

Graph class key: (round(log2 n), round(log2 m), skew bucket), where skew =
max out-degree / mean out-degree of the non-isolated vertices, bucketed by
powers of 4 (a grid lands in bucket 0, RMAT graphs in high buckets).
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import threading

import numpy as np

from . import _check, _stream_ptr, gg_options, load

FIELDS = ["policy", "direction", "lb_mode", "warp_threshold", "cta_threshold", "pull_alpha", "pull_beta", "delta"]
BATCH_FIELDS = ["light_heavy", "delta"]
_lock = threading.Lock()
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "gg_autotune.json")


def graph_class(row_offsets) -> str:
    ro = np.asarray(row_offsets, np.int64)
    n = ro.shape[0] - 1
    m = int(ro[-1])
    deg = np.diff(ro)
    nz = deg[deg > 0]
    skew = float(nz.max() / nz.mean()) if nz.size else 1.0
    bucket = int(math.log(max(skew, 1.0), 4))
    return f"n{round(math.log2(max(n, 1)))}_m{round(math.log2(max(m, 1)))}_s{bucket}"


def options_to_dict(o: gg_options, fields=FIELDS) -> dict:
    return {k: int(getattr(o, k)) for k in fields}


def dict_to_kwargs(d: dict, fields=FIELDS) -> dict:
    return {k: int(v) for k, v in d.items() if k in fields}


def _read(cache_path):
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def _write(cache_path, key, d, ms):
    if not cache_path:
        return
    with _lock:
        cache = _read(cache_path)
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        field = "ms_per_call" if key.startswith("batch:") else "ms_per_source"
        cache[key] = {"options": d, field: float(ms)}
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)


def autotune(graph, row_offsets, sources, cache_path: str | None = DEFAULT_CACHE, retune: bool = False,
             stream=None) -> dict:
    """Best single-source options for `graph` (a Graph) as keyword arguments
    for Graph.sssp / make_options.  Cached per graph class in cache_path."""
    import torch
    key = graph_class(row_offsets)
    cache = _read(cache_path)
    if key in cache and not retune:
        return dict_to_kwargs(cache[key]["options"])
    srcs = np.ascontiguousarray(sources, dtype=np.uint32)
    scratch = torch.empty(graph.n, dtype=torch.uint32, device="cuda")
    best = gg_options()
    ms = ctypes.c_float()
    _check(load().gg_autotune(graph.handle, srcs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), srcs.shape[0],
                              scratch.data_ptr(), ctypes.byref(best), ctypes.byref(ms), _stream_ptr(stream)),
           "gg_autotune")
    d = options_to_dict(best)
    _write(cache_path, key, d, ms.value)
    return dict_to_kwargs(d)


def autotune_batch(graph, row_offsets, sources, cache_path: str | None = DEFAULT_CACHE, retune: bool = False,
                   stream=None) -> dict:
    """Best batched options (light_heavy schedule and width) for `graph` and
    this many sources, as keyword arguments for Graph.sssp_batch.  Cached per
    graph class and source count (key "batch:<class>_k<k>")."""
    import torch
    srcs = np.ascontiguousarray(sources, dtype=np.uint32)
    key = f"batch:{graph_class(row_offsets)}_k{srcs.shape[0]}"
    cache = _read(cache_path)
    if key in cache and not retune:
        return dict_to_kwargs(cache[key]["options"], BATCH_FIELDS)
    scratch = torch.empty(graph.n * srcs.shape[0], dtype=torch.uint32, device="cuda")
    best = gg_options()
    ms = ctypes.c_float()
    _check(load().gg_autotune_batch(graph.handle, srcs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), srcs.shape[0],
                                    scratch.data_ptr(), ctypes.byref(best), ctypes.byref(ms), _stream_ptr(stream)),
           "gg_autotune_batch")
    d = options_to_dict(best, BATCH_FIELDS)
    _write(cache_path, key, d, ms.value)
    return dict_to_kwargs(d, BATCH_FIELDS)
