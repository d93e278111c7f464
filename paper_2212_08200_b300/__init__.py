"""Python binding of the B300 frontier SSSP library (libgg.so, include/gg.h).

Argument marshalling only: every step of an SSSP run executes in the CUDA
kernels of libgg.so.  PyTorch supplies device memory and streams.  There is
no CPU fallback: importing a function that needs the library raises
``ImportError`` when libgg.so is missing, and every failing C call raises
``GGError`` carrying the library's status and message.

The functions keep the C names (``gg_graph_create_csr``, ``gg_sssp``, ...);
``Graph`` wraps a handle with a destructor.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = [
    "GGError", "GG_INF", "GG_DEVICE_PTRS", "GG_SYMMETRIC", "GG_NO_VALIDATE",
    "GG_POLICY_BSP_GRAPH", "GG_POLICY_ASYNC_PERSISTENT", "GG_POLICY_BSP_HOST", "GG_POLICY_BSP_PERSISTENT",
    "GG_DIR_AUTO", "GG_DIR_PUSH", "GG_DIR_PULL", "GG_LB_AUTO", "GG_LB_MERGE_PATH", "GG_LB_BINS", "GG_LB_WARP", "GG_LB_LOCAL", "GG_DELTA_NONE",
    "GG_LH_AUTO", "GG_LH_OFF", "GG_LH_ROUNDS",
    "gg_graph_create_csr", "gg_graph_destroy", "gg_graph_info", "gg_graph_check", "gg_sssp", "gg_sssp_ex",
    "gg_bfs", "gg_bfs_ex", "GG_FLOAT_WEIGHTS", "GG_FLT_MAX_BITS",
    "gg_sssp_batch", "gg_sssp_multi", "gg_sssp_tree", "Server",
    "gg_status_string", "gg_last_error", "gg_abi_version", "gg_sssp_noalloc", "GG_NOALLOC_MAX_VERTICES",
    "Graph", "lib_path", "load",
]

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(HERE, "libgg.so")
_lib = None
_lock = threading.Lock()

GG_INF = 0xFFFFFFFF
GG_DEVICE_PTRS, GG_SYMMETRIC, GG_NO_VALIDATE, GG_NO_PACK, GG_FLOAT_WEIGHTS = 0x1, 0x2, 0x4, 0x8, 0x10
GG_FLT_MAX_BITS = 0x7F7FFFFF   # "unreached" for binary32 distances (FLT_MAX)
GG_POLICY_BSP_GRAPH, GG_POLICY_ASYNC_PERSISTENT, GG_POLICY_BSP_HOST, GG_POLICY_BSP_PERSISTENT = 0, 1, 2, 3
GG_DIR_AUTO, GG_DIR_PUSH, GG_DIR_PULL = 0, 1, 2
GG_LB_AUTO, GG_LB_MERGE_PATH, GG_LB_BINS, GG_LB_WARP, GG_LB_LOCAL = 0, 1, 2, 3, 4
GG_DELTA_NONE = 0xFFFFFFFF
GG_LH_AUTO, GG_LH_OFF, GG_LH_ROUNDS = 0, 1, 2

STATUS = {0: "GG_OK", 1: "GG_ERR_INVALID_ARG", 2: "GG_ERR_OUT_OF_MEMORY", 3: "GG_ERR_CUDA",
          4: "GG_ERR_TIMEOUT", 5: "GG_ERR_BUSY", 6: "GG_ERR_NOT_READY", 7: "GG_ERR_OVERFLOW",
          8: "GG_ERR_INTERNAL", 9: "GG_ERR_NOT_SUPPORTED"}


class GGError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        self.status_name = STATUS.get(status, str(status))
        super().__init__(f"{where}: {self.status_name}: {msg}")


class gg_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_uint32), ("pull_iterations", ctypes.c_uint32),
                ("edges_scanned", ctypes.c_uint64), ("frontier_total", ctypes.c_uint64),
                ("max_frontier", ctypes.c_uint32), ("device_status", ctypes.c_uint32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class gg_options(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("policy", ctypes.c_int), ("direction", ctypes.c_int),
                ("lb_mode", ctypes.c_int), ("warp_threshold", ctypes.c_uint32), ("cta_threshold", ctypes.c_uint32),
                ("pull_alpha", ctypes.c_uint32), ("pull_beta", ctypes.c_uint32),
                ("max_iterations", ctypes.c_uint32), ("watchdog_ns", ctypes.c_uint64),
                ("stats", ctypes.POINTER(gg_stats)), ("trace", ctypes.c_void_p), ("trace_cap", ctypes.c_uint32),
                ("delta", ctypes.c_uint32), ("light_heavy", ctypes.c_uint32)]


class gg_server_config(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("max_slots", ctypes.c_uint32),
                ("max_graph_vertices", ctypes.c_uint32), ("supersteps_per_launch", ctypes.c_uint32),
                ("max_vertices_in_flight", ctypes.c_uint64), ("hbm_reserve_bytes", ctypes.c_uint64),
                ("delta", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class gg_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("vertex_budget", ctypes.c_uint64), ("queued", ctypes.c_uint32), ("running", ctypes.c_uint32),
                ("max_running", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("p50_us", ctypes.c_double),
                ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double), ("max_us", ctypes.c_double)]

    def as_dict(self):
        return {k: (float(getattr(self, k)) if t is ctypes.c_double else int(getattr(self, k)))
                for k, t in self._fields_ if k != "reserved"}


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Loads libgg.so (built by paper_2212_08200_b300.build).  Raises
    ImportError when it is missing: there is no fallback path."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"libgg.so not built at {_LIB_PATH}; run python -m paper_2212_08200_b300.build")
        lib = ctypes.CDLL(_LIB_PATH)
        vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        P32 = ctypes.POINTER(ctypes.c_uint32)
        sig = {
            "gg_graph_create_csr": (ctypes.c_int, [u32, u64, vp, vp, vp, u32, vp, ctypes.POINTER(vp)]),
            "gg_graph_destroy": (ctypes.c_int, [vp]),
            "gg_graph_info": (ctypes.c_int, [vp, P32, ctypes.POINTER(u64), ctypes.POINTER(u64)]),
            "gg_graph_check": (ctypes.c_int, [vp]),
            "gg_options_default": (None, [ctypes.POINTER(gg_options)]),
            "gg_sssp": (ctypes.c_int, [vp, u32, vp, vp]),
            "gg_sssp_ex": (ctypes.c_int, [vp, u32, vp, ctypes.POINTER(gg_options), vp]),
            "gg_bfs": (ctypes.c_int, [vp, u32, vp, vp]),
            "gg_bfs_ex": (ctypes.c_int, [vp, u32, vp, ctypes.POINTER(gg_options), vp]),
            "gg_sssp_noalloc": (ctypes.c_int, [u32, u64, vp, vp, vp, u32, vp, vp]),
            "gg_sssp_batch": (ctypes.c_int, [vp, P32, u32, vp, vp]),
            "gg_sssp_batch_ex": (ctypes.c_int, [vp, P32, u32, vp, ctypes.POINTER(gg_options), vp]),
            "gg_sssp_multi": (ctypes.c_int, [ctypes.POINTER(vp), P32, u32, ctypes.POINTER(vp), vp]),
            "gg_sssp_multi_ex": (ctypes.c_int, [ctypes.POINTER(vp), P32, u32, ctypes.POINTER(vp), u32, vp]),
            "gg_server_config_default": (None, [ctypes.POINTER(gg_server_config)]),
            "gg_server_create": (ctypes.c_int, [ctypes.POINTER(gg_server_config), ctypes.POINTER(vp)]),
            "gg_server_submit": (ctypes.c_int, [vp, vp, u32, vp, ctypes.POINTER(u64)]),
            "gg_server_poll": (ctypes.c_int, [vp, u64, ctypes.POINTER(ctypes.c_int)]),
            "gg_server_wait": (ctypes.c_int, [vp, u64, u32, ctypes.POINTER(ctypes.c_int)]),
            "gg_server_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(gg_server_stats)]),
            "gg_server_reset_stats": (ctypes.c_int, [vp]),
            "gg_server_destroy": (ctypes.c_int, [vp]),
            "gg_autotune": (ctypes.c_int, [vp, P32, u32, vp, ctypes.POINTER(gg_options),
                                           ctypes.POINTER(ctypes.c_float), vp]),
            "gg_autotune_batch": (ctypes.c_int, [vp, P32, u32, vp, ctypes.POINTER(gg_options),
                                                 ctypes.POINTER(ctypes.c_float), vp]),
            "gg_sssp_tree": (ctypes.c_int, [vp, u32, vp, vp, vp, u64, ctypes.POINTER(u64), vp]),
            "gg_part_create": (ctypes.c_int, [u32, u32, u32, u32, vp, vp, vp, vp, vp, ctypes.POINTER(vp)]),
            "gg_part_destroy": (ctypes.c_int, [vp]),
            "gg_part_info": (ctypes.c_int, [vp, P32, ctypes.POINTER(u64)]),
            "gg_part_begin": (ctypes.c_int, [vp, u32, vp]),
            "gg_part_advance": (ctypes.c_int, [vp, vp, vp, u64, ctypes.POINTER(u64)]),
            "gg_part_apply": (ctypes.c_int, [vp, vp, u64, vp, P32]),
            "gg_part_distances": (ctypes.c_int, [vp, vp, vp]),
            "gg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "gg_last_error": (ctypes.c_char_p, []),
            "gg_abi_version": (u32, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc: int, where: str):
    if rc != 0:
        raise GGError(rc, where, load().gg_last_error().decode(errors="replace"))


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(a):
    """(address, is_device) of a numpy array or torch tensor of uint32/int32."""
    if isinstance(a, np.ndarray):
        if a.dtype not in (np.uint32, np.int32) or not a.flags.c_contiguous:
            raise TypeError("numpy arrays must be contiguous uint32")
        return a.ctypes.data, False
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype not in (torch.uint32, torch.int32) or not a.is_contiguous():
            raise TypeError("tensors must be contiguous uint32/int32")
        return a.data_ptr(), a.is_cuda
    raise TypeError(f"unsupported array type {type(a)}")


def gg_status_string(s: int) -> str:
    return load().gg_status_string(s).decode()


def gg_last_error() -> str:
    return load().gg_last_error().decode(errors="replace")


def gg_abi_version() -> int:
    return int(load().gg_abi_version())


def gg_graph_create_csr(row_offsets, col_indices, weights, symmetric: bool = False, validate: bool = True,
                        stream=None, pack: bool = True, float_weights: bool = False) -> int:
    """Handle (int) for a CSR given as numpy arrays (host) or CUDA tensors
    (device).  All three must live on the same side.  float_weights: the
    weights are IEEE binary32 (a float32 array is passed by its bit pattern)."""
    lib = load()
    if float_weights and isinstance(weights, np.ndarray) and weights.dtype == np.float32:
        weights = weights.view(np.uint32)
    ro, ro_dev = _ptr(row_offsets)
    col, col_dev = _ptr(col_indices)
    w, w_dev = _ptr(weights)
    if len({ro_dev, col_dev, w_dev}) != 1:
        raise ValueError("row_offsets, col_indices and weights must all be host or all be device")
    n = int(row_offsets.shape[0]) - 1
    m = int(col_indices.shape[0])
    if int(weights.shape[0]) != m:
        raise ValueError("weights and col_indices differ in length")
    flags = ((GG_DEVICE_PTRS if ro_dev else 0) | (GG_SYMMETRIC if symmetric else 0) |
             (0 if validate else GG_NO_VALIDATE) | (0 if pack else GG_NO_PACK) |
             (GG_FLOAT_WEIGHTS if float_weights else 0))
    h = ctypes.c_void_p()
    _check(lib.gg_graph_create_csr(n, m, ro, col if m else None, w if m else None, flags,
                                   _stream_ptr(stream) if (stream is not None or ro_dev) else 0,
                                   ctypes.byref(h)), "gg_graph_create_csr")
    return h.value


def gg_graph_destroy(handle: int):
    _check(load().gg_graph_destroy(handle), "gg_graph_destroy")


def gg_graph_info(handle: int):
    n = ctypes.c_uint32()
    m = ctypes.c_uint64()
    b = ctypes.c_uint64()
    _check(load().gg_graph_info(handle, ctypes.byref(n), ctypes.byref(m), ctypes.byref(b)), "gg_graph_info")
    return int(n.value), int(m.value), int(b.value)


def gg_graph_check(handle: int):
    _check(load().gg_graph_check(handle), "gg_graph_check")


def make_options(policy=GG_POLICY_BSP_GRAPH, direction=GG_DIR_AUTO, lb_mode=GG_LB_AUTO, warp_threshold=0,
                 cta_threshold=0, pull_alpha=0, pull_beta=0, max_iterations=0, watchdog_ns=0, stats=None,
                 trace=None, trace_cap=0, delta=0, light_heavy=0) -> gg_options:
    o = gg_options()
    load().gg_options_default(ctypes.byref(o))
    o.policy, o.direction, o.lb_mode = policy, direction, lb_mode
    o.warp_threshold, o.cta_threshold = warp_threshold, cta_threshold
    o.pull_alpha, o.pull_beta, o.max_iterations, o.watchdog_ns = pull_alpha, pull_beta, max_iterations, watchdog_ns
    o.delta = delta
    o.light_heavy = light_heavy
    if stats is not None:
        o.stats = ctypes.pointer(stats)
    if trace is not None:
        o.trace = _ptr(trace)[0]
        o.trace_cap = trace_cap or int(trace.numel()) // 4
    return o


def gg_sssp(handle: int, src: int, dist_out, stream=None):
    """Distances from src into dist_out (CUDA uint32 tensor of n), async."""
    p, dev = _ptr(dist_out)
    if not dev:
        raise ValueError("dist_out must be a CUDA tensor")
    _check(load().gg_sssp(handle, src, p, _stream_ptr(stream)), "gg_sssp")


def gg_sssp_ex(handle: int, src: int, dist_out, options: gg_options | None = None, stream=None):
    p, dev = _ptr(dist_out)
    if not dev:
        raise ValueError("dist_out must be a CUDA tensor")
    _check(load().gg_sssp_ex(handle, src, p, ctypes.byref(options) if options is not None else None,
                             _stream_ptr(stream)), "gg_sssp_ex")


def gg_bfs(handle: int, src: int, depth_out, stream=None, options: gg_options | None = None):
    """Hop counts from src into depth_out (CUDA uint32 tensor of n), async."""
    p, dev = _ptr(depth_out)
    if not dev:
        raise ValueError("depth_out must be a CUDA tensor")
    if options is None:
        _check(load().gg_bfs(handle, src, p, _stream_ptr(stream)), "gg_bfs")
    else:
        _check(load().gg_bfs_ex(handle, src, p, ctypes.byref(options), _stream_ptr(stream)), "gg_bfs_ex")


def gg_sssp_batch(handle: int, srcs, dist_out, stream=None, options: gg_options | None = None):
    """Distances from every source in srcs (host uint32 array of k) into
    dist_out (CUDA uint32 tensor of n*k, dist_out[v*k + s]), async."""
    srcs = np.ascontiguousarray(srcs, dtype=np.uint32)
    p, dev = _ptr(dist_out)
    if not dev:
        raise ValueError("dist_out must be a CUDA tensor")
    sp = srcs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    if options is None:
        _check(load().gg_sssp_batch(handle, sp, srcs.shape[0], p, _stream_ptr(stream)), "gg_sssp_batch")
    else:
        _check(load().gg_sssp_batch_ex(handle, sp, srcs.shape[0], p, ctypes.byref(options), _stream_ptr(stream)),
               "gg_sssp_batch_ex")


def gg_sssp_multi(handles, srcs, dist_outs, stream=None, delta: int | None = None):
    """One query per (handles[i], srcs[i]) into dist_outs[i] (CUDA uint32
    tensors), all advanced together, async."""
    k = len(handles)
    if not (len(srcs) == len(dist_outs) == k):
        raise ValueError("handles, srcs and dist_outs differ in length")
    hs = (ctypes.c_void_p * k)(*handles)
    sp = np.ascontiguousarray(srcs, dtype=np.uint32)
    ptrs = []
    for d in dist_outs:
        p, dev = _ptr(d)
        if not dev:
            raise ValueError("dist_outs must be CUDA tensors")
        ptrs.append(p)
    dp = (ctypes.c_void_p * k)(*ptrs)
    spp = sp.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    if delta is None:
        _check(load().gg_sssp_multi(hs, spp, k, dp, _stream_ptr(stream)), "gg_sssp_multi")
    else:
        _check(load().gg_sssp_multi_ex(hs, spp, k, dp, delta, _stream_ptr(stream)), "gg_sssp_multi_ex")


def gg_sssp_tree(handle: int, src: int, dist, parent_out, tight_out=None, stream=None) -> int:
    """The edge-frontier program: parent_out (CUDA uint32 tensor of n) gets
    each reached vertex's smallest tight predecessor, tight_out (optional
    CUDA uint32 tensor) the tight edges' CSR positions; returns the number of
    tight edges.  Synchronous."""
    ptrs = [_ptr(a) for a in (dist, parent_out)]
    if not all(dev for _, dev in ptrs):
        raise ValueError("dist and parent_out must be CUDA tensors")
    tp, cap = None, 0
    if tight_out is not None:
        p, dev = _ptr(tight_out)
        if not dev:
            raise ValueError("tight_out must be a CUDA tensor")
        tp, cap = p, int(tight_out.numel())
    cnt = ctypes.c_uint64()
    _check(load().gg_sssp_tree(handle, src, ptrs[0][0], ptrs[1][0], tp, cap, ctypes.byref(cnt), _stream_ptr(stream)),
           "gg_sssp_tree")
    return int(cnt.value)


class Server:
    """Continuous-batching query server (gg_server_*).  Submit returns a
    ticket; results are written to the caller's CUDA tensor."""

    def __init__(self, max_graph_vertices: int, max_slots: int = 64, supersteps_per_launch: int = 8,
                 max_vertices_in_flight: int = 0, hbm_reserve_bytes: int = 1 << 30, delta: int = 0):
        lib = load()
        c = gg_server_config()
        lib.gg_server_config_default(ctypes.byref(c))
        c.max_graph_vertices = max_graph_vertices
        c.max_slots = max_slots
        c.supersteps_per_launch = supersteps_per_launch
        c.max_vertices_in_flight = max_vertices_in_flight
        c.hbm_reserve_bytes = hbm_reserve_bytes
        c.delta = delta
        h = ctypes.c_void_p()
        _check(lib.gg_server_create(ctypes.byref(c), ctypes.byref(h)), "gg_server_create")
        self.handle = h.value
        self._keep = {}

    def submit(self, graph, src: int, dist_out) -> int:
        p, dev = _ptr(dist_out)
        if not dev:
            raise ValueError("dist_out must be a CUDA tensor")
        t = ctypes.c_uint64()
        gh = graph.handle if isinstance(graph, Graph) else graph
        _check(load().gg_server_submit(self.handle, gh, src, p, ctypes.byref(t)), "gg_server_submit")
        self._keep[t.value] = dist_out
        return t.value

    def poll(self, ticket: int):
        """None while pending, else the query's status code (0 = GG_OK)."""
        r = ctypes.c_int()
        rc = load().gg_server_poll(self.handle, ticket, ctypes.byref(r))
        if rc == 6:
            return None
        _check(rc, "gg_server_poll")
        self._keep.pop(ticket, None)
        return r.value

    def wait(self, ticket: int, timeout_ms: int = 60000):
        r = ctypes.c_int()
        rc = load().gg_server_wait(self.handle, ticket, timeout_ms, ctypes.byref(r))
        if rc == 6:
            return None
        _check(rc, "gg_server_wait")
        self._keep.pop(ticket, None)
        return r.value

    def stats(self) -> dict:
        st = gg_server_stats()
        _check(load().gg_server_get_stats(self.handle, ctypes.byref(st)), "gg_server_get_stats")
        return st.as_dict()

    def reset_stats(self):
        _check(load().gg_server_reset_stats(self.handle), "gg_server_reset_stats")

    def close(self):
        if getattr(self, "handle", None):
            _check(load().gg_server_destroy(self.handle), "gg_server_destroy")
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


GG_NOALLOC_MAX_VERTICES = 1 << 20


def gg_sssp_noalloc(row_offsets, col_indices, weights, src: int, dist_out, stream=None):
    """Distances from src computed straight from a device CSR (CUDA uint32
    tensors) without allocating any device memory; returns when dist_out is
    complete.  For callers that must not allocate (see include/gg.h).

    The C call trusts the sizes it is given, so the lengths are checked here:
    weights must hold exactly as many entries as col_indices, dist_out at
    least n, and all four tensors must sit on one GPU.  The call runs with
    that GPU current (its built-in scratch array is the current device's)."""
    ptrs = [_ptr(a) for a in (row_offsets, col_indices, weights, dist_out)]
    if not all(dev for _, dev in ptrs):
        raise ValueError("gg_sssp_noalloc takes CUDA tensors only")
    devices = {a.device for a in (row_offsets, col_indices, weights, dist_out)}
    if len(devices) != 1:
        raise ValueError(f"gg_sssp_noalloc: row_offsets, col_indices, weights and dist_out are on "
                         f"different devices {sorted(str(d) for d in devices)}")
    if row_offsets.dim() != 1 or int(row_offsets.shape[0]) < 2:
        raise ValueError("row_offsets must be a 1-D tensor of n + 1 >= 2 entries")
    n = int(row_offsets.shape[0]) - 1
    m = int(col_indices.numel())
    if int(weights.numel()) != m:
        raise ValueError(f"weights has {int(weights.numel())} entries, col_indices {m}: they must match")
    if int(dist_out.numel()) < n:
        raise ValueError(f"dist_out has {int(dist_out.numel())} entries, fewer than n = {n}")
    import torch
    with torch.cuda.device(row_offsets.device):
        _check(load().gg_sssp_noalloc(n, m, ptrs[0][0], ptrs[1][0] if m else None, ptrs[2][0] if m else None,
                                      src, ptrs[3][0], _stream_ptr(stream)), "gg_sssp_noalloc")


class Graph:
    """Owning wrapper of a gg_graph_t."""

    def __init__(self, row_offsets, col_indices, weights, symmetric: bool = False, validate: bool = True,
                 stream=None, pack: bool = True, float_weights: bool = False):
        self.handle = gg_graph_create_csr(row_offsets, col_indices, weights, symmetric, validate, stream, pack,
                                          float_weights)
        self.n, self.m, _ = gg_graph_info(self.handle)
        self.float_weights = float_weights

    def bfs(self, src: int, depth_out=None, stream=None, **opts):
        """Hop counts from src (uint32 CUDA tensor; unreachable = GG_INF)."""
        import torch
        if depth_out is None:
            depth_out = torch.empty(self.n, dtype=torch.uint32, device="cuda")
        gg_bfs(self.handle, src, depth_out, stream, make_options(**opts) if opts else None)
        return depth_out

    def sssp(self, src: int, dist_out=None, stream=None, **opts):
        import torch
        if dist_out is None:
            dist_out = torch.empty(self.n, dtype=torch.uint32, device="cuda")
        if opts:
            gg_sssp_ex(self.handle, src, dist_out, make_options(**opts), stream)
        else:
            gg_sssp(self.handle, src, dist_out, stream)
        return dist_out

    def sssp_batch(self, srcs, dist_out=None, stream=None, **opts):
        """(n, k) view of the vertex-major distance matrix."""
        import torch
        k = len(srcs)
        if dist_out is None:
            dist_out = torch.empty(self.n * k, dtype=torch.uint32, device="cuda")
        gg_sssp_batch(self.handle, srcs, dist_out, stream, make_options(**opts) if opts else None)
        return dist_out.view(self.n, k)

    def check(self):
        gg_graph_check(self.handle)

    @property
    def device_bytes(self) -> int:
        return gg_graph_info(self.handle)[2]

    def close(self):
        if getattr(self, "handle", None):
            gg_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
