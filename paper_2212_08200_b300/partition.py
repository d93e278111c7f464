"""Single-source SSSP over a 1D vertex partition, one part per rank.

Sec. III-D (with Table I) names partitioning as the way a graph is spread
over processors; the simplest is a random vertex partition.  Here every rank
(one process, one GPU) holds a part made by ``part_of``: the out-edges of the
vertices it owns, with global column ids, and a route word per global vertex
(owner rank << 24 | index among the owner's vertices).  ``sssp`` then runs the
bulk-synchronous loop of the C ABI's gg_part_* calls:

    advance   (gg_part_advance, CUDA) relax the part's frontier; updates to
              other ranks' vertices come back grouped by destination;
    exchange  (``exchange_pairs``) the groups move between ranks with
              point-to-point collectives of torch.distributed (NCCL for
              device tensors, gloo through host memory);
    apply     (gg_part_apply, CUDA) relax the received pairs and close the
              superstep;
    converge  one all-reduce of the ranks' next frontier sizes.

Every relaxation runs in the library's kernels; this module only builds the
host-side partition, moves buffers and counts, and drives the loop.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _check, _ptr, _stream_ptr, load

MAX_RANKS = 256
MAX_LOCAL = 1 << 24


def random_owner(n: int, nranks: int, seed: int = 1) -> np.ndarray:
    """owner[v] uniform over the ranks (seeded; the same on every rank)."""
    if not 1 <= nranks <= MAX_RANKS:
        raise ValueError("nranks must be in [1, 256]")
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, nranks, n).astype(np.uint32)


def routes(owner: np.ndarray, nranks: int) -> np.ndarray:
    """route[v] = (owner << 24) | index of v among its owner's vertices
    (ascending global id)."""
    owner = np.asarray(owner, np.uint32)
    local = np.empty(owner.shape[0], np.uint32)
    for r in range(nranks):
        ids = np.flatnonzero(owner == r)
        if ids.shape[0] > MAX_LOCAL:
            raise ValueError("a part would hold more than 2^24 vertices")
        local[ids] = np.arange(ids.shape[0], dtype=np.uint32)
    return (owner << np.uint32(24)) | local


def part_of(ro, col, w, owner: np.ndarray, rank: int, nranks: int):
    """(route, vertices, row_offsets, cols, weights) of rank's part: its owned
    vertices in ascending id order with their out-edges (global columns)."""
    ro = np.asarray(ro, np.int64)
    verts = np.flatnonzero(np.asarray(owner) == rank).astype(np.uint32)
    deg = ro[verts.astype(np.int64) + 1] - ro[verts.astype(np.int64)]
    lro = np.zeros(verts.shape[0] + 1, np.int64)
    np.cumsum(deg, out=lro[1:])
    total = int(lro[-1])
    # the global position of every edge of the part: row start + offset in the row
    idx = np.repeat(ro[verts.astype(np.int64)] - lro[:-1], deg) + np.arange(total, dtype=np.int64)
    return (routes(owner, nranks), verts, lro.astype(np.uint32), np.asarray(col, np.uint32)[idx],
            np.asarray(w, np.uint32)[idx])


class PartGraph:
    """Owning wrapper of a gg_part_t (this rank's part on the current GPU)."""

    def __init__(self, n_global: int, rank: int, nranks: int, route, row_offsets, cols, weights, stream=None):
        lib = load()
        arrs = [np.ascontiguousarray(a, np.uint32) for a in (route, row_offsets, cols, weights)]
        n_local = arrs[1].shape[0] - 1
        h = ctypes.c_void_p()
        _check(lib.gg_part_create(n_global, rank, nranks, n_local, *[a.ctypes.data for a in arrs],
                                  _stream_ptr(stream), ctypes.byref(h)), "gg_part_create")
        self.handle, self.lib = h.value, lib
        self.n_global, self.rank, self.nranks, self.n_local = n_global, rank, nranks, n_local
        self.m_local = int(arrs[1][-1])

    def close(self):
        if getattr(self, "handle", None):
            _check(self.lib.gg_part_destroy(self.handle), "gg_part_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def exchange_pairs(send, send_counts, group=None):
    """Moves each rank's pairs to their destination ranks.  send: u32 tensor
    of 2 * sum(send_counts) entries, destination d's pairs from offset
    2 * sum(send_counts[:d]); send_counts: nranks ints.  Returns (recv, total
    pairs received), recv on send's device.  Device tensors go over the
    process group directly; a gloo group gets host copies."""
    import torch
    import torch.distributed as dist
    world, me = dist.get_world_size(group), dist.get_rank(group)
    dev = send.device
    host = dist.get_backend(group) == "gloo"
    cnt = torch.tensor([int(c) for c in send_counts], dtype=torch.int64)
    allc = [torch.zeros(world, dtype=torch.int64) for _ in range(world)]
    if host:
        dist.all_gather(allc, cnt, group=group)
    else:
        allc_d = [c.to(dev) for c in allc]
        dist.all_gather(allc_d, cnt.to(dev), group=group)
        allc = [c.cpu() for c in allc_d]
    recv_counts = [int(allc[s][me]) for s in range(world)]
    total = sum(recv_counts)
    buf_dev = "cpu" if host else dev
    sbuf = send.view(torch.int32).to(buf_dev) if host else send.view(torch.int32)
    rbuf = torch.empty(max(2 * total, 1), dtype=torch.int32, device=buf_dev)
    ops = []
    off = 0
    for d in range(world):
        c = int(send_counts[d])
        if d != me and c:
            ops.append(dist.P2POp(dist.isend, sbuf[2 * off:2 * (off + c)], d, group=group))
        off += c
    off = 0
    for s in range(world):
        c = recv_counts[s]
        if s != me and c:
            ops.append(dist.P2POp(dist.irecv, rbuf[2 * off:2 * (off + c)], s, group=group))
        off += c
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    return rbuf.to(dev).view(torch.uint32), total


def sssp(part: PartGraph, src: int, group=None, stream=None, max_supersteps: int | None = None):
    """Distances from global vertex src to this rank's vertices (device u32
    tensor, local order) and the number of supersteps.  Every rank of the
    group calls it with the same src; without a process group (or with one
    rank) there is nothing to exchange."""
    import torch
    import torch.distributed as dist
    grouped = group is not None or (dist.is_available() and dist.is_initialized())
    world = dist.get_world_size(group) if grouped else 1
    lib = part.lib
    sp = _stream_ptr(stream)
    _check(lib.gg_part_begin(part.handle, src, sp), "gg_part_begin")
    cap = max(part.m_local, 1)
    send = torch.empty(2 * cap, dtype=torch.uint32, device="cuda")
    counts = (ctypes.c_uint64 * part.nranks)()
    nxt = ctypes.c_uint32()
    steps = 0
    limit = max_supersteps if max_supersteps is not None else 4 * part.n_global + 16
    while True:
        _check(lib.gg_part_advance(part.handle, sp, _ptr(send)[0], cap, counts), "gg_part_advance")
        sent = [int(counts[d]) for d in range(part.nranks)]
        if world > 1:
            recv, total = exchange_pairs(send[:2 * sum(sent)], sent, group)
        else:
            recv, total = send[:0], 0
        _check(lib.gg_part_apply(part.handle, _ptr(recv)[0] if total else None, total, sp, ctypes.byref(nxt)),
               "gg_part_apply")
        steps += 1
        left = int(nxt.value)
        if world > 1:
            t = torch.tensor([left], dtype=torch.int64,
                             device="cpu" if dist.get_backend(group) == "gloo" else "cuda")
            dist.all_reduce(t, group=group)
            left = int(t.item())
        if left == 0 or steps >= limit:
            break
    out = torch.empty(max(part.n_local, 1), dtype=torch.uint32, device="cuda")
    _check(lib.gg_part_distances(part.handle, _ptr(out)[0], sp), "gg_part_distances")
    torch.cuda.synchronize()
    return out[:part.n_local], steps
