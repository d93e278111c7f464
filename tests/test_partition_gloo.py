"""Host logic of the partitioned single-source loop on CPU (no GPU): the 1D
random partition reassembles the graph, the pair exchange delivers every
group to its destination under a world-size 2 and 3 gloo group, and a CPU
model of the loop (relaxations emulated in numpy, exchange through the real
exchange_pairs) reaches the oracle's distances."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import graphgen
import oracle
from paper_2212_08200_b300 import partition as P

INF = 0xFFFFFFFF


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("nranks", [1, 2, 3, 5])
def test_parts_reassemble_the_graph(nranks):
    ro, col, w = graphgen.rmat(10, 16, seed=4, W=255)
    n = ro.shape[0] - 1
    owner = P.random_owner(n, nranks, seed=7)
    seen = np.zeros(n, np.int64)
    edges = []
    for r in range(nranks):
        route, verts, lro, lcol, lw = P.part_of(ro, col, w, owner, r, nranks)
        assert np.all(route[verts] >> 24 == r)
        np.testing.assert_array_equal(route[verts] & 0xFFFFFF, np.arange(verts.shape[0]))
        seen[verts] += 1
        for i, v in enumerate(verts):
            edges += [(int(v), int(c), int(x)) for c, x in zip(lcol[lro[i]:lro[i + 1]], lw[lro[i]:lro[i + 1]])]
    assert np.all(seen == 1)                                 # every vertex owned exactly once
    rows = np.repeat(np.arange(n), np.diff(ro.astype(np.int64)))
    assert sorted(edges) == sorted(zip(rows.tolist(), col.tolist(), w.tolist()))


def _exchange_worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.Generator(np.random.PCG64(100 + rank))
        counts = [0 if d == rank else int(rng.integers(0, 5)) for d in range(world)]
        pairs = np.concatenate([np.stack([np.full(c, 1000 * rank + d), rng.integers(0, 99, c)], 1).ravel()
                                for d, c in enumerate(counts)]).astype(np.uint32)
        np.save(os.path.join(out_dir, f"sent{rank}.npy"), pairs)
        np.save(os.path.join(out_dir, f"counts{rank}.npy"), np.array(counts))
        recv, total = P.exchange_pairs(torch.from_numpy(pairs.view(np.int32)).view(torch.uint32), counts)
        np.save(os.path.join(out_dir, f"recv{rank}.npy"), recv.view(torch.int32).numpy()[:2 * total].view(np.uint32))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_delivers_every_group(tmp_path, world):
    mp.spawn(_exchange_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    sent = [np.load(tmp_path / f"sent{r}.npy").reshape(-1, 2) for r in range(world)]
    counts = [np.load(tmp_path / f"counts{r}.npy") for r in range(world)]
    for me in range(world):
        expect = []
        for s in range(world):
            off = int(counts[s][:me].sum())
            expect.append(sent[s][off:off + int(counts[s][me])])
        got = np.load(tmp_path / f"recv{me}.npy").reshape(-1, 2)
        np.testing.assert_array_equal(got, np.concatenate(expect))   # sender order, each group intact


def _model_worker(rank, world, port, out_dir):
    """The loop of partition.sssp with its two device calls emulated in numpy."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ro, col, w = graphgen.random_graph(400, 1600, 30, seed=5, wmin=0)
        n = ro.shape[0] - 1
        owner = P.random_owner(n, world, seed=3)
        route, verts, lro, lcol, lw = P.part_of(ro, col, w, owner, rank, world)
        nl = verts.shape[0]
        dist_l = np.full(nl, 1 << 40, np.int64)
        src = 0
        front = []
        if route[src] >> 24 == rank:
            dist_l[route[src] & 0xFFFFFF] = 0
            front = [int(route[src] & 0xFFFFFF)]
        while True:
            nxt, out = set(), [[] for _ in range(world)]
            for u in front:                                  # advance
                for e in range(lro[u], lro[u + 1]):
                    r = int(route[lcol[e]])
                    nd = dist_l[u] + int(lw[e])
                    if r >> 24 == rank:
                        if nd < dist_l[r & 0xFFFFFF]:
                            dist_l[r & 0xFFFFFF] = nd
                            nxt.add(r & 0xFFFFFF)
                    else:
                        out[r >> 24] += [r & 0xFFFFFF, nd]
            counts = [len(o) // 2 for o in out]
            send = np.array(sum(out, []), np.uint32)
            recv, total = P.exchange_pairs(torch.from_numpy(send.view(np.int32)).view(torch.uint32), counts)
            pr = recv.view(torch.int32).numpy()[:2 * total].view(np.uint32).reshape(-1, 2)
            for lv, nd in pr:                                 # apply
                if nd < dist_l[lv]:
                    dist_l[lv] = nd
                    nxt.add(int(lv))
            front = sorted(nxt)
            t = torch.tensor([len(front)], dtype=torch.int64)
            dist.all_reduce(t)
            if int(t.item()) == 0:
                break
        np.save(os.path.join(out_dir, f"d{rank}.npy"), np.stack([verts, np.where(dist_l >= 1 << 40, INF, dist_l)]))
    finally:
        dist.destroy_process_group()


def test_partitioned_loop_model_reaches_the_oracle(tmp_path):
    world = 2
    mp.spawn(_model_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    ro, col, w = graphgen.random_graph(400, 1600, 30, seed=5, wmin=0)
    got = np.full(ro.shape[0] - 1, 7, np.int64)
    for r in range(world):
        v, d = np.load(tmp_path / f"d{r}.npy")
        got[v] = d
    np.testing.assert_array_equal(got.astype(np.uint32), oracle.dijkstra(ro, col, w, 0))
