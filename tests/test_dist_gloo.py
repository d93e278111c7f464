"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the query
shards are disjoint and complete, the timing reductions take the max / sum
over ranks, and each rank's share of a batched-source workload, answered by
the CPU oracle, reassembles into the single-rank answer.  No GPU needed."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import graphgen
import oracle


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        queries = list(range(2000))
        mine = bench.shard(queries, rank, world)
        t_max = bench.reduce_over_ranks(1.0 + rank, "max", dist)
        n_sum = bench.reduce_over_ranks(len(mine), "sum", dist)
        ro, col, w = graphgen.rmat(10, 8, seed=3, W=255)
        srcs = graphgen.sample_sources(ro, 8, seed=1)
        my_srcs = bench.shard(list(srcs), rank, world)
        d = oracle.dijkstra_many(ro, col, w, np.array(my_srcs, np.uint32))
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), d)
        np.save(os.path.join(out_dir, f"meta{rank}.npy"), np.array([t_max, n_sum] + mine[:3], np.float64))
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_and_reductions(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    m0 = np.load(tmp_path / "meta0.npy")
    m1 = np.load(tmp_path / "meta1.npy")
    assert m0[0] == m1[0] == 2.0                      # max over ranks of (1 + rank)
    assert m0[1] == m1[1] == 2000                     # shards cover every query once
    assert list(m0[2:]) == [0, 2, 4] and list(m1[2:]) == [1, 3, 5]
    ro, col, w = graphgen.rmat(10, 8, seed=3, W=255)
    srcs = graphgen.sample_sources(ro, 8, seed=1)
    full = oracle.dijkstra_many(ro, col, w, srcs)
    d0, d1 = np.load(tmp_path / "rank0.npy"), np.load(tmp_path / "rank1.npy")
    np.testing.assert_array_equal(full[0::2], d0)
    np.testing.assert_array_equal(full[1::2], d1)


def test_shard_single_rank_is_identity():
    assert bench.shard([1, 2, 3], 0, 1) == [1, 2, 3]
    assert bench.reduce_over_ranks(3.5, "max", None) == 3.5
