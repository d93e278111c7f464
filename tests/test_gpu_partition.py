"""GPU parity of single-source SSSP over a 1D random vertex partition
(gg_part_* through partition.sssp) against the oracle, bit-exact.

World size 1 runs in-process.  World sizes 2 and 3 run as processes on the
one GPU of the box, exchanging through a gloo group in host memory: every
kernel of a rank finishes before its host exchanges, and no kernel waits on
another rank's, so the ranks need not run at the same time."""
import os
import socket

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def graphs():
    yield "rmat14", graphgen.rmat(14, 16, seed=1, W=255), None
    yield "grid64", graphgen.grid(64, 64, 1), 0
    ro, col, w = graphgen.random_graph(3000, 9000, 20, seed=2, wmin=0)   # directed: sinks, zero weights
    yield "directed", (ro, col, w), None


def run_rank(rank, world, ro, col, w, src, group=None):
    from paper_2212_08200_b300 import partition as P
    n = ro.shape[0] - 1
    owner = P.random_owner(n, world, seed=11)
    route, verts, lro, lcol, lw = P.part_of(ro, col, w, owner, rank, world)
    part = P.PartGraph(n, rank, world, route, lro, lcol, lw)
    d, steps = P.sssp(part, src, group=group)
    part.close()
    return verts, d.cpu().numpy(), steps


def _src(name, ro, fixed):
    return fixed if fixed is not None else int(graphgen.max_degree_vertex(ro))


def test_one_rank_matches_oracle():
    for name, (ro, col, w), fixed in graphs():
        src = _src(name, ro, fixed)
        verts, d, steps = run_rank(0, 1, ro, col, w, src)
        np.testing.assert_array_equal(verts, np.arange(ro.shape[0] - 1))
        np.testing.assert_array_equal(d, oracle.dijkstra(ro, col, w, src), err_msg=name)
        assert steps >= 1


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for name, (ro, col, w), fixed in graphs():
            verts, d, steps = run_rank(rank, world, ro, col, w, _src(name, ro, fixed))
            np.save(os.path.join(out_dir, f"{name}_{rank}.npy"), np.stack([verts, d]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_on_one_gpu_match_oracle(tmp_path, world):
    import torch.multiprocessing as mp
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for name, (ro, col, w), fixed in graphs():
        src = _src(name, ro, fixed)
        got = np.full(ro.shape[0] - 1, 7, np.uint32)
        owned = np.zeros(ro.shape[0] - 1, np.int64)
        for r in range(world):
            v, d = np.load(tmp_path / f"{name}_{r}.npy")
            got[v] = d
            owned[v] += 1
        assert np.all(owned == 1)
        np.testing.assert_array_equal(got, oracle.dijkstra(ro, col, w, src), err_msg=name)


def test_part_argument_errors():
    import paper_2212_08200_b300 as gg
    from paper_2212_08200_b300 import partition as P
    ro, col, w = graphgen.grid(8, 5, 1)
    n = ro.shape[0] - 1
    owner = P.random_owner(n, 2, seed=1)
    route, verts, lro, lcol, lw = P.part_of(ro, col, w, owner, 0, 2)
    with pytest.raises(gg.GGError):                   # rank >= nranks
        P.PartGraph(n, 2, 2, route, lro, lcol, lw)
    with pytest.raises(gg.GGError):                   # the other rank's vertex count
        P.PartGraph(n, 1, 2, route, lro, lcol, lw)
    bad = lcol.copy()
    bad[0] = n
    with pytest.raises(gg.GGError):                   # a column >= n_global
        P.PartGraph(n, 0, 2, route, lro, bad, lw)
