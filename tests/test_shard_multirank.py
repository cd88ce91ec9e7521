"""Splitting one problem along the horizontal axis over ranks (the bench's
`--shard columns` mode), checked on CPU with world size 2 (gloo).

Every step of Algorithms 1 and 2 separates along the horizontal axis
(Section IV-C; Section V), so ranks that each solve a contiguous set of image
columns, with the whole k-space, together compute exactly the whole
reconstruction.  Here each rank runs the FP64 oracle on its column shard
and the shards are gathered on rank 0, which compares them with the oracle's
solve of the whole problem: the two must agree to rounding.
"""

import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_column_shards_cover_every_column_once():
    sys.path.insert(0, ROOT)
    import bench
    for Nx in (1, 7, 64, 256, 1023):
        for world in (1, 2, 3, 4, 8):
            if world > Nx:
                continue
            spans = [bench.column_shard(Nx, world, r) for r in range(world)]
            assert spans[0][0] == 0
            for (a, w), (b, _) in zip(spans, spans[1:]):
                assert b == a + w
            assert spans[-1][0] + spans[-1][1] == Nx
            widths = [w for _, w in spans]
            assert max(widths) - min(widths) <= 1 and min(widths) >= 1


def _rank(rank, world, port, prior, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import synthdata
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    c = synthdata.make_case("tiny", Nx=18, Ny=32, Nt=5, Nc=3, iters=12)
    i0, w = bench.column_shard(18, world, rank)
    prob = oracle.Problem(c.kspace, c.sens, c.mask, c.mu, np.arange(i0, i0 + w))
    x, _ = prob.solve(prior, c.lam, c.mu, c.rho, c.iters, objective=False)
    parts = [None] * world
    dist.all_gather_object(parts, (i0, x))
    if rank == 0:
        whole = np.concatenate([p[1] for p in sorted(parts, key=lambda p: p[0])], axis=2)
        ref, _ = oracle.Problem(c.kspace, c.sens, c.mask, c.mu).solve(prior, c.lam, c.mu, c.rho, c.iters,
                                                                       objective=False)
        q.put(float(np.linalg.norm(whole - ref) / np.linalg.norm(ref)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("prior", ["tv", "dft"])
def test_two_column_shards_equal_the_whole(prior):
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, prior, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(300)
        assert p.exitcode == 0
    err = q.get(timeout=10)
    assert err < 1e-12, err
