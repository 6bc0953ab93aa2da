"""Row sharding of the 2D scan over 2 and 3 ranks (gloo on CPU, no GPU).

Each rank computes its block of t1 rows (here with the FP64 oracle standing in
for the GPU row kernel), the blocks are gathered, and the assembled R_I, R_II
must equal the single-process result exactly.  With more ranks than t1 rows the
ranks without rows compute nothing and still take part in the gather.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import workloads as W
from paper_2601_20550_gb300.shard import response_2d_sharded, row_range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out, n1=5):
    import torch.distributed as dist
    from oracle import heom as OH
    from oracle import model as OM
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    model = W.small_two_mode(n1=2, n2=2, depth_L=2)
    grid = W.grid(0.5, 2, n1, 4, (0.0, 2.0), t_eq_fs=4.0)
    prob = OM.Problem(model)
    rho_eq, _, _ = OH.equilibrate(prob, grid["dt_fs"], t_eq_fs=grid["t_eq_fs"])
    full_I, full_II = OH.response_2d(prob, rho_eq, grid)

    def rows_fn(j0, j1):
        assert j1 > j0   # the row kernel rejects an empty block
        return full_I[:, j0:j1], full_II[:, j0:j1]

    RI, RII = response_2d_sharded(None, None, grid, dist=dist, rows_fn=rows_fn)
    ok = np.array_equal(RI, full_I) and np.array_equal(RII, full_II)
    out[rank] = 1 if ok else 0
    dist.destroy_process_group()


def test_row_range_partition():
    for n1 in (1, 5, 64, 127):
        for world in (1, 2, 3, 8):
            blocks = [row_range(n1, world, r) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n1
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("world, n1", [(2, 5), (3, 2)])
def test_sharded_gather_gloo(world, n1):
    ctx = mp.get_context("spawn")
    out = ctx.Array("i", world)
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out, n1)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs)
    assert list(out) == [1] * world
