"""The multi-process path of bench.py on CPU (gloo, world_size 2): each rank
draws its own batch of the same shape (chains are independent, no data-path
collective), and timing is reduced as the max over ranks after a barrier."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    from paper_2010_08482_gb300 import workloads as w
    w_, r_, l_ = bench.dist_setup()
    assert (w_, r_, l_) == (world, rank, rank)
    b = w.batch_t2g(32, rank=rank)
    first = torch.tensor(b.tau[:4].copy())
    gathered = [torch.zeros(4, dtype=first.dtype) for _ in range(world)]
    dist.all_gather(gathered, first)
    bench.barrier(world)
    local = 1.0 + rank  # a per-rank elapsed time
    m = bench.max_over_ranks(world, local, "cpu")
    out[rank] = (b.n_chains, m, [g.numpy().tolist() for g in gathered])
    dist.destroy_process_group()


def test_two_rank_gloo_weak_scaling_logic():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 32
    assert out[0][1] == out[1][1] == 2.0  # max over ranks
    g = out[0][2]
    assert not np.allclose(g[0], g[1])  # independent batches per rank
