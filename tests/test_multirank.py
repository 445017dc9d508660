"""The multi-rank (weak-scaling) path of bench.py on CPU: two gloo ranks shard
the k_par points without overlap and agree on the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n_k, steps, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ks = bench.shard_kpoints(rank, world, n_k, steps, first_step=3)
    gathered = [None] * world
    dist.all_gather_object(gathered, ks)
    tmax = bench.reduce_max(10.0 + rank, world, "cpu")
    dist.destroy_process_group()
    q.put((rank, gathered, tmax))


def test_two_gloo_ranks_shard_disjointly_and_reduce_max():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, n_k, steps = 2, 32, 5
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_k, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, tmax in res:
        assert tmax == 11.0
        per_step = list(zip(*gathered))
        for ks in per_step:                       # one step: ranks hold different k
            assert len(set(ks)) == world
        flat = [k for g in gathered for k in g]
        assert len(set(flat)) == world * steps    # no k repeated within the run
