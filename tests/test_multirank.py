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


def _worker_uneven(rank, world, port, q):
    import numpy as np
    import torch.distributed as dist
    import bench
    from synthetic import uneven_batch
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    insts = uneven_batch(2048)[:96]
    w = [bench.instance_weight(x) for x in insts]
    mine = bench.shard_instances(w, rank, world)
    # a stand-in per-instance T and gradient (the exchange, not the physics, is under test)
    T = {i: 1.0 + np.sin(i) for i in mine}
    g = sum((np.cos(np.arange(5) * (i + 1)) for i in mine), np.zeros(5))
    tot = bench.reduce_sum([sum(T.values())], world, "cpu")[0]
    gsum = bench.reduce_sum(g, world, "cpu")
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    dist.destroy_process_group()
    q.put((rank, gathered, tot, gsum.tolist(), w))


def test_uneven_instances_shard_by_weight_and_sum_on_the_host():
    """Two gloo ranks split the first 96 uneven instances by n^3 (N_s + 1):
    disjoint, complete, loads within the largest single weight of each other;
    the host-side sums of the summed T and of a gradient vector equal the
    serial sums on both ranks."""
    import numpy as np
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world = 2
    port = _free_port()
    procs = [ctx.Process(target=_worker_uneven, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    serial_T = sum(1.0 + np.sin(i) for i in range(96))
    serial_g = sum((np.cos(np.arange(5) * (i + 1)) for i in range(96)), np.zeros(5))
    for rank, gathered, tot, gsum, w in res:
        flat = sorted(i for g in gathered for i in g)
        assert flat == list(range(96))
        loads = [sum(w[i] for i in g) for g in gathered]
        assert abs(loads[0] - loads[1]) <= max(w) + 1e-6
        assert abs(tot - serial_T) < 1e-9
        assert np.allclose(gsum, serial_g, rtol=0, atol=1e-9)
