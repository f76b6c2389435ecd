"""Receiver sharding over 2 ranks (gloo, CPU processes): the MINLOC exchange gives
the unsharded loss and argmin, and the summed per-rank gradients give the full
gradient (powers and gradients from the FP64 oracle)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2401_11882_gb300.dist import shard


def test_shard_covers_everything_once():
    for n in (0, 1, 7, 64, 1001):
        for world in (1, 2, 3, 8):
            blocks = [shard(n, world, r) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(blocks[i][1] == blocks[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2401_11882_gb300 import scenes
    from paper_2401_11882_gb300.dist import shard, sharded_min_loss, sum_allreduce
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = scenes.clutter_scene(6, 5, seed=3, max_order=1, alpha=40.0, smoothing="sigmoid")
        a, b = shard(sc.n_rx, world, rank)
        P = oracle.power(sc.walls, sc.tx, sc.rx[a:b], 1, 40.0, "sigmoid", threads=1)
        loss, arg = sharded_min_loss(P, a)
        g = np.zeros(b - a)
        if a <= arg < b:
            g[arg - a] = -1.0
        grad = oracle.gradient(sc.walls, sc.tx, sc.rx[a:b], 1, 40.0, "sigmoid", g, "tx", threads=1)
        total = sum_allreduce(torch.tensor(grad))
        out[rank] = (loss, arg, total.numpy().tolist())
    finally:
        dist.destroy_process_group()


def test_two_rank_min_loss_and_gradient(oracle_mod):
    from paper_2401_11882_gb300 import scenes
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    sc = scenes.clutter_scene(6, 5, seed=3, max_order=1, alpha=40.0, smoothing="sigmoid")
    P = oracle_mod.power(sc.walls, sc.tx, sc.rx, 1, 40.0, "sigmoid")
    loss, arg = oracle_mod.loss(P)
    g = np.zeros(sc.n_rx)
    g[arg] = -1.0
    grad = oracle_mod.gradient(sc.walls, sc.tx, sc.rx, 1, 40.0, "sigmoid", g, "tx")
    for r in range(world):
        l_r, a_r, g_r = out[r]
        assert a_r == arg and l_r == pytest.approx(loss, rel=1e-15)
        np.testing.assert_allclose(g_r, grad, rtol=1e-13)
