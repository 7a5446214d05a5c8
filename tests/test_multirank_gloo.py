"""Shot-parallel FWI gradient across ranks (world size 2, gloo, CPU).

Each rank computes the FP64 oracle gradient of its own shots and the ranks
sum them with one all-reduce; the result must equal the single-process sum
exactly up to the order of two float64 additions."""
import os

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1609_03361_gb300.shots import allreduce_gradient, shard


def _problem():
    import oracle
    from paper_1609_03361_gb300 import workloads as W
    shape, h, p = (22, 18), 10.0, 4
    v = np.full(shape, 1.5)
    v[:, 9:] = 2.0
    dt = 0.8 * oracle.dt_max(2, h, p, 2.0)
    nt = 90
    s = oracle.Setup(shape, h, p, 5, dt, nt)
    M = oracle.extend_model(s, 1 / v ** 2)
    eta = oracle.damping(s, 2.0)
    rec = np.array([[x, 20.0] for x in np.linspace(0, 210, 7)])
    srcs = [np.array([[x, 30.0]]) for x in (30.0, 80.0, 130.0, 180.0, 200.0)]
    q = W.ricker(25.0, dt, nt)[:, None]
    rng = np.random.default_rng(1)
    d = rng.standard_normal((nt, rec.shape[0]))
    return s, M, eta, srcs, q, rec, d


def _shot_gradient(i):
    import oracle
    s, M, eta, srcs, q, rec, d = _problem()
    r = oracle.forward(s, M, eta, srcs[i], q, rec) - d
    return oracle.gradient(s, M, eta, srcs[i], q, rec, r)


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = torch.zeros(_problem()[1].shape, dtype=torch.float64)
    for i in shard(5, rank, world):
        g += torch.from_numpy(_shot_gradient(i))
    g = allreduce_gradient(g)
    if rank == 0:
        torch.save(g, out)
    dist.destroy_process_group()


def test_shard_round_robin():
    assert shard(5, 0, 2) == [0, 2, 4] and shard(5, 1, 2) == [1, 3]
    assert sorted(sum((shard(7, r, 3) for r in range(3)), [])) == list(range(7))
    with pytest.raises(ValueError):
        shard(4, 2, 2)


def test_two_rank_gradient_sum(tmp_path):
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    out = str(tmp_path / "g.pt")
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    g2 = torch.load(out).numpy()
    g1 = sum(_shot_gradient(i) for i in range(5))
    assert np.allclose(g2, g1, rtol=1e-13, atol=1e-13 * np.abs(g1).max())
