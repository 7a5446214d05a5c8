"""Host logic of the single-shot domain decomposition (no GPU): slab ranges,
neighbours, and the ghost-plane swap between gloo ranks (world size 3)."""
import os
import socket

import pytest
import torch
import torch.multiprocessing as mp

from paper_1609_03361_gb300.decomp import exchange_with_neighbours, neighbours, slab_ranges


@pytest.mark.parametrize("nx,parts,r", [(336, 2, 4), (336, 3, 4), (181, 4, 2), (17, 2, 8), (9, 1, 8)])
def test_slab_ranges_cover_and_balance(nx, parts, r):
    rg = slab_ranges(nx, parts, r)
    assert rg[0][0] == 0 and rg[-1][1] == nx
    assert all(a[1] == b[0] for a, b in zip(rg[:-1], rg[1:]))
    sizes = [e - b for b, e in rg]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= r


def test_slab_ranges_reject_thin_slabs():
    with pytest.raises(ValueError):
        slab_ranges(15, 2, 8)
    with pytest.raises(ValueError):
        slab_ranges(10, 0, 1)


def test_neighbours():
    assert neighbours(0, 1) == (None, None)
    assert neighbours(0, 3) == (None, 1)
    assert neighbours(1, 3) == (0, 2)
    assert neighbours(2, 3) == (1, None)


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 7
    send_lo = torch.full((n,), 10.0 * rank + 1)
    send_hi = torch.full((n,), 10.0 * rank + 2)
    recv_lo = torch.full((n,), -1.0)
    recv_hi = torch.full((n,), -1.0)
    exchange_with_neighbours(send_lo, send_hi, recv_lo, recv_hi, rank, world)
    torch.save((recv_lo, recv_hi), os.path.join(out, f"r{rank}.pt"))
    dist.destroy_process_group()


def test_ghost_swap_between_three_ranks(tmp_path):
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    mp.start_processes(_worker, args=(3, port, str(tmp_path)), nprocs=3, join=True,
                       start_method="spawn")
    got = [torch.load(tmp_path / f"r{r}.pt") for r in range(3)]
    # recv_lo of rank r = send_hi of rank r-1; recv_hi of rank r = send_lo of rank r+1
    assert torch.all(got[0][0] == -1) and torch.all(got[0][1] == 11)
    assert torch.all(got[1][0] == 2) and torch.all(got[1][1] == 21)
    assert torch.all(got[2][0] == 12) and torch.all(got[2][1] == -1)
