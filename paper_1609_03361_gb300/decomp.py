"""Single-shot domain decomposition along x: one grid cut into slabs of
computational x planes, each advanced by the CUDA library (``fdw_create_slab``,
``fdw_step``), with the r ghost planes on either side of a slab refreshed from
its neighbours after every time step.

Two drivers share the same slabs and schedule:

- ``SlabForward``: all slabs in this process (on one or several devices); the
  exchange is a device copy per neighbour pair (``fdw_exchange_ghosts``).
- ``slab_forward_distributed``: one slab per ``torch.distributed`` rank; the
  exchange copies the send planes out (``fdw_halo_copy``), swaps them with
  the neighbouring ranks point to point and copies the received planes into
  the ghost planes; the traces are summed over ranks (every receiver is
  recorded by exactly one slab, the others hold zeros in its column).

Each slab computes its planes with exactly the arithmetic of the whole-grid
step, so the decomposed traces and wavefield equal the whole-grid ones bit for
bit.  The paper (Sec. 6) names MPI parallelism only between whole inversion
operators; splitting one grid is an extension.
"""
from __future__ import annotations

from . import fdwave as fw


def slab_ranges(nx: int, nparts: int, r: int) -> list[tuple[int, int]]:
    """Contiguous, balanced ranges [x_begin, x_end) covering the nx
    computational planes, each at least r planes (a slab sends r planes)."""
    if nparts < 1 or nx < nparts * max(r, 1):
        raise ValueError(f"cannot cut {nx} planes into {nparts} slabs of at least {r}")
    base, extra = divmod(nx, nparts)
    out, x = [], 0
    for p in range(nparts):
        n = base + (1 if p < extra else 0)
        out.append((x, x + n))
        x += n
    return out


def neighbours(rank: int, world: int) -> tuple[int | None, int | None]:
    """Ranks of the lower and upper neighbour slab (None at the grid edges)."""
    return (rank - 1 if rank > 0 else None, rank + 1 if rank + 1 < world else None)


class SlabForward:
    """Forward modelling of one shot on `nparts` slabs held by this process.

    devices: one CUDA device per slab (default: all on device 0)."""

    def __init__(self, shape, spacing, space_order, nbl, dt, nt, vmax, nparts, devices=None):
        self.nt = int(nt)
        nx = int(shape[0]) + 2 * int(nbl)
        self.ranges = slab_ranges(nx, nparts, int(space_order) // 2)
        devices = devices or [0] * nparts
        self.slabs = [fw.Solver(shape, spacing, space_order, nbl, dt, nt, vmax, device=d, slab=rg)
                      for rg, d in zip(self.ranges, devices)]

    def set_model(self, m, layout="physical", dtype="f32"):
        for s in self.slabs:
            s.set_model(m, layout, dtype)

    def set_sources(self, xyz):
        for s in self.slabs:
            s.set_sources(xyz)

    def set_receivers(self, xyz):
        for s in self.slabs:
            s.set_receivers(xyz)

    def forward(self, qs, recs):
        """qs, recs: one device wavelet [nt][nsrc] and one zero-filled device
        trace array [nt][nrec] per slab (on the slab's device).  Returns recs;
        their sum is the whole grid's traces."""
        for n in range(self.nt - 1):
            for s, q, r in zip(self.slabs, qs, recs):
                s.step(n, q, r)
            for lo, hi in zip(self.slabs[:-1], self.slabs[1:]):
                fw.fdw_exchange_ghosts(lo.ctx, hi.ctx, n, None, hi.device)
        for s, q, r in zip(self.slabs, qs, recs):   # the last time level's samples
            s.step(self.nt - 1, q, r)
        return recs

    def close(self):
        for s in self.slabs:
            s.close()


def exchange_with_neighbours(send_lo, send_hi, recv_lo, recv_hi, rank, world):
    """Point-to-point swap of ghost planes between neighbouring ranks: this
    rank's send_lo goes to the lower neighbour's recv_hi and its send_hi to
    the upper neighbour's recv_lo.  Tensors of equal size (device tensors with
    NCCL, host tensors with gloo)."""
    import torch.distributed as dist
    lower, upper = neighbours(rank, world)
    ops = []
    if lower is not None:
        ops.append(dist.P2POp(dist.isend, send_lo, lower))
        ops.append(dist.P2POp(dist.irecv, recv_lo, lower))
    if upper is not None:
        ops.append(dist.P2POp(dist.isend, send_hi, upper))
        ops.append(dist.P2POp(dist.irecv, recv_hi, upper))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


def slab_forward_distributed(solver, q, rec, rank, world):
    """One slab per rank (``solver`` built with ``slab=``): time loop with a
    ghost-plane swap after every step, then the traces summed over ranks.
    q, rec are device tensors on the solver's device (rec zero-filled)."""
    import torch
    import torch.distributed as dist
    cnt = fw.fdw_halo_planes(solver.ctx, 0)[4]
    dev = torch.device("cuda", solver.device)
    bufs = [torch.zeros(cnt, dtype=torch.float32, device=dev) for _ in range(4)]
    send_lo, send_hi, recv_lo, recv_hi = bufs
    lower, upper = neighbours(rank, world)
    for n in range(solver.nt - 1):
        solver.step(n, q, rec)
        fw.fdw_halo_copy(solver.ctx, n, 0, send_lo, send_hi, None, solver.device)
        torch.cuda.current_stream(dev).synchronize()
        exchange_with_neighbours(send_lo, send_hi, recv_lo, recv_hi, rank, world)
        fw.fdw_halo_copy(solver.ctx, n, 1, recv_lo if lower is not None else None,
                         recv_hi if upper is not None else None, None, solver.device)
    solver.step(solver.nt - 1, q, rec)
    dist.all_reduce(rec, op=dist.ReduceOp.SUM)
    return rec
