"""Halo exchange between ranks that each hold one y slab of a lattice.

The processors command (Sec. Commands; Sec. Parallelization) splits a
lattice over a grid of processes.  Here each rank (one process, one GPU)
holds one y slab (``Lattice.processor_rank``) and after every iteration
sends its first and last rows to the ranks below and above (periodic in y)
and receives their rows into its ghost rows.  The library packs and unpacks
the rows on the device (``lb_halo_pack`` / ``lb_halo_unpack``); this module
only moves the packed buffers between ranks with ``torch.distributed``
point-to-point operations (NCCL on GPUs, gloo on CPU) and sums the thermo
records.  It holds no step of the method.

Message schedule, per iteration, for rank r of W:
  face 1 (high y) rows -> rank (r + 1) % W, received there into face 0;
  face 0 (low y) rows  -> rank (r - 1) % W, received there into face 1.
With W = 2 both messages go to the same peer; NCCL matches them in the
order they are posted, gloo by tag (0: towards +y, 1: towards -y).
"""
from __future__ import annotations

from typing import Dict, Sequence

# thermo keys that add up over slabs (the others, step, are equal on all)
ADDITIVE = ("mass1", "mass2", "momx", "momy", "momx1", "momy1", "momx2", "momy2", "mass_eq1",
            "mass_eq2", "solute", "bsum", "removed1", "removed2", "removed_solute", "nsolid",
            "nfluid", "flips")


def exchange_buffers(dist, rank: int, world: int, send: Sequence, recv: Sequence) -> None:
    """Move send[1] (this rank's face-1 rows) to rank + 1's recv[0] and
    send[0] (face-0 rows) to rank - 1's recv[1], for every rank at once;
    returns when this rank's receives are complete."""
    if world == 1:
        recv[0].copy_(send[1])
        recv[1].copy_(send[0])
        return
    up, down = (rank + 1) % world, (rank - 1) % world
    if dist.get_backend() == "nccl":
        ops = [dist.P2POp(dist.isend, send[1], up), dist.P2POp(dist.irecv, recv[0], down),
               dist.P2POp(dist.isend, send[0], down), dist.P2POp(dist.irecv, recv[1], up)]
        reqs = dist.batch_isend_irecv(ops)
    else:
        reqs = [dist.isend(send[1], up, tag=0), dist.irecv(recv[0], down, tag=0),
                dist.isend(send[0], down, tag=1), dist.irecv(recv[1], up, tag=1)]
    for r in reqs:
        r.wait()


class SlabExchange:
    """Per-rank halo exchange of a slab: device buffers sized by the
    library, packed and unpacked by it, moved by ``exchange_buffers``.

    ``slab`` needs halo_size(), halo_pack(face, buf), halo_unpack(face, buf)
    (``lb2d.Lattice`` after processor_rank)."""

    def __init__(self, slab, dist, rank: int, world: int, device):
        import torch
        n = slab.halo_size()
        self.slab, self.dist, self.rank, self.world = slab, dist, rank, world
        self.send = [torch.empty(n, dtype=torch.uint8, device=device) for _ in range(2)]
        self.recv = [torch.empty(n, dtype=torch.uint8, device=device) for _ in range(2)]

    def __call__(self) -> None:
        for face in (0, 1):
            self.slab.halo_pack(face, self.send[face])
        exchange_buffers(self.dist, self.rank, self.world, self.send, self.recv)
        for face in (0, 1):
            self.slab.halo_unpack(face, self.recv[face])

    @property
    def bytes_per_iteration(self) -> int:
        return 2 * self.send[0].numel()


def reduce_thermo(dist, world: int, record: Dict[str, float], device=None) -> Dict[str, float]:
    """The lattice's thermo record from the slabs' own records: FP64 sums of
    the additive quantities over all ranks (all_reduce)."""
    import torch
    out = dict(record)
    if world == 1:
        return out
    keys = [k for k in ADDITIVE if k in record]
    t = torch.tensor([float(record[k]) for k in keys], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    for k, v in zip(keys, t.tolist()):
        out[k] = v
    return out
