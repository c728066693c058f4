"""The halo-exchange schedule of a lattice split over ranks (processors
command, Sec. Parallelization) on CPU with the gloo backend: world sizes 2,
3 and 4, each rank one y slab with ghost rows.

Each rank streams the nine populations of its slab (pull from x - e_i,
periodic; the streaming step of the method without the collision, in numpy)
and exchanges its halo rows through ``halo.exchange_buffers`` with the
library's message layout (face 1 rows to rank + 1, face 0 rows to rank - 1);
after several iterations every slab must hold exactly the rows of the same
streaming applied to the whole array.  The thermo sums of the slabs must add
up to the whole lattice's.  No GPU: the packing the library does on the
device is done here on host arrays."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
NX, NY, STEPS = 13, 29, 7


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _stream(f):
    """pull streaming of [9][ny][nx] populations, periodic"""
    return np.stack([np.roll(np.roll(f[i], EY[i], axis=0), EX[i], axis=1) for i in range(9)])


class HostSlab:
    """Rows [y0, y0 + n) of a [9][NY][NX] array with H ghost rows per side,
    with the halo calls of the library (face 0 low y, face 1 high y; the
    message holds H rows of every plane)."""

    def __init__(self, full, rank, world, H):
        self.H = H
        self.y0 = rank * NY // world
        self.n = (rank + 1) * NY // world - self.y0
        rows = [(self.y0 - H + k) % NY for k in range(self.n + 2 * H)]
        self.f = full[:, rows, :].copy()

    def halo_size(self):
        return 9 * self.H * NX * 8

    def _rows(self, face, ghost):
        H, n = self.H, self.n
        if face == 0:
            return slice(0, H) if ghost else slice(H, 2 * H)
        return slice(H + n, 2 * H + n) if ghost else slice(n, H + n)

    def halo_pack(self, face, buf):
        buf.numpy()[:] = np.ascontiguousarray(self.f[:, self._rows(face, False), :]).view(np.uint8).ravel()

    def halo_unpack(self, face, buf):
        self.f[:, self._rows(face, True), :] = buf.numpy().view(np.float64).reshape(9, self.H, NX)

    def step(self):
        # stream the held rows; only the own rows are exact afterwards
        g = _stream(self.f)
        self.f[:, self.H:self.H + self.n, :] = g[:, self.H:self.H + self.n, :]

    def own(self):
        return self.f[:, self.H:self.H + self.n, :]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1202_0442_gb300 import halo
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(5)
        full = rng.random((9, NY, NX))
        ok = True
        for H in (1, 2):
            s = HostSlab(full, rank, world, H)
            ex = halo.SlabExchange(s, dist, rank, world, "cpu")
            ref = full.copy()
            for _ in range(STEPS):
                s.step()
                ex()
                ref = _stream(ref)
                # ghost rows hold the neighbours' rows of this iteration
                rows = [(s.y0 - H + k) % NY for k in range(s.n + 2 * H)]
                ok &= bool(np.array_equal(s.f, ref[:, rows, :]))
            ok &= bool(np.array_equal(s.own(), ref[:, s.y0:s.y0 + s.n, :]))
        # thermo: each slab sums its own nodes; the all-reduce gives the lattice's
        rec = {"step": STEPS, "mass1": float(s.own().sum()), "nfluid": float(s.n * NX), "momx": float(rank)}
        tot = halo.reduce_thermo(dist, world, rec)
        ok &= abs(tot["mass1"] - float(full.sum())) <= 1e-12 * float(full.sum())
        ok &= tot["nfluid"] == NX * NY and tot["step"] == STEPS
        ok &= tot["momx"] == world * (world - 1) / 2
        out.put((rank, ok))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3, 4])
def test_slab_exchange_schedule_gloo(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    got = dict(q.get(timeout=5) for _ in range(world))
    assert got == {r: True for r in range(world)}


def test_single_rank_exchange_is_periodic():
    """World size 1: the slab is its own neighbour."""
    sys.path.insert(0, ROOT)
    from paper_1202_0442_gb300 import halo
    full = np.random.default_rng(1).random((9, NY, NX))
    s = HostSlab(full, 0, 1, 2)
    ex = halo.SlabExchange(s, None, 0, 1, "cpu")
    ref = full.copy()
    for _ in range(STEPS):
        s.step()
        ex()
        ref = _stream(ref)
    assert np.array_equal(s.own(), ref)
