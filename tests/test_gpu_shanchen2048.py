"""The two-component Shan-Chen recipe at its stated size, 2048 x 2048,
against the oracle node by node for 200 iterations (interforce command,
Sec. Phase separation; adhesiveforce).

The oracle cannot run the whole lattice for hundreds of iterations in a
test, so it runs windows: the update of a node reads the populations of its
neighbours (the pull) and the densities of its neighbours after streaming
(the interforce and adhesion sums), so after T iterations a node depends
only on the initial state within 2T nodes of it.  A window of the periodic
lattice, cut out and run as a periodic lattice of its own, therefore gives
the exact (FP64) result of the whole lattice on every node more than
2T + 2 nodes from its edge.  The library runs the whole 2048^2 lattice as
the benchmark would (FP32 storage); the windows' centres are compared:
max relative error in each component's density and in the Eq. (4)
velocity (normalised by the largest oracle velocity over the compared
nodes) below 1e-5, masks equal.  The windows sit on the droplet's edge,
on the adhesive ring (inside and outside) and in the bulk.  The oracle
windows run in spawned worker processes, one per window."""
import multiprocessing as mp
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu

N = 2048
T = 200
CORE = 24                      # compared nodes per side of a window
MARGIN = 2 * T + 2
W = CORE + 2 * MARGIN


def _windows():
    """(x0, y0) lower corners of the compared cores, wrapped"""
    c = N // 2
    ri = 600
    dc, dr = N // 10, 100
    centres = [(dc + dr, dc),            # edge of the free droplet
               (c + ri - 4, c),          # inside the ring, beside the wall
               (c, c + ri + 6),          # outside the ring, beside the wall
               (c + 320, c - 250)]       # bulk of fluid 1 inside the ring
    return [((x - CORE // 2) % N, (y - CORE // 2) % N) for x, y in centres]


def _crop(a, x0, y0, size):
    ys = (np.arange(size) + y0) % N
    xs = (np.arange(size) + x0) % N
    return a[np.ix_(ys, xs)]


def _oracle_window(args):
    """Worker: the oracle on the window around core (x0, y0), T iterations;
    returns the core's densities, velocity and mask."""
    x0, y0 = args
    sys.path.insert(0, ROOT)
    from oracle import orc
    from oracle.drive import oracle_from_workload
    from paper_1202_0442_gb300 import synth
    orc.build()
    w = synth.shan_chen2(N)
    wx, wy = (x0 - MARGIN) % N, (y0 - MARGIN) % N
    w.solid = _crop(w.solid, wx, wy, W)
    w.rho = [_crop(r, wx, wy, W) for r in w.rho]
    w.nx = w.ny = W
    o = oracle_from_workload(w)
    o.step(T)
    sl = (slice(MARGIN, MARGIN + CORE), slice(MARGIN, MARGIN + CORE))
    ux, uy = o.velocity()
    return {"rho1": o.fields(0)[0][sl], "rho2": o.fields(1)[0][sl], "ux": ux[sl], "uy": uy[sl],
            "solid": o.solid()[sl]}


def test_shan_chen_2048_windows_200_iterations():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wins = _windows()
    # the oracle windows start first, in spawned processes (no CUDA in them)
    pool = mp.get_context("spawn").Pool(len(wins))
    try:
        pending = pool.map_async(_oracle_window, wins)
        from paper_1202_0442_gb300 import build, lb2d, synth
        torch.cuda.set_device(0)
        build.build()
        w = synth.shan_chen2(N)
        lt = lb2d.from_workload(w, "fp32")
        lt.iteration(T)
        r1, r2 = lt.fields(1)[0], lt.fields(2)[0]
        _, ugx, ugy = lt.velocity_f32()
        mask = lt.mask()
        ref = pending.get(timeout=1800)
    finally:
        pool.close()
        pool.join()
    e1 = e2 = du = 0.0
    umax = 0.0
    for (x0, y0), o in zip(wins, ref):
        fl = o["solid"] == 0
        assert np.array_equal(_crop(mask, x0, y0, CORE), o["solid"])
        e1 = max(e1, float(np.max(np.abs(_crop(r1, x0, y0, CORE) - o["rho1"])[fl] / o["rho1"][fl])))
        e2 = max(e2, float(np.max(np.abs(_crop(r2, x0, y0, CORE) - o["rho2"])[fl] / o["rho2"][fl])))
        du = max(du, float(np.max(np.abs(_crop(ugx, x0, y0, CORE) - o["ux"])[fl])),
                 float(np.max(np.abs(_crop(ugy, x0, y0, CORE) - o["uy"])[fl])))
        umax = max(umax, float(np.max(np.abs(o["ux"][fl]))), float(np.max(np.abs(o["uy"][fl]))))
    assert umax > 0
    assert e1 < 1e-5 and e2 < 1e-5 and du / umax < 1e-5, (e1, e2, du / umax, umax)
