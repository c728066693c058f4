"""Seeded synthetic workloads shaped like the paper's lattice Boltzmann cases.

This module only draws geometry, parameters and initial macroscopic fields
(density, velocity, concentration).  It holds none of the method's
arithmetic: each consumer turns the fields into populations with its own
equilibrium.  Both the GPU library's tests/benchmark and the CPU oracle's
harness read the same ``Workload`` objects, which is why this is the only
module the two sides share.

Random numbers come from numpy's PCG64 (``numpy.random.default_rng``), so a
seed gives the same workload on every machine.

Workloads (sizes in nodes; a paper script's lattice(N_x, N_y) has N_x + 1):

- ``channel``: force-driven channel between solid rows (Sec. Poiseuille
  flow): 64 x 32, walls y = 0 and y = 31, tau = 1, aveforce g_x = 1e-6.
- ``porous``: random non-overlapping discs at a target porosity with a
  density drop between a Zou-He dirichlet inlet (x = 0) and outlet
  (x = nx-1), periodic in y: 1024 x 1024, r in 8..24, porosity 0.7,
  tau = 0.8, rho_in = 1.001, rho_out = 1.0.
- ``shan_chen2``: two periodic fluid components with interforce G = 0.9 and
  an adhesive solid ring (adhesiveforce +-0.3): 2048 x 2048, ring
  600 <= r < 604, fluid 1 rich (1.0/0.03) inside the ring and in a free
  droplet, fluid 2 rich (0.03/1.0) elsewhere, +-1 % noise.
- ``reactive``: channel with random discs, uniform-velocity inlet
  u_x = 0.02, dirichlet outlet rho = 1, solute with inlet concentration 1,
  adiabatic outlet, surface reaction k_r = 1e-3, C_s = 0, b0 = 0,
  b_max = 1: 1024 x 512, 40 discs r in 8..24, tau = 0.9, tau_s = 0.7.
- ``batch``: 256 periodic force-driven porous lattices, sides 64..512 in
  steps of 32, porosity U[0.4, 0.9], tau U[0.6, 1.5], g_x = 1e-6.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# --------------------------------------------------------------------------
# workload description
# --------------------------------------------------------------------------


@dataclass
class Opening:
    """An inlet or outlet on one wall, spanning a0..a1 along it."""
    wall: str                      # "xlo" | "xhi" | "ylo" | "yhi"
    a0: int
    a1: int
    kind: str                      # "inlet" | "outlet"
    # per component: (style, v, rho); style in poiseuille/uniform/dirichlet/gradient
    momentum: List[Tuple[str, float, float]] = field(default_factory=list)
    # (style, C) with style in dirichlet/adiabatic, ("flux", C0, v), or None
    solute: Optional[Tuple] = None


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    solid: np.ndarray                                   # uint8 [ny, nx]
    rho: List[np.ndarray]                               # per component [ny, nx]
    ux: Optional[np.ndarray] = None                     # [ny, nx] initial velocity
    uy: Optional[np.ndarray] = None
    tau: Sequence[float] = (1.0,)
    alpha: Sequence[float] = (4.0 / 9.0,)
    aveforce: Sequence[Tuple[float, float]] = ((0.0, 0.0),)
    aveacceleration: Sequence[Tuple[float, float]] = ((0.0, 0.0),)
    interforce: Optional[Tuple[float, float, float]] = None      # (G, psi0, rho0)
    adhesive: Sequence[Optional[Tuple[float, float, float]]] = (None,)
    openings: List[Opening] = field(default_factory=list)
    solute_q: int = 0
    taus: float = 1.0
    C: Optional[np.ndarray] = None                      # initial concentration
    reaction: Optional[Tuple[float, float, float, float, int]] = None  # kr, Cs, b0, bmax, seed
    intersolute: Optional[Tuple[float, float, float]] = None    # (G, psi0, C0)
    # boundary_style per component: None (noslip), R (slip 1, mixed 0 < R < 1)
    # or an [ny][nx] array of R on the solid nodes (hybrid)
    slip: Optional[Sequence] = None
    steps: int = 1
    rho_ref: Sequence[float] = (1.0,)                   # typical density per component
    info: dict = field(default_factory=dict)

    @property
    def ncomp(self) -> int:
        return len(self.rho)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny

    @property
    def fluid_nodes(self) -> int:
        return int(self.nodes - int(self.solid.sum()))


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------


def rect_mask(nx: int, ny: int, x0: int, x1: int, y0: int, y1: int) -> np.ndarray:
    """obstacle(rectangle, x0, x1, y0, y1): inclusive bounds."""
    m = np.zeros((ny, nx), np.uint8)
    m[max(y0, 0):min(y1, ny - 1) + 1, max(x0, 0):min(x1, nx - 1) + 1] = 1
    return m


def circle_mask(nx: int, ny: int, xc: int, yc: int, r: int,
                periodic: bool = True) -> np.ndarray:
    """obstacle(circle, xc, yc, r): (x-xc)^2 + (y-yc)^2 <= r^2 in integers."""
    y, x = np.mgrid[0:ny, 0:nx]
    dx = x - xc
    dy = y - yc
    if periodic:
        dx = (dx + nx // 2) % nx - nx // 2
        dy = (dy + ny // 2) % ny - ny // 2
    return ((dx * dx + dy * dy) <= r * r).astype(np.uint8)


def _disc_stamp(m: np.ndarray, xc: int, yc: int, r: int, periodic_x: bool,
                periodic_y: bool) -> int:
    """Mark the disc solid; return how many nodes became solid."""
    ny, nx = m.shape
    added = 0
    for dy in range(-r, r + 1):
        w = int(np.floor(np.sqrt(r * r - dy * dy)))
        yy = yc + dy
        if periodic_y:
            yy %= ny
        elif not (0 <= yy < ny):
            continue
        xs = np.arange(xc - w, xc + w + 1)
        if periodic_x:
            xs %= nx
        else:
            xs = xs[(xs >= 0) & (xs < nx)]
        added += int(len(xs) - int(m[yy, xs].sum()))
        m[yy, xs] = 1
    return added


def random_discs(nx: int, ny: int, seed: int, rmin: int, rmax: int, *,
                 porosity: Optional[float] = None, count: Optional[int] = None,
                 gap: int = 2, margin_x: int = 0, margin_y: int = 0,
                 periodic_x: bool = True, periodic_y: bool = True,
                 overlap: bool = False, base: Optional[np.ndarray] = None,
                 max_tries: int = 200000):
    """Random sequential addition of discs with integer centres and radii.

    Without ``overlap`` two discs keep centre distance >= r1 + r2 + gap
    (minimum image on periodic axes).  Discs stay ``margin_x`` nodes from
    x = 0 and x = nx-1 when x is not periodic (same for y).  Stops when the
    solid fraction reaches 1 - porosity, or after ``count`` discs.
    Returns (mask, list of (xc, yc, r), achieved porosity).
    """
    rng = np.random.default_rng(seed)
    m = np.zeros((ny, nx), np.uint8) if base is None else base.copy()
    discs: List[Tuple[int, int, int]] = []
    target_solid = None if porosity is None else (1.0 - porosity) * nx * ny
    solid_count = int(m.sum())
    # placed discs bucketed on a grid of cells at least as wide as the
    # largest exclusion distance, so a candidate is checked against the
    # discs of its 3 x 3 cells only
    cell = 2 * rmax + gap
    gx, gy = max(1, nx // cell), max(1, ny // cell)
    buckets = {}
    tries = 0
    while tries < max_tries:
        if count is not None and len(discs) >= count:
            break
        if target_solid is not None and solid_count >= target_solid:
            break
        tries += 1
        r = int(rng.integers(rmin, rmax + 1))
        lox = 0 if periodic_x else margin_x + r
        hix = nx - 1 if periodic_x else nx - 1 - margin_x - r
        loy = 0 if periodic_y else margin_y + r
        hiy = ny - 1 if periodic_y else ny - 1 - margin_y - r
        if hix < lox or hiy < loy:
            continue
        xc = int(rng.integers(lox, hix + 1))
        yc = int(rng.integers(loy, hiy + 1))
        ok = True
        cx, cy = min(xc * gx // nx, gx - 1), min(yc * gy // ny, gy - 1)
        if not overlap:
            near = []
            for ddy in (-1, 0, 1):
                for ddx in (-1, 0, 1):
                    kx, ky = cx + ddx, cy + ddy
                    if periodic_x:
                        kx %= gx
                    if periodic_y:
                        ky %= gy
                    near.extend(buckets.get((kx, ky), ()))
            for (x2, y2, r2) in (discs if gx < 3 or gy < 3 else near):
                dx = xc - x2
                dy = yc - y2
                if periodic_x:
                    dx = (dx + nx // 2) % nx - nx // 2
                if periodic_y:
                    dy = (dy + ny // 2) % ny - ny // 2
                lim = r + r2 + gap
                if dx * dx + dy * dy < lim * lim:
                    ok = False
                    break
        if not ok:
            continue
        discs.append((xc, yc, r))
        buckets.setdefault((cx, cy), []).append((xc, yc, r))
        solid_count += _disc_stamp(m, xc, yc, r, periodic_x, periodic_y)
    por = 1.0 - float(m.sum()) / (nx * ny)
    return m, discs, por


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------


def channel(nx: int = 64, ny: int = 32, tau: float = 1.0, gx: float = 1e-6,
            steps: int = 2000) -> Workload:
    """Force-driven channel, solid rows y = 0 and y = ny-1, periodic in x."""
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = 1
    solid[ny - 1, :] = 1
    rho = np.where(solid, 0.0, 1.0)
    return Workload(name=f"channel_{nx}x{ny}", nx=nx, ny=ny, solid=solid,
                    rho=[rho], tau=(tau,), aveforce=((gx, 0.0),), steps=steps,
                    rho_ref=(1.0,), info={"H": ny - 2, "gx": gx})


def porous(nx: int = 1024, ny: int = 1024, seed: int = 1, porosity: float = 0.7,
           rmin: int = 8, rmax: int = 24, tau: float = 0.8,
           rho_in: float = 1.001, rho_out: float = 1.0,
           steps: int = 10000) -> Workload:
    """Pressure-driven flow through random discs, Zou-He dirichlet openings
    on the full x = 0 and x = nx-1 columns, periodic in y."""
    solid, discs, por = random_discs(nx, ny, seed, rmin, rmax, porosity=porosity,
                                     gap=2, margin_x=3, periodic_x=False,
                                     periodic_y=True)
    x = np.arange(nx, dtype=np.float64)
    prof = rho_in + (rho_out - rho_in) * x / max(nx - 1, 1)
    rho = np.where(solid, 0.0, np.broadcast_to(prof, (ny, nx)))
    ops = [Opening("xlo", 0, ny - 1, "inlet", [("dirichlet", 0.0, rho_in)]),
           Opening("xhi", 0, ny - 1, "outlet", [("dirichlet", 0.0, rho_out)])]
    return Workload(name=f"porous_{nx}x{ny}", nx=nx, ny=ny, solid=solid,
                    rho=[rho], tau=(tau,), openings=ops, steps=steps,
                    rho_ref=(0.5 * (rho_in + rho_out),),
                    info={"porosity": por, "discs": len(discs), "seed": seed,
                          "rho_in": rho_in, "rho_out": rho_out})


def shan_chen2(n: int = 2048, seed: int = 1, G: float = 0.9, gads: float = 0.3,
               r_in: int = 600, r_out: int = 604, rich: float = 1.0,
               lean: float = 0.03, drop_r: int = 100, noise: float = 0.01,
               tau: float = 1.0, steps: int = 20000) -> Workload:
    """Two periodic components with an adhesive solid ring.

    The ring is solid where r_in^2 <= d^2 < r_out^2 about the centre.
    Fluid 1 is rich inside the ring and in a free droplet of radius drop_r
    centred at (n/10, n/10); fluid 2 is rich elsewhere.  Densities carry
    multiplicative noise U[-noise, +noise].  Sizes scale with n (the ring
    radius is r_in * n / 2048 when n differs from 2048)."""
    rng = np.random.default_rng(seed)
    s = n / 2048.0
    ri, ro = int(round(r_in * s)), int(round(r_out * s))
    ro = max(ro, ri + 2)
    dr = max(int(round(drop_r * s)), 3)
    y, x = np.mgrid[0:n, 0:n]
    c = n // 2
    d2 = (x - c) ** 2 + (y - c) ** 2
    solid = ((d2 >= ri * ri) & (d2 < ro * ro)).astype(np.uint8)
    inside = d2 < ri * ri
    dc = n // 10
    ddx = (x - dc + n // 2) % n - n // 2
    ddy = (y - dc + n // 2) % n - n // 2
    drop = (ddx * ddx + ddy * ddy) <= dr * dr
    one = inside | drop
    rho1 = np.where(one, rich, lean) * (1.0 + rng.uniform(-noise, noise, (n, n)))
    rho2 = np.where(one, lean, rich) * (1.0 + rng.uniform(-noise, noise, (n, n)))
    rho1 = np.where(solid, 0.0, rho1)
    rho2 = np.where(solid, 0.0, rho2)
    mid = 0.5 * (rich + lean)
    return Workload(name=f"shan_chen2_{n}", nx=n, ny=n, solid=solid,
                    rho=[rho1, rho2], tau=(tau, tau), alpha=(4 / 9, 4 / 9),
                    aveforce=((0.0, 0.0), (0.0, 0.0)),
                    aveacceleration=((0.0, 0.0), (0.0, 0.0)),
                    interforce=(G, 0.0, 0.0),
                    adhesive=((gads, 0.0, 0.0), (-gads, 0.0, 0.0)),
                    steps=steps, rho_ref=(mid, mid),
                    info={"ring": (ri, ro), "drop": (dc, dc, dr), "G": G,
                          "seed": seed})


def reactive(nx: int = 1024, ny: int = 512, seed: int = 1, ndiscs: int = 40,
             rmin: int = 8, rmax: int = 24, tau: float = 0.9, u_in: float = 0.02,
             rho_out: float = 1.0, q: int = 9, taus: float = 0.7,
             C_in: float = 1.0, kr: float = 1e-3, Cs: float = 0.0,
             b0: float = 0.0, bmax: float = 1.0, growth_seed: int = 1,
             steps: int = 50000, inlet: str = "velocity", rho_in: float = 1.005,
             C_init: Optional[float] = None) -> Workload:
    """Solute transport with surface reaction and growth in a disc-filled
    channel (solid rows y = 0 and y = ny-1; openings on y = 1..ny-2).

    inlet "velocity": uniform inlet speed u_in (the stated recipe);
    "pressure": dirichlet rho_in at the inlet, the initial density linear
    between rho_in and rho_out.  C_init: initial concentration of the fluid
    nodes (default C_in)."""
    wall = np.zeros((ny, nx), np.uint8)
    wall[0, :] = 1
    wall[ny - 1, :] = 1
    # discs keep a fluid gap of >= 3 nodes to each other, the walls and
    # the openings, so no fluid node sees solid on two opposite sides
    solid, discs, por = random_discs(nx, ny, seed, rmin, rmax, count=ndiscs,
                                     gap=4, margin_x=5, margin_y=5,
                                     periodic_x=False, periodic_y=False,
                                     base=wall)
    if inlet == "velocity":
        rho = np.where(solid, 0.0, 1.0)
        mom_in = ("uniform", u_in, 1.0)
    else:
        x = np.arange(nx, dtype=np.float64)
        prof = rho_in + (rho_out - rho_in) * x / max(nx - 1, 1)
        rho = np.where(solid, 0.0, np.broadcast_to(prof, (ny, nx)))
        mom_in = ("dirichlet", 0.0, rho_in)
    C = np.where(solid, 0.0, C_in if C_init is None else C_init)
    ops = [Opening("xlo", 1, ny - 2, "inlet", [mom_in],
                   solute=("dirichlet", C_in)),
           Opening("xhi", 1, ny - 2, "outlet", [("dirichlet", 0.0, rho_out)],
                   solute=("adiabatic", C_in))]
    return Workload(name=f"reactive_{nx}x{ny}_q{q}" + ("" if inlet == "velocity" else "_pressure"),
                    nx=nx, ny=ny, solid=solid,
                    rho=[rho], tau=(tau,), openings=ops, solute_q=q, taus=taus,
                    C=C, reaction=(kr, Cs, b0, bmax, growth_seed), steps=steps,
                    rho_ref=(1.0,),
                    info={"porosity": por, "discs": len(discs), "seed": seed})


def batch(count: int = 256, seed0: int = 0, smin: int = 64, smax: int = 512,
          step: int = 32, gx: float = 1e-6, steps: int = 5000,
          sizes_seed: int = 12345) -> List[Workload]:
    """Independent periodic force-driven porous lattices of uneven sizes.

    Instance k draws its sides, porosity and tau from a generator seeded
    with sizes_seed + k and its discs with seed seed0 + k; discs may overlap
    (the target porosity goes down to 0.4, below what non-overlapping
    discs can reach)."""
    sides = np.arange(smin, smax + 1, step)
    out = []
    for k in range(count):
        rng = np.random.default_rng(sizes_seed + k)
        nx = int(rng.choice(sides))
        ny = int(rng.choice(sides))
        por = float(rng.uniform(0.4, 0.9))
        tau = float(rng.uniform(0.6, 1.5))
        rmax = max(4, min(nx, ny) // 16)
        solid, discs, got = random_discs(nx, ny, seed0 + k, 3, rmax,
                                         porosity=por, overlap=True)
        rho = np.where(solid, 0.0, 1.0)
        out.append(Workload(name=f"batch{k}_{nx}x{ny}", nx=nx, ny=ny,
                            solid=solid, rho=[rho], tau=(tau,),
                            aveforce=((gx, 0.0),), steps=steps, rho_ref=(1.0,),
                            info={"porosity": got, "target": por, "discs": len(discs)}))
    return out


# --------------------------------------------------------------------------
# small generic inputs for the parity tests
# --------------------------------------------------------------------------


def random_mask(nx: int, ny: int, seed: int, frac: float) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return (rng.random((ny, nx)) < frac).astype(np.uint8)


def random_populations(q: int, nx: int, ny: int, seed: int, base: Sequence[float],
                       spread: float, solid: Optional[np.ndarray] = None) -> np.ndarray:
    """Positive random populations base[i] * (1 + U[-spread, spread]),
    zero on solid nodes.  Not an equilibrium: used to exercise every term."""
    rng = np.random.default_rng(seed)
    b = np.asarray(base, np.float64).reshape(q, 1, 1)
    f = b * (1.0 + rng.uniform(-spread, spread, (q, ny, nx)))
    if solid is not None:
        f = np.where(solid[None, :, :] != 0, 0.0, f)
    return f


def noise_field(nx: int, ny: int, seed: int, lo: float, hi: float) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, (ny, nx))
