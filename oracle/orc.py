"""Python handle on the FP64 CPU oracle (``lb2d_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the checker the GPU library is
compared against: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module.  It never imports the
product package and the product package never imports it.

``build()`` compiles the C source with gcc (ISO C99, no FMA contraction, so
the x86 build container and the Arm GPU host give the same bits).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb2d_oracle.c")
_HDR = os.path.join(_HERE, "lb2d_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liblb2d_oracle.so")

XLO, XHI, YLO, YHI = 0, 1, 2, 3
INLET, OUTLET = 0, 1
M_NONE, M_POISEUILLE, M_UNIFORM, M_DIRICHLET, M_GRADIENT = 0, 1, 2, 3, 4
S_NONE, S_DIRICHLET, S_ADIABATIC, S_FLUX = 0, 1, 2, 3
WALLS = {"xlo": XLO, "xhi": XHI, "ylo": YLO, "yhi": YHI}
MSTYLES = {"poiseuille": M_POISEUILLE, "uniform": M_UNIFORM,
           "dirichlet": M_DIRICHLET, "gradient": M_GRADIENT}
SSTYLES = {"dirichlet": S_DIRICHLET, "adiabatic": S_ADIABATIC, "flux": S_FLUX}

THERMO_KEYS = ["mass1", "mass2", "momx", "momy", "mass_eq1", "mass_eq2",
               "solute", "bsum", "removed1", "removed2", "removed_solute",
               "nsolid", "nfluid", "momx1", "momy1", "momx2", "momy2"]

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liblb2d_oracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    P, I, D, U64 = C.c_void_p, C.c_int, C.c_double, C.c_uint64
    dp = C.POINTER(C.c_double)
    u8p = C.POINTER(C.c_uint8)
    sig = {
        "orc_create": (P, [I, I, I, I]),
        "orc_destroy": (None, [P]),
        "orc_set_tau": (I, [P, I, D]),
        "orc_set_alpha": (I, [P, I, D]),
        "orc_set_taus": (I, [P, D]),
        "orc_set_solid": (I, [P, u8p]),
        "orc_get_solid": (I, [P, u8p]),
        "orc_set_f": (I, [P, I, dp]),
        "orc_get_f": (I, [P, I, dp]),
        "orc_set_equilibrium": (I, [P, I, dp, dp, dp]),
        "orc_set_g": (I, [P, dp]),
        "orc_get_g": (I, [P, dp]),
        "orc_set_solute_equilibrium": (I, [P, dp, dp, dp]),
        "orc_set_b": (I, [P, dp]),
        "orc_get_b": (I, [P, dp]),
        "orc_set_aveforce": (I, [P, I, D, D]),
        "orc_set_aveacceleration": (I, [P, I, D, D]),
        "orc_set_interforce": (I, [P, D, D, D]),
        "orc_set_adhesiveforce": (I, [P, I, D, D, D]),
        "orc_add_opening": (I, [P, I, I, I, I]),
        "orc_set_opening_momentum": (I, [P, I, I, I, D, D]),
        "orc_set_opening_solute": (I, [P, I, I, D, D]),
        "orc_set_intersolute": (I, [P, D, D, D]),
        "orc_set_slip": (I, [P, I, D, dp]),
        "orc_set_margin_eps": (I, [P, D, I]),
        "orc_get_margin_events": (I, [P, C.POINTER(C.c_int64), dp, I]),
        "orc_set_reaction": (I, [P, D, D, D, D, U64]),
        "orc_step": (I, [P]),
        "orc_time": (C.c_long, [P]),
        "orc_set_time": (I, [P, C.c_long]),
        "orc_get_fields": (I, [P, I, dp, dp, dp, dp]),
        "orc_get_solute_C": (I, [P, dp]),
        "orc_get_thermo": (I, [P, dp]),
        "orc_get_flips": (I, [P, C.POINTER(C.c_int64), I]),
        "orc_feq": (None, [D, D, D, D, dp]),
        "orc_zouhe": (I, [I, I, I, D, D, dp, dp, dp]),
        "orc_reaction_link": (None, [I, I, D, D, D, dp, dp]),
        "orc_splitmix64": (U64, [U64]),
        "orc_poiseuille_v": (D, [D, I, I, I]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, shape) -> np.ndarray:
    out = np.ascontiguousarray(np.broadcast_to(np.asarray(a, np.float64), shape))
    return out


def _check(rc: int, what: str) -> None:
    if rc < 0:
        raise ValueError(f"oracle rejected {what} (rc={rc})")


# ---------------------------------------------------------------------------
# single-node pieces
# ---------------------------------------------------------------------------

def feq(rho: float, ux: float, uy: float, alpha: float = 4.0 / 9.0) -> np.ndarray:
    out = np.zeros(9)
    _load().orc_feq(rho, ux, uy, alpha, _dp(out))
    return out


def zouhe(wall: str, kind: str, style: str, f: np.ndarray, v: float = 0.0,
          rho: float = 0.0):
    """Apply one opening rule to a copy of ``f``; returns (f, rho, v)."""
    g = np.array(f, dtype=np.float64).copy()
    r = np.zeros(1)
    vv = np.zeros(1)
    rc = _load().orc_zouhe(WALLS[wall], INLET if kind == "inlet" else OUTLET,
                           MSTYLES[style], v, rho, _dp(g), _dp(r), _dp(vv))
    _check(rc, "zouhe")
    return g, float(r[0]), float(vv[0])


def reaction_link(q: int, i: int, g_out: float, kr: float, Cs: float):
    ci = np.zeros(1)
    gi = np.zeros(1)
    _load().orc_reaction_link(q, i, g_out, kr, Cs, _dp(ci), _dp(gi))
    return float(ci[0]), float(gi[0])


def splitmix64(x: int) -> int:
    return int(_load().orc_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


def poiseuille_v(vmax: float, a0: int, a1: int, coord: int) -> float:
    return float(_load().orc_poiseuille_v(vmax, a0, a1, coord))


# ---------------------------------------------------------------------------
# lattice
# ---------------------------------------------------------------------------

class Oracle:
    """One lattice of the FP64 oracle; all arrays are SoA numpy arrays."""

    def __init__(self, nx: int, ny: int, ncomp: int = 1, solute_q: int = 0):
        self._l = _load()
        self.nx, self.ny, self.ncomp, self.q = nx, ny, ncomp, solute_q
        self._h = self._l.orc_create(nx, ny, ncomp, solute_q)
        if not self._h:
            raise ValueError("oracle: bad lattice")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._l.orc_destroy(h)
            self._h = None

    # -- parameters --------------------------------------------------------
    def set_tau(self, tau: float, comp: int = 0):
        _check(self._l.orc_set_tau(self._h, comp, tau), "tau")

    def set_alpha(self, alpha: float, comp: int = 0):
        _check(self._l.orc_set_alpha(self._h, comp, alpha), "alpha")

    def set_taus(self, taus: float):
        _check(self._l.orc_set_taus(self._h, taus), "taus")

    def set_solid(self, mask: np.ndarray):
        m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(self.ny, self.nx)
        self._l.orc_set_solid(self._h, m.ctypes.data_as(C.POINTER(C.c_uint8)))

    def solid(self) -> np.ndarray:
        m = np.zeros((self.ny, self.nx), np.uint8)
        self._l.orc_get_solid(self._h, m.ctypes.data_as(C.POINTER(C.c_uint8)))
        return m

    def set_aveforce(self, fx: float, fy: float, comp: int = 0):
        _check(self._l.orc_set_aveforce(self._h, comp, fx, fy), "aveforce")

    def set_aveacceleration(self, ax: float, ay: float, comp: int = 0):
        _check(self._l.orc_set_aveacceleration(self._h, comp, ax, ay), "accel")

    def set_interforce(self, G: float, psi0: float = 0.0, rho0: float = 0.0):
        _check(self._l.orc_set_interforce(self._h, G, psi0, rho0), "interforce")

    def set_adhesiveforce(self, G: float, psi0: float = 0.0, rho0: float = 0.0,
                          comp: int = 0):
        _check(self._l.orc_set_adhesiveforce(self._h, comp, G, psi0, rho0),
               "adhesiveforce")

    def add_opening(self, wall: str, a0: int, a1: int, kind: str) -> int:
        rc = self._l.orc_add_opening(self._h, WALLS[wall], a0, a1,
                                     INLET if kind == "inlet" else OUTLET)
        _check(rc, "opening")
        return rc

    def set_opening_momentum(self, opening: int, style: str, v: float = 0.0,
                             rho: float = 0.0, comp: int = 0):
        _check(self._l.orc_set_opening_momentum(self._h, opening, comp,
                                                MSTYLES[style], v, rho),
               "opening momentum")

    def set_opening_solute(self, opening: int, style: str, Cbar: float = 0.0, v: float = 0.0):
        """Cbar: dirichlet concentration or the flux style's C0; v: the flux
        style's velocity."""
        _check(self._l.orc_set_opening_solute(self._h, opening, SSTYLES[style],
                                              Cbar, v), "opening solute")

    def set_slip(self, R_all: float = 0.0, R_map=None, comp: int = 0):
        """boundary_style slip (R = 1), mixed (0 < R < 1) or, with R_map
        ([ny][nx], read on solid nodes), hybrid."""
        m = None if R_map is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(R_map, np.float64), (self.ny, self.nx)))
        _check(self._l.orc_set_slip(self._h, comp, R_all, None if m is None else _dp(m)), "slip")

    def set_intersolute(self, G: float, psi0: float, C0: float):
        _check(self._l.orc_set_intersolute(self._h, G, psi0, C0), "intersolute")

    def set_reaction(self, kr: float, Cs: float, b0: float, bmax: float,
                     seed: int):
        _check(self._l.orc_set_reaction(self._h, kr, Cs, b0, bmax,
                                        seed & 0xFFFFFFFFFFFFFFFF), "reaction")

    # -- state -------------------------------------------------------------
    def set_f(self, f: np.ndarray, comp: int = 0):
        a = _f64(f, (9, self.ny, self.nx))
        _check(self._l.orc_set_f(self._h, comp, _dp(a)), "f")

    def f(self, comp: int = 0) -> np.ndarray:
        a = np.zeros((9, self.ny, self.nx))
        _check(self._l.orc_get_f(self._h, comp, _dp(a)), "f")
        return a

    def set_equilibrium(self, rho, ux=0.0, uy=0.0, comp: int = 0):
        sh = (self.ny, self.nx)
        r, u, v = _f64(rho, sh), _f64(ux, sh), _f64(uy, sh)
        _check(self._l.orc_set_equilibrium(self._h, comp, _dp(r), _dp(u), _dp(v)),
               "equilibrium")

    def set_g(self, g: np.ndarray):
        a = _f64(g, (self.q, self.ny, self.nx))
        _check(self._l.orc_set_g(self._h, _dp(a)), "g")

    def g(self) -> np.ndarray:
        a = np.zeros((self.q, self.ny, self.nx))
        _check(self._l.orc_get_g(self._h, _dp(a)), "g")
        return a

    def set_solute_equilibrium(self, C, ux=0.0, uy=0.0):
        sh = (self.ny, self.nx)
        c, u, v = _f64(C, sh), _f64(ux, sh), _f64(uy, sh)
        _check(self._l.orc_set_solute_equilibrium(self._h, _dp(c), _dp(u), _dp(v)),
               "solute equilibrium")

    def set_b(self, b):
        a = _f64(b, (self.ny, self.nx))
        self._l.orc_set_b(self._h, _dp(a))

    def b(self) -> np.ndarray:
        a = np.zeros((self.ny, self.nx))
        self._l.orc_get_b(self._h, _dp(a))
        return a

    # -- run and read ------------------------------------------------------
    def step(self, n: int = 1):
        for _ in range(n):
            _check(self._l.orc_step(self._h), "step")

    @property
    def t(self) -> int:
        return int(self._l.orc_time(self._h))

    def set_t(self, t: int):
        """Step counter (a run resumed from a restart file continues it)."""
        _check(self._l.orc_set_time(self._h, t), "time")

    def fields(self, comp: int = 0):
        sh = (self.ny, self.nx)
        r, px, py, req = (np.zeros(sh) for _ in range(4))
        _check(self._l.orc_get_fields(self._h, comp, _dp(r), _dp(px), _dp(py),
                                      _dp(req)), "fields")
        return r, px, py, req

    def velocity(self):
        """Solvent velocity of Eq. (4): sum_s (j_s + F_s/2) / sum_s rho_s."""
        rs = np.zeros((self.ny, self.nx))
        pxs = np.zeros_like(rs)
        pys = np.zeros_like(rs)
        for s in range(self.ncomp):
            r, px, py, _ = self.fields(s)
            rs += r
            pxs += px
            pys += py
        with np.errstate(invalid="ignore", divide="ignore"):
            ux = np.where(rs > 0, pxs / np.where(rs > 0, rs, 1), 0.0)
            uy = np.where(rs > 0, pys / np.where(rs > 0, rs, 1), 0.0)
        return ux, uy

    def solute_C(self) -> np.ndarray:
        a = np.zeros((self.ny, self.nx))
        _check(self._l.orc_get_solute_C(self._h, _dp(a)), "C")
        return a

    def thermo(self) -> dict:
        a = np.zeros(len(THERMO_KEYS))
        self._l.orc_get_thermo(self._h, _dp(a))
        return dict(zip(THERMO_KEYS, a.tolist()))

    def set_margin_eps(self, eps: float, cap: int = 4096):
        _check(self._l.orc_set_margin_eps(self._h, eps, cap), "margin eps")

    def margin_events(self):
        """(node indices, b - bmax) of the growth decisions of the last
        iteration that lay within the margin set by set_margin_eps"""
        n = self._l.orc_get_margin_events(self._h, None, None, 0)
        idx = np.zeros(max(n, 1), np.int64)
        val = np.zeros(max(n, 1))
        self._l.orc_get_margin_events(self._h, idx.ctypes.data_as(C.POINTER(C.c_int64)), _dp(val), n)
        return idx[:n], val[:n]

    def flips(self) -> np.ndarray:
        n = self._l.orc_get_flips(self._h, None, 0)
        a = np.zeros(max(n, 1), np.int64)
        self._l.orc_get_flips(self._h, a.ctypes.data_as(C.POINTER(C.c_int64)), n)
        return a[:n]
