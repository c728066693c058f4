"""ctypes binding of the C ABI in ``include/lb2d.h``.

Argument marshalling only: every step of the lattice Boltzmann update runs
in the CUDA kernels of ``_lib/liblb2d.so``.  There is no CPU fallback; if
the library has not been built this module raises on first use.

PyTorch supplies the CUDA stream (the current stream of the device) so the
library's work orders with the caller's torch work.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence, Tuple

import numpy as np

from . import synth

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblb2d.so")

LB_OK, LB_E_ORDER, LB_E_ARG, LB_E_UNSUPPORTED, LB_E_CUDA, LB_E_NAN, LB_E_NOMEM, LB_E_TIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7
LB_DEBUG_POISON, LB_DEBUG_GUARDS = 0x1, 0x2
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}
LB_STOCHASTIC_ROUNDING = 0x100
LB_PRECISE_MOMENTUM = 0x200
_CODES = {LB_E_ORDER: "LB_E_ORDER", LB_E_ARG: "LB_E_ARG", LB_E_UNSUPPORTED: "LB_E_UNSUPPORTED",
          LB_E_CUDA: "LB_E_CUDA", LB_E_NAN: "LB_E_NAN", LB_E_NOMEM: "LB_E_NOMEM",
          LB_E_TIMEOUT: "LB_E_TIMEOUT"}


class LBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_CODES.get(code, code)}: {msg}")
        self.code = code


class Thermo(C.Structure):
    _fields_ = [("step", C.c_int64), ("mass", C.c_double * 2), ("mom", C.c_double * 2),
                ("mom_comp", (C.c_double * 2) * 2), ("mass_eq", C.c_double * 2),
                ("solute", C.c_double), ("bsum", C.c_double), ("removed", C.c_double * 2),
                ("removed_solute", C.c_double), ("nsolid", C.c_int64), ("nfluid", C.c_int64),
                ("flips", C.c_int64)]

    def as_dict(self) -> dict:
        return {"step": self.step, "mass1": self.mass[0], "mass2": self.mass[1],
                "momx": self.mom[0], "momy": self.mom[1],
                "momx1": self.mom_comp[0][0], "momy1": self.mom_comp[0][1],
                "momx2": self.mom_comp[1][0], "momy2": self.mom_comp[1][1],
                "mass_eq1": self.mass_eq[0], "mass_eq2": self.mass_eq[1],
                "solute": self.solute, "bsum": self.bsum, "removed1": self.removed[0],
                "removed2": self.removed[1], "removed_solute": self.removed_solute,
                "nsolid": self.nsolid, "nfluid": self.nfluid, "flips": self.flips}


_lib = None

# name -> (restype, argtypes); every function of include/lb2d.h
P, I, D, S, U64, SZ = C.c_void_p, C.c_int, C.c_double, C.c_char_p, C.c_uint64, C.c_size_t
DP, FP, U8P = C.POINTER(C.c_double), C.POINTER(C.c_float), C.POINTER(C.c_uint8)
SIGNATURES = {
    "lb_create": (I, [I, P, C.POINTER(P)]),
    "lb_destroy": (I, [P]),
    "lb_last_error": (S, [P]),
    "lb_launch_count": (I, [P, C.POINTER(C.c_uint64)]),
    "lb_lattice": (I, [P, S, I, I, D]),
    "lb_processors": (I, [P, I, I]),
    "lb_processor_rank": (I, [P, I]),
    "lb_halo_size": (I, [P, C.POINTER(SZ)]),
    "lb_halo_pack": (I, [P, I, P]),
    "lb_halo_unpack": (I, [P, I, P]),
    "lb_exchange": (I, [C.POINTER(P), I]),
    "lb_fluids": (I, [P, D, D, D, D]),
    "lb_solute": (I, [P, D, I]),
    "lb_set_storage": (I, [P, I, DP, D]),
    "lb_boundary_style": (I, [P, S, D]),
    "lb_obstacle_rect": (I, [P, I, I, I, I]),
    "lb_obstacle_circle": (I, [P, I, I, I]),
    "lb_obstacle_mask": (I, [P, U8P]),
    "lb_obstacle_rect_styled": (I, [P, I, I, I, I, S, D, S, D]),
    "lb_obstacle_circle_styled": (I, [P, I, I, I, S, D, S, D]),
    "lb_obstacle_mask_hybrid": (I, [P, U8P, DP]),
    "lb_inlet": (I, [P, S, I, I, S, S]),
    "lb_outlet": (I, [P, S, I, I, S, S]),
    "lb_inlet_momentum": (I, [P, S, S, D, D]),
    "lb_outlet_momentum": (I, [P, S, S, D, D]),
    "lb_inlet_solute": (I, [P, S, S, D, D]),
    "lb_outlet_solute": (I, [P, S, S, D, D]),
    "lb_surface_reaction": (I, [P, D, D, S, D, D, U64]),
    "lb_position0_rect": (I, [P, I, I, I, I]),
    "lb_position0_circle": (I, [P, I, I, I]),
    "lb_momentum0": (I, [P, I, D, I]),
    "lb_concentration0": (I, [P, D]),
    "lb_set_equilibrium": (I, [P, I, DP, DP, DP]),
    "lb_set_solute_equilibrium": (I, [P, DP, DP, DP]),
    "lb_set_populations": (I, [P, I, DP]),
    "lb_set_solute_populations": (I, [P, DP]),
    "lb_set_precipitate": (I, [P, DP]),
    "lb_aveforce": (I, [P, I, D, I]),
    "lb_aveforce_xy": (I, [P, D, D, I]),
    "lb_aveacceleration": (I, [P, I, D, I]),
    "lb_aveacceleration_xy": (I, [P, D, D, I]),
    "lb_interforce": (I, [P, D, D, D]),
    "lb_intersolute": (I, [P, D, D, D]),
    "lb_adhesiveforce": (I, [P, D, D, D, I]),
    "lb_set_kernel": (I, [P, S]),
    "lb_set_wait_limit": (I, [P, C.c_int64]),
    "lb_set_debug": (I, [P, I]),
    "lb_debug_check": (I, [P, C.POINTER(C.c_int64)]),
    "lb_thermo": (I, [P, I]),
    "lb_thermo_deferred": (I, [P, I]),
    "lb_output": (I, [P, I]),
    "lb_iteration": (I, [P, I]),
    "lb_get_thermo": (I, [P, C.POINTER(Thermo)]),
    "lb_thermo_static": (I, [P, C.POINTER(Thermo)]),
    "lb_get_fields": (I, [P, I, DP, DP, DP, DP]),
    "lb_get_velocity_f32": (I, [P, FP, FP, FP]),
    "lb_get_populations": (I, [P, I, DP]),
    "lb_get_solute": (I, [P, DP, DP, DP]),
    "lb_get_mask": (I, [P, U8P]),
    "lb_get_flips": (I, [P, C.POINTER(C.c_int64), I, C.POINTER(I)]),
    "lb_buffer_size": (I, [P, S, C.POINTER(SZ)]),
    "lb_set_step": (I, [P, C.c_int64]),
    "lb_bind": (I, [P, S, P, SZ]),
    "lb_current_buffer": (I, [P, C.POINTER(I)]),
    "lb_state_size": (I, [P, C.POINTER(C.c_size_t)]),
    "lb_save_state": (I, [P, P, SZ]),
    "lb_load_state": (I, [P, P, SZ]),
    "lb_write_restart": (I, [P, S, I]),
    "lb_write_data": (I, [P, S]),
    "lb_read_data": (I, [P, S, S]),
    "lb_lattice_info": (I, [P, C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(I),
                            C.POINTER(I)]),
    "lb_batch_create": (I, [C.POINTER(P), I, C.POINTER(P)]),
    "lb_batch_destroy": (I, [P]),
    "lb_batch_iteration": (I, [P, I, I]),
    "lb_batch_autotune": (I, [P, S]),
    "lb_batch_last_error": (S, [P]),
    "lb_batch_launch_count": (I, [P, C.POINTER(C.c_uint64)]),
}


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run __graft_entry__.build() "
                               "(or python -m paper_1202_0442_gb300.build); there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _dp(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(DP)


def _f64(a, shape) -> np.ndarray:
    return np.ascontiguousarray(np.broadcast_to(np.asarray(a, np.float64), shape))


def _b(s: Optional[str]):
    return None if s is None else s.encode()


def current_stream_handle(device: int = 0) -> int:
    import torch
    return int(torch.cuda.current_stream(device).cuda_stream)


class Lattice:
    """One lattice on one GPU; methods follow the paper's command names."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        self._L = lib()
        if stream is None:
            stream = current_stream_handle(device)
        h = P()
        rc = self._L.lb_create(device, C.c_void_p(stream), C.byref(h))
        if rc != LB_OK:
            raise LBError(rc, "lb_create failed (no CUDA device?)")
        self._h = h
        self.device = device
        self._bound = {}  # name -> caller tensor kept alive while bound
        self.nx = self.ny = 0
        self.ncomp = 1
        self.q = 0
        self._py, self._rank = 1, -1

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.lb_destroy(h)
            self._h = None

    def close(self):
        self.__del__()
        self._bound = {}

    def _ck(self, rc: int):
        if rc != LB_OK:
            raise LBError(rc, self._L.lb_last_error(self._h).decode())

    @property
    def handle(self):
        return self._h

    # -- initialization commands -------------------------------------------
    def lattice(self, nx: int, ny: int, tau: float, style: str = "d2q9"):
        self._ck(self._L.lb_lattice(self._h, _b(style), nx, ny, tau))
        self.nx, self.ny = nx, ny

    def processors(self, px: int, py: int):
        self._ck(self._L.lb_processors(self._h, px, py))
        self._py = py

    def processor_rank(self, rank: int):
        """Hold slab ``rank`` of the lattice split by processors(1, py)."""
        self._ck(self._L.lb_processor_rank(self._h, rank))
        self._rank = rank

    @property
    def rows(self):
        """(first row, row count) of the rows this context updates and
        returns: the whole lattice, or its slab."""
        if self._rank < 0:
            return 0, self.ny
        y0 = self._rank * self.ny // self._py
        return y0, (self._rank + 1) * self.ny // self._py - y0

    def halo_size(self) -> int:
        n = SZ()
        self._ck(self._L.lb_halo_size(self._h, C.byref(n)))
        return n.value

    def halo_pack(self, face: int, buf) -> None:
        """Rows for the neighbour across ``face`` (0 low y, 1 high y) into
        the CUDA tensor ``buf`` (halo_size() bytes)."""
        self._ck(self._L.lb_halo_pack(self._h, face, C.c_void_p(buf.data_ptr())))

    def halo_unpack(self, face: int, buf) -> None:
        """Ghost rows on ``face`` from the CUDA tensor ``buf``."""
        self._ck(self._L.lb_halo_unpack(self._h, face, C.c_void_p(buf.data_ptr())))

    def fluids(self, tau1: float, tau2: float, alpha1: float = 4 / 9, alpha2: float = 4 / 9):
        self._ck(self._L.lb_fluids(self._h, tau1, tau2, alpha1, alpha2))
        self.ncomp = 2

    def solute(self, taus: float, q: int = 4):
        self._ck(self._L.lb_solute(self._h, taus, q))
        self.q = q

    def set_storage(self, storage: str = "fp32", rho_ref: Sequence[float] = (1.0,), h_max: float = 0.0,
                    rounding: str = "nearest", precise: bool = False):
        r = np.array(list(rho_ref) + [rho_ref[0]] * (2 - len(rho_ref)), np.float64)
        code = (STORAGE[storage] | (LB_STOCHASTIC_ROUNDING if rounding == "stochastic" else 0)
                | (LB_PRECISE_MOMENTUM if precise else 0))
        self._ck(self._L.lb_set_storage(self._h, code, _dp(r), h_max))

    def boundary_style(self, style: str = "noslip", R: float = 0.0):
        self._ck(self._L.lb_boundary_style(self._h, _b(style), R))

    def obstacle_rect_styled(self, x0, x1, y0, y1, style1=None, arg1=0.0, style2=None, arg2=0.0):
        self._ck(self._L.lb_obstacle_rect_styled(self._h, x0, x1, y0, y1, _b(style1), arg1, _b(style2), arg2))

    def obstacle_circle_styled(self, xc, yc, r, style1=None, arg1=0.0, style2=None, arg2=0.0):
        self._ck(self._L.lb_obstacle_circle_styled(self._h, xc, yc, r, _b(style1), arg1, _b(style2), arg2))

    def obstacle_mask_hybrid(self, mask: np.ndarray, R: Optional[np.ndarray] = None):
        """mask [ny][nx]; R [ncomp][ny][nx] (or [ny][nx] for one component)"""
        m = np.ascontiguousarray(mask, np.uint8).reshape(self.ny, self.nx)
        r = None if R is None else np.ascontiguousarray(R, np.float64).reshape(-1, self.ny, self.nx)
        self._ck(self._L.lb_obstacle_mask_hybrid(self._h, m.ctypes.data_as(U8P), _dp(r)))

    def obstacle_rect(self, x0, x1, y0, y1):
        self._ck(self._L.lb_obstacle_rect(self._h, x0, x1, y0, y1))

    def obstacle_circle(self, xc, yc, r):
        self._ck(self._L.lb_obstacle_circle(self._h, xc, yc, r))

    def obstacle_mask(self, mask: np.ndarray):
        m = np.ascontiguousarray(mask, np.uint8).reshape(self.ny, self.nx)
        self._ck(self._L.lb_obstacle_mask(self._h, m.ctypes.data_as(U8P)))

    def inlet(self, wall, a0, a1, label1, label2=None):
        self._ck(self._L.lb_inlet(self._h, _b(wall), a0, a1, _b(label1), _b(label2)))

    def outlet(self, wall, a0, a1, label1, label2=None):
        self._ck(self._L.lb_outlet(self._h, _b(wall), a0, a1, _b(label1), _b(label2)))

    def inlet_momentum(self, label, style, v=0.0, rho=1.0):
        self._ck(self._L.lb_inlet_momentum(self._h, _b(label), _b(style), v, rho))

    def outlet_momentum(self, label, style, v=0.0, rho=1.0):
        self._ck(self._L.lb_outlet_momentum(self._h, _b(label), _b(style), v, rho))

    def inlet_solute(self, label, style, C=0.0, v=0.0):
        self._ck(self._L.lb_inlet_solute(self._h, _b(label), _b(style), C, v))

    def outlet_solute(self, label, style, C=0.0, v=0.0):
        self._ck(self._L.lb_outlet_solute(self._h, _b(label), _b(style), C, v))

    def surface_reaction(self, kr, Cs, b0, bmax, seed=1, style="growth"):
        self._ck(self._L.lb_surface_reaction(self._h, kr, Cs, _b(style), b0, bmax, seed & (2 ** 64 - 1)))

    def position0_rect(self, x0, x1, y0, y1):
        self._ck(self._L.lb_position0_rect(self._h, x0, x1, y0, y1))

    def position0_circle(self, xc, yc, r):
        self._ck(self._L.lb_position0_circle(self._h, xc, yc, r))

    def momentum0(self, mode: int, value: float, fluid: int = 1):
        self._ck(self._L.lb_momentum0(self._h, mode, value, fluid))

    def concentration0(self, value: float):
        self._ck(self._L.lb_concentration0(self._h, value))

    def set_equilibrium(self, rho, ux=None, uy=None, fluid: int = 1):
        sh = (self.ny, self.nx)
        r = _f64(rho, sh)
        u = None if ux is None else _f64(ux, sh)
        v = None if uy is None else _f64(uy, sh)
        self._ck(self._L.lb_set_equilibrium(self._h, fluid, _dp(r), _dp(u), _dp(v)))

    def set_solute_equilibrium(self, Cf, ux=None, uy=None):
        sh = (self.ny, self.nx)
        c = _f64(Cf, sh)
        u = None if ux is None else _f64(ux, sh)
        v = None if uy is None else _f64(uy, sh)
        self._ck(self._L.lb_set_solute_equilibrium(self._h, _dp(c), _dp(u), _dp(v)))

    def set_populations(self, f, fluid: int = 1):
        a = _f64(f, (9, self.ny, self.nx))
        self._ck(self._L.lb_set_populations(self._h, fluid, _dp(a)))

    def set_solute_populations(self, g):
        a = _f64(g, (self.q, self.ny, self.nx))
        self._ck(self._L.lb_set_solute_populations(self._h, _dp(a)))

    def set_precipitate(self, b):
        a = _f64(b, (self.ny, self.nx))
        self._ck(self._L.lb_set_precipitate(self._h, _dp(a)))

    def set_step(self, t: int):
        """Iterations done so far (the growth pick and thermo schedule use it)."""
        self._ck(self._L.lb_set_step(self._h, int(t)))

    # -- force fields --------------------------------------------------------
    def aveforce(self, mode: int, value: float, fluid: int = 1):
        self._ck(self._L.lb_aveforce(self._h, mode, value, fluid))

    def aveforce_xy(self, fx: float, fy: float, fluid: int = 1):
        self._ck(self._L.lb_aveforce_xy(self._h, fx, fy, fluid))

    def aveacceleration(self, mode: int, value: float, fluid: int = 1):
        self._ck(self._L.lb_aveacceleration(self._h, mode, value, fluid))

    def aveacceleration_xy(self, ax: float, ay: float, fluid: int = 1):
        self._ck(self._L.lb_aveacceleration_xy(self._h, ax, ay, fluid))

    def interforce(self, G: float, psi0: float = 0.0, rho0: float = 0.0):
        self._ck(self._L.lb_interforce(self._h, G, psi0, rho0))

    def intersolute(self, G: float, psi0: float, C0: float):
        self._ck(self._L.lb_intersolute(self._h, G, psi0, C0))

    def adhesiveforce(self, G: float, psi0: float = 0.0, rho0: float = 0.0, fluid: int = 1):
        self._ck(self._L.lb_adhesiveforce(self._h, G, psi0, rho0, fluid))

    # -- output and action -----------------------------------------------------
    def set_kernel(self, name: str = "auto"):
        self._ck(self._L.lb_set_kernel(self._h, _b(name)))

    def set_debug(self, flags: int = 0):
        """LB_DEBUG_POISON: NaN in every buffer an iteration writes, before
        it; LB_DEBUG_GUARDS: NaN guard zones around the buffers allocated
        afterwards."""
        self._ck(self._L.lb_set_debug(self._h, flags))

    def debug_check(self) -> int:
        """Guard bytes overwritten so far (LB_DEBUG_GUARDS)."""
        n = C.c_int64()
        self._ck(self._L.lb_debug_check(self._h, C.byref(n)))
        return int(n.value)

    def set_wait_limit(self, cycles: int = -1):
        """Clock-cycle limit of the TMA kernel's waits (-1: default)."""
        self._ck(self._L.lb_set_wait_limit(self._h, int(cycles)))

    def output(self, Nf: int):
        """output command: node fields every Nf iterations (0: off)."""
        self._ck(self._L.lb_output(self._h, Nf))

    def thermo(self, Nf: int):
        self._ck(self._L.lb_thermo(self._h, Nf))

    def thermo_deferred(self, on: bool = True):
        """Thermo records read by the next thermo evaluation or get_thermo
        instead of waited for at each thermo step (lb_thermo_deferred)."""
        self._ck(self._L.lb_thermo_deferred(self._h, 1 if on else 0))

    def iteration(self, Nt: int):
        self._ck(self._L.lb_iteration(self._h, Nt))

    def get_thermo(self) -> dict:
        t = Thermo()
        self._ck(self._L.lb_get_thermo(self._h, C.byref(t)))
        return t.as_dict()

    def thermo_static(self) -> dict:
        """Thermo record recomputed by lb_thermo_static, which allocates
        nothing (its scratch is a fixed array of the library)."""
        t = Thermo()
        self._ck(self._L.lb_thermo_static(self._h, C.byref(t)))
        return t.as_dict()

    def fields(self, fluid: int = 1):
        sh = (self.rows[1], self.nx)
        r, px, py, req = (np.zeros(sh) for _ in range(4))
        self._ck(self._L.lb_get_fields(self._h, fluid, _dp(r), _dp(px), _dp(py), _dp(req)))
        return r, px, py, req

    def velocity_f32(self, out=None):
        """Total density and solvent velocity (FP32) of the last iteration;
        ``out`` may be three preallocated (pinned) float32 arrays."""
        sh = (self.rows[1], self.nx)
        if out is None:
            out = tuple(np.zeros(sh, np.float32) for _ in range(3))
        r, u, v = out
        fp = lambda a: C.cast(C.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data), FP)
        self._ck(self._L.lb_get_velocity_f32(self._h, fp(r), fp(u), fp(v)))
        return out

    def populations(self, fluid: int = 1) -> np.ndarray:
        a = np.zeros((9, self.rows[1], self.nx))
        self._ck(self._L.lb_get_populations(self._h, fluid, _dp(a)))
        return a

    def solute_state(self, g=True, Cf=True, b=True):
        sh = (self.rows[1], self.nx)
        ga = np.zeros((self.q, self.rows[1], self.nx)) if g else None
        ca = np.zeros(sh) if Cf else None
        ba = np.zeros(sh) if b else None
        self._ck(self._L.lb_get_solute(self._h, _dp(ga), _dp(ca), _dp(ba)))
        return ga, ca, ba

    def mask(self) -> np.ndarray:
        m = np.zeros((self.rows[1], self.nx), np.uint8)
        self._ck(self._L.lb_get_mask(self._h, m.ctypes.data_as(U8P)))
        return m

    def buffer_size(self, what: str) -> int:
        """Bytes the named state buffer ("f0", "f1", "g0", "g1", "fields",
        "u") needs under the current setup."""
        n = SZ()
        self._ck(self._L.lb_buffer_size(self._h, what.encode(), C.byref(n)))
        return n.value

    def bind(self, what: str, tensor) -> None:
        """Use a caller-owned CUDA tensor (contiguous, on this device, at
        least buffer_size(what) bytes) as the named state buffer; the
        library writes it in place and the lattice keeps a reference.
        ``None`` unbinds.  Before the first iteration."""
        if tensor is None:
            self._ck(self._L.lb_bind(self._h, what.encode(), None, 0))
            self._bound.pop(what, None)
            return
        if not tensor.is_cuda or not tensor.is_contiguous():
            raise ValueError("bind needs a contiguous CUDA tensor")
        nbytes = tensor.numel() * tensor.element_size()
        self._ck(self._L.lb_bind(self._h, what.encode(), C.c_void_p(tensor.data_ptr()), nbytes))
        self._bound[what] = tensor

    def current_buffer(self) -> int:
        """k such that f<k> (and g<k>) hold the current state."""
        k = I()
        self._ck(self._L.lb_current_buffer(self._h, C.byref(k)))
        return k.value

    def flips(self) -> np.ndarray:
        """Node indices (y*nx + x, ascending) that growth turned solid in
        the last iteration executed."""
        n = I()
        self._ck(self._L.lb_get_flips(self._h, None, 0, C.byref(n)))
        out = np.zeros(max(n.value, 1), np.int64)
        self._ck(self._L.lb_get_flips(self._h, out.ctypes.data_as(C.POINTER(C.c_int64)), n.value, C.byref(n)))
        return out[:n.value]

    def state_size(self) -> int:
        n = C.c_size_t()
        self._ck(self._L.lb_state_size(self._h, C.byref(n)))
        return n.value

    def save_state(self, buf) -> None:
        """Copy the raw state into ``buf`` (numpy uint8 array or torch tensor
        of state_size() bytes, pinned for full copy speed)."""
        ptr, n = _buffer(buf)
        self._ck(self._L.lb_save_state(self._h, C.c_void_p(ptr), n))

    def load_state(self, buf) -> None:
        ptr, n = _buffer(buf)
        self._ck(self._L.lb_load_state(self._h, C.c_void_p(ptr), n))

    def write_restart(self, file: str, Nf: int) -> None:
        """write_restart command: input-data text files "<file>.<t>" (plus
        ".fluid1"/".fluid2", ".solute") every Nf iterations; 0 stops."""
        self._ck(self._L.lb_write_restart(self._h, _b(file), Nf))

    def write_data(self, file: str) -> None:
        """The current state as input-data text files named after ``file``."""
        self._ck(self._L.lb_write_data(self._h, _b(file)))

    def read_data(self, file: str, *args: str) -> None:
        """read_data command: args from "fluids", "solute", "equilibrium"."""
        self._ck(self._L.lb_read_data(self._h, _b(file), _b(",".join(args)) if args else None))
        v = [I() for _ in range(6)]
        self._ck(self._L.lb_lattice_info(self._h, *[C.byref(x) for x in v]))
        self.nx, self.ny, self.ncomp, self.q, _, self._py = (x.value for x in v)

    def launch_count(self) -> int:
        n = C.c_uint64()
        self._ck(self._L.lb_launch_count(self._h, C.byref(n)))
        return int(n.value)

    def velocity(self):
        """Solvent velocity of Eq. (4) as the library computes it
        (lb_get_velocity_f32), as float64 arrays [ny][nx]."""
        _, ux, uy = self.velocity_f32()
        return ux.astype(np.float64), uy.astype(np.float64)


def exchange(lattices: Sequence["Lattice"]) -> None:
    """Halo exchange of the slabs of one lattice held in this process on one
    device and stream (lattices[r] holds slab r), lb_exchange."""
    arr = (P * len(lattices))(*[lt.handle for lt in lattices])
    rc = lattices[0]._L.lb_exchange(arr, len(lattices))
    if rc != LB_OK:
        msgs = [lt._L.lb_last_error(lt.handle).decode() for lt in lattices]
        raise LBError(rc, "lb_exchange: " + " | ".join(m for m in msgs if m))


def _buffer(buf):
    if hasattr(buf, "data_ptr"):
        return buf.data_ptr(), buf.numel() * buf.element_size()
    a = np.asarray(buf)
    return a.ctypes.data, a.nbytes


class Batch:
    """Several single-component periodic lattices advanced by one launch per
    iteration (lb_batch_*)."""

    def __init__(self, lattices: Sequence[Lattice]):
        self._L = lib()
        self.lattices = list(lattices)
        arr = (P * len(self.lattices))(*[lt.handle for lt in self.lattices])
        h = P()
        rc = self._L.lb_batch_create(arr, len(self.lattices), C.byref(h))
        if rc != LB_OK:
            msg = self.lattices[0]._L.lb_last_error(self.lattices[0].handle).decode()
            raise LBError(rc, "lb_batch_create: " + msg)
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.lb_batch_destroy(h)
            self._h = None

    def _ck(self, rc):
        if rc != LB_OK:
            raise LBError(rc, self._L.lb_batch_last_error(self._h).decode())

    def iteration(self, Nt: int, use_graph: bool = True):
        self._ck(self._L.lb_batch_iteration(self._h, Nt, 1 if use_graph else 0))

    def autotune(self, cache_json: Optional[str] = None):
        self._ck(self._L.lb_batch_autotune(self._h, _b(cache_json)))

    def launch_count(self) -> int:
        n = C.c_uint64()
        self._ck(self._L.lb_batch_launch_count(self._h, C.byref(n)))
        return int(n.value)


# ---------------------------------------------------------------------------
# workload -> command sequence
# ---------------------------------------------------------------------------

def from_workload(w: "synth.Workload", storage: str = "fp32", h_max: float = 0.0,
                  device: int = 0, stream: Optional[int] = None, thermo: int = 0,
                  rounding: str = "nearest", kernel: str = "auto", precise: bool = False,
                  bind: Optional[dict] = None, step: int = 0,
                  slab: Optional[Tuple[int, int]] = None, debug: int = 0) -> Lattice:
    """Issue the command sequence that sets up workload ``w``.  ``bind``:
    state buffer name -> caller-owned CUDA tensor (Lattice.bind); ``step``:
    iterations already done (a state that continues another run); ``slab``:
    (py, rank) to hold one y slab of the lattice (processors command);
    ``debug``: LB_DEBUG_* flags, set before any device buffer exists."""
    lt = Lattice(device, stream)
    if debug:
        lt.set_debug(debug)
    lt.lattice(w.nx, w.ny, w.tau[0])
    if slab is not None:
        lt.processors(1, slab[0])
        lt.processor_rank(slab[1])
    if step:
        lt.set_step(step)
    if w.ncomp == 2:
        al = list(w.alpha) + [4.0 / 9.0] * (2 - len(w.alpha))
        lt.fluids(w.tau[0], w.tau[1], al[0], al[1])
    if w.solute_q:
        lt.solute(w.taus, w.solute_q)
    lt.set_storage(storage, list(w.rho_ref), h_max, rounding, precise)
    for name, tensor in (bind or {}).items():
        lt.bind(name, tensor)
    slip = list(getattr(w, "slip", None) or ())
    if any(np.ndim(R) > 0 for R in slip if R is not None):
        # hybrid: per-node coefficients, per component
        lt.boundary_style("hybrid")
        Rm = np.stack([np.zeros((w.ny, w.nx)) if (s >= len(slip) or slip[s] is None)
                       else np.broadcast_to(np.asarray(slip[s], np.float64), (w.ny, w.nx))
                       for s in range(w.ncomp)])
        lt.obstacle_mask_hybrid(w.solid, Rm)
    else:
        Rs = {float(R) for R in slip if R is not None}
        if len(Rs) > 1 or (Rs and len([R for R in slip if R is not None]) != w.ncomp):
            raise ValueError("components with different uniform coefficients need per-node maps")
        R = Rs.pop() if Rs else 0.0
        lt.boundary_style("noslip" if R == 0.0 else "slip" if R == 1.0 else "mixed", R)
        if w.solid.any():
            lt.obstacle_mask(w.solid)
    for k, op in enumerate(w.openings):
        labels = [f"o{k}f{s}" for s in range(w.ncomp)]
        (lt.inlet if op.kind == "inlet" else lt.outlet)(op.wall, op.a0, op.a1, labels[0],
                                                        labels[1] if w.ncomp == 2 else None)
        for s, (style, v, rho) in enumerate(op.momentum):
            (lt.inlet_momentum if op.kind == "inlet" else lt.outlet_momentum)(labels[s], style, v, rho)
        if op.solute is not None and w.solute_q:
            sv = op.solute[2] if len(op.solute) > 2 else 0.0
            (lt.inlet_solute if op.kind == "inlet" else lt.outlet_solute)(labels[0], op.solute[0], op.solute[1], sv)
    if w.reaction is not None and w.solute_q:
        kr, Cs, b0, bmax, seed = w.reaction
        lt.surface_reaction(kr, Cs, b0, bmax, seed)
    for s in range(w.ncomp):
        fx, fy = w.aveforce[s] if s < len(w.aveforce) else (0.0, 0.0)
        if fx or fy:
            lt.aveforce_xy(fx, fy, s + 1)
        ax, ay = w.aveacceleration[s] if s < len(w.aveacceleration) else (0.0, 0.0)
        if ax or ay:
            lt.aveacceleration_xy(ax, ay, s + 1)
        ad = w.adhesive[s] if s < len(w.adhesive) else None
        if ad is not None:
            lt.adhesiveforce(ad[0], ad[1], ad[2], s + 1)
    if w.interforce is not None:
        lt.interforce(*w.interforce)
    if getattr(w, "intersolute", None) is not None and w.solute_q:
        lt.intersolute(*w.intersolute)
    lt.thermo(thermo)
    lt.set_kernel(kernel)
    for s in range(w.ncomp):
        lt.set_equilibrium(w.rho[s], w.ux, w.uy, s + 1)
    if w.solute_q:
        Cf = np.zeros((w.ny, w.nx)) if w.C is None else w.C
        lt.set_solute_equilibrium(Cf, w.ux, w.uy)
    return lt
