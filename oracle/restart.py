"""The paper's input-data / restart text files read into the oracle
(read_data and write_restart commands, Sec. Commands).

TEST INFRASTRUCTURE ONLY (tests).  A plain reader written from the command
descriptions, independent of the GPU library's reader: a fluid file holds
the sections relaxation_time (tau, and alpha for two components), domain
(Nx Ny: sites 0..Nx, 0..Ny), processors (px py), inlet/outlet (wall x0 x1
label style arguments), boundary (periodic, noslip, slip, mixed R, hybrid), field
(force / acceleration as e<k> value pairs, interforce G psi0 rho0,
adhesiveforce G psi0 rho0), density (x y rho style; rho = -11 marks a solid
site) and momentum (x y f0 .. f8); a solute file holds relaxation_time,
inlet/outlet, reaction (surface kr Cs style bmax), field (intersolute G
psi0 C0), concentration (x y C [b]) and solute_modes (x y g ...).  Order
rules checked: domain before processors, field after relaxation_time,
processors before density and momentum, boundary before density, reaction
before concentration.

Readings where the command leaves room (stated the same way for the
library): every site is listed in density and, when present, momentum,
concentration and solute_modes; a mixed site may carry its R after the
style word; the reaction line may carry b0 and the growth seed after bmax;
a D2Q9 solute line carries g_0 .. g_8; without a momentum (solute_modes)
section, or with the argument "equilibrium", the state starts at the
equilibrium of the densities (concentrations) read and of the velocity the
populations read carry (zero without populations); the solute's velocity is
that of the solvent, sum_s j_s / sum_s rho_s.
"""
from __future__ import annotations

import numpy as np

from .orc import Oracle

FLUID_SECTIONS = ("relaxation_time", "domain", "processors", "inlet", "outlet", "boundary", "field",
                  "density", "momentum")
SOLUTE_SECTIONS = ("relaxation_time", "inlet", "outlet", "reaction", "field", "concentration",
                   "solute_modes")
EX = (0, 1, 0, -1, 0, 1, -1, -1, 1)
EY = (0, 0, 1, 0, -1, 1, 1, -1, -1)
SOLID = -11.0


class DataError(ValueError):
    pass


def sections(path, names):
    """{name: [token lists]} and the order the sections appear in."""
    out, order, cur = {}, [], None
    with open(path) as fh:
        for no, line in enumerate(fh, 1):
            tok = line.split()
            if not tok:
                continue
            if len(tok) == 1 and tok[0] in names:
                if tok[0] in out:
                    raise DataError(f"{path}:{no}: section {tok[0]} repeated")
                cur = tok[0]
                out[cur] = []
                order.append(cur)
                continue
            if cur is None:
                raise DataError(f"{path}:{no}: data before the first section")
            out[cur].append(tok)
    return out, order


def _before(order, a, b):
    return a not in order or b not in order or order.index(a) < order.index(b)


def _sites(rows, nx, ny, width, what, path):
    """rows 'x y v...' -> values [width][ny][nx] (every site once)"""
    a = np.zeros((width, ny, nx))
    seen = np.zeros((ny, nx), bool)
    for r in rows:
        x, y = int(r[0]), int(r[1])
        if not (0 <= x < nx and 0 <= y < ny):
            raise DataError(f"{path}: site ({x},{y}) outside the lattice")
        vals = [float(v) for v in r[2:2 + width]]
        if len(vals) != width:
            raise DataError(f"{path}: {what} line with {len(vals)} values")
        a[:, y, x] = vals
        seen[y, x] = True
    if not seen.all():
        raise DataError(f"{path}: the section {what} lists {int(seen.sum())} of {nx * ny} sites")
    return a


def read_fluid(path):
    s, order = sections(path, FLUID_SECTIONS)
    if not _before(order, "domain", "processors"):
        raise DataError(f"{path}: domain must precede processors")
    if "field" in order and not ("relaxation_time" in order and _before(order, "relaxation_time", "field")):
        raise DataError(f"{path}: field must follow relaxation_time")
    if not (_before(order, "processors", "density") and _before(order, "processors", "momentum")):
        raise DataError(f"{path}: processors must precede density and momentum")
    if not _before(order, "boundary", "density"):
        raise DataError(f"{path}: boundary must precede density")
    d = {"path": path}
    if s.get("relaxation_time"):
        t = [float(v) for v in s["relaxation_time"][0]]
        d["tau"] = t[0]
        d["alpha"] = t[1] if len(t) > 1 else None
    if s.get("domain"):
        d["Nx"], d["Ny"] = (int(v) for v in s["domain"][0])
    if s.get("processors"):
        d["px"], d["py"] = (int(v) for v in s["processors"][0])
    d["open"] = []
    for kind in ("inlet", "outlet"):
        for r in s.get(kind, []):
            d["open"].append({"kind": kind, "wall": r[0], "a0": int(r[1]), "a1": int(r[2]), "label": r[3],
                              "style": r[4] if len(r) > 4 else None, "args": [float(v) for v in r[5:]]})
    d["boundary"] = s["boundary"][0] if s.get("boundary") else ["periodic"]
    F = np.zeros(2)
    A = np.zeros(2)
    for r in s.get("field", []):
        if r[0] in ("force", "acceleration"):
            acc = F if r[0] == "force" else A
            for m, v in zip(r[1::2], r[2::2]):
                k = int(m[1:])
                acc += float(v) * np.array([EX[k], EY[k]])
        elif r[0] in ("interforce", "adhesiveforce"):
            d[r[0]] = tuple(float(v) for v in r[1:4])
        else:
            raise DataError(f"{path}: unknown field item {r[0]}")
    d["force"], d["acceleration"] = tuple(F), tuple(A)
    d["_s"] = s
    return d


def _fluid_sites(d, nx, ny, mixedR):
    s, path = d["_s"], d["path"]
    if s.get("density"):
        rho = _sites(s["density"], nx, ny, 1, "density", path)[0]
        R = np.zeros((ny, nx))
        for r in s["density"]:
            x, y = int(r[0]), int(r[1])
            st = r[3] if len(r) > 3 else "noslip"
            if st == "slip":
                R[y, x] = 1.0
            elif st == "mixed":
                R[y, x] = float(r[4]) if len(r) > 4 else mixedR
        d["rho"], d["solid"], d["R"] = rho, (rho == SOLID).astype(np.uint8), R
    if s.get("momentum"):
        d["f"] = _sites(s["momentum"], nx, ny, 9, "momentum", path)
    if "rho" not in d and "f" not in d:
        raise DataError(f"{path}: neither density nor momentum")


def read_solute(path, nx, ny):
    s, order = sections(path, SOLUTE_SECTIONS)
    if "field" in order and not ("relaxation_time" in order and _before(order, "relaxation_time", "field")):
        raise DataError(f"{path}: field must follow relaxation_time")
    if not _before(order, "reaction", "concentration"):
        raise DataError(f"{path}: reaction must precede concentration")
    d = {"path": path, "open": []}
    if s.get("relaxation_time"):
        d["taus"] = float(s["relaxation_time"][0][0])
    for kind in ("inlet", "outlet"):
        for r in s.get(kind, []):
            d["open"].append({"kind": kind, "wall": r[0], "a0": int(r[1]), "a1": int(r[2]), "label": r[3],
                              "style": r[4], "args": [float(v) for v in r[5:]]})
    for r in s.get("reaction", []):
        d["reaction"] = {"kr": float(r[1]), "Cs": float(r[2]), "style": r[3], "bmax": float(r[4]),
                         "b0": float(r[5]) if len(r) > 5 else None, "seed": int(r[6]) if len(r) > 6 else None}
    for r in s.get("field", []):
        if r[0] != "intersolute":
            raise DataError(f"{path}: unknown field item {r[0]}")
        d["intersolute"] = tuple(float(v) for v in r[1:4])
    if s.get("concentration"):
        rows = s["concentration"]
        d["C"] = _sites(rows, nx, ny, 1, "concentration", path)[0]
        if any(len(r) > 3 for r in rows):
            d["b"] = np.zeros((ny, nx))
            for r in rows:
                if len(r) > 3:
                    d["b"][int(r[1]), int(r[0])] = float(r[3])
    if s.get("solute_modes"):
        q = len(s["solute_modes"][0]) - 2
        if q not in (4, 9):
            raise DataError(f"{path}: {q} solute modes")
        d["g"] = _sites(s["solute_modes"], nx, ny, q, "solute_modes", path)
    if "C" not in d and "g" not in d:
        raise DataError(f"{path}: neither concentration nor solute_modes")
    return d


def oracle_from_data(file, *args, b0=0.0, seed=0):
    """An oracle set up from input-data files as read_data(file, args)
    would: args from "fluids", "solute", "equilibrium".  b0 and seed stand
    in for a reaction line that does not carry them."""
    fluids, solute, equilibrium = "fluids" in args, "solute" in args, "equilibrium" in args
    names = [f"{file}.fluid1", f"{file}.fluid2"] if fluids else [file]
    D = [read_fluid(n) for n in names]
    Nx, Ny = D[0]["Nx"], D[0]["Ny"]
    if any((d["Nx"], d["Ny"]) != (Nx, Ny) for d in D):
        raise DataError("the fluid files give different domains")
    nx, ny = Nx + 1, Ny + 1
    b = D[0]["boundary"]
    mixedR = float(b[1]) if b[0] == "mixed" else 0.0
    for d in D:
        _fluid_sites(d, nx, ny, mixedR)
    S = read_solute(f"{file}.solute", nx, ny) if solute else None
    q = 0
    if S is not None:
        q = S["g"].shape[0] if "g" in S else 4
    o = Oracle(nx, ny, len(D), q)
    solid = D[0]["solid"] if "solid" in D[0] else np.zeros((ny, nx), np.uint8)
    o.set_solid(solid)
    for c, d in enumerate(D):
        if "tau" in d:
            o.set_tau(d["tau"], c)
        # the density-ratio parameter applies to multicomponent runs only
        if d.get("alpha") is not None and len(D) == 2:
            o.set_alpha(d["alpha"], c)
        o.set_aveforce(*d["force"], c)
        o.set_aveacceleration(*d["acceleration"], c)
        if "adhesiveforce" in d:
            o.set_adhesiveforce(*d["adhesiveforce"], c)
        if b[0] == "slip":
            o.set_slip(1.0, None, c)
        elif b[0] == "mixed":
            o.set_slip(mixedR, None, c)
        elif b[0] == "hybrid":
            o.set_slip(0.0, np.where(solid != 0, d["R"], 0.0), c)
    if "interforce" in D[0]:
        o.set_interforce(*D[0]["interforce"])
    where = {}
    for k, op in enumerate(D[0]["open"]):
        i = o.add_opening(op["wall"], op["a0"], op["a1"], op["kind"])
        where[(op["kind"], op["wall"], op["a0"], op["a1"])] = i
        for c, d in enumerate(D):
            m = [p for p in d["open"] if (p["kind"], p["wall"], p["a0"], p["a1"]) == (op["kind"], op["wall"], op["a0"], op["a1"])]
            if not m:
                raise DataError(f"{d['path']}: no line for the opening at {op['wall']} {op['a0']} {op['a1']}")
            p = m[0]
            if p["style"] is None:
                continue
            a = p["args"]
            v, rho = (a[0], a[1]) if p["style"] in ("poiseuille", "uniform") else (0.0, a[0])
            o.set_opening_momentum(i, p["style"], v, rho, c)
    # the state
    rs = np.zeros((ny, nx))
    jx = np.zeros((ny, nx))
    jy = np.zeros((ny, nx))
    fl = solid == 0
    for c, d in enumerate(D):
        if "f" in d and not equilibrium:
            f = np.where(fl, d["f"], 0.0)
            o.set_f(f, c)
            rho_c, px, py = f.sum(0), np.tensordot(EX, f, 1), np.tensordot(EY, f, 1)
        else:
            f = d.get("f")
            px = np.tensordot(EX, f, 1) if f is not None else np.zeros((ny, nx))
            py = np.tensordot(EY, f, 1) if f is not None else np.zeros((ny, nx))
            rho_c = d["rho"] if "rho" in d else f.sum(0)
            rho_c = np.where(fl, rho_c, 0.0)
            safe = np.where(fl, rho_c, 1.0)
            o.set_equilibrium(rho_c, np.where(fl, px / safe, 0.0), np.where(fl, py / safe, 0.0), c)
            px, py = np.where(fl, px, 0.0), np.where(fl, py, 0.0)
        rs += np.where(fl, rho_c, 0.0)
        jx += px
        jy += py
    if S is None:
        return o
    if "taus" in S:
        o.set_taus(S["taus"])
    for op in S["open"]:
        key = (op["kind"], op["wall"], op["a0"], op["a1"])
        if key not in where:
            raise DataError(f"{S['path']}: the solute opening has no fluid opening")
        a = op["args"]
        if op["style"] == "flux":
            o.set_opening_solute(where[key], "flux", a[1], a[0])
        else:
            o.set_opening_solute(where[key], op["style"], a[0], 0.0)
    if "intersolute" in S:
        o.set_intersolute(*S["intersolute"])
    if "reaction" in S:
        r = S["reaction"]
        o.set_reaction(r["kr"], r["Cs"], r["b0"] if r["b0"] is not None else b0, r["bmax"],
                       r["seed"] if r["seed"] is not None else seed)
    if "g" in S and not equilibrium:
        o.set_g(np.where(fl, S["g"], 0.0))
    else:
        C = S["C"] if "C" in S else S["g"].sum(0)
        safe = np.where(rs > 0, rs, 1.0)
        o.set_solute_equilibrium(np.where(fl, C, 0.0), np.where(rs > 0, jx / safe, 0.0),
                                 np.where(rs > 0, jy / safe, 0.0))
    if "b" in S:
        o.set_b(S["b"])
    return o
