"""Long runs: every workload at its stated iteration count, the GPU library
against the FP64 oracle.

The oracle needs minutes to hours for these (config 4 alone about two
hours on one core), so this is a script run by hand, not part of the
pytest suites:

    python tests/long_parity.py gpu <dir> [case ...]      # on a GPU
    python tests/long_parity.py oracle <dir> [case ...]   # on CPU cores
    python tests/long_parity.py compare <gpu_dir> <oracle_dir>
    python tests/long_parity.py report <dir>              # config 3 at 2048^2, GPU only
    python tests/long_parity.py owindows <dir> [case ...]  # oracle states + flips for windows
    python tests/long_parity.py gwindows <odir> <dir> [case ...]  # GPU restarted in each window

`gpu` runs the library (one lattice, or the batched launch for the batch
case) and writes <dir>/<case>_<storage>.npz; `oracle` runs the oracle,
one process per case, and writes <dir>/<case>.npz; `compare` prints one
markdown table row per (case, storage): relative errors in rho and u,
masks, mass drift of both sides, and the case's own physics numbers.
No value produced here is stored as an expected value anywhere.

`owindows` / `gwindows` compare growth decisions along the whole run by
restarting the GPU from the oracle's state: the oracle saves, at a few
window starts, its state as the GPU stores it (population deviations and
solute populations rounded to FP32, FP64 deposits, the mask) together
with its flips and near-threshold decisions for the next WINDOW steps;
the GPU restarts there (`lb_set_step`) and every step's flip set is
compared until the first difference, which must sit at a decision within
rounding of the threshold.  Nothing of the GPU run enters the oracle.
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1202_0442_gb300 import synth  # noqa: E402

BATCH_PICK = (0, 37, 73, 109, 146, 182, 219, 255)


def _batch_workloads():
    ws = synth.batch()
    return [ws[k] for k in BATCH_PICK]


CASES = {
    # name: (workload factory, iterations, storages, checkpoints)
    "channel": (lambda: synth.channel(), 2000, ("fp32", "fp16", "bf16"), ()),
    "porous": (lambda: synth.porous(), 10000, ("fp32", "fp16", "bf16"), ()),
    "shan_chen2_256": (lambda: synth.shan_chen2(256), 20000, ("fp32", "fp16"), (2000,)),
    # the stated recipe (uniform velocity inlet) diverges in the oracle and
    # on the GPU alike once growth closes cells at the inlet (about 1700
    # iterations); the long run uses the pressure-driven version, solute
    # entering from the inlet
    "reactive_q9": (lambda: synth.reactive(q=9, inlet="pressure", C_init=0.0), 50000, ("fp32",), ()),
    "reactive_q4": (lambda: synth.reactive(q=4, inlet="pressure", C_init=0.0), 50000, ("fp32",), ()),
    "batch8": (_batch_workloads, 5000, ("fp32", "fp32+pm", "fp16"), ()),
}
H_MAX = {"channel": 2e-3, "porous": 2e-3, "shan_chen2_256": 1.2, "batch8": 5e-3}
# config 3 at its stated size: the oracle runs the whole 2048^2 lattice to
# 2000 iterations (about 1.5 h on one core) and the comparison is node by
# node on 16 bands of 32 rows (a quarter of the lattice, crossing the free
# droplet, the ring and the bulk); the GPU goes on to 20 000 iterations,
# where its component masses are compared with the initial ones (the
# oracle's own drift, FP64, stays below 1e-11 at 20 000 on the 256^2 ring)
CASES["shan_chen2_2048"] = (lambda: synth.shan_chen2(2048), 20000, ("fp32",), (2000,))
ORACLE_STEPS = {"shan_chen2_2048": 2000}
ROWS = {"shan_chen2_2048": np.concatenate([np.arange(k * 128, k * 128 + 32) for k in range(16)])}


def _snapshot_gpu(lt, w, rows=None):
    sel = (lambda a: a) if rows is None else (lambda a: a[rows])
    out = {"mask": sel(lt.mask().astype(np.uint8))}
    for c in range(1, w.ncomp + 1):
        r, px, py, _ = lt.fields(c)
        out[f"rho{c}"] = sel(r.astype(np.float32))
    ux, uy = lt.velocity()
    out["ux"], out["uy"] = sel(ux.astype(np.float32)), sel(uy.astype(np.float32))
    if w.solute_q:
        _, Cf, b = lt.solute_state(g=False)
        out["C"], out["b"] = Cf.astype(np.float32), b
    out["thermo"] = np.array(json.dumps(lt.get_thermo()))
    return out


EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], float)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], float)


def _snapshot_pops(f, mask, w):
    """Density, velocity (j + F/2)/rho and mass from the populations of a
    single-component lattice with aveforce/aveacceleration (the batched
    lattices, whose kernel writes no field planes)."""
    fl = mask == 0
    rho = np.where(fl, f.sum(0), 0.0)
    fx, fy = w.aveforce[0] if w.aveforce else (0.0, 0.0)
    ax, ay = w.aveacceleration[0] if w.aveacceleration else (0.0, 0.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        ux = np.where(fl, (np.tensordot(EX, f, 1) + 0.5 * (fx + rho * ax)) / np.where(fl, rho, 1), 0.0)
        uy = np.where(fl, (np.tensordot(EY, f, 1) + 0.5 * (fy + rho * ay)) / np.where(fl, rho, 1), 0.0)
    return {"mask": mask.astype(np.uint8), "rho1": rho, "ux": ux, "uy": uy,
            "thermo": np.array(json.dumps({"mass1": float(rho[fl].sum())}))}


def _snapshot_oracle(o, w, rows=None):
    sel = (lambda a: a) if rows is None else (lambda a: a[rows])
    out = {"mask": sel(o.solid().astype(np.uint8))}
    for c in range(w.ncomp):
        out[f"rho{c + 1}"] = sel(o.fields(c)[0])
    ux, uy = o.velocity()
    out["ux"], out["uy"] = sel(ux), sel(uy)
    if w.solute_q:
        out["C"], out["b"] = o.solute_C(), o.b()
    out["thermo"] = np.array(json.dumps(o.thermo()))
    return out


def run_gpu(outdir, names):
    import torch
    from paper_1202_0442_gb300 import build, lb2d
    build.build()
    torch.cuda.set_device(0)
    os.makedirs(outdir, exist_ok=True)
    for name in names:
        make, steps, storages, cps = CASES[name]
        for st in storages:
            # "+pm": exact FP32 momentum pairs (LB_PRECISE_MOMENTUM)
            kw = {"h_max": H_MAX.get(name, 0.0), "precise": st.endswith("+pm")}
            if not st.startswith("fp32"):
                kw["rounding"] = "stochastic"
            storage = st.split("+")[0]
            t0 = time.time()
            if name == "batch8":
                ws = make()
                lts = [lb2d.from_workload(w, storage, thermo=0, **kw) for w in ws]
                b = lb2d.Batch(lts)
                b.iteration(steps)
                torch.cuda.synchronize()
                res = {}
                for k, (w, lt) in enumerate(zip(ws, lts)):
                    snap = _snapshot_pops(lt.populations(), lt.mask(), w)
                    for key, v in snap.items():
                        res[f"l{k}_{key}"] = v
            else:
                w = make()
                lt = lb2d.from_workload(w, storage, thermo=0, **kw)
                res, done = {}, 0
                for cp in tuple(cps) + (steps,):
                    lt.iteration(cp - done)
                    done = cp
                    tag = "" if cp == steps else f"t{cp}_"
                    for key, v in _snapshot_gpu(lt, w, ROWS.get(name)).items():
                        res[tag + key] = v
            torch.cuda.synchronize()
            res = {k: (v.astype(np.float32) if v.dtype == np.float64 and not k.endswith("b") else v)
                   for k, v in res.items()}
            res["seconds"] = np.array(time.time() - t0)
            np.savez_compressed(os.path.join(outdir, f"{name}_{st}.npz"), **res)
            print(f"{name} {st}: {steps} iterations, {time.time() - t0:.1f} s", flush=True)


def _oracle_one(args):
    name, outdir = args
    sys.path.insert(0, ROOT)
    from oracle.drive import oracle_from_workload
    make, steps, _, cps = CASES[name]
    t0 = time.time()
    res = {}
    if name == "batch8":
        for k, w in enumerate(make()):
            o = oracle_from_workload(w)
            o.step(steps)
            for key, v in _snapshot_pops(o.f(0), o.solid(), w).items():
                res[f"l{k}_{key}"] = v
    else:
        w = make()
        o = oracle_from_workload(w)
        done = 0
        last = ORACLE_STEPS.get(name, steps)
        for cp in [c for c in tuple(cps) + (steps,) if c <= last]:
            o.step(cp - done)
            done = cp
            tag = "" if cp == steps else f"t{cp}_"
            for key, v in _snapshot_oracle(o, w, ROWS.get(name)).items():
                res[tag + key] = v
    res["seconds"] = np.array(time.time() - t0)
    np.savez_compressed(os.path.join(outdir, f"{name}.npz"), **res)
    return name, time.time() - t0


def run_oracle(outdir, names):
    os.makedirs(outdir, exist_ok=True)
    with mp.get_context("spawn").Pool(len(names)) as pool:
        for name, dt in pool.imap_unordered(_oracle_one, [(n, outdir) for n in names]):
            print(f"oracle {name}: {dt:.0f} s", flush=True)


def _rel(a, b, fl):
    den = max(float(np.max(np.abs(b[fl]))), 1e-300)
    return float(np.max(np.abs(a[fl].astype(np.float64) - b[fl])) / den)


def _compare_one(g, o, w, prefix="", rows=None):
    mg, mo = g[prefix + "mask"], o[prefix + "mask"]
    fl = (mo == 0) & (mg == 0)
    row = {"mask_equal": bool(np.array_equal(mg, mo)), "mask_diff": int((mg != mo).sum())}
    for c in range(1, w.ncomp + 1):
        row[f"rho{c}"] = _rel(g[prefix + f"rho{c}"], o[prefix + f"rho{c}"], fl)
    den = max(float(np.max(np.abs(o[prefix + "ux"][fl]))), float(np.max(np.abs(o[prefix + "uy"][fl]))), 1e-300)
    row["u"] = max(float(np.max(np.abs(g[prefix + "ux"][fl] - o[prefix + "ux"][fl]))),
                   float(np.max(np.abs(g[prefix + "uy"][fl] - o[prefix + "uy"][fl])))) / den
    tg = json.loads(str(g[prefix + "thermo"]))
    to = json.loads(str(o[prefix + "thermo"]))
    m0 = [float(np.sum(np.where(w.solid != 0, 0.0, r))) for r in w.rho]
    for c in range(1, w.ncomp + 1):
        row[f"drift{c}_gpu"] = (tg[f"mass{c}"] - m0[c - 1]) / m0[c - 1]
        row[f"drift{c}_oracle"] = (to[f"mass{c}"] - m0[c - 1]) / m0[c - 1]
        row[f"mass{c}_vs_oracle"] = abs(tg[f"mass{c}"] - to[f"mass{c}"]) / abs(to[f"mass{c}"])
    if rows is not None:
        row["rows_compared"] = int(len(rows))
    if w.solute_q:
        row["C"] = _rel(g[prefix + "C"], o[prefix + "C"], fl)
        row["b"] = float(np.max(np.abs(g[prefix + "b"] - o[prefix + "b"])) / max(float(np.max(o[prefix + "b"])), 1e-300))
        row["grown_gpu"] = int((mg != w.solid).sum())
        row["grown_oracle"] = int((mo != w.solid).sum())
        for k in ("solute", "bsum", "removed_solute"):
            row[f"{k}_vs_oracle"] = abs(tg[k] - to[k]) / max(abs(to[k]), 1e-300)
    return row


def _laplace(d, w, prefix=""):
    """Laplace report: pressure p = (rho1 + rho2)/3 + G rho1 rho2 / 3 inside
    the free droplet (mean over its inner half radius) and far outside
    (a 17 x 17 window at (0.9 n, 0.1 n), clear of the droplet and the ring),
    and the droplet's radius from its area (rho1 above the mean of the two
    phase densities within 1.5 initial radii of the initial centre)."""
    G = w.interforce[0]
    r1, r2 = d[prefix + "rho1"].astype(np.float64), d[prefix + "rho2"].astype(np.float64)
    p = (r1 + r2) / 3 + G * r1 * r2 / 3
    dc, _, dr = w.info["drop"]
    n = w.nx
    y, x = np.mgrid[0:n, 0:n]
    ddx = (x - dc + n // 2) % n - n // 2
    ddy = (y - dc + n // 2) % n - n // 2
    near = ddx * ddx + ddy * ddy <= (1.5 * dr) ** 2
    drop = near & (r1 > w.rho_ref[0]) & (w.solid == 0)
    area = int(drop.sum())
    R = float(np.sqrt(area / np.pi)) if area else 0.0
    inner = drop & (ddx * ddx + ddy * ddy <= (0.5 * R) ** 2)
    px, py = int(0.9 * n), int(0.1 * n)
    win = p[py - 8:py + 9, px - 8:px + 9]
    p_in = float(p[inner].mean()) if inner.any() else float("nan")
    p_out = float(win.mean())
    return {"p_in": p_in, "p_out": p_out, "dp": p_in - p_out, "R": R, "dp_R": (p_in - p_out) * R,
            "drop_r0": dr}

def _permeability(d, w, prefix=""):
    """Darcy permeability k = mu q / |grad p| with q the superficial mean
    u_x over all nodes, p = rho / 3, mu = rho_mean nu, nu = (tau - 1/2)/3,
    the gradient from the held densities over the length nx - 1."""
    nu = (w.tau[0] - 0.5) / 3.0
    fl = w.solid == 0
    r = d[prefix + "rho1"].astype(np.float64)
    q = float(np.sum(np.where(fl, d[prefix + "ux"], 0.0))) / (w.nx * w.ny)
    dp = (w.info["rho_in"] - w.info["rho_out"]) / 3.0 / (w.nx - 1)
    return q * float(r[fl].mean()) * nu / dp


def compare(gdir, odir):
    rows = []
    for name, (make, steps, storages, cps) in CASES.items():
        op = os.path.join(odir, f"{name}.npz")
        if not os.path.exists(op):
            continue
        o = np.load(op)
        for st in storages:
            gp = os.path.join(gdir, f"{name}_{st}.npz")
            if not os.path.exists(gp):
                continue
            g = np.load(gp)
            if name == "batch8":
                ws = make()
                worst = {}
                for k, w in enumerate(ws):
                    r = _compare_one(g, o, w, prefix=f"l{k}_")
                    for key, v in r.items():
                        if isinstance(v, bool):
                            worst[key] = worst.get(key, True) and v
                        else:
                            worst[key] = max(worst.get(key, v), v, key=abs) if "drift" in key else max(worst.get(key, 0), v)
                rows.append((name, st, steps, worst))
                continue
            w = make()
            for cp in cps:
                rows.append((name, st, cp, _compare_one(g, o, w, prefix=f"t{cp}_", rows=ROWS.get(name))))
            if ORACLE_STEPS.get(name, steps) < steps:
                # past the oracle's run: the GPU's component masses against
                # the initial ones (the method keeps them exactly)
                tg = json.loads(str(g["thermo"]))
                m0 = [float(np.sum(np.where(w.solid != 0, 0.0, r))) for r in w.rho]
                rows.append((name, st, steps, {f"drift{c}_gpu": (tg[f"mass{c}"] - m0[c - 1]) / m0[c - 1]
                                               for c in range(1, w.ncomp + 1)}))
                continue
            r = _compare_one(g, o, w)
            if name == "porous":
                r["permeability_gpu"] = _permeability(g, w)
                r["permeability_oracle"] = _permeability(o, w)
            if name.startswith("shan_chen"):
                r.update({f"gpu_{k}": v for k, v in _laplace(g, w).items()})
                r.update({f"oracle_{k}": v for k, v in _laplace(o, w).items()})
            rows.append((name, st, steps, r))
    for name, st, t, r in rows:
        items = ", ".join(f"{k} {v:.3g}" if isinstance(v, float) else f"{k} {v}" for k, v in r.items())
        print(f"| {name} | {st} | {t} | {items} |")


REACTIVE = ("reactive_q4", "reactive_q9")


WINDOW_STARTS = (10000, 25000, 40000)
WINDOW = 1000


def _owindows_one(args):
    name, outdir = args
    sys.path.insert(0, ROOT)
    from oracle.drive import oracle_from_workload
    make = CASES[name][0]
    w = make()
    o = oracle_from_workload(w)
    o.set_margin_eps(1e-4, 1 << 16)
    bmax = abs(w.reaction[3])
    s = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    rho_ref = float(np.float32(w.rho_ref[0]))
    t0 = time.time()
    for ws in WINDOW_STARTS:
        o.step(ws - o.t)
        f = o.f(0)
        solid = o.solid()
        # the state as the library holds it: deviations from s_i rho_ref and
        # the solute populations in FP32, the deposits in FP64
        h32 = np.where(solid[None] != 0, 0.0, f - s * rho_ref).astype(np.float32)
        g32 = o.g().astype(np.float32)
        b = o.b()
        ts, nodes, mt, mn, mv = [], [], [], [], []
        for t in range(ws + 1, ws + WINDOW + 1):
            o.step(1)
            fl = o.flips()
            ts.append(np.full(fl.size, t, np.int32))
            nodes.append(fl.astype(np.int32))
            idx, val = o.margin_events()
            mt.append(np.full(idx.size, t, np.int32))
            mn.append(idx.astype(np.int32))
            mv.append(val / bmax)
        np.savez_compressed(os.path.join(outdir, f"{name}_w{ws}.npz"), h32=h32, g32=g32, b=b,
                            solid=solid.astype(np.uint8), t0=np.array(ws), ft=np.concatenate(ts),
                            fn=np.concatenate(nodes), mt=np.concatenate(mt), mn=np.concatenate(mn),
                            mv=np.concatenate(mv))
        print(f"oracle {name}: window {ws} saved, {time.time() - t0:.0f} s", flush=True)
    return name, time.time() - t0


def run_owindows(outdir, names):
    os.makedirs(outdir, exist_ok=True)
    names = [n for n in names if n in REACTIVE] or list(REACTIVE)
    with mp.get_context("spawn").Pool(len(names)) as pool:
        for name, dt in pool.imap_unordered(_owindows_one, [(n, outdir) for n in names]):
            print(f"oracle {name}: {dt:.0f} s", flush=True)


def run_gwindows(odir, outdir, names):
    import copy as _copy
    import torch
    from paper_1202_0442_gb300 import build, lb2d
    build.build()
    torch.cuda.set_device(0)
    os.makedirs(outdir, exist_ok=True)
    names = [n for n in names if n in REACTIVE] or list(REACTIVE)
    report = {}
    for name in names:
        w = CASES[name][0]()
        s = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
        rho_ref = float(np.float32(w.rho_ref[0]))
        for ws in WINDOW_STARTS:
            path = os.path.join(odir, f"{name}_w{ws}.npz")
            if not os.path.exists(path):
                continue
            d = np.load(path)
            ww = _copy.copy(w)
            ww.solid = d["solid"]
            lt = lb2d.from_workload(ww, "fp32", thermo=0, step=int(d["t0"]))
            # f = h + s rho_ref in FP64: the library's FP64 subtraction gives h back exactly
            lt.set_populations(np.where(d["solid"][None] != 0, 0.0, d["h32"].astype(np.float64) + s * rho_ref))
            lt.set_solute_populations(d["g32"].astype(np.float64))
            lt.set_precipitate(d["b"])
            ft, fn, mt, mn, mv = d["ft"], d["fn"], d["mt"], d["mn"], d["mv"]
            rep = {"compared": 0, "matched_flips": 0, "oracle_flips": int(fn.size), "first_diff": None}
            for t in range(ws + 1, ws + WINDOW + 1):
                lt.iteration(1)
                fg = lt.flips()
                fo = np.sort(fn[ft == t]).astype(np.int64)
                rep["compared"] += 1
                if np.array_equal(fg, fo):
                    rep["matched_flips"] += int(fo.size)
                    continue
                margins = {int(n): float(v) for n, v in zip(mn[mt == t], mv[mt == t])}
                diff = []
                for n in np.setxor1d(fg, fo):
                    y, x = divmod(int(n), w.nx)
                    near = {m: margins[m] for m in ((yy % w.ny) * w.nx + (xx % w.nx)
                                                    for yy in (y - 1, y, y + 1) for xx in (x - 1, x, x + 1))
                            if m in margins}
                    diff.append({"node": int(n), "in": "gpu" if n in set(fg.tolist()) else "oracle",
                                 "near_triggers": near})
                rep["first_diff"] = {"t": t, "diff": diff}
                break
            report[f"{name}@{ws}"] = rep
            print(name, ws, json.dumps(rep)[:1500], flush=True)
    with open(os.path.join(outdir, "windows.json"), "w") as fh:
        json.dump(report, fh, indent=1)


def run_report(outdir):
    """Config 3 at full size (2048^2, two components, 20000 iterations):
    component masses, their drift, and the pressures of the Laplace
    report, FP32 and FP16 storage.  GPU only (the oracle would need hours;
    its parity is checked on the 256^2 version of the same recipe)."""
    import torch
    from paper_1202_0442_gb300 import build, lb2d
    build.build()
    torch.cuda.set_device(0)
    os.makedirs(outdir, exist_ok=True)
    out = {}
    runs = [("stated", synth.shan_chen2(2048), ("fp32", "fp16"))]
    for R in (100, 200, 300):
        runs.append((f"x2.2_drop{R}", synth.shan_chen2(2048, rich=2.2, lean=0.066, drop_r=R), ("fp32",)))
    for tag, w, storages in runs:
        _report_one(out, tag, w, storages)
    with open(os.path.join(outdir, "shan_chen2_2048_report.json"), "w") as fh:
        json.dump(out, fh, indent=1)


def _report_one(out, tag, w, storages):
    import torch
    from paper_1202_0442_gb300 import lb2d
    m0 = [float(np.sum(np.where(w.solid != 0, 0.0, r))) for r in w.rho]
    for st in storages:
        kw = {"h_max": 1.2}
        if st != "fp32":
            kw["rounding"] = "stochastic"
        lt = lb2d.from_workload(w, st, thermo=0, **kw)
        t0 = time.time()
        lt.iteration(w.steps)
        torch.cuda.synchronize()
        dt = time.time() - t0
        th = lt.get_thermo()
        d = {"rho1": lt.fields(1)[0], "rho2": lt.fields(2)[0]}
        rep = {"iterations": w.steps, "seconds": dt,
               "mlups": w.nx * w.ny * w.steps / dt / 1e6,
               "mass1": th["mass1"], "mass2": th["mass2"],
               "drift1": (th["mass1"] - m0[0]) / m0[0], "drift2": (th["mass2"] - m0[1]) / m0[1]}
        rep.update(_laplace(d, w))
        out[f"{tag}/{st}"] = rep
        print(tag, st, rep, flush=True)


def main(argv):
    if len(argv) < 2:
        print(__doc__)
        return 2
    mode = argv[0]
    if mode == "compare":
        compare(argv[1], argv[2])
        return 0
    if mode == "report":
        run_report(argv[1])
        return 0
    if mode == "gwindows":
        run_gwindows(argv[1], argv[2], argv[3:])
        return 0
    if mode == "owindows":
        run_owindows(argv[1], argv[2:])
        return 0
    names = argv[2:] or list(CASES)
    if mode == "gpu":
        run_gpu(argv[1], names)
    elif mode == "oracle":
        run_oracle(argv[1], names)
    else:
        print(__doc__)
        return 2
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
