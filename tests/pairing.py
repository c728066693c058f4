"""Helpers that run one workload on the GPU library and on the FP64 oracle
and measure their differences (used by the -m gpu parity tests)."""
import numpy as np

from oracle.drive import oracle_from_workload
from paper_1202_0442_gb300 import lb2d

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def run_pair(w, steps, storage="fp32", h_max=0.0, thermo=0, oracle_steps=None, **kw):
    lt = lb2d.from_workload(w, storage, h_max=h_max, thermo=thermo, **kw)
    o = oracle_from_workload(w)
    if steps:
        lt.iteration(steps)
        o.step(steps if oracle_steps is None else oracle_steps)
    return lt, o


def rel_rho(lt, o, w, comp=1):
    fl = w.solid == 0 if lt is None else (o.solid() == 0)
    rg = lt.fields(comp)[0]
    ro = o.fields(comp - 1)[0]
    return float(np.max(np.abs(rg[fl] - ro[fl])) / np.max(np.abs(ro[fl])))


def rel_u(lt, o):
    fl = o.solid() == 0
    ug, vg = lt.velocity()
    uo, vo = o.velocity()
    den = max(np.max(np.abs(uo[fl])), np.max(np.abs(vo[fl])), 1e-300)
    return float(max(np.max(np.abs(ug[fl] - uo[fl])), np.max(np.abs(vg[fl] - vo[fl]))) / den)


def pop_err(lt, o, comp=1, rho_ref=1.0):
    """max |f_gpu - f_oracle| over the scale of the deviations from rest."""
    fg = lt.populations(comp)
    fo = o.f(comp - 1)
    fl = (o.solid() == 0)[None, :, :]
    dev = np.abs(fo - W9[:, None, None] * rho_ref)
    scale = max(float(np.max(np.where(fl, dev, 0.0))), 1e-300)
    return float(np.max(np.where(fl, np.abs(fg - fo), 0.0)) / scale), scale


def thermo_err(lt, o, keys):
    tg = lt.get_thermo()
    to = o.thermo()
    out = {}
    for k in keys:
        den = max(abs(to[k]), 1e-300)
        out[k] = abs(tg[k] - to[k]) / den
    return out, tg, to
