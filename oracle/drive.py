"""Set up the FP64 oracle from a workload description.

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline).  The workload
is read by attribute (duck typing), so this module does not import the GPU
package; ``paper_1202_0442_gb300.synth.Workload`` is the usual argument.
"""
from __future__ import annotations

import numpy as np

from .orc import Oracle


def oracle_from_workload(w, solute_q=None) -> Oracle:
    q = w.solute_q if solute_q is None else solute_q
    o = Oracle(w.nx, w.ny, w.ncomp, q)
    o.set_solid(w.solid)
    for s in range(w.ncomp):
        o.set_tau(w.tau[s], s)
        o.set_alpha(w.alpha[s] if s < len(w.alpha) else 4.0 / 9.0, s)
        fx, fy = w.aveforce[s] if s < len(w.aveforce) else (0.0, 0.0)
        o.set_aveforce(fx, fy, s)
        ax, ay = (w.aveacceleration[s] if s < len(w.aveacceleration)
                  else (0.0, 0.0))
        o.set_aveacceleration(ax, ay, s)
        ad = w.adhesive[s] if s < len(w.adhesive) else None
        if ad is not None:
            o.set_adhesiveforce(ad[0], ad[1], ad[2], s)
    if w.interforce is not None:
        o.set_interforce(*w.interforce)
    for s, R in enumerate(getattr(w, "slip", None) or ()):
        if R is None:
            continue
        if np.ndim(R) == 0:
            o.set_slip(float(R), None, s)
        else:
            o.set_slip(0.0, R, s)
    for op in w.openings:
        k = o.add_opening(op.wall, op.a0, op.a1, op.kind)
        for s, (style, v, rho) in enumerate(op.momentum):
            o.set_opening_momentum(k, style, v, rho, s)
        if op.solute is not None and q:
            v = op.solute[2] if len(op.solute) > 2 else 0.0
            o.set_opening_solute(k, op.solute[0], op.solute[1], v)
    ux = 0.0 if w.ux is None else w.ux
    uy = 0.0 if w.uy is None else w.uy
    for s in range(w.ncomp):
        o.set_equilibrium(w.rho[s], ux, uy, s)
    if q:
        o.set_taus(w.taus)
        if getattr(w, "intersolute", None) is not None:
            o.set_intersolute(*w.intersolute)
        C = np.zeros((w.ny, w.nx)) if w.C is None else w.C
        o.set_solute_equilibrium(C, ux, uy)
        if w.reaction is not None:
            kr, Cs, b0, bmax, seed = w.reaction
            o.set_reaction(kr, Cs, b0, bmax, seed)
            o.set_b(np.where(w.solid != 0, b0, 0.0))
    return o
