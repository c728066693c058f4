"""A small, self-contained run of one kernel for ncu captures.

    python profile_target.py porous4096 fp32
    python profile_target.py shanchen2048 fp32
    python profile_target.py reactive fp32
    python profile_target.py batch256 fp32

Sets up the named workload on cuda:0, runs a fixed number of iterations
(thermo off, so every launch is the same kernel sequence) and exits 0.
Under ``ncu -k regex:<kernel> -s <skip> -c 1`` it gives one launch of that
kernel on a lattice larger than L2 while keeping the device footprint to a
few GB.
"""
from __future__ import annotations

import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None) -> int:
    argv = sys.argv[1:] if argv is None else argv
    name = argv[0] if argv else "porous4096"
    storage = argv[1] if len(argv) > 1 else "fp32"
    iters = int(argv[2]) if len(argv) > 2 else 8
    import torch

    from paper_1202_0442_gb300 import build, lb2d, synth
    build.build()
    torch.cuda.set_device(0)
    if name == "porous4096":
        w = synth.porous(4096, 4096, seed=1)
    elif name == "porous1024":
        w = synth.porous()
    elif name == "shanchen2048":
        w = synth.shan_chen2(2048)
    elif name == "reactive":
        w = synth.reactive()
    elif name == "batch256":
        # the 256 lattices of the batched workload, one launch per iteration
        ws = synth.batch()
        kw = {"h_max": 5e-3, "rounding": "stochastic"} if storage != "fp32" else {"precise": True}
        lats = [lb2d.from_workload(x, storage, **kw) for x in ws]
        for lt in lats:
            lt.thermo(1 << 30)
        b = lb2d.Batch(lats)
        b.iteration(iters, use_graph=False)
        torch.cuda.synchronize()
        print(f"batch256 {storage}: {iters} iterations, {sum(x.nodes for x in ws)} nodes, "
              f"{b.launch_count()} launches")
        return 0
    else:
        raise SystemExit(f"unknown workload {name}")
    lt = lb2d.from_workload(w, storage, h_max=2e-3,
                            rounding="stochastic" if storage != "fp32" else "nearest")
    lt.thermo(1 << 30)
    lt.iteration(iters)
    torch.cuda.synchronize()
    print(f"{name} {storage}: {iters} iterations, {w.nodes} nodes, {w.fluid_nodes} fluid, "
          f"{lt.launch_count()} launches")
    return 0


if __name__ == "__main__":
    sys.exit(main())
