"""The library's own Eq. (4) output against the oracle.

lb_get_velocity_f32 is the call the end-to-end benchmark reads: total
density and the solvent velocity u = sum_s (j_s + F_s/2) / sum_s rho_s
(Eq. (4), output command) formed by the library's export kernel.  Here it is
compared node by node with the oracle's Eq. (4) velocity on full-size
1024 x 1024 lattices, one and two components, with and without forces,
into page-locked and into ordinary host buffers.  Tolerance: FP32 storage,
max |u - u_ref| / max |u_ref| and max |rho - rho_ref| / rho_ref over fluid
nodes below 1e-5.
"""
import copy

import numpy as np
import pytest

from oracle.drive import oracle_from_workload
from paper_1202_0442_gb300 import lb2d, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1202_0442_gb300 import build
    build.build()
    yield


def _porous_forced():
    """The benchmark's disc medium, periodic on all edges, driven by a body
    force instead of the density drop."""
    w = copy.deepcopy(synth.porous())
    w.openings = []
    w.rho = [np.where(w.solid != 0, 0.0, 1.0)]
    w.aveforce = ((2e-6, -5e-7),)
    return w


def _two_components_forced():
    """The two-component Shan-Chen recipe at 1024^2: interforce G = 0.9 and
    an adhesive ring (+-0.3) drive the flow."""
    return synth.shan_chen2(1024)


def _two_components_unforced():
    """Two miscible components (0.6 / 0.4 with +-1 % seeded noise) in the
    benchmark's disc medium, periodic, no force of any kind: the flow is the
    decay of the initial density noise."""
    w = copy.deepcopy(synth.porous())
    fl = w.solid == 0
    n1 = synth.noise_field(w.nx, w.ny, 11, -0.01, 0.01)
    n2 = synth.noise_field(w.nx, w.ny, 12, -0.01, 0.01)
    w.openings = []
    w.rho = [np.where(fl, 0.6 * (1 + n1), 0.0), np.where(fl, 0.4 * (1 + n2), 0.0)]
    w.tau = (0.8, 1.1)
    w.alpha = (4 / 9, 4 / 9)
    w.aveforce = ((0.0, 0.0), (0.0, 0.0))
    w.aveacceleration = ((0.0, 0.0), (0.0, 0.0))
    w.adhesive = (None, None)
    w.rho_ref = (0.6, 0.4)
    return w


CASES = {
    "porous_pressure": (synth.porous, 30),
    "porous_force": (_porous_forced, 30),
    "two_components_interforce_adhesion": (_two_components_forced, 10),
    "two_components_no_force": (_two_components_unforced, 10),
}


@pytest.mark.parametrize("case", list(CASES))
def test_velocity_f32_against_oracle(case):
    make, steps = CASES[case]
    w = make()
    lt = lb2d.from_workload(w, "fp32", thermo=0)
    lt.iteration(steps)
    o = oracle_from_workload(w)
    o.step(steps)
    # ordinary host arrays (staging copy) and page-locked ones (written by
    # the export kernel over the host link): the same bits
    plain = lt.velocity_f32()
    pinned = tuple(torch.zeros((w.ny, w.nx), dtype=torch.float32).pin_memory() for _ in range(3))
    lt.velocity_f32(pinned)
    for a, b in zip(plain, pinned):
        assert np.array_equal(a, b.numpy())
    rho_g, ux_g, uy_g = (a.astype(np.float64) for a in plain)
    fl = o.solid() == 0
    assert np.array_equal(fl, w.solid == 0)
    rho_o = sum(o.fields(c)[0] for c in range(w.ncomp))
    ux_o, uy_o = o.velocity()
    assert np.all(rho_g[~fl] == 0) and np.all(ux_g[~fl] == 0) and np.all(uy_g[~fl] == 0)
    e_rho = float(np.max(np.abs(rho_g[fl] - rho_o[fl]) / rho_o[fl]))
    den = max(np.max(np.abs(ux_o[fl])), np.max(np.abs(uy_o[fl])))
    assert den > 0
    e_u = float(max(np.max(np.abs(ux_g[fl] - ux_o[fl])), np.max(np.abs(uy_g[fl] - uy_o[fl]))) / den)
    assert e_rho < TOL32 and e_u < TOL32, (case, e_rho, e_u)
