"""Reads of unwritten memory, checked with poisoned buffers (the checking
aid that stands in for a memory sanitizer).

With LB_DEBUG_POISON the library fills, before every iteration, every
buffer that iteration writes with NaN bit patterns: the next state's
populations (solid slots and row padding included, which the kernels leave
unwritten where a whole 32-byte sector holds no fluid node), the solute
populations, deposit shares, solvent-velocity and concentration planes and,
on thermo or output steps, the node-field planes.  A kernel that read a
slot no kernel of the iteration wrote would carry NaN into the fluid state,
the exports or the thermo sums.  Each workload below runs with and without
the flag; populations, solute state, deposits, mask, Eq. (4) velocity and
thermo records must be equal bit for bit and finite.  The poisoned runs
also allocate every library buffer between zones of NaN patterns
(LB_DEBUG_GUARDS): a read past a buffer's end would carry NaN in, and the
zones must be intact at the end (no write out of bounds).  Every fluid kernel
variant is reached: the streaming kernel (FP32, FP16, BF16; noslip, slip
map, mixed; openings of every style incl. gradient), two components
(mass-exact), Shan-Chen with one and two components (and with openings), the fused fluid-solute
kernel with reaction and growth (D2Q9, D2Q4), the separate solute kernel
under a two-component fluid, intersolute, the TMA kernel, slabs with
their halo exchange and the batched launch."""
import copy

import numpy as np
import pytest

from paper_1202_0442_gb300 import lb2d, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1202_0442_gb300 import build
    build.build()
    yield


def _channel(out_style):
    nx, ny = 40, 14
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = solid[-1, :] = 1
    ops = [synth.Opening("xlo", 1, ny - 2, "inlet", [("poiseuille", 0.04, 1.0)]),
           synth.Opening("xhi", 1, ny - 2, "outlet", [out_style])]
    return synth.Workload(name="ch", nx=nx, ny=ny, solid=solid, rho=[np.where(solid, 0, 1.0)], tau=(0.8,),
                          openings=ops)


def _slip_map():
    nx, ny = 72, 40
    mask = synth.random_mask(nx, ny, 3, 0.25)
    R = np.random.default_rng(2).choice([0.0, 0.3, 1.0], size=(ny, nx))
    return synth.Workload(name="slip", nx=nx, ny=ny, solid=mask, rho=[np.where(mask, 0, 1.0)], tau=(0.8,),
                          aveforce=((1e-4, -5e-5),), slip=[R])


def _mixed():
    w = copy.deepcopy(synth.porous(100, 60, seed=4, rmin=4, rmax=8))
    w.slip = (0.4,)
    return w


def _sc_one():
    nx, ny = 64, 48
    rho = 200.0 + synth.noise_field(nx, ny, 2, 0.0, 1.0)
    return synth.Workload(name="sc1", nx=nx, ny=ny, solid=np.zeros((ny, nx), np.uint8), rho=[rho], tau=(1.0,),
                          interforce=(-120.0, 4.0, 200.0), rho_ref=(200.0,))


def _two_no_sc():
    w = copy.deepcopy(synth.shan_chen2(128))
    w.interforce = None
    return w


def _two_with_solute():
    nx, ny = 48, 32
    mask = synth.random_mask(nx, ny, 4, 0.1)
    y, x = np.mgrid[0:ny, 0:nx]
    blob = (x - 20) ** 2 + (y - 14) ** 2 < 64
    return synth.Workload(name="2cs", nx=nx, ny=ny, solid=mask,
                          rho=[np.where(mask, 0, np.where(blob, 1.0, 0.05)),
                               np.where(mask, 0, np.where(blob, 0.05, 1.0))],
                          tau=(0.8, 1.1), alpha=(4 / 9, 4 / 9), aveforce=((2e-5, 0.0), (2e-5, 0.0)),
                          interforce=(0.9, 0.0, 0.0), rho_ref=(0.5, 0.5), solute_q=9, taus=0.7,
                          C=np.where(mask, 0, synth.noise_field(nx, ny, 6, 0.5, 1.5)))


def _intersolute():
    nx, ny = 64, 40
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = solid[-1, :] = 1
    solid[15:22, 20:27] = 1
    C = np.where(solid, 0.0, synth.noise_field(nx, ny, 4, 0.2, 1.0))
    return synth.Workload(name="is", nx=nx, ny=ny, solid=solid, rho=[np.where(solid, 0.0, 1.0)], tau=(0.9,),
                          aveforce=((1e-5, 0.0),), solute_q=4, taus=0.8, C=C, intersolute=(-0.05, 1.0, 0.3))


def _sc_openings():
    nx, ny = 48, 30
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = solid[-1, :] = 1
    ops = [synth.Opening("xlo", 1, ny - 2, "inlet", [("uniform", 0.02, 0.7), ("dirichlet", 0.0, 0.41)]),
           synth.Opening("xhi", 1, ny - 2, "outlet", [("dirichlet", 0.0, 0.7), ("uniform", 0.01, 0.4)])]
    return synth.Workload(name="sco", nx=nx, ny=ny, solid=solid,
                          rho=[np.where(solid, 0, 0.7), np.where(solid, 0, 0.4)], tau=(0.8, 1.1),
                          alpha=(4 / 9, 4 / 9), rho_ref=(0.7, 0.4), openings=ops, interforce=(0.3, 0.0, 0.0))


def _reactive(q):
    return synth.reactive(128, 64, seed=3, ndiscs=4, rmin=4, rmax=8, q=q, kr=0.02, bmax=0.3, growth_seed=7)


FP16 = {"h_max": 2e-3, "rounding": "stochastic"}
CASES = {
    "porous_fp32": (lambda: synth.porous(130, 96, seed=2, rmin=4, rmax=10), "fp32", {}, None, 40),
    "porous_fp16": (lambda: synth.porous(130, 96, seed=2, rmin=4, rmax=10), "fp16", FP16, None, 40),
    "porous_bf16": (lambda: synth.porous(130, 96, seed=2, rmin=4, rmax=10), "bf16", FP16, None, 40),
    "channel_gradient_outlet": (lambda: _channel(("gradient", 0.0, 1.0)), "fp32", {}, None, 60),
    "channel_uniform_outlet": (lambda: _channel(("uniform", 0.01, 1.0)), "fp32", {}, None, 60),
    "slip_map_hybrid": (_slip_map, "fp32", {}, None, 40),
    "mixed": (_mixed, "fp32", {}, None, 40),
    "two_components": (_two_no_sc, "fp32", {}, None, 30),
    "shan_chen_one": (_sc_one, "fp32", {}, None, 30),
    "shan_chen_two_fp32": (lambda: synth.shan_chen2(128), "fp32", {}, None, 30),
    "shan_chen_two_fp16": (lambda: synth.shan_chen2(128), "fp16", {"h_max": 1.2, "rounding": "stochastic"}, None, 30),
    "shan_chen_two_openings": (_sc_openings, "fp32", {}, None, 30),
    "reactive_q9_fused": (lambda: _reactive(9), "fp32", {}, None, 150),
    "reactive_q4_fused": (lambda: _reactive(4), "fp32", {}, None, 150),
    "reactive_q9_separate": (lambda: _reactive(9), "fp32", {}, "streaming", 150),
    "two_components_solute": (_two_with_solute, "fp32", {}, None, 60),
    "intersolute": (_intersolute, "fp32", {}, None, 60),
    "tma": (lambda: synth.porous(128, 96, seed=2, rmin=4, rmax=10), "fp32", {}, "tma", 40),
}


def _state(lt, w):
    out = [lt.mask()]
    for c in range(1, w.ncomp + 1):
        out.append(lt.populations(c))
    out.extend(lt.velocity_f32())
    if w.solute_q:
        out.extend(lt.solute_state())
    return out


@pytest.mark.parametrize("case", list(CASES))
def test_poisoned_buffers_change_nothing(case):
    make, storage, kw, kernel, steps = CASES[case]
    w = make()
    runs = []
    for poison in (False, True):
        dbg = (lb2d.LB_DEBUG_POISON | lb2d.LB_DEBUG_GUARDS) if poison else 0
        lt = lb2d.from_workload(w, storage, thermo=7, kernel=kernel or "auto", debug=dbg, **kw)
        recs = []
        for k in range(steps // 10):
            lt.iteration(10)
            recs.append(lt.get_thermo())
        runs.append((_state(lt, w), recs))
        if poison:
            assert lt.debug_check() == 0
    (a, ra), (b, rb) = runs
    assert ra == rb
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
        assert np.all(np.isfinite(x))


def test_poisoned_slabs():
    """Slabs with surface reaction (three ghost rows, two computed
    redundantly) and their halo exchange, poisoned, against the unpoisoned
    whole lattice: bit for bit."""
    w = _reactive(9)
    whole = lb2d.from_workload(w, thermo=9)
    slabs = [lb2d.from_workload(w, thermo=9, slab=(3, r), debug=lb2d.LB_DEBUG_POISON | lb2d.LB_DEBUG_GUARDS)
             for r in range(3)]
    for _ in range(90):
        whole.iteration(1)
        for s in slabs:
            s.iteration(1)
        lb2d.exchange(slabs)
    cat = lambda arrs: np.concatenate(arrs, axis=-2)
    assert np.array_equal(cat([s.populations(1) for s in slabs]), whole.populations(1))
    for a, b in zip(zip(*[s.solute_state() for s in slabs]), whole.solute_state()):
        assert np.array_equal(cat(list(a)), b)
    assert np.array_equal(cat([s.mask() for s in slabs]), whole.mask())
    assert all(s.debug_check() == 0 for s in slabs)


def test_debug_flag_errors():
    lt = lb2d.Lattice(0)
    with pytest.raises(lb2d.LBError) as e:
        lt.set_debug(0x10)
    assert e.value.code == lb2d.LB_E_ARG
    lt.set_debug(0)


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_poisoned_batch(storage):
    """The batched launch over lattices of uneven sizes, poisoned (direct
    launches) against unpoisoned (graph replays): bit for bit."""
    ws = [synth.porous(nx, ny, seed=s, rmin=3, rmax=7) for s, (nx, ny) in enumerate([(64, 96), (96, 64), (160, 128)])]
    for w in ws:
        w.openings = []
        w.aveforce = ((1e-5, 0.0),)
    kw = {"h_max": 5e-3, "rounding": "stochastic"} if storage == "fp16" else {}
    out = []
    for poison in (False, True):
        dbg = (lb2d.LB_DEBUG_POISON | lb2d.LB_DEBUG_GUARDS) if poison else 0
        lats = [lb2d.from_workload(w, storage, debug=dbg, **kw) for w in ws]
        for lt in lats:
            lt.thermo(1 << 30)
        b = lb2d.Batch(lats)
        b.iteration(45, use_graph=True)
        torch.cuda.synchronize()
        out.append([lt.populations(1) for lt in lats])
        if poison:
            assert all(lt.debug_check() == 0 for lt in lats)
        del b
    for x, y in zip(*out):
        assert np.array_equal(x, y)
        assert np.all(np.isfinite(x))
