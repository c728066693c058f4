"""Input-data and restart text files through the library (read_data and
write_restart commands, Sec. Commands), against the oracle's own reader.

- The library reads ``golden/read_data_channel.dat`` (a file laid out as
  the read_data command describes) and runs: its populations right after
  reading and after 40 iterations match the oracle set up by the oracle's
  reader from the same file (FP32 storage: the populations to the FP32
  rounding of their deviations; after the run, rho and u to 1e-5).
- The library writes its state (write_data / write_restart) for one fluid
  with openings, two fluids with interforce and adhesion, two fluids under
  the hybrid boundary style (per-site styles per fluid), a channel under the
  mixed style, and a solute with surface reaction and growth (D2Q9 and
  D2Q4); the oracle's reader takes the
  files and must hold exactly the populations, solute modes, deposits and
  mask the library exports; both then continue and agree to 1e-5 (growth
  decisions equal).
- The library reads its own files back: the populations equal the original
  ones (a deviation below about 1e-9 of its population can move by one last
  bit through the 17-digit text; the binary snapshot is the bitwise
  restart), and the continued runs agree to a few FP32 last bits (such a
  last bit shifts later roundings).
- write_restart writes the step-numbered files every Nf iterations; the
  errors of misplaced sections, late calls and slabs.
"""
import copy
import os

import numpy as np
import pytest

from oracle.restart import oracle_from_data
from paper_1202_0442_gb300 import lb2d, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "read_data_channel.dat")
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1202_0442_gb300 import build
    build.build()
    yield


def _compare_flow(lt, o, ncomp):
    """max relative error of the total density and of the Eq. (4) velocity"""
    fl = o.solid() == 0
    assert np.array_equal(lt.mask() != 0, ~fl)
    rho_o = sum(o.fields(c)[0] for c in range(ncomp))
    ux_o, uy_o = o.velocity()
    rho_g, ux_g, uy_g = (a.astype(np.float64) for a in lt.velocity_f32())
    e_rho = float(np.max(np.abs(rho_g[fl] - rho_o[fl]) / rho_o[fl]))
    den = max(np.max(np.abs(ux_o[fl])), np.max(np.abs(uy_o[fl])))
    e_u = float(max(np.max(np.abs(ux_g[fl] - ux_o[fl])), np.max(np.abs(uy_g[fl] - uy_o[fl]))) / den)
    return e_rho, e_u


def test_library_reads_the_golden_file():
    lt = lb2d.Lattice(0)
    lt.read_data(GOLDEN)
    lt.iteration(0)
    o = oracle_from_data(GOLDEN)
    f_o, f_g = o.f(), lt.populations(1)
    fl = o.solid() == 0
    assert np.array_equal(lt.mask() != 0, ~fl)
    assert np.all(f_g[:, ~fl] == 0)
    # FP32 storage of the deviations from w_i rho_ref
    assert np.max(np.abs(f_g - f_o)) < 1e-8
    lt.iteration(40)
    o.step(40)
    e_rho, e_u = _compare_flow(lt, o, 1)
    assert e_rho < TOL32 and e_u < TOL32, (e_rho, e_u)


def test_library_reads_the_golden_file_at_equilibrium():
    lt = lb2d.Lattice(0)
    lt.read_data(GOLDEN, "equilibrium")
    lt.iteration(0)
    o = oracle_from_data(GOLDEN, "equilibrium")
    assert np.max(np.abs(lt.populations(1) - o.f())) < 1e-8


def test_momentum0_after_read_data_repaints_its_region_only():
    """position0/momentum0 after read_data reinitialise the region they
    mark; every other site keeps the populations read"""
    lt = lb2d.Lattice(0)
    lt.read_data(GOLDEN)
    lt.position0_rect(1, 2, 1, 1)
    for m, v in enumerate([0.4, 0.1, 0.1, 0.1, 0.1, 0.03, 0.03, 0.03, 0.03]):
        lt.momentum0(m, v)
    lt.iteration(0)
    want = oracle_from_data(GOLDEN).f()
    want[:, 1, 1:3] = np.array([0.4, 0.1, 0.1, 0.1, 0.1, 0.03, 0.03, 0.03, 0.03])[:, None]
    assert np.max(np.abs(lt.populations(1) - want)) < 1e-8


def test_obstacle_after_read_data_overrides_the_sites_read():
    """obstacle commands after read_data turn the sites they cover solid
    (their populations read are dropped); the run then matches the oracle
    read from the same file with the same sites made solid"""
    lt = lb2d.Lattice(0)
    lt.read_data(GOLDEN)
    lt.boundary_style("noslip")
    lt.obstacle_rect(2, 2, 1, 1)
    lt.iteration(0)
    o = oracle_from_data(GOLDEN)
    solid = o.solid()
    solid[1, 2] = 1
    o.set_solid(solid)
    f = o.f()
    f[:, 1, 2] = 0.0
    o.set_f(f)
    assert np.array_equal(lt.mask() != 0, solid != 0)
    assert np.max(np.abs(lt.populations(1) - o.f())) < 1e-8
    lt.iteration(30)
    o.step(30)
    e_rho, e_u = _compare_flow(lt, o, 1)
    assert e_rho < TOL32 and e_u < TOL32, (e_rho, e_u)


def _porous_open():
    return synth.porous(128, 96, seed=2, rmin=4, rmax=10)


def _two_fluids():
    return synth.shan_chen2(128)


def _reactive(q):
    return synth.reactive(128, 64, seed=3, ndiscs=4, rmin=4, rmax=8, q=q, kr=0.02, bmax=0.3, growth_seed=7)


def _hybrid_two_fluids():
    """hybrid boundary style: per-site coefficients per fluid (noslip/slip
    for fluid 1, noslip/mixed 0.5 for fluid 2) with interforce"""
    nx, ny = 64, 48
    mask = synth.random_mask(nx, ny, 5, 0.15)
    rng = np.random.default_rng(7)
    R1 = rng.choice([0.0, 1.0], size=(ny, nx))
    R2 = rng.choice([0.0, 0.5], size=(ny, nx))
    r1 = np.where(mask, 0, synth.noise_field(nx, ny, 1, 0.6, 0.8))
    r2 = np.where(mask, 0, synth.noise_field(nx, ny, 2, 0.2, 0.4))
    return synth.Workload(name="hyb2", nx=nx, ny=ny, solid=mask, rho=[r1, r2], tau=(0.9, 1.2),
                          aveforce=((1e-4, 0.0), (0.0, 1e-4)), interforce=(0.5, 0.0, 0.0),
                          slip=[R1, R2], rho_ref=(0.7, 0.3))


def _mixed_channel():
    """mixed boundary style (R = 0.7) in a channel with dirichlet openings"""
    nx, ny = 96, 26
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = solid[-1, :] = 1
    solid[10:16, 40:46] = 1
    return synth.Workload(name="mixch", nx=nx, ny=ny, solid=solid, rho=[np.where(solid, 0, 1.0)], tau=(0.7,),
                          openings=[synth.Opening("xlo", 1, ny - 2, "inlet", [("dirichlet", 0.0, 1.002)]),
                                    synth.Opening("xhi", 1, ny - 2, "outlet", [("dirichlet", 0.0, 1.0)])],
                          slip=[0.7])


def _args(w):
    a = []
    if w.ncomp == 2:
        a.append("fluids")
    if w.solute_q:
        a.append("solute")
    return a


CASES = {"porous_openings": (_porous_open, 40, 30),
         "two_fluids_interforce_adhesion": (_two_fluids, 40, 20),
         "hybrid_two_fluids": (_hybrid_two_fluids, 40, 30),
         "mixed_channel_openings": (_mixed_channel, 60, 30),
         "reactive_q9": (lambda: _reactive(9), 120, 20),
         "reactive_q4": (lambda: _reactive(4), 120, 20)}


@pytest.mark.parametrize("case", list(CASES))
def test_oracle_reads_what_the_library_writes(case, tmp_path):
    make, n0, n1 = CASES[case]
    w = make()
    lt = lb2d.from_workload(w, "fp32")
    lt.iteration(n0)
    base = str(tmp_path / "state")
    lt.write_data(base)
    o = oracle_from_data(base, *_args(w))
    o.set_t(n0)
    assert np.array_equal(o.solid(), (lt.mask() != 0).astype(np.uint8))
    for c in range(w.ncomp):
        assert np.array_equal(o.f(c), lt.populations(c + 1)), c
    if w.solute_q:
        g, _, b = lt.solute_state()
        assert np.array_equal(o.g(), g)
        assert np.array_equal(o.b(), b)
    for _ in range(n1):
        lt.iteration(1)
        o.step(1)
        if w.solute_q:
            assert np.array_equal(np.sort(lt.flips()), np.sort(o.flips()))
    e_rho, e_u = _compare_flow(lt, o, w.ncomp)
    assert e_rho < TOL32 and e_u < TOL32, (case, e_rho, e_u)


@pytest.mark.parametrize("case,storage", [("porous_openings", "fp32"), ("two_fluids_interforce_adhesion", "fp32"),
                                          ("reactive_q9", "fp32"), ("porous_openings", "fp16")])
def test_library_reads_its_own_files(case, storage, tmp_path):
    make, n0, n1 = CASES[case]
    w = make()
    kw = {"h_max": 2e-3, "rounding": "stochastic"} if storage == "fp16" else {}
    a = lb2d.from_workload(w, storage, **kw)
    a.iteration(n0)
    base = str(tmp_path / "state")
    a.write_data(base)
    # the storage format is the caller's choice, not part of the file: set
    # it up as for the lattice that wrote the file, then read
    b = lb2d.Lattice(0)
    b.lattice(w.nx, w.ny, w.tau[0])
    if w.ncomp == 2:
        b.fluids(w.tau[0], w.tau[1])
    if w.solute_q:
        b.solute(w.taus, w.solute_q)
    b.set_storage(storage, list(w.rho_ref), kw.get("h_max", 0.0), kw.get("rounding", "nearest"))
    b.read_data(base, *_args(w))
    b.set_step(n0)
    b.iteration(0)
    assert np.array_equal(a.mask(), b.mask())
    for c in range(1, w.ncomp + 1):
        fa, fb = a.populations(c), b.populations(c)
        same = fa == fb
        assert same.mean() > 0.999, (c, same.mean())
        assert np.max(np.abs(fa - fb)) < 1e-15
    a.iteration(n1)
    b.iteration(n1)
    # a last-bit difference moves later FP32 roundings by a few last bits:
    # of the stored deviations f - w rho_ref (fluid), of the stored values
    # themselves (solute, kept unshifted)
    for c in range(1, w.ncomp + 1):
        fa, fb = a.populations(c), b.populations(c)
        assert np.max(np.abs(fa - fb)) <= 1e-9 * np.max(np.abs(fa))
    if w.solute_q:
        for x, y in zip(a.solute_state(), b.solute_state()):
            assert np.max(np.abs(x - y)) <= 8 * 2.0 ** -23 * max(np.max(np.abs(x)), 1e-30)


def test_write_restart_every_nf(tmp_path):
    w = _porous_open()
    a = lb2d.from_workload(w, "fp32")
    a.write_restart(str(tmp_path / "r"), 10)
    a.iteration(25)
    assert sorted(os.listdir(tmp_path)) == ["r.10", "r.20"]
    b = lb2d.from_workload(w, "fp32")
    b.iteration(20)
    b.write_data(str(tmp_path / "direct"))
    assert open(tmp_path / "r.20").read() == open(tmp_path / "direct").read()
    a.write_restart("", 0)
    a.iteration(10)
    assert sorted(os.listdir(tmp_path)) == ["direct", "r.10", "r.20"]
    # the command precedes the iteration command (write_data writes now)
    with pytest.raises(lb2d.LBError) as e:
        a.write_restart(str(tmp_path / "late"), 10)
    assert e.value.code == lb2d.LB_E_ORDER


def _bad(tmp_path, edit):
    lines = open(GOLDEN).read().split("\n")
    p = tmp_path / "bad.dat"
    p.write_text("\n".join(edit(lines)) + "\n")
    return str(p)


def test_read_data_errors(tmp_path):
    lt = lb2d.Lattice(0)
    with pytest.raises(lb2d.LBError) as e:
        lt.read_data(str(tmp_path / "missing"))
    assert e.value.code == lb2d.LB_E_ARG
    # boundary after density
    def swap(L):
        i, j = L.index("boundary"), L.index("density")
        blk = L[i:i + 3]
        rest = L[:i] + L[i + 3:]
        k = rest.index("momentum")
        return rest[:k] + blk + rest[k:]
    with pytest.raises(lb2d.LBError) as e:
        lt.read_data(_bad(tmp_path, swap))
    assert e.value.code == lb2d.LB_E_ARG
    # a site missing from momentum
    with pytest.raises(lb2d.LBError) as e:
        lt.read_data(_bad(tmp_path, lambda L: [x for x in L if not x.startswith("3 2 0.4465")]))
    assert e.value.code == lb2d.LB_E_ARG
    with pytest.raises(lb2d.LBError) as e:
        lt.read_data(GOLDEN, "fluid")
    assert e.value.code == lb2d.LB_E_ARG
    # after the first iteration
    ok = lb2d.Lattice(0)
    ok.read_data(GOLDEN)
    ok.iteration(1)
    with pytest.raises(lb2d.LBError) as e:
        ok.read_data(GOLDEN)
    assert e.value.code == lb2d.LB_E_ORDER
    # a slab
    s = lb2d.from_workload(_porous_open(), slab=(2, 0))
    with pytest.raises(lb2d.LBError) as e:
        s.write_data(str(tmp_path / "slab"))
    assert e.value.code == lb2d.LB_E_UNSUPPORTED
