"""A lattice split into y slabs (processors command, Sec. Parallelization)
runs bit for bit like the whole lattice, on one GPU.

Each slab is a context that holds its rows and ghost rows
(lb_processor_rank); after every iteration the slabs' halo rows are
exchanged device to device (lb_exchange), or through packed device buffers
(lb_halo_pack / lb_halo_unpack, the messages a multi-GPU run sends over
NCCL).  After every step the slabs' own rows must equal the whole lattice's
rows exactly: populations, node fields, the Eq. (4) velocity and the mask;
the slabs' thermo sums add up to the lattice's to rounding (FP64 sums in
another order).  Cases: the benchmark's porous 1024^2 lattice (x-wall
openings) in 2 and 4 slabs, FP16 storage with stochastic rounding in 3
uneven slabs, two components with interforce and adhesion (two ghost
rows), a partial-slip wall (two ghost rows), y-wall openings (velocity,
pressure and gradient outlets on the first and last slab), a solute
carried by the flow (fused fluid-solute kernel), solute with surface
reaction and growth, a single slab that is its own neighbour."""
import copy

import numpy as np
import pytest

from paper_1202_0442_gb300 import halo, lb2d, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

THERMO_KEYS = ("mass1", "mass2", "momx", "momy", "mass_eq1", "solute", "bsum", "removed1", "removed_solute",
               "nsolid", "nfluid")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1202_0442_gb300 import build
    build.build()
    yield


def _kw(storage, w=None):
    if storage == "fp32":
        return {}
    # deviations of two phase-separated components reach about 1/2
    return {"h_max": 1.2 if (w is not None and w.ncomp == 2) else 4e-3, "rounding": "stochastic"}


def _run(w, py, steps, storage="fp32", via_buffers=False, check_every=None):
    """The whole lattice and its py slabs side by side; compares them after
    the last step (and every check_every steps)."""
    whole = lb2d.from_workload(w, storage, **_kw(storage, w))
    slabs = [lb2d.from_workload(w, storage, slab=(py, r), **_kw(storage, w)) for r in range(py)]
    bufs = None
    if via_buffers:
        n = slabs[0].halo_size()
        bufs = [[torch.empty(n, dtype=torch.uint8, device="cuda") for _ in range(2)] for _ in slabs]
    done = 0
    while done < steps:
        k = min(check_every or steps, steps - done)
        whole.iteration(k)
        for _ in range(k):
            for s in slabs:
                s.iteration(1)
            if via_buffers:
                for s, b in zip(slabs, bufs):
                    s.halo_pack(0, b[0])
                    s.halo_pack(1, b[1])
                for r, s in enumerate(slabs):
                    s.halo_unpack(0, bufs[(r - 1) % py][1])
                    s.halo_unpack(1, bufs[(r + 1) % py][0])
            else:
                lb2d.exchange(slabs)
        done += k
        _compare(w, whole, slabs)
    return whole, slabs


def _compare(w, whole, slabs):
    cat = lambda arrs: np.concatenate(arrs, axis=-2)
    assert [s.rows for s in slabs] == sorted(s.rows for s in slabs)
    assert sum(s.rows[1] for s in slabs) == w.ny
    assert np.array_equal(cat([s.mask() for s in slabs]), whole.mask())
    for c in range(1, w.ncomp + 1):
        assert np.array_equal(cat([s.populations(c) for s in slabs]), whole.populations(c)), c
        for a, b in zip(zip(*[s.fields(c) for s in slabs]), whole.fields(c)):
            assert np.array_equal(cat(list(a)), b)
    for a, b in zip(zip(*[s.velocity_f32() for s in slabs]), whole.velocity_f32()):
        assert np.array_equal(cat(list(a)), b)
    if w.solute_q:
        for a, b in zip(zip(*[s.solute_state() for s in slabs]), whole.solute_state()):
            assert np.array_equal(cat(list(a)), b)
    tw = whole.get_thermo()
    ts = [s.get_thermo() for s in slabs]
    assert all(t["step"] == tw["step"] for t in ts)
    for k in THERMO_KEYS:
        tot = sum(t[k] for t in ts)
        assert abs(tot - tw[k]) <= 1e-12 * max(abs(tw[k]), 1.0), (k, tot, tw[k])


@pytest.mark.parametrize("py", [2, 4])
def test_porous_1024_slabs(py):
    """The benchmark lattice (Zou-He dirichlet openings on the full x walls,
    periodic in y) in py slabs."""
    _run(synth.porous(), py, 12, check_every=6)


def test_porous_fp16_three_uneven_slabs():
    """FP16 storage, stochastic rounding: the dither of a node is drawn from
    its place in the whole lattice, so the slabs round like it; 200 rows in
    3 slabs of 66, 67, 67."""
    _run(synth.porous(256, 200, seed=3, rmin=4, rmax=12), 3, 20, storage="fp16", check_every=10)


@pytest.mark.parametrize("py,storage", [(2, "fp32"), (4, "fp32"), (3, "fp16"), (2, "bf16")])
def test_two_components_interforce_slabs(py, storage):
    """Interforce needs the neighbours' densities after streaming: two
    ghost rows; mass-exact collision (its random last bit per node), and
    with 16-bit storage a random dither per store, both drawn from the
    node's place in the whole lattice."""
    _run(synth.shan_chen2(256), py, 16, storage=storage, check_every=8)


def test_slip_wall_slabs():
    """A partial-slip obstacle (mirror sources two rows away): two ghost rows."""
    w = copy.deepcopy(synth.porous(160, 96, seed=4, rmin=4, rmax=8))
    w.slip = (0.5,)
    _run(w, 2, 20, check_every=10)


@pytest.mark.parametrize("out_style", [("dirichlet", 0.0, 1.0), ("gradient", 0.0, 1.0)])
def test_y_wall_openings_slabs(out_style):
    """Inlet on the low y wall (slab 0), outlet on the high y wall (the last
    slab), the flow crossing every slab boundary."""
    ny, nx = 48, 14
    solid = np.zeros((ny, nx), np.uint8)
    solid[:, 0] = solid[:, -1] = 1
    ops = [synth.Opening("ylo", 1, nx - 2, "inlet", [("poiseuille", 0.04, 1.0)]),
           synth.Opening("yhi", 1, nx - 2, "outlet", [out_style])]
    w = synth.Workload(name="ychan", nx=nx, ny=ny, solid=solid, rho=[np.where(solid, 0, 1.0)], tau=(0.8,),
                       openings=ops)
    _run(w, 3, 60, check_every=20)


@pytest.mark.parametrize("q", [4, 9])
def test_solute_slabs(q):
    """A solute carried by the flow, dirichlet inlet and adiabatic outlet
    (the fused fluid-solute kernel), no surface reaction."""
    w = copy.deepcopy(synth.reactive(128, 64, seed=3, ndiscs=4, rmin=4, rmax=8, q=q))
    w.reaction = None
    _run(w, 4, 30, check_every=15)


@pytest.mark.parametrize("q,py,storage", [(9, 2, "fp32"), (9, 4, "fp32"), (4, 3, "fp32"), (9, 2, "fp16")])
def test_reactive_growth_slabs(q, py, storage):
    """Solute, surface reaction, precipitation and growth (App. C) in slabs:
    each slab also updates the two ghost rows next to its own rows, so the
    deposits its boundary solids gather and the growth decisions one row
    out are its own; the mask and deposit rows travel with the halo.  The
    slabs' populations, solute, deposits, masks and every step's grown
    nodes equal the whole lattice's bit for bit."""
    # pressure-driven (with the velocity inlet, growth closing the channel
    # makes the run diverge beyond any 16-bit range)
    w = synth.reactive(128, 64, seed=3, ndiscs=4, rmin=4, rmax=8, q=q, kr=0.02, bmax=0.3, growth_seed=7,
                       inlet="pressure")
    whole, slabs = _run(w, py, 120, storage=storage, check_every=40)
    for _ in range(20):
        whole.iteration(1)
        for s in slabs:
            s.iteration(1)
        lb2d.exchange(slabs)
        fw = whole.flips()
        fs = np.sort(np.concatenate([s.flips() + s.rows[0] * w.nx for s in slabs]))
        assert np.array_equal(fw, fs)
    _compare(w, whole, slabs)
    tw = whole.get_thermo()
    assert tw["flips"] > 0 and tw["flips"] == sum(s.get_thermo()["flips"] for s in slabs)


def test_growth_surface_list_equals_row_scan_full_size():
    """The growth step over the surface list (a whole lattice: gather,
    decisions and flips in one launch) against the scan of every row with
    the separate flip kernel (the same lattice held as one slab, processors
    1 x 1), on the full 1024 x 512 reactive channel: every step's grown
    nodes, then populations, solute state, deposits, mask and thermo bit
    for bit after 300 iterations with growth events."""
    w = synth.reactive(seed=1, kr=0.02, bmax=0.3, growth_seed=7, inlet="pressure")
    whole = lb2d.from_workload(w, thermo=50)
    one = lb2d.from_workload(w, thermo=50, slab=(1, 0))
    grown = 0
    for _ in range(300):
        whole.iteration(1)
        one.iteration(1)
        fw = whole.flips()
        assert np.array_equal(fw, np.sort(one.flips()))
        grown += len(fw)
    assert grown > 0
    assert np.array_equal(whole.mask(), one.mask())
    assert np.array_equal(whole.populations(1), one.populations(1))
    for a, b in zip(whole.solute_state(), one.solute_state()):
        assert np.array_equal(a, b)
    assert whole.get_thermo() == one.get_thermo()
    assert whole.get_thermo()["flips"] == grown


def test_halo_messages_through_buffers():
    """The exchange through packed device buffers (the messages a
    multi-GPU run sends over NCCL) gives the same bits."""
    _run(synth.shan_chen2(128), 2, 10, via_buffers=True, check_every=5)


def test_single_slab_is_its_own_neighbour():
    w = synth.porous(96, 64, seed=2, rmin=3, rmax=6)
    whole = lb2d.from_workload(w, thermo=7)
    one = lb2d.from_workload(w, thermo=7, slab=(1, 0))
    whole.iteration(23)
    one.iteration(23)
    assert np.array_equal(one.populations(1), whole.populations(1))
    assert one.get_thermo() == whole.get_thermo()


def test_slab_exchange_object_single_rank():
    """halo.SlabExchange with one rank (its own neighbour), as bench.py's
    split mode runs it at N = 1."""
    w = synth.porous(96, 64, seed=2, rmin=3, rmax=6)
    whole = lb2d.from_workload(w)
    one = lb2d.from_workload(w, slab=(1, 0))
    ex = halo.SlabExchange(one, None, 0, 1, "cuda")
    whole.iteration(9)
    for _ in range(9):
        one.iteration(1)
        ex()
    assert np.array_equal(one.populations(1), whole.populations(1))


def test_slab_errors():
    w = synth.porous(64, 48, seed=2, rmin=3, rmax=6)
    lt = lb2d.Lattice(0)
    lt.lattice(64, 48, 0.8)
    with pytest.raises(lb2d.LBError):
        lt.processor_rank(1)                 # the grid is 1 x 1 until processors says otherwise
    lt.processors(2, 2)                      # slabs split y only
    with pytest.raises(lb2d.LBError) as e:
        lt.processor_rank(1)
    assert e.value.code == lb2d.LB_E_UNSUPPORTED
    lt.processors(1, 2)
    with pytest.raises(lb2d.LBError):
        lt.processor_rank(2)
    # more than one iteration per call on a slab of several
    s = lb2d.from_workload(w, slab=(2, 1))
    with pytest.raises(lb2d.LBError) as e:
        s.iteration(2)
    assert e.value.code == lb2d.LB_E_ORDER
    s.iteration(1)
    # too few rows for the ghost rows
    with pytest.raises(lb2d.LBError) as e:
        lb2d.from_workload(w, slab=(24, 3))
    assert e.value.code == lb2d.LB_E_ARG
    # intersolute is not built for slabs
    r = copy.deepcopy(synth.reactive(128, 64, seed=3, ndiscs=4, rmin=4, rmax=8))
    r.reaction = None
    r.intersolute = (-0.5, 1.0, 1.0)
    with pytest.raises(lb2d.LBError) as e:
        lb2d.from_workload(r, slab=(2, 0))
    assert e.value.code == lb2d.LB_E_UNSUPPORTED
    # slabs of different lattices
    a = lb2d.from_workload(w, slab=(2, 0))
    b = lb2d.from_workload(synth.porous(64, 48, seed=3, rmin=3, rmax=6), slab=(2, 1))
    a.iteration(1)
    b.iteration(1)
    lb2d.exchange([a, b])                    # same sizes: accepted (the caller's lattice)
    c = lb2d.from_workload(w, slab=(2, 1))
    with pytest.raises(lb2d.LBError):
        lb2d.exchange([a, c])                # c is one step behind
