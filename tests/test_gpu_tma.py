"""The persistent TMA-pipelined fluid kernel: same per-node arithmetic as
the streaming kernel, so the two agree bit for bit; and both match the
FP64 oracle.  Sizes cover one tile column, several with a partial last
one, periodic wrap in x and y, and every wall opening."""
import numpy as np
import pytest

from oracle.drive import oracle_from_workload
from paper_1202_0442_gb300 import lb2d, synth
from pairing import W9, pop_err, rel_rho, rel_u

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1202_0442_gb300 import build
    build.build()
    yield


def _both(w, steps, storage="fp32", **kw):
    out = []
    for k in ("streaming", "tma"):
        lt = lb2d.from_workload(w, storage, kernel=k, **kw)
        lt.iteration(steps)
        out.append(lt)
    return out


@pytest.mark.parametrize("nx,ny", [(64, 32), (96, 40), (264, 100), (1024, 48)])
def test_tma_equals_streaming_and_oracle(nx, ny):
    mask = synth.random_mask(nx, ny, nx + ny, 0.15)
    f = synth.random_populations(9, nx, ny, 7, W9, 0.2, mask)
    w = synth.Workload(name="t", nx=nx, ny=ny, solid=mask, rho=[np.where(mask, 0, 1.0)], tau=(0.85,),
                       aveforce=((1e-4, -2e-4),), aveacceleration=((3e-5, 1e-5),))
    a = lb2d.from_workload(w, kernel="streaming")
    b = lb2d.from_workload(w, kernel="tma")
    a.set_populations(f)
    b.set_populations(f)
    a.iteration(40)
    b.iteration(40)
    assert np.array_equal(a.populations(), b.populations())
    assert a.get_thermo() == b.get_thermo()
    o = oracle_from_workload(w)
    o.set_f(f)
    o.step(40)
    e, _ = pop_err(b, o)
    assert e < 1e-5


@pytest.mark.parametrize("axis", ["x", "y"])
def test_tma_openings(axis):
    import test_gpu_parity as T
    for pair in T.STYLE_PAIRS:
        w = T._opening_channel(axis, *pair, n_along=136, n_across=24)
        a, b = _both(w, 150)
        assert np.array_equal(a.populations(), b.populations())
        o = oracle_from_workload(w)
        o.step(150)
        tol = T.GRADIENT_TOL if pair[1][0] == "gradient" else 1e-5
        assert rel_u(b, o) < tol and rel_rho(b, o, w) < tol


def test_tma_porous_and_adhesion():
    w = synth.porous(256, 128, seed=4, rmin=4, rmax=10)
    a, b = _both(w, 200)
    assert np.array_equal(a.populations(), b.populations())
    o = oracle_from_workload(w)
    o.step(200)
    assert rel_u(b, o) < 1e-5
    nx, ny = 128, 48
    mask = np.zeros((ny, nx), np.uint8)
    mask[0, :] = mask[-1, :] = 1
    mask[10:20, 30:60] = 1
    rho = np.where(mask, 0, 200.0 + synth.noise_field(nx, ny, 2, 0.0, 1.0))
    w2 = synth.Workload(name="ads", nx=nx, ny=ny, solid=mask, rho=[rho], tau=(1.0,),
                        adhesive=((-250.0, 4.0, 200.0),), rho_ref=(200.0,))
    a, b = _both(w2, 60)
    assert np.array_equal(a.populations(), b.populations())


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_tma_16bit(storage):
    w = synth.channel(128, 32, 1.0, 1e-6)
    a, b = _both(w, 500, storage, h_max=2e-3, rounding="stochastic")
    assert np.array_equal(a.populations(), b.populations())


def test_tma_with_solute_coupling():
    """The fluid of a reactive run (one component + solute) goes through
    the TMA kernel and hands its velocity to the solute kernel."""
    w = synth.reactive(256, 64, seed=3, ndiscs=5, rmin=4, rmax=8, q=4, kr=0.02, bmax=0.3)
    a, b = _both(w, 300)
    assert np.array_equal(a.mask(), b.mask())
    assert np.array_equal(a.solute_state(Cf=False, b=False)[0], b.solute_state(Cf=False, b=False)[0])
    o = oracle_from_workload(w)
    o.step(300)
    assert np.array_equal(b.mask(), o.solid())


def test_tma_rejects_unsupported_width():
    w = synth.channel(66, 16, 1.0, 1e-6)
    lt = lb2d.from_workload(w, kernel="tma")
    with pytest.raises(lb2d.LBError) as ei:
        lt.iteration(1)
    assert ei.value.code == lb2d.LB_E_UNSUPPORTED


def test_bounded_wait_runs_out_and_recovers():
    """Failure detection without a GPU fault: with the wait limit at 0 every
    CTA of the TMA kernel gives up at its first wait; it records that, lets
    its issued copies land and returns, and the
    next thermo evaluation reports LB_E_TIMEOUT.  With the default limit
    restored and the state restored from a snapshot the lattice runs on
    normally, bit for bit like an undisturbed run."""
    w = synth.porous(256, 96, seed=4, rmin=4, rmax=10)
    lt = lb2d.from_workload(w, kernel="tma")
    ref = lb2d.from_workload(w, kernel="tma")
    snap = np.zeros(lt.state_size(), np.uint8)
    lt.save_state(snap)
    lt.set_wait_limit(0)
    with pytest.raises(lb2d.LBError) as e:
        lt.iteration(3)
    assert e.value.code == lb2d.LB_E_TIMEOUT
    lt.set_wait_limit(-1)
    lt.load_state(snap)
    lt.iteration(7)
    ref.iteration(7)
    assert np.array_equal(lt.populations(), ref.populations())
    assert lt.get_thermo() == ref.get_thermo()
