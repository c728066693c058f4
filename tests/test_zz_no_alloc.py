"""lb_thermo_static, the entry point that allocates nothing.

It exists for callers that cannot let the library allocate device memory
(a framework's caching allocator owns the free memory, a loop cannot pay for
an allocation or the synchronisation a free may imply, or the program
forbids allocation after start-up).  It recomputes the thermo record from a
context's fields using a fixed device array of the library for its partial
sums; the record must equal the one lb_get_thermo returns after the same
iteration, call after call.  This file is collected last so that a run that
stops at its first failure has run every other test before it.
"""
import numpy as np
import pytest

from paper_1202_0442_gb300 import lb2d, synth

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


def _same(a: dict, b: dict):
    assert a.keys() == b.keys()
    for k in a:
        assert a[k] == b[k] or (np.isnan(a[k]) and np.isnan(b[k])), (k, a[k], b[k])


@pytest.mark.parametrize("case", ["porous", "two_components", "reactive"])
def test_static_thermo_equals_allocating_thermo(case):
    if case == "porous":
        w = synth.porous(160, 96, seed=2, rmin=3, rmax=8)
    elif case == "two_components":
        w = synth.shan_chen2(128)
    else:
        w = synth.reactive(128, 64, seed=3, ndiscs=4, rmin=4, rmax=8, q=9, kr=0.02, bmax=0.3)
    lt = lb2d.from_workload(w)
    for steps in (30, 17):
        lt.iteration(steps)
        ref = lt.get_thermo()
        first = lt.thermo_static()
        second = lt.thermo_static()
        _same(first, ref)
        _same(second, ref)
        assert first["nfluid"] + first["nsolid"] == w.nodes


def test_static_thermo_refuses_fields_of_another_state():
    """With thermo every 7 iterations, a run that stops between thermo steps
    leaves field planes of an earlier step while the mask and deposits move
    on: the call must refuse rather than mix the two.  So must it after a
    snapshot round trip, until an iteration ends with a thermo step."""
    w = synth.reactive(128, 64, seed=3, ndiscs=4, rmin=4, rmax=8, q=9, kr=0.02, bmax=0.3)
    lt = lb2d.from_workload(w, thermo=7)
    lt.iteration(17)                        # thermo at 7 and 14, not at 17
    with pytest.raises(lb2d.LBError) as e:
        lt.thermo_static()
    assert e.value.code == lb2d.LB_E_ORDER
    lt.iteration(4)                         # 21: a thermo step
    _same(lt.thermo_static(), lt.get_thermo())
    buf = np.zeros(lt.state_size(), np.uint8)
    lt.save_state(buf)
    lt.load_state(buf)
    with pytest.raises(lb2d.LBError) as e:
        lt.thermo_static()
    assert e.value.code == lb2d.LB_E_ORDER
    lt.iteration(7)                         # 28: a thermo step again
    ref = lt.get_thermo()
    assert ref["step"] == 28
    for _ in range(2):
        _same(lt.thermo_static(), ref)


def test_static_thermo_reads_deferred_record_first():
    """With deferred thermo records the call reads the record still waiting
    in host memory before it checks and recomputes: called first after the
    iteration, it still equals lb_get_thermo's record."""
    w = synth.reactive(128, 64, seed=3, ndiscs=4, rmin=4, rmax=8, q=9, kr=0.02, bmax=0.3)
    lt = lb2d.from_workload(w)
    lt.thermo_deferred(True)
    for steps in (30, 17):
        lt.iteration(steps)
        first = lt.thermo_static()
        _same(first, lt.get_thermo())
        assert first["step"] == 30 if steps == 30 else first["step"] == 47

