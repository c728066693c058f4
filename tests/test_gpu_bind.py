"""Caller-owned device buffers (lb_bind): a lattice whose state lives in
torch tensors runs bit for bit like one whose buffers the library owns,
and the tensors hold the state in the documented layout."""
import numpy as np
import pytest

from paper_1202_0442_gb300 import lb2d, synth

from pairing import W9

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _tensors(lt_probe, names):
    return {n: torch.zeros(lt_probe.buffer_size(n), dtype=torch.uint8, device="cuda") for n in names}


def _probe(w, storage="fp32"):
    lt = lb2d.Lattice(0)
    lt.lattice(w.nx, w.ny, w.tau[0])
    if w.solute_q:
        lt.solute(w.taus, w.solute_q)
    lt.set_storage(storage, list(w.rho_ref), 2e-3 if storage != "fp32" else 0.0)
    return lt


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_bound_populations_bitwise(storage):
    w = synth.porous(100, 70, seed=5)
    probe = _probe(w, storage)
    bufs = _tensors(probe, ["f0", "f1", "fields"])
    probe.close()
    kw = {"h_max": 2e-3, "rounding": "stochastic"} if storage != "fp32" else {}
    a = lb2d.from_workload(w, storage, thermo=5, bind=bufs, **kw)
    b = lb2d.from_workload(w, storage, thermo=5, **kw)
    a.iteration(23)
    b.iteration(23)
    assert np.array_equal(a.populations(1), b.populations(1))
    assert a.get_thermo() == b.get_thermo()
    # the current buffer, read straight from the tensor: deviations from
    # w_i rho_ref in [9][ny][pitch] of the storage type
    k = a.current_buffer()
    pitch = (w.nx + 31) // 32 * 32
    dt = torch.float32 if storage == "fp32" else torch.float16
    h = bufs[f"f{k}"].view(dt).reshape(9, w.ny, pitch)[:, :, :w.nx].double().cpu().numpy()
    if storage != "fp32":
        # stored as h * 2^s, s the largest integer with h_max 2^s <= 2^14
        s = 0
        while 2e-3 * 2.0 ** (s + 1) <= 2.0 ** 14:
            s += 1
        h = h * 2.0 ** -s
    fl = w.solid == 0
    # the reference density as the library holds it: rounded to FP32
    f = h + W9[:, None, None] * float(np.float32(w.rho_ref[0]))
    fa = a.populations(1)
    assert np.array_equal(np.where(fl, f, 0.0), np.where(fl, fa, 0.0))


def test_bound_solute_buffers_and_velocity():
    w = synth.reactive(128, 64, seed=3, ndiscs=4, rmin=4, rmax=8, q=9, kr=0.02, bmax=0.3, growth_seed=7)
    probe = _probe(w)
    names = ["f0", "f1", "g0", "g1", "fields", "u"]
    bufs = _tensors(probe, names)
    probe.close()
    a = lb2d.from_workload(w, bind=bufs)
    b = lb2d.from_workload(w)
    a.iteration(150)
    b.iteration(150)
    assert np.array_equal(a.populations(1), b.populations(1))
    ga, _, ba = a.solute_state()
    gb, _, bb = b.solute_state()
    assert np.array_equal(ga, gb) and np.array_equal(ba, bb)
    assert np.array_equal(a.mask(), b.mask())
    k = a.current_buffer()
    pitch = (w.nx + 31) // 32 * 32
    g = bufs[f"g{k}"].view(torch.float32).reshape(9, w.ny, pitch)[:, :, :w.nx].double().cpu().numpy()
    fl = a.mask() == 0
    assert np.array_equal(np.where(fl, g, 0.0), np.where(fl, ga, 0.0))


def test_bind_errors():
    w = synth.porous(64, 48, seed=2)
    lt = _probe(w)
    need = lt.buffer_size("f0")
    assert need == 9 * 48 * 64 * 4
    assert lt.buffer_size("u") == 0
    small = torch.zeros(need - 4, dtype=torch.uint8, device="cuda")
    with pytest.raises(lb2d.LBError):
        lt.bind("f0", small)
    odd = torch.zeros(need + 64, dtype=torch.uint8, device="cuda")[16:]
    with pytest.raises(lb2d.LBError):
        lt.bind("f0", odd)
    with pytest.raises(lb2d.LBError):
        lt.bind("nonsense", torch.zeros(need, dtype=torch.uint8, device="cuda"))
    with pytest.raises(ValueError):
        lt.bind("f0", torch.zeros(need, dtype=torch.uint8))
    ok = torch.zeros(need, dtype=torch.uint8, device="cuda")
    lt.bind("f0", ok)
    with pytest.raises(lb2d.LBError):
        lt.bind("f1", ok)  # the same memory twice
    # a storage change after binding that needs more bytes fails when the
    # device state is created (here by the state upload)
    lt.set_storage("fp16", [1.0], 2e-3)
    lt.bind("f1", torch.zeros(lt.buffer_size("f1"), dtype=torch.uint8, device="cuda"))
    lt.set_storage("fp32", [1.0], 0.0)
    with pytest.raises(lb2d.LBError):
        lt.set_equilibrium(np.ones((48, 64)), np.zeros((48, 64)), np.zeros((48, 64)), 1)


def test_velocity_f32_paths():
    """lb_get_velocity_f32 into page-locked buffers (the export kernel writes
    them directly) and into ordinary host arrays (staging copy) gives the
    same bits, and both equal rho = rho_ref + drho, u = p / rho formed in
    FP32 from the node fields."""
    w = synth.porous(100, 70, seed=5)
    lt = lb2d.from_workload(w, "fp32", thermo=0)
    lt.iteration(17)
    plain = lt.velocity_f32()
    pinned = tuple(torch.zeros((w.ny, w.nx), dtype=torch.float32).pin_memory() for _ in range(3))
    lt.velocity_f32(pinned)
    for a, b in zip(plain, pinned):
        assert np.array_equal(a, b.numpy())
    rho64, px, py, _ = lt.fields()
    fl = w.solid == 0
    # the fields hold rho - rho_ref in FP32; FP64 gives it back exactly
    r0 = np.float32(w.rho_ref[0])
    drho = (rho64 - float(r0)).astype(np.float32)
    rho = np.where(fl, r0 + drho, np.float32(1))  # solid nodes: no division by 0
    ux = px.astype(np.float32) / rho
    uy = py.astype(np.float32) / rho
    assert np.array_equal(np.where(fl, rho, 0), plain[0])
    assert np.array_equal(np.where(fl, ux, 0), plain[1])
    assert np.array_equal(np.where(fl, uy, 0), plain[2])


def test_new_entry_point_errors():
    """Argument and order errors of lb_set_step, lb_get_flips and the
    fused kernel choice."""
    w = synth.porous(64, 48, seed=2)
    lt = lb2d.from_workload(w, "fp32")
    with pytest.raises(lb2d.LBError):
        lt.set_step(-1)
    assert lt.flips().size == 0            # no surface reaction: nothing grows
    lt.iteration(2)
    assert lt.flips().size == 0
    with pytest.raises(lb2d.LBError):
        lt.set_kernel("bogus")
    lt.set_kernel("fused")                 # no solute: the iteration refuses it
    with pytest.raises(lb2d.LBError) as e:
        lt.iteration(1)
    assert "LB_E_UNSUPPORTED" in str(e.value)
    lt.set_kernel("auto")
    lt.iteration(1)
    lt.set_step(1000)                      # the step count is the caller's to set
    lt.iteration(1)
    assert lt.get_thermo()["step"] == 1001


def test_output_command_fields_without_thermo():
    """output command: node fields every Nf iterations without the thermo
    sums; the fields equal those a thermo step writes, bit for bit, and no
    thermo record exists until a thermo step runs."""
    w = synth.porous(100, 70, seed=5)
    a = lb2d.from_workload(w, "fp32")
    b = lb2d.from_workload(w, "fp32")
    a.thermo(1 << 30)
    a.output(1)
    b.thermo(1)
    a.iteration(9)
    b.iteration(9)
    for x, y in zip(a.velocity_f32(), b.velocity_f32()):
        assert np.array_equal(x, y)
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)
    with pytest.raises(lb2d.LBError) as e:
        a.get_thermo()
    assert e.value.code == lb2d.LB_E_ORDER
    with pytest.raises(lb2d.LBError) as e:
        a.thermo_static()
    assert e.value.code == lb2d.LB_E_ORDER
    with pytest.raises(lb2d.LBError):
        a.output(-1)


def test_contexts_on_two_threads():
    """Two contexts on two streams driven from two host threads at once (as
    the end-to-end benchmark leg runs them): every snapshot upload,
    iteration and velocity download gives the bits the same calls give
    one after the other."""
    import threading
    w = synth.porous(256, 192, seed=4, rmin=4, rmax=10)
    streams = [torch.cuda.Stream() for _ in range(2)]
    lts = [lb2d.from_workload(w, "fp32", stream=s.cuda_stream) for s in streams]
    lts[1].iteration(7)  # a different state in each context
    snaps = []
    for lt in lts:
        snaps.append(torch.empty(lt.state_size(), dtype=torch.uint8, pin_memory=True))
        lt.save_state(snaps[-1])
        lt.output(1)
    want = []
    for lt, snap in zip(lts, snaps):
        lt.load_state(snap)
        lt.iteration(3)
        want.append([a.copy() for a in lt.velocity_f32()])
    got = [[], []]

    def run(i):
        outs = tuple(torch.empty((w.ny, w.nx), dtype=torch.float32, pin_memory=True) for _ in range(3))
        for _ in range(10):
            lts[i].load_state(snaps[i])
            lts[i].iteration(3)
            lts[i].velocity_f32(outs)
            got[i].append([o.numpy().copy() for o in outs])

    th = [threading.Thread(target=run, args=(i,)) for i in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for i in range(2):
        assert len(got[i]) == 10
        for rec in got[i]:
            for a, b in zip(rec, want[i]):
                assert np.array_equal(a, b)
    assert not np.array_equal(want[0][1], want[1][1])
