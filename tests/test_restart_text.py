"""The oracle's reader of input-data files (read_data command, Sec.
Commands), on CPU.

``golden/read_data_channel.dat`` is a 5 x 4 channel laid out as the
read_data command describes a fluid file: the nine sections (in an order
the command allows), solid walls marked by density -11, one dirichlet inlet
and outlet, a force given as two velocity modes, populations listed site by
site.  The reader must give the state and setup written there: checked
against an oracle set up by hand from the same numbers (same bits after
several iterations), and each order rule of the command must reject a file
that breaks it.
"""
import os

import numpy as np
import pytest

from oracle.orc import Oracle
from oracle.restart import DataError, oracle_from_data, read_fluid

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "read_data_channel.dat")
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def _listed_populations():
    """the momentum section's numbers, read here line by line"""
    lines = open(GOLDEN).read().split("\n")
    k = lines.index("momentum")
    f = np.zeros((9, 4, 5))
    for ln in lines[k + 1:]:
        t = ln.split()
        if t:
            f[:, int(t[1]), int(t[0])] = [float(v) for v in t[2:]]
    return f


def _by_hand():
    """the channel of the fixture set up through the oracle's own calls"""
    o = Oracle(5, 4)
    solid = np.zeros((4, 5), np.uint8)
    solid[0, :] = solid[3, :] = 1
    o.set_solid(solid)
    o.set_tau(0.8)
    # force e1 1e-5 e5 2e-6: e1 = (1, 0), e5 = (1, 1)
    o.set_aveforce(1e-5 + 2e-6, 2e-6)
    k = o.add_opening("xlo", 1, 2, "inlet")
    o.set_opening_momentum(k, "dirichlet", 0.0, 1.002)
    k = o.add_opening("xhi", 1, 2, "outlet")
    o.set_opening_momentum(k, "dirichlet", 0.0, 1.0)
    o.set_f(_listed_populations())
    return o


def test_golden_channel_reads_as_written():
    o = oracle_from_data(GOLDEN)
    assert (o.nx, o.ny, o.ncomp) == (5, 4, 1)
    solid = o.solid()
    assert solid[0].all() and solid[3].all() and not solid[1:3].any()
    assert np.array_equal(o.f(), _listed_populations())
    ref = _by_hand()
    o.step(25)
    ref.step(25)
    assert np.array_equal(o.f(), ref.f())


def test_golden_channel_equilibrium_argument():
    """'equilibrium': f = f_eq(rho of the density section, u carried by
    the populations)"""
    o = oracle_from_data(GOLDEN, "equilibrium")
    f_list = _listed_populations()
    rho_sec = np.zeros((4, 5))
    for ln in open(GOLDEN).read().split("density")[1].split("momentum")[0].strip().split("\n"):
        t = ln.split()
        rho_sec[int(t[1]), int(t[0])] = float(t[2])
    f = o.f()
    fl = o.solid() == 0
    assert np.allclose(f.sum(0)[fl], rho_sec[fl], rtol=0, atol=1e-15)
    jx, jy = np.tensordot(EX, f_list, 1), np.tensordot(EY, f_list, 1)
    rs = f_list.sum(0)
    # the momentum the equilibrium carries: rho_sec * (j / sum f)
    assert np.allclose(np.tensordot(EX, f, 1)[fl], (rho_sec * jx / np.where(fl, rs, 1))[fl], atol=1e-15)
    assert np.allclose(np.tensordot(EY, f, 1)[fl], (rho_sec * jy / np.where(fl, rs, 1))[fl], atol=1e-15)
    assert np.all(f[:, ~fl] == 0)


def _variant(tmp_path, edit):
    lines = open(GOLDEN).read().split("\n")
    p = tmp_path / "v.dat"
    p.write_text("\n".join(edit(lines)) + "\n")
    return str(p)


def _move_section(lines, name, after):
    """the section `name` (with its data) moved behind section `after`"""
    heads = [i for i, ln in enumerate(lines) if ln.strip() and len(ln.split()) == 1 and ln.strip() in (
        "relaxation_time", "domain", "processors", "inlet", "outlet", "boundary", "field", "density", "momentum")]
    blocks = {}
    for a, b in zip(heads, heads[1:] + [len(lines)]):
        blocks[lines[a].strip()] = lines[a:b]
    order = [lines[h].strip() for h in heads]
    order.remove(name)
    order.insert(order.index(after) + 1, name)
    return [ln for s in order for ln in blocks[s]]


@pytest.mark.parametrize("name,after", [("processors", "density"),       # processors before density
                                        ("processors", "momentum"),      # ... and momentum
                                        ("boundary", "density"),         # boundary before density
                                        ("domain", "processors"),        # domain before processors
                                        ("relaxation_time", "field")])   # field after relaxation_time
def test_order_rules(tmp_path, name, after):
    with pytest.raises(DataError):
        read_fluid(_variant(tmp_path, lambda L: _move_section(L, name, after)))


def test_allowed_reordering(tmp_path):
    """inlet/outlet may come anywhere"""
    p = _variant(tmp_path, lambda L: _move_section(_move_section(L, "inlet", "momentum"), "outlet", "relaxation_time"))
    o = oracle_from_data(p)
    assert np.array_equal(o.f(), _listed_populations())


def test_missing_site_and_stray_data(tmp_path):
    with pytest.raises(DataError):
        oracle_from_data(_variant(tmp_path, lambda L: [ln for ln in L if ln != "2 1 1.0025 noslip"]))
    with pytest.raises(DataError):
        read_fluid(_variant(tmp_path, lambda L: ["0.5"] + L))
