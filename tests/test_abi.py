"""The C-ABI library builds, loads and exports every function its header
declares; the Python binding knows every one of them.  No GPU needed."""
import os
import re
import subprocess

import pytest

from paper_1202_0442_gb300 import build, lb2d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lb2d.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(lb_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_declares_the_command_set():
    names = declared_functions()
    for cmd in ("lattice", "processors", "fluids", "solute", "inlet", "outlet", "inlet_momentum",
                "outlet_momentum", "inlet_solute", "outlet_solute", "boundary_style", "obstacle_rect",
                "obstacle_circle", "surface_reaction", "position0_rect", "momentum0", "concentration0",
                "aveforce", "aveacceleration", "interforce", "adhesiveforce", "thermo", "iteration"):
        assert f"lb_{cmd}" in names, cmd


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    assert set(declared_functions()) == set(lb2d.SIGNATURES)
    L = lb2d.lib()
    for name in declared_functions():
        assert getattr(L, name) is not None
