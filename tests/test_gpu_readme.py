"""The README's usage example runs as written and gives a plausible force-
driven channel (mass kept, flow along +x)."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_example_runs(capsys):
    text = open(os.path.join(ROOT, "README.md")).read()
    code = re.search(r"```python\n(.*?)```", text, re.S).group(1)
    ns = {}
    exec(compile(code, "README.md", "exec"), ns)
    th, px, nx, ny = ns["th"], ns["px"], ns["nx"], ns["ny"]
    fluid = nx * (ny - 2)
    assert abs(th["mass1"] - fluid) < 1e-6 * fluid
    assert px[ny // 2].min() > 0
