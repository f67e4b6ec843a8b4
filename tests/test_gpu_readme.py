"""The usage example of the README runs as written."""
import os
import re

import pytest

from gpu_helpers import rs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_python_example_runs():
    rs()  # built
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, flags=re.S)
    assert blocks
    ns = {}
    exec(compile(blocks[0], "README.md", "exec"), ns)
    assert ns["counts"].shape == (1024, 1024)
    assert ns["lc_mu"].numel() == 2000 and ns["zoomed"].shape == (1024, 1024)
