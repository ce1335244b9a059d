"""The README's usage snippet runs as written (public Python API on a GPU)."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_python_snippet_runs():
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, flags=re.S)
    assert blocks, "README has no python block"
    scope = {}
    exec(compile(blocks[0], "README.md", "exec"), scope)
    rows, counts = scope["rows"], scope["counts"]
    assert rows.shape[0] == counts.shape[0] == 4096 and int(counts.min()) > 0
    assert scope["xyz"].grad is not None and scope["eps"].grad is not None
    assert scope["nl64"].max_count > 0
