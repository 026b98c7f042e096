"""The Python example in README.md runs as written (documentation that works)."""
import os
import re

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_example_runs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_3297_gb300 import build
    build.build_library()
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, flags=re.S)
    assert blocks, "README has a Python example"
    scope = {}
    try:
        exec(compile(blocks[0], "README.md", "exec"), scope)
        assert scope["composites"] > 0
        assert int(scope["primes"].sum().item()) == (1024 << 20) - scope["composites"]
    finally:
        if "ctx" in scope:
            scope["ctx"].close()
