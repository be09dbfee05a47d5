"""The Python examples of README.md run as written (on a GPU)."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu


def test_readme_examples_run():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1112_5588_gb300 import build
    build.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "README.md")) as fh:
        blocks = re.findall(r"```python\n(.*?)```", fh.read(), flags=re.S)
    assert len(blocks) >= 2
    ns = {}
    for code in blocks:
        exec(compile(code, "README.md", "exec"), ns)
    torch.cuda.synchronize()
    # the first example's product is finite and the batch wrote its outputs
    assert torch.isfinite(ns["y"]).all()
    assert all(torch.isfinite(t).all() for t in ns["ys"])
    assert ns["choice"]["source"] in ("model", "sweep") and ns["choice"]["b"] in (32, 64, 128, 256)
    assert torch.isfinite(ns["y_ceiling"]).all()
