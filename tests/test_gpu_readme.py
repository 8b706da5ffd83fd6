"""The README's quick start runs as written (GPU)."""
import os
import re

import pytest

from tests.gpu_common import requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def test_readme_quick_start_runs():
    import torch
    text = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, re.S)
    assert blocks, "no python block in the README"
    env = {}
    exec(compile(blocks[0], "README.md", "exec"), env)
    rgb, depth = env["rgb"], env["depth"]
    assert rgb.shape == (640000, 3) and depth.shape == (640000,)
    assert torch.isfinite(rgb).all() and torch.isfinite(depth).all()
    assert env["feats"].grad is not None and env["params"].grad is not None
    assert float(env["params"].grad.abs().sum()) > 0.0
