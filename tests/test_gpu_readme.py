"""The usage example of the repository's README runs as written."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_example_runs(capsys):
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, flags=re.S)
    assert blocks
    ns = {}
    exec(compile(blocks[0], "README.md", "exec"), ns)
    out = capsys.readouterr().out.split()
    psnr, bpppb, ssim = float(out[0]), float(out[1]), float(out[2])
    assert 30 < psnr < 80 and 0 < bpppb < 8 and 0.5 < ssim <= 1.0
    ns["ctx"].close()
