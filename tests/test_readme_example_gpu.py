"""The Python usage example of README.md runs as written (three flavours, 262,144 beams, mixed
precision, adaptive exact propagators from the neutrino sphere to 1000 km) and gives sane
survival probabilities."""
import os
import re

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_python_example(xf):
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, flags=re.S)
    assert len(blocks) == 1
    env = {}
    exec(compile(blocks[0], "README.md", "exec"), env)
    s, pee, mean = env["s"], env["pee"], env["mean"]
    assert s.stats().r_km == 1000.0 and s.stats().status == 0
    assert pee.shape == (2 * 256 * 512,) and np.all((pee >= -1e-6) & (pee <= 1 + 1e-6))
    assert 0.5 < mean <= 1.0 and pee.min() < 0.5         # the MSW conversions of the low energies
    snap = env["snap"]
    assert snap["r_km"] == 1000.0 and snap["pee_nu"].shape == (512, 256)
    assert np.allclose(np.concatenate([snap["pee_nu"].ravel(), snap["pee_nubar"].ravel()]), pee)
