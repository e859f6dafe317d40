"""The Python examples of README.md run as written (in order, one namespace) and give
consistent results: the two solvers' energies agree, the batched ground states converge,
and E2[Q] = E2[W] - E2[P]."""
import os
import re

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_examples(gpu):
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, flags=re.S)
    assert len(blocks) >= 4
    ns = {}
    for b in blocks:
        exec(compile(b, "README.md", "exec"), ns)
    assert np.allclose(ns["r64"].energies.cpu().numpy(), ns["rmix"].energies.cpu().numpy(), atol=1e-9)
    assert ns["res"].converged.all()
    assert np.allclose(ns["E2_Q"], ns["E2_W"] - ns["E2_P"], rtol=1e-12, atol=1e-12)
    assert ns["g1"].shape == (60, 60)
