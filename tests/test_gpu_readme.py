"""The Python examples of README.md run as written (in order, one namespace) and give
consistent results: the two solvers' energies agree, the batched ground states converge,
and E2[Q] = E2[W] - E2[P]."""
import os
import re
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_readme_examples(gpu, monkeypatch):
    import torch.distributed as dist

    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, flags=re.S)
    assert len(blocks) >= 4
    # the row-split example runs as a one-rank torchrun job would
    for k, v in {"RANK": "0", "LOCAL_RANK": "0", "WORLD_SIZE": "1",
                 "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(_free_port())}.items():
        monkeypatch.setenv(k, v)
    was_initialized = dist.is_initialized()
    ns = {}
    try:
        for b in blocks:
            exec(compile(b, "README.md", "exec"), ns)
    finally:
        if dist.is_initialized() and not was_initialized:
            dist.destroy_process_group()
    S_ref = ns["H"].sigma(ns["C"]).cpu().numpy()
    assert np.array_equal(ns["S_split"].cpu().numpy().shape, S_ref.shape)
    assert np.allclose(ns["S_split"].cpu().numpy(), S_ref, rtol=1e-12, atol=1e-12)
    assert np.allclose(ns["r64"].energies.cpu().numpy(), ns["rmix"].energies.cpu().numpy(), atol=1e-9)
    assert ns["res"].converged.all()
    assert np.allclose(ns["E2_Q"], ns["E2_W"] - ns["E2_P"], rtol=1e-12, atol=1e-12)
    assert ns["g1"].shape == (60, 60)
