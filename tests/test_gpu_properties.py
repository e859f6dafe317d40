"""Properties of the GPU sigma that hold at any size, checked on the full bench spaces
without the oracle.

- Hermiticity: <x, H y> = <H x, y> for seeded random x, y on the 2M-determinant real
  space and the 1M-determinant complex spinor space (H = H^+, Eq. Hamiltonian), in every
  precision mode that computes in FP64-class arithmetic.
- alpha/beta swap symmetry: on a space closed under exchanging the spin labels (a 200k
  selected space of the 30-orbital recipe united with its swapped copy, about 400k
  determinants), sigma(P c) = P sigma(c).  Spin-free integrals with n_alpha = n_beta make
  H invariant under the swap; every determinant takes the same sign (-1)^(n_alpha n_beta).
"""
import dataclasses

import numpy as np
import pytest

from paper_2501_18185_gb300 import sci
from paper_2501_18185_gb300 import workloads as W

pytestmark = pytest.mark.gpu

_cache = {}


def _ham(name):
    if name not in _cache:
        w = W.selected_30o() if name == "sel_30o" else W.selected_spinor_64()
        _cache[name] = (w, sci.Hamiltonian.from_workload(w))
    return _cache[name]


@pytest.mark.parametrize("name,prec", [("sel_30o", sci.SCI_PREC_F64), ("sel_30o", sci.SCI_PREC_F64_DS),
                                       ("sel_64s", sci.SCI_PREC_F64), ("sel_64s", sci.SCI_PREC_F64_DS)])
def test_hermiticity_full_size(gpu, name, prec):
    torch = gpu
    w, H = _ham(name)
    rng = np.random.default_rng(11)
    X = rng.normal(size=(w.M, 2))
    if w.ints.complex_:
        X = X + 1j * rng.normal(size=(w.M, 2))
    Xd = torch.from_numpy(X).cuda()
    S = H.sigma(Xd, prec=prec)
    x, y, hx, hy = Xd[:, 0], Xd[:, 1], S[:, 0], S[:, 1]
    lhs = complex(torch.sum(x.conj() * hy).item())     # <x, H y>
    rhs = complex(torch.sum(hx.conj() * y).item())     # <H x, y>
    scale = float(torch.linalg.vector_norm(x) * torch.linalg.vector_norm(hy))
    assert abs(lhs - rhs) < 1e-12 * scale, (lhs, rhs, scale)


def _spin_swap(keys, n):
    keys = np.asarray(keys, dtype=np.uint64)
    mask = np.uint64((1 << n) - 1)
    return (keys >> np.uint64(n)) | ((keys & mask) << np.uint64(n))


def test_alpha_beta_swap_symmetry_selected_400k(gpu):
    torch = gpu
    w = W.selected_30o(M=200_000)
    keys = np.unique(np.concatenate([w.keys, _spin_swap(w.keys, w.n)]))
    rng = np.random.default_rng(5)
    c = rng.normal(size=(len(keys), 2))
    ws = dataclasses.replace(w, name="sel_30o_swap_closed", keys=keys, c=c)
    H = sci.Hamiltonian.from_workload(ws)
    perm = np.searchsorted(keys, _spin_swap(keys, w.n))
    assert np.array_equal(keys[perm], _spin_swap(keys, w.n))
    pc = np.empty_like(c)
    pc[perm] = c
    s = H.sigma(torch.from_numpy(c).cuda()).cpu().numpy()
    ps = H.sigma(torch.from_numpy(pc).cuda()).cpu().numpy()
    assert np.linalg.norm(ps[perm] - s) < 1e-12 * np.linalg.norm(s)
