"""Host logic of the batched Davidson (batch_davidson.py) on the CPU.

The batched sigma launch, the segmented products and the batched eigensolver are
replaced by plain per-instance torch arithmetic on dense symmetric matrices, so what is
tested here is the solver around them:
- every instance reaches the lowest eigenvalue of its matrix (numpy eigvalsh), with
  instances of 1, 2 and 9 rows (spaces exhausted after a few columns) next to larger
  ones, with and without restarts;
- the returned vectors have unit norm and the residual the solver reports;
- one launch per start vector and per unconverged iteration; the active set in each
  launch never grows, and keeping converged instances in the launch gives the same
  energies;
- the start block: unit vectors on the lowest diagonal entries, seeded noise.
"""
import numpy as np
import pytest
import torch

from paper_2501_18185_gb300 import batch_davidson as BD
from paper_2501_18185_gb300 import sci


class _Seg:
    """Segmented products by per-instance torch arithmetic."""

    def __init__(self, offsets, kmax, device=None, stream=None):
        self.off = np.asarray(offsets)
        self.nseg, self.kmax = len(self.off) - 1, kmax

    def close(self):
        pass

    def tn(self, A, t, out=None):
        A2 = A if A.dim() == 2 else A.view(1, -1)
        assert A2.shape[0] <= self.kmax
        r = torch.zeros((self.nseg, A2.shape[0]), dtype=torch.float64)
        for s in range(self.nseg):
            a, b = self.off[s], self.off[s + 1]
            r[s] = A2[:, a:b] @ t[a:b]
        return r

    def nn(self, y, beta=None, A1=None, c1=None, alpha1=1.0, A2=None, c2=None, alpha2=1.0, dg=None, shift=None):
        for s in range(self.nseg):
            a, b = self.off[s], self.off[s + 1]
            bs = 0.0 if beta is None else float(beta[s])
            acc = bs * y[a:b] if bs != 0.0 else torch.zeros(b - a, dtype=torch.float64)
            if A1 is not None and A1.shape[0]:
                acc = acc + alpha1 * (c1[s] @ A1[:, a:b])
            if A2 is not None and A2.shape[0]:
                acc = acc + alpha2 * (c2[s] @ A2[:, a:b])
            if dg is not None:
                den = shift[s] - dg[a:b]
                acc = acc / torch.where(den.abs() < 1e-8, torch.full_like(den, 1e-8), den)
            y[a:b] = acc
        return y


class _Ham:
    def __init__(self, H):
        self.H = torch.from_numpy(H)
        self.M = H.shape[0]

    def diagonal(self):
        return self.H.diagonal().clone()


class _Batch:
    """Block-diagonal H applied to fixed buffers; records the instances each replay computes."""

    def __init__(self, hams):
        self.hams, self.device = hams, torch.device("cpu")
        self.offsets, o = [], 0
        for h in hams:
            self.offsets.append(o)
            o += h.M
        self.M = o
        self.active = np.ones(len(hams), dtype=bool)
        self.computed = []

    def plan(self, schedule, C, S):
        self.active[:] = True

    def capture(self, C, S):
        self.C, self.S = C, S

    def set_active(self, a):
        a = np.asarray(a)
        assert a.shape == (len(self.hams),)
        self.active = a != 0

    def replay(self):
        self.S.zero_()
        self.computed.append(int(self.active.sum()))
        for h, o, on in zip(self.hams, self.offsets, self.active):
            if on:
                self.S[o:o + h.M] = h.H @ self.C[o:o + h.M]


def _matrices(sizes, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for M in sizes:
        A = rng.normal(size=(M, M))
        out.append(_Ham(0.05 * (A + A.T) + np.diag(np.sort(rng.normal(size=M)) * 3)))
    return out


def _syev(G, n=None, w=None, V=None, max_sweeps=30):
    """Eigenpairs of the symmetrised leading n x n blocks (torch's CPU eigh)."""
    n = G.shape[1] if n is None else n
    Gs = G[:, :n, :n]
    return torch.linalg.eigh(0.5 * (Gs + Gs.transpose(1, 2)))


@pytest.fixture
def fake_seg(monkeypatch):
    monkeypatch.setattr(sci, "Segments", _Seg)
    monkeypatch.setattr(sci, "syev_batched", _syev)


@pytest.mark.parametrize("max_space,keep,nstart", [(24, 2, 4), (6, 2, 2), (5, 3, 4)])
def test_ground_states_match_dense(fake_seg, max_space, keep, nstart):
    hams = _matrices([9, 16, 300, 50, 1, 2, 120])
    B = _Batch(hams)
    r = BD.davidson_batched(B, tol=1e-8, max_iter=600, max_space=max_space, keep=keep, nstart=nstart)
    assert r.converged.all()
    nst = min(nstart, max_space - 1)
    assert r.sigma_launches == nst + r.iterations - 1 == len(B.computed)
    assert r.active_per_launch == B.computed
    assert all(a >= b for a, b in zip(B.computed, B.computed[1:])) and B.computed[-1] < len(hams)
    for i, (h, o) in enumerate(zip(hams, B.offsets)):
        ref = np.linalg.eigvalsh(h.H.numpy())[0]
        assert abs(r.energies[i] - ref) < 1e-10, (i, r.energies[i], ref)
        x = r.vectors[o:o + h.M]
        assert abs(float(torch.linalg.vector_norm(x)) - 1.0) < 1e-10
        assert float(torch.linalg.vector_norm(h.H @ x - r.energies[i] * x)) < 1.5e-8
    assert B.active.all()          # the batch is left with every instance active


def test_keeping_converged_instances_changes_nothing(fake_seg):
    hams = _matrices([40, 7, 200, 3], seed=3)
    r1 = BD.davidson_batched(_Batch(hams), tol=1e-9, max_iter=400)
    B2 = _Batch(hams)
    r2 = BD.davidson_batched(B2, tol=1e-9, max_iter=400, drop_converged=False)
    assert set(B2.computed) == {len(hams)}
    assert r1.iterations == r2.iterations
    assert np.abs(r1.energies - r2.energies).max() < 1e-12


def test_start_block():
    off = np.array([0, 5, 5, 7, 20])
    diag = np.concatenate([[3.0, -1.0, 2.0, -5.0, 0.0], [1.0, 0.5], np.arange(13.0)])
    T = BD.start_block(off, diag, 3)
    assert T.shape == (3, 20)
    assert np.array_equal(T, BD.start_block(off, diag, 3))          # seeded
    # instance 0: lowest diagonals at rows 3, 1, 4
    for j, row in enumerate([3, 1, 4]):
        assert abs(T[j, row] - 1.0) < 0.01
    # instance 2 (2 rows): two unit vectors, the third column is noise only
    assert abs(T[0, 6] - 1.0) < 0.01 and abs(T[1, 5] - 1.0) < 0.01
    assert np.abs(T[2, 5:7]).max() < 0.01
    noise = T.copy()
    noise[np.abs(noise) > 0.5] -= 1.0
    assert 0 < np.abs(noise).max() < 0.01


def test_space_limit():
    """The batched eigensolver takes matrices up to 64 x 64: larger spaces are refused
    before any work (no batch method is called)."""
    for bad in (1, 65):
        with pytest.raises(ValueError):
            BD.davidson_batched(object(), max_space=bad)


def test_cleanup_on_failure(fake_seg, monkeypatch):
    """A launch that fails mid-solve leaves the batch with every instance active again and
    the segment workspace closed."""
    closed = []
    monkeypatch.setattr(_Seg, "close", lambda self: closed.append(True))
    hams = _matrices([30, 12, 80], seed=4)
    B = _Batch(hams)
    orig = B.replay

    def failing():
        if len(B.computed) == 10:
            raise RuntimeError("launch failed")
        orig()

    B.replay = failing
    with pytest.raises(RuntimeError):
        BD.davidson_batched(B, tol=1e-12, max_iter=50)
    assert B.active.all() and closed == [True]
