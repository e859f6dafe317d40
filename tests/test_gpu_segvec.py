"""Segmented block-vector products (sci_seg_tn / sci_seg_nn) against numpy per instance,
and the active-instance mask of the batched sigma (sci_batch_set_active).

Segments: empty ones, one row, sizes that span several 2048-row items with ragged tails;
widths from 1 to kmax (several 8-column passes); leading dimensions above the row count.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2501_18185_gb300 import sci
from paper_2501_18185_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SIZES = [0, 1, 2047, 2048, 2049, 5000, 0, 31, 12289, 7]


def _case(torch, k, seed=0, ld_pad=5):
    rng = np.random.default_rng(seed)
    off = np.concatenate([[0], np.cumsum(SIZES)]).astype(np.int64)
    M = int(off[-1])
    Abuf = rng.normal(size=(k, M + ld_pad))
    t = rng.normal(size=M)
    A = torch.from_numpy(Abuf).cuda()[:, :M]     # row stride M + ld_pad
    return rng, off, M, Abuf[:, :M], A, t, torch.from_numpy(t).cuda()


@pytest.mark.parametrize("k", [1, 3, 8, 13, 40])
def test_seg_tn(gpu, k):
    torch = gpu
    rng, off, M, An, A, t, td = _case(torch, k, seed=k)
    sg = sci.Segments(off, kmax=64)
    got = sg.tn(A, td).cpu().numpy()
    for s in range(len(SIZES)):
        a, b = off[s], off[s + 1]
        ref = An[:, a:b] @ t[a:b]
        assert np.allclose(got[s], ref, rtol=1e-12, atol=1e-12 * max(1.0, np.abs(An[:, a:b]).sum() ** 0.5)), s
        if a == b:
            assert np.all(got[s] == 0.0)
    again = sg.tn(A, td).cpu().numpy()
    assert np.array_equal(got, again)        # fixed reduction order


@pytest.mark.parametrize("k1,k2", [(0, 0), (5, 0), (0, 9), (17, 24)])
def test_seg_nn_and_preconditioner(gpu, k1, k2):
    torch = gpu
    rng, off, M, An, A, t, td = _case(torch, max(k1, k2, 1), seed=10 + k1 + k2)
    nseg = len(SIZES)
    B1 = rng.normal(size=(k1, M))
    B2 = rng.normal(size=(k2, M))
    c1 = rng.normal(size=(nseg, k1))
    c2 = rng.normal(size=(nseg, k2))
    beta = rng.normal(size=nseg)
    beta[3] = 0.0
    y0 = rng.normal(size=M)
    for s in range(nseg):                       # y is not read where beta = 0
        if beta[s] == 0.0:
            y0[off[s]:off[s + 1]] = np.nan
    dg = rng.normal(size=M)
    shift = rng.normal(size=nseg)
    dg[off[2] + 5] = shift[2] + 1e-10           # a clamped denominator
    sg = sci.Segments(off, kmax=32)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    for with_prec in (False, True):
        y = cu(y0.copy())
        sg.nn(y, cu(beta), A1=cu(B1) if k1 else None, c1=cu(c1) if k1 else None, alpha1=0.5,
              A2=cu(B2) if k2 else None, c2=cu(c2) if k2 else None, alpha2=-2.0,
              dg=cu(dg) if with_prec else None, shift=cu(shift) if with_prec else None)
        got = y.cpu().numpy()
        for s in range(nseg):
            a, b = off[s], off[s + 1]
            ref = (beta[s] * y0[a:b] if beta[s] != 0 else np.zeros(b - a)) + 0.5 * (c1[s] @ B1[:, a:b]) - 2.0 * (c2[s] @ B2[:, a:b])
            if with_prec:
                den = shift[s] - dg[a:b]
                den = np.where(np.abs(den) < 1e-8, 1e-8, den)
                ref = ref / den
            assert np.allclose(got[a:b], ref, rtol=1e-12, atol=1e-12), (s, with_prec)
    y = cu(np.zeros(M))
    sg.nn(y, None)                               # beta NULL, nothing else: y = 0
    assert float(y.abs().max()) == 0.0


def test_seg_errors(gpu):
    torch = gpu
    with pytest.raises(sci.SciError):
        sci.Segments(np.array([0, 5, 3]), kmax=4)           # decreasing offsets
    with pytest.raises(sci.SciError):
        sci.Segments(np.array([0, 5]), kmax=300)            # kmax above 256
    sg = sci.Segments(np.array([0, 5, 9]), kmax=4)
    A = torch.zeros((5, 9), dtype=torch.float64, device="cuda")
    t = torch.zeros(9, dtype=torch.float64, device="cuda")
    with pytest.raises(sci.SciError) as e:
        sci.sci_seg_tn(sg.sg, 5, A, 9, t, torch.zeros(10, dtype=torch.float64, device="cuda"))   # k > kmax
    assert e.value.code == sci.SCI_ERR_ARG
    with pytest.raises(sci.SciError):
        sci.sci_seg_tn(sg.sg, 2, A, 8, t, torch.zeros(4, dtype=torch.float64, device="cuda"))    # lda < rows


def test_batch_active_mask(gpu):
    """Inactive instances get S = 0 and cost nothing; active ones are unchanged, in plain
    launches and in replays of a graph captured before the mask changed."""
    torch = gpu
    ws = [W.random_small(401 + i, "spin_orbitals", 7 + i % 3, 3, 2 + i % 2) for i in range(6)]
    hams = [sci.Hamiltonian.from_workload(w) for w in ws]
    C = torch.from_numpy(np.concatenate([w.c[:, 0] for w in ws])).cuda()
    B = sci.Batch(hams)
    B.plan(sci.SCI_SCHED_AUTO, C, torch.empty_like(C))
    full = B.sigma(C).cpu().numpy()
    for i, w in enumerate(ws):
        ref = Oracle.from_workload(w).sigma(w.c)[:, 0]
        assert np.linalg.norm(full[B.offsets[i]:B.offsets[i] + w.M] - ref) < 1e-11 * np.linalg.norm(ref)
    S = torch.empty_like(C)
    B.capture(C, S)
    mask = np.array([1, 0, 1, 1, 0, 0], dtype=np.int32)
    B.set_active(mask)
    for run in (lambda: B.sigma(C, out=S), B.replay):
        S.fill_(np.nan)
        run()
        got = S.cpu().numpy()
        for i, w in enumerate(ws):
            sl = slice(B.offsets[i], B.offsets[i] + w.M)
            if mask[i]:
                assert np.array_equal(got[sl], full[sl]) or np.allclose(got[sl], full[sl], rtol=1e-13, atol=1e-14)
            else:
                assert np.all(got[sl] == 0.0)
    with pytest.raises(sci.SciError):
        B.set_active(np.ones(5, dtype=np.int32))   # one flag per instance
    B.plan(sci.SCI_SCHED_TILE)                     # a new plan makes every instance active
    got = B.sigma(C).cpu().numpy()
    assert np.allclose(got, full, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 24, 27, 32, 33, 64])
def test_syev_batched_random(gpu, n):
    """Eigenvalues against numpy eigvalsh, eigenvector residuals and orthonormality."""
    torch = gpu
    rng = np.random.default_rng(100 + n)
    nb = 7
    A = rng.normal(size=(nb, n, n))
    A = A + A.transpose(0, 2, 1) + np.diag(np.linspace(-5, 5, n))[None]
    w, V = sci.syev_batched(torch.from_numpy(A).cuda())
    w, V = w.cpu().numpy(), V.cpu().numpy()
    for b in range(nb):
        ref = np.linalg.eigvalsh(A[b])
        scale = np.abs(A[b]).sum()
        assert np.abs(w[b] - ref).max() < 1e-13 * scale
        assert np.all(np.diff(w[b]) >= 0)
        assert np.abs(A[b] @ V[b] - V[b] * w[b][None, :]).max() < 1e-13 * scale
        assert np.abs(V[b].T @ V[b] - np.eye(n)).max() < 1e-13 * max(1, n)


def test_syev_batched_leading_block_degenerate_and_symmetrised(gpu):
    """The leading n x n block of a larger strided buffer, as the batched solver uses it;
    a degenerate pair and a decoupled large diagonal entry (a null column's penalty); an
    input that is not symmetric is symmetrised."""
    torch = gpu
    rng = np.random.default_rng(7)
    cap, n, nb = 24, 17, 5
    G = rng.normal(size=(nb, cap, cap))
    G = G + G.transpose(0, 2, 1)
    G[1, :n, :n] = np.diag(np.r_[[1.0, 1.0], np.arange(2.0, n + 0.0)])   # degenerate pair
    G[2, 10, :] = G[2, :, 10] = 0.0
    G[2, 10, 10] = 1000.0                                                  # decoupled penalty
    G[3, :n, :n] += np.triu(rng.normal(size=(n, n)), 1)                    # not symmetric
    Gd = torch.from_numpy(G).cuda()
    wbuf = torch.full((nb, cap), np.nan, dtype=torch.float64, device="cuda")
    Vbuf = torch.full((nb, cap, cap), np.nan, dtype=torch.float64, device="cuda")
    w, V = sci.syev_batched(Gd, n=n, w=wbuf, V=Vbuf)
    w, V = w.cpu().numpy(), V.cpu().numpy()
    for b in range(nb):
        S = 0.5 * (G[b, :n, :n] + G[b, :n, :n].T)
        assert np.abs(w[b] - np.linalg.eigvalsh(S)).max() < 1e-12 * np.abs(S).sum()
        assert np.abs(S @ V[b] - V[b] * w[b][None, :]).max() < 1e-12 * np.abs(S).sum()
    assert w[2, -1] == 1000.0 and abs(abs(V[2][10, -1]) - 1.0) < 1e-15
    assert np.isnan(wbuf[:, n:].cpu().numpy()).all()          # nothing written past n


def test_syev_batched_errors(gpu):
    torch = gpu
    G = torch.zeros((2, 65, 65), dtype=torch.float64, device="cuda")
    with pytest.raises(sci.SciError):
        sci.syev_batched(G)                                    # n above 64
    with pytest.raises(sci.SciError):
        sci.sci_syev_batched(0, 2, 4, G, 3, 65 * 65, G, 65, G, 65, 65 * 65)   # lda < n


def test_syev_batched_sweep_limit_counts_unconverged(gpu):
    """One sweep does not diagonalise a dense 24 x 24 matrix: every matrix is counted in
    not_converged, and the result is still an orthogonal similarity (w from V^T A V)."""
    torch = gpu
    rng = np.random.default_rng(9)
    A = rng.normal(size=(3, 24, 24))
    A = A + A.transpose(0, 2, 1)
    Ad = torch.from_numpy(A).cuda()
    w = torch.empty((3, 24), dtype=torch.float64, device="cuda")
    V = torch.empty((3, 24, 24), dtype=torch.float64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    sci.sci_syev_batched(0, 3, 24, Ad, 24, 24 * 24, w, 24, V, 24, 24 * 24, 1, cnt,
                         torch.cuda.current_stream().cuda_stream)
    assert int(cnt.item()) == 3
    Vn = V.cpu().numpy()
    for b in range(3):
        assert np.abs(Vn[b].T @ Vn[b] - np.eye(24)).max() < 1e-13
    cnt.zero_()
    sci.sci_syev_batched(0, 3, 24, Ad, 24, 24 * 24, w, 24, V, 24, 24 * 24, 30, cnt,
                         torch.cuda.current_stream().cuda_stream)
    assert int(cnt.item()) == 0
