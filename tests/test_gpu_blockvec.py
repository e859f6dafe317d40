"""libsci block-vector kernels (sci_bv_gemm_tn / sci_bv_gemm_nn) against torch FP64 products.

Tolerances: the FP64 policy differs from cuBLAS only in summation order (relative 1e-13
of sum |a_i b_i|); the paired-FP32 policy carries inputs to 2^-47 relative and sums in
paired FP32 folded to FP64, so 1e-12 of sum |a_i b_i|.
"""
import numpy as np
import pytest

from paper_2501_18185_gb300 import sci

pytestmark = pytest.mark.gpu

PRECS = [("f64", sci.SCI_PREC_F64, 1e-13), ("ds", sci.SCI_PREC_F64_DS, 1e-12)]


@pytest.fixture(scope="module")
def ctx(gpu):
    c = sci.sci_create(0, gpu.cuda.current_stream().cuda_stream)
    yield c
    sci.sci_destroy(c)


def _buf(torch, M, width, cap, seed, scale_rows=False):
    """A view [M, width] into a [M, cap] buffer (row stride cap), values of mixed size."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    B = torch.randn((M, cap), generator=g, dtype=torch.float64)
    if scale_rows:
        B *= torch.exp(-torch.rand((M, 1), generator=g, dtype=torch.float64) * 20)
    return B.cuda(), B.cuda()[:, :width]


@pytest.mark.parametrize("name,prec,rtol", PRECS)
@pytest.mark.parametrize("M,k,a", [(1, 1, 1), (31, 5, 3), (100_003, 96, 8), (65_537, 200, 8), (40_000, 128, 16),
                                   (9_999, 17, 13)])
def test_tn_matches_torch(gpu, ctx, name, prec, rtol, M, k, a):
    torch = gpu
    _, A = _buf(torch, M, k, k + 7, 1, scale_rows=True)
    _, B = _buf(torch, M, a, a + 3, 2)
    P = torch.empty((k, a), dtype=torch.float64, device="cuda")
    sci.sci_bv_gemm_tn(ctx, M, k, a, A, A.stride(0), B, B.stride(0), P, prec)
    ref = A.T @ B
    scale = A.abs().T @ B.abs()
    err = ((P - ref).abs() / scale.clamp_min(1e-300)).max().item()
    assert err < rtol, err
    # deterministic: a second call gives the same bits
    P2 = torch.empty_like(P)
    sci.sci_bv_gemm_tn(ctx, M, k, a, A, A.stride(0), B, B.stride(0), P2, prec)
    assert torch.equal(P, P2)


@pytest.mark.parametrize("name,prec,rtol", PRECS)
@pytest.mark.parametrize("M,k1,k2,a", [(1, 1, 0, 1), (33, 0, 4, 5), (100_003, 96, 96, 8), (50_001, 120, 16, 16),
                                       (7_777, 3, 250, 11)])
def test_nn_matches_torch(gpu, ctx, name, prec, rtol, M, k1, k2, a):
    torch = gpu
    g = torch.Generator(device="cpu").manual_seed(3)
    _, A1 = _buf(torch, M, max(k1, 1), max(k1, 1) + 2, 4, scale_rows=True)
    _, A2 = _buf(torch, M, max(k2, 1), max(k2, 1) + 5, 5)
    S1 = torch.randn((k1, a), generator=g, dtype=torch.float64).cuda()
    S2 = torch.randn((k2, a), generator=g, dtype=torch.float64).cuda()
    Cbuf, C = _buf(torch, M, a, a + 1, 6)
    C0 = C.clone()
    beta = -0.75
    sci.sci_bv_gemm_nn(ctx, M, a, A1 if k1 else None, A1.stride(0), k1, S1 if k1 else None, A2 if k2 else None,
                       A2.stride(0), k2, S2 if k2 else None, beta, C, C.stride(0), None, None, None, prec)
    ref = beta * C0
    scale = abs(beta) * C0.abs()
    if k1:
        ref = ref + A1[:, :k1] @ S1
        scale = scale + A1[:, :k1].abs() @ S1.abs()
    if k2:
        ref = ref + A2[:, :k2] @ S2
        scale = scale + A2[:, :k2].abs() @ S2.abs()
    err = ((C - ref).abs() / scale.clamp_min(1e-300)).max().item()
    assert err < rtol, err
    # the column beyond a is untouched
    assert torch.equal(Cbuf[:, a], _buf(torch, M, a, a + 1, 6)[0][:, a])


@pytest.mark.parametrize("name,prec,rtol", PRECS)
def test_nn_in_place_and_residual_epilogue(gpu, ctx, name, prec, rtol):
    """C aliasing A2 (the Gram-Schmidt update of a block inside the search-space buffer),
    and the residual epilogue: column sums of squares and the preconditioned output."""
    torch = gpu
    M, k, a, cap = 123_457, 40, 6, 64
    g = torch.Generator(device="cpu").manual_seed(7)
    V = torch.randn((M, cap), generator=g, dtype=torch.float64).cuda()
    V0 = V.clone()
    S1 = torch.randn((k, a), generator=g, dtype=torch.float64).cuda()
    Z = torch.randn((a, a - 2), generator=g, dtype=torch.float64).cuda()   # the block narrows
    S1n = S1[:, :a - 2].contiguous()
    sci.sci_bv_gemm_nn(ctx, M, a - 2, V[:, :k], cap, k, S1n, V[:, k:], cap, a, Z, 0.0, V[:, k:], cap,
                       None, None, None, prec)
    ref = V0[:, :k] @ S1n + V0[:, k:k + a] @ Z
    scale = V0[:, :k].abs() @ S1n.abs() + V0[:, k:k + a].abs() @ Z.abs()
    assert ((V[:, k:k + a - 2] - ref).abs() / scale).max().item() < rtol
    assert torch.equal(V[:, :k], V0[:, :k]) and torch.equal(V[:, k + a - 2:], V0[:, k + a - 2:])

    # residual: R = W Y - V (Y theta), colsq = ||R_j||^2, output R / (theta_j - d_m)
    W = torch.randn((M, k), generator=g, dtype=torch.float64).cuda()
    Y = torch.randn((k, a), generator=g, dtype=torch.float64).cuda()
    theta = torch.linspace(-3, -1, a, dtype=torch.float64).cuda()
    d = torch.randn(M, generator=g, dtype=torch.float64).cuda() - 2.0
    d[:5] = theta[0]                                   # exact hits take the 1e-8 clamp
    out = torch.empty((M, a), dtype=torch.float64, device="cuda")
    cs = torch.zeros(a, dtype=torch.float64, device="cuda")
    sci.sci_bv_gemm_nn(ctx, M, a, W, k, k, Y, V0, cap, k, -(Y * theta[None, :]), 0.0, out, a, d, theta, cs, prec)
    R = W @ Y - V0[:, :k] @ (Y * theta[None, :])
    assert torch.allclose(cs, (R * R).sum(0), rtol=1e-11, atol=0)
    den = theta[None, :] - d[:, None]
    den = torch.where(den.abs() < 1e-8, torch.full_like(den, 1e-8), den)
    # the quotient is taken in FP32
    assert ((out - R / den).abs() / (R / den).abs().clamp_min(1e-300)).max().item() < 2e-6


def test_bv_rejects_bad_arguments(gpu, ctx):
    torch = gpu
    A = torch.zeros((10, 4), dtype=torch.float64, device="cuda")
    P = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    for args in [(10, 4, 0), (10, 4, 17), (10, 300, 4), (10, 129, 16), (-1, 4, 4)]:
        with pytest.raises(sci.SciError) as e:
            sci.sci_bv_gemm_tn(ctx, *args, A, 4, A, 4, P, sci.SCI_PREC_F64)
        assert e.value.code == sci.SCI_ERR_ARG
    with pytest.raises(sci.SciError):
        sci.sci_bv_gemm_tn(ctx, 10, 4, 4, A, 3, A, 4, P, sci.SCI_PREC_F64)        # lda < k
    with pytest.raises(sci.SciError):
        sci.sci_bv_gemm_tn(ctx, 10, 4, 4, A, 4, A, 4, P, sci.SCI_PREC_F32_STORE_F64_ACC)
    with pytest.raises(sci.SciError):
        sci.sci_bv_gemm_nn(ctx, 10, 4, A, 4, 200, P, A, 4, 100, P, 0.0, A, 4, None, None, None, sci.SCI_PREC_F64)
    # M = 0: P is zeroed, nothing else happens
    P.fill_(1.0)
    sci.sci_bv_gemm_tn(ctx, 0, 4, 4, None, 4, None, 4, P, sci.SCI_PREC_F64)
    torch.cuda.synchronize()
    assert float(P.abs().sum()) == 0.0


@pytest.mark.parametrize("arith", ["f64", "ds"])
def test_davidson_block_kernels_match_torch_ops(gpu, arith):
    """The solver on libsci block kernels reaches the same energies as on torch products
    (dense stand-in for sigma, CI-like spectrum)."""
    torch = gpu
    from paper_2501_18185_gb300.davidson import TorchBlockOps, davidson

    n = 3000
    rng = np.random.default_rng(11)
    A = rng.normal(scale=0.05, size=(n, n))
    A = 0.5 * (A + A.T)
    A[np.diag_indices(n)] = np.sort(rng.uniform(-5.0, 5.0, n))
    At = torch.from_numpy(A).cuda()
    d = At.diagonal().contiguous()
    ref = np.linalg.eigvalsh(A)[:4]
    r1 = davidson(lambda X: At @ X, d, nroots=4, tol=1e-9, arith=arith)
    r2 = davidson(lambda X: At @ X, d, nroots=4, tol=1e-9, ops=TorchBlockOps())
    assert r1.converged and r2.converged
    assert np.abs(r1.energies.cpu().numpy() - ref).max() < 1e-10
    assert np.abs(r2.energies.cpu().numpy() - ref).max() < 1e-10
    X = r1.vectors
    assert float(torch.linalg.vector_norm(At @ X - X * r1.energies, dim=0).max()) <= 1e-9
    # orthonormal Ritz vectors
    assert float((X.T @ X - torch.eye(4, dtype=torch.float64, device="cuda")).abs().max()) < 1e-12


def test_block_ops_wider_than_one_call(gpu):
    """SciBlockOps cuts products wider than one kernel call (blocks of more than 16
    columns, more than 256 operand columns) into several calls; the results equal torch's."""
    torch = gpu
    from paper_2501_18185_gb300.davidson import SciBlockOps

    ops = SciBlockOps("cuda")
    g = torch.Generator(device="cpu").manual_seed(13)
    M = 20_011
    A = torch.randn((M, 300), generator=g, dtype=torch.float64).cuda()
    B = torch.randn((M, 37), generator=g, dtype=torch.float64).cuda()
    P = ops.tn(A, B)
    ref = (A.T @ B).cpu().numpy()
    assert np.abs(P - ref).max() < 1e-12 * np.abs(ref).max()
    S1 = np.random.default_rng(1).normal(size=(300, 21))
    S2 = np.random.default_rng(2).normal(size=(37, 21))
    C = torch.randn((M, 25), generator=g, dtype=torch.float64).cuda()
    C0 = C.clone()
    d = torch.randn(M, generator=g, dtype=torch.float64).cuda()
    sh = np.linspace(-2.0, -1.0, 21)
    cs = ops.nn(C, 21, A1=A, S1=S1, A2=B, S2=S2, beta=0.5, dg=d, shift=sh, colsq=True)
    R = A @ torch.from_numpy(S1).cuda() + B @ torch.from_numpy(S2).cuda() + 0.5 * C0[:, :21]
    assert np.allclose(cs, (R * R).sum(0).cpu().numpy(), rtol=1e-11)
    den = torch.from_numpy(sh).cuda()[None, :] - d[:, None]
    assert float(((C[:, :21] - R / den).abs() / (R / den).abs().clamp_min(1e-300)).max()) < 2e-6
    assert torch.equal(C[:, 21:], C0[:, 21:])


@pytest.mark.parametrize("nroots,max_space", [(20, None), (4, 200)])
def test_davidson_many_roots_and_wide_space(gpu, nroots, max_space):
    """More roots than one block call takes (20 > 16), and a search space wider than one
    residual call (2 x 200 > 256 columns): energies as dense eigh."""
    torch = gpu
    from paper_2501_18185_gb300.davidson import davidson

    n = 2500
    rng = np.random.default_rng(17)
    A = rng.normal(scale=0.05, size=(n, n))
    A = 0.5 * (A + A.T)
    A[np.diag_indices(n)] = np.sort(rng.uniform(-5.0, 5.0, n))
    At = torch.from_numpy(A).cuda()
    ref = np.linalg.eigvalsh(A)[:nroots]
    r = davidson(lambda X: At @ X, At.diagonal().contiguous(), nroots=nroots, tol=1e-8, max_space=max_space,
                 max_iter=500)
    assert r.converged
    assert np.abs(r.energies.cpu().numpy() - ref).max() < 1e-9
