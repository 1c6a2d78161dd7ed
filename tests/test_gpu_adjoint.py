"""The differentiable solve: hand-written adjoint (grad_B = A^-T G, grad_A =
-grad_B X^T on the saved mixed-precision factor) against central finite
differences in FP64, the CPU oracle's adjoint and closed forms."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


def test_adjoint_matches_finite_differences_n64(hpl, orc):
    import torch
    n, nrhs, nb = 64, 3, 32
    A = hpl.generate(21, hpl.STREAM_A, n, n, hpl.GEN_DIAG_DOMINANT)
    B = hpl.generate(21, hpl.STREAM_B, n, nrhs)
    G = torch.from_numpy(np.random.default_rng(5).standard_normal((n, nrhs))).cuda()
    A_ = A.clone().requires_grad_(True)
    B_ = B.clone().requires_grad_(True)
    X = hpl.solve(A_, B_, nb=nb)
    (X * G).sum().backward()
    gA, gB = _np(A_.grad), _np(B_.grad)

    def f(Am, Bm):
        Xm = hpl.solve(torch.from_numpy(np.asfortranarray(Am)).cuda().t().contiguous().t(),
                       torch.from_numpy(Bm).cuda(), nb=nb)
        return float((Xm * G).sum())

    A0, B0 = _np(A).copy(), _np(B).copy()
    for (i, j) in [(0, 0), (5, 40), (63, 2), (17, 17)]:
        h = 1e-6 * max(1.0, abs(A0[i, j]))
        Ap, Am = A0.copy(), A0.copy()
        Ap[i, j] += h
        Am[i, j] -= h
        fd = (f(Ap, B0) - f(Am, B0)) / (2 * h)
        assert abs(fd - gA[i, j]) <= 1e-6 * max(1.0, abs(gA[i, j])) + 1e-9, (i, j, fd, gA[i, j])
    for (i, c) in [(0, 0), (33, 2)]:
        h = 1e-6
        Bp, Bm = B0.copy(), B0.copy()
        Bp[i, c] += h
        Bm[i, c] -= h
        fd = (f(A0, Bp) - f(A0, Bm)) / (2 * h)
        assert abs(fd - gB[i, c]) <= 1e-6 * max(1.0, abs(gB[i, c])), (i, c, fd, gB[i, c])


@pytest.mark.parametrize("refine", [1, 0])     # GMRES per column; classic refinement on the block
@pytest.mark.parametrize("n,nrhs,nb", [(512, 4, 128), (1000, 2, 256), (777, 70, 128)])
def test_adjoint_matches_oracle(hpl, orc, n, nrhs, nb, refine):
    import torch
    A = hpl.generate(22, hpl.STREAM_A, n, n, hpl.GEN_DIAG_DOMINANT)
    B = hpl.generate(22, hpl.STREAM_B, n, nrhs)
    G = torch.from_numpy(np.random.default_rng(6).standard_normal((n, nrhs))).cuda()
    X, info, ws = hpl.mxp_solve(A, B, nb=nb, refine=refine)
    gB, gA, binfo = hpl.lu_solve_backward(A, X, G, ws, nb=nb, refine=refine)
    torch.cuda.synchronize()
    assert info.read()["status"] == 0 and binfo.read()["status"] == 0
    ogB, ogA = orc.adjoint(_np(A), _np(X), _np(G))
    assert np.abs(_np(gB) - ogB).max() <= 1e-9 * np.abs(ogB).max()
    assert np.abs(_np(gA) - ogA).max() <= 1e-9 * np.abs(ogA).max()


@pytest.mark.parametrize("refine", [1, 0])
def test_adjoint_closed_forms(hpl, refine):
    import torch
    n, nrhs = 48, 2
    d = torch.tensor([2.0 ** (k % 5 - 2) for k in range(n)], dtype=torch.float64, device="cuda")
    A = hpl.colmajor(n, n)
    A.zero_()
    A.diagonal().copy_(d)
    G = torch.arange(n * nrhs, dtype=torch.float64, device="cuda").reshape(n, nrhs) / 7.0
    B = torch.ones(n, nrhs, dtype=torch.float64, device="cuda")
    X, info, ws = hpl.mxp_solve(A, B, nb=16, refine=refine)
    gB, gA, _ = hpl.lu_solve_backward(A, X, G, ws, nb=16, refine=refine)
    torch.cuda.synchronize()
    assert torch.allclose(gB, G / d[:, None], rtol=1e-12, atol=0)
    assert torch.allclose(gA, -gB @ X.t(), rtol=1e-14, atol=1e-300)


@pytest.mark.slow
@pytest.mark.parametrize("refine", [1, 0])
def test_adjoint_n4096_64rhs(hpl, orc, refine):
    """The differentiable-solve configuration: n = 4096 dominant A, 64 right-hand
    sides, forward BF16 factor + FP64 refinement, backward on the saved factor,
    compared with the oracle's FP64 adjoint."""
    import torch
    n, nrhs, nb = 4096, 64, 2048
    A = hpl.generate(23, hpl.STREAM_A, n, n, hpl.GEN_DIAG_DOMINANT)
    B = hpl.generate(23, hpl.STREAM_B, n, nrhs)
    G = torch.from_numpy(np.random.default_rng(7).standard_normal((n, nrhs))).cuda()
    X, info, ws = hpl.mxp_solve(A, B, nb=nb, refine=refine)
    gB, gA, binfo = hpl.lu_solve_backward(A, X, G, ws, nb=nb, refine=refine)
    torch.cuda.synchronize()
    assert info.read()["status"] == 0 and binfo.read()["status"] == 0
    ogB, ogA = orc.adjoint(_np(A), _np(X), _np(G))
    assert np.abs(_np(gB) - ogB).max() <= 1e-9 * np.abs(ogB).max()
    assert np.abs(_np(gA) - ogA).max() <= 1e-9 * np.abs(ogA).max()
