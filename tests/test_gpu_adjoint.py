"""The differentiable solve: hand-written adjoint (grad_B = A^-T G, grad_A =
-grad_B X^T on the saved mixed-precision factor) against central finite
differences in FP64, the CPU oracle's adjoint and closed forms."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("nrhs", [3, 1])
def test_adjoint_matches_finite_differences_n64(hpl, orc, nrhs):
    """The differentiable-solve check at n = 64: every entry of the GPU's
    grad_A and grad_B (through the autograd layer) within 1e-6 relative of
    central finite differences in FP64 (numpy's LAPACK solve on the CPU), with
    no absolute floor."""
    import torch
    from _parity import fd_gradients, max_rel_err
    n, nb = 64, 32
    A = hpl.generate(21, hpl.STREAM_A, n, n, hpl.GEN_DIAG_DOMINANT)
    B = hpl.generate(21, hpl.STREAM_B, n, nrhs)
    Gn = np.random.default_rng(5).standard_normal((n, nrhs))
    G = torch.from_numpy(Gn).cuda()
    A_ = A.clone().requires_grad_(True)
    B_ = B.clone().requires_grad_(True)
    X = hpl.solve(A_, B_, nb=nb)
    (X * G).sum().backward()
    torch.cuda.synchronize()
    gA, gB = _np(A_.grad), _np(B_.grad)
    fdA, fdB = fd_gradients(_np(A), _np(B), Gn)
    ea, eb = max_rel_err(gA, fdA), max_rel_err(gB, fdB)
    assert ea <= 1e-6, ea
    assert eb <= 1e-6, eb


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
