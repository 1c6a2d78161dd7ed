"""GPU parity of the mixed-precision (HPL-MxP) solve against the CPU oracle,
through the C ABI: the block factor (D_k^-1, L21, updated blocks), the
refined solution, the scaled residual and the refinement iteration counts."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


def _np(t):
    return t.detach().cpu().numpy()


def _system(hpl, n, seed):
    A = hpl.generate(seed, hpl.STREAM_A, n, n, hpl.GEN_DIAG_DOMINANT)
    b = hpl.generate(seed, hpl.STREAM_B, n, 1)[:, 0].contiguous()
    return A, b


@pytest.mark.parametrize("n,nb", [(256, 64), (512, 128), (1000, 256), (300, 100), (7, 64), (1, 8), (2048, 512)])
def test_mxp_factor_matches_oracle(hpl, orc, n, nb):
    import torch
    A, b = _system(hpl, n, 3)
    x, info, ws = hpl.mxp_solve(A, b, nb=nb)
    torch.cuda.synchronize()
    F, Dinv = hpl.mxp_factor_views(ws, n, nb)
    Fg, Dg = _np(F).astype(np.float64), _np(Dinv).astype(np.float64)
    Fo, Do, info_o = orc.mxp_factor(_np(A), min(nb, n), orc.PREC_BF16)
    Fo, Do = Fo.astype(np.float64), Do.astype(np.float64)
    # diagonal inverses: split-BF16 Newton-Schulz on both sides, ~1e-5 accurate
    # (only the kb x kb part of each block slot is defined; a short last block
    # leaves the rest of its slot unused)
    nbe = min(nb, n)
    for k0 in range(0, n, nbe):
        kb = min(nbe, n - k0)
        dg, do = Dg[k0:k0 + kb, :kb], Do[k0:k0 + kb, :kb]
        assert np.abs(dg - do).max() <= 5e-5 * np.abs(do).max(), k0
    # L21 / updated blocks: operands rounded to BF16 on both sides; a rounding
    # decision may flip on values that differ in their last FP32 bits
    off = ~np.eye(n, dtype=bool)
    if n > 1:
        assert np.abs(Fg - Fo)[off].max() <= 2.0 ** -7 * np.abs(Fo[off]).max()
    assert np.abs(np.diag(Fg) - np.diag(Fo)).max() <= 1e-5 * np.abs(np.diag(Fo)).max()


@pytest.mark.parametrize("refine", [0, 1])
@pytest.mark.parametrize("n,nb", [(512, 128), (1536, 256), (2000, 512)])
def test_mxp_solution_matches_fp64(hpl, orc, n, nb, refine):
    import torch
    A, b = _system(hpl, n, 5)
    A0, b0 = _np(A).copy(order="F"), _np(b).copy()
    x, info, ws = hpl.mxp_solve(A, b, nb=nb, refine=refine)
    torch.cuda.synchronize()
    rec = info.read()
    assert rec["status"] == 0, rec
    xg = _np(x)[:, 0]
    sr = orc.scaled_residual(A0, xg, b0)              # independent FP64 check on the CPU
    assert sr < 16 and rec["scaled_residual"] < 16
    x64, _ = orc.solve(A0, b0)
    bound = 2 * 16 * n * EPS * np.linalg.cond(A0, np.inf)
    assert np.abs(xg - x64).max() / np.abs(x64).max() < bound
    emu = orc.mxp_solve(A0, b0, nb, prec=orc.PREC_BF16, refine=refine)
    assert abs(rec["iters"] - emu["iters"]) <= 2, (rec, emu["iters"])


def test_mxp_multiple_rhs(hpl, orc):
    import torch
    n, nb, nrhs = 768, 256, 3
    A = hpl.generate(8, hpl.STREAM_A, n, n, hpl.GEN_DIAG_DOMINANT)
    B = hpl.generate(8, hpl.STREAM_B, n, nrhs)
    X, info, _ = hpl.mxp_solve(A, B, nb=nb)
    torch.cuda.synchronize()
    assert info.read()["status"] == 0
    A0, B0, X0 = _np(A), _np(B), _np(X)
    for c in range(nrhs):
        assert orc.scaled_residual(A0, X0[:, c], B0[:, c]) < 16


def test_mxp_not_converged_reports_status(hpl):
    import torch
    n = 256
    A = hpl.generate(4, hpl.STREAM_A, n, n, hpl.GEN_DIAG_DOMINANT)
    b = hpl.generate(4, hpl.STREAM_B, n, 1)[:, 0].contiguous()
    x, info, _ = hpl.mxp_solve(A, b, nb=64, refine=0, max_iter=1, tol=1e-30)
    torch.cuda.synchronize()
    rec = info.read()
    assert rec["status"] == 4 and rec["iters"] == 1


def test_mxp_rejects_invalid(hpl):
    import ctypes
    import torch
    lib = hpl.load()
    opts = hpl.make_opts(nb=64, prec=7)                # no such precision: refused before any launch
    assert lib.mxp_solve(64, 1, 8, 64, 0, 8, 64, 8, 64, ctypes.byref(opts), 8, 1 << 30, 8, None) == 1
    opts = hpl.make_opts(nb=64)
    assert lib.mxp_solve(64, 1, None, 64, 0, 8, 64, 8, 64, ctypes.byref(opts), 8, 1 << 30, 8, None) == 1
    assert lib.mxp_solve(64, 1, 8, 64, 0, 8, 64, 8, 64, ctypes.byref(opts), 8, 16, 8, None) == 6


@pytest.mark.slow
def test_mxp_full_size_n98304(hpl, orc):
    """n = 98304, NB = 1536: the oracle cannot factor this size; it checks the
    GPU solution through the scaled residual computed on the CPU with A
    regenerated from the seed."""
    import torch
    n, nb, seed = 98304, 1536, 1
    A = hpl.generate(seed, hpl.STREAM_A, n, n, hpl.GEN_DIAG_DOMINANT)
    b = hpl.generate(seed, hpl.STREAM_B, n, 1)[:, 0].contiguous()
    x, info, ws = hpl.mxp_solve(A, b, nb=nb)
    torch.cuda.synchronize()
    rec = info.read()
    assert rec["status"] == 0 and rec["scaled_residual"] < 16, rec
    del ws, A
    torch.cuda.empty_cache()
    assert orc.scaled_residual_gen(seed, n, True, _np(x)[:, 0], _np(b)) < 16


@pytest.mark.parametrize("n,nb", [(512, 128), (1000, 256)])
def test_mxp_fp8_variant(hpl, orc, n, nb):
    """FP8 E4M3 trailing update: factor blocks vs the oracle's FP8 emulation,
    FP64 solution, and iteration counts (reported; within 2 of the oracle)."""
    import torch
    A, b = _system(hpl, n, 12)
    A0, b0 = _np(A).copy(order="F"), _np(b).copy()
    x, info, ws = hpl.mxp_solve(A, b, nb=nb, prec=hpl.PREC_FP8_E4M3)
    torch.cuda.synchronize()
    rec = info.read()
    assert rec["status"] == 0, rec
    xg = _np(x)[:, 0]
    assert orc.scaled_residual(A0, xg, b0) < 16
    x64, _ = orc.solve(A0, b0)
    assert np.abs(xg - x64).max() / np.abs(x64).max() < 2 * 16 * n * EPS * np.linalg.cond(A0, np.inf)
    F, _ = hpl.mxp_factor_views(ws, n, nb)
    Fo, _, _ = orc.mxp_factor(A0, nb, orc.PREC_FP8)
    Fg = _np(F).astype(np.float64)
    off = ~np.eye(n, dtype=bool)
    # updated entries: FP8 rounding decisions may differ on nearly equal inputs
    assert np.abs(Fg - Fo)[off].max() <= 2.0 ** -3 * np.abs(Fo[off]).max()
    assert np.abs(np.diag(Fg) - np.diag(Fo)).max() <= 1e-4 * np.abs(np.diag(Fo)).max()
    emu = orc.mxp_solve(A0, b0, nb, prec=orc.PREC_FP8, refine=1)
    assert abs(rec["iters"] - emu["iters"]) <= 2
