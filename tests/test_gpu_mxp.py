"""GPU parity of the mixed-precision (HPL-MxP) solve against the CPU oracle,
through the C ABI: the block factor (D_k^-1, L21, updated blocks), the
refined solution, the scaled residual and the refinement iteration counts."""
import numpy as np
import pytest
from _parity import (BLOCK_VS_PLAIN_BERR, assert_blocks_close, block_lu_backward_error,
                     plain_lu_backward_error)

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53
# Per-part tolerances of the GPU block factor against the oracle's block
# emulation, each relative to the largest entry of the same part of the same
# step (L21, U12, the off-diagonal and the diagonal of D_k). Operands are
# rounded to the low precision on both sides, and a rounding decision may flip
# on values that differ in their last FP32 bits: one flip moves an entry by
# one unit in the last place of the operand format, relative to that entry.
TOL_BF16 = dict(l21=2.0 ** -7, u12=2.0 ** -7, doff=2.0 ** -7, ddiag=1e-5)
TOL_FP8 = dict(l21=2.0 ** -7, u12=2.0 ** -3, doff=2.0 ** -3, ddiag=1e-4)    # L21 keeps BF16 operands
TOL_FP16 = dict(l21=2.0 ** -10, u12=2.0 ** -10, doff=2.0 ** -10, ddiag=1e-5)
TOL_TF32 = TOL_FP16                  # the same 10 fraction bits, FP32's exponent range
# BF16 storage rounds every stored value (L21 and the updated trailing matrix)
# to BF16 after each step, so a rounding flip in an earlier step carries into
# the inputs of later ones: a few units of BF16's 2^-8 relative spacing
# (measured: 1.35 x 2^-7 on L21 of the third step at n = 1000, NB = 256).
TOL_BF16_STORAGE = dict(l21=2.0 ** -6, u12=2.0 ** -6, doff=2.0 ** -6, ddiag=2.0 ** -7)


def _check_against_plain(orc, A0, Fg, nb, prec):
    """The GPU block factor against the plain LU of the paper's order (FP32
    panel and U12 solve, rounded update operands, FP32 accumulation): its
    backward error within the stated factor of the plain factor's, and not
    below a quarter of it (the low precision really is used)."""
    Fp, _ = orc.mxp_lu_plain(A0, nb, prec)
    ep = plain_lu_backward_error(A0, Fp)
    eg = block_lu_backward_error(A0, Fg, nb)
    assert ep / 4 <= eg <= BLOCK_VS_PLAIN_BERR[prec] * ep, (eg, ep)


def _np(t):
    return t.detach().cpu().numpy()


def _system(hpl, n, seed):
    A = hpl.generate(seed, hpl.STREAM_A, n, n, hpl.GEN_DIAG_DOMINANT)
    b = hpl.generate(seed, hpl.STREAM_B, n, 1)[:, 0].contiguous()
    return A, b


@pytest.mark.parametrize("n,nb", [(256, 64), (512, 128), (1000, 256), (300, 100), (7, 64), (1, 8), (2048, 512),
                                  (2560, 256)])     # updates of >= 76 tiles of 256 x 256: the pair kernel
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
    # L21, U12 and D_k, each against its own scale
    assert_blocks_close(Fg, Fo, nbe, **TOL_BF16)
    if n > nbe:                      # one block: no low-precision product at all
        _check_against_plain(orc, _np(A), Fg, nbe, 0)


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
    plain = orc.mxp_solve_plain(A0, b0, nb, prec=orc.PREC_BF16, refine=refine)
    assert plain["status"] == 0
    assert abs(rec["iters"] - plain["iters"]) <= 2, (rec, plain["iters"])


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
    """Argument errors are refused on the host before anything is launched.
    Every call gets real device buffers large enough for the call, so that
    even a missing check could not make a kernel touch memory it does not own."""
    import ctypes
    import torch
    lib = hpl.load()
    n = 64
    A, b = _system(hpl, n, 2)
    x = hpl.colmajor(n, 1)
    info = hpl.Info()
    opts = hpl.make_opts(nb=64)
    need = lib.mxp_workspace_size(n, 1, ctypes.byref(opts))
    ws = hpl.workspace(need + 512, A.device)
    st = torch.cuda.current_stream().cuda_stream
    args = lambda o, ldb=n, wp=ws.data_ptr(), wb=need: (
        n, 1, A.data_ptr(), n, 0, b.data_ptr(), ldb, x.data_ptr(), n, ctypes.byref(o), wp, wb, info.ptr(), st)
    bad = hpl.make_opts(nb=64, prec=7)                 # no such precision
    assert lib.mxp_solve(*args(bad)) == 1
    assert lib.mxp_solve(*args(opts, ldb=n - 1)) == 1  # ldb < n
    assert lib.mxp_solve(*args(opts, wb=16)) == 6      # workspace too small
    assert lib.mxp_solve(*args(opts, wp=ws.data_ptr() + 8)) == 1    # workspace not 256-byte aligned
    torch.cuda.synchronize()


@pytest.mark.slow
@pytest.mark.parametrize("prec,stored,storage", [(0, True, 0), (1, True, 0), (2, True, 0), (0, False, 0), (0, True, 1),
                                                (0, False, 1)])
def test_mxp_full_size_n98304(hpl, orc, prec, stored, storage):
    """n = 98304, NB = 3072 (the benchmark's launch configuration), BF16, FP8
    and FP16 updates, FP32 or BF16 storage, A stored or regenerated by the library: the oracle cannot
    factor this size; it checks the GPU solution through the scaled residual
    computed on the CPU with A regenerated from the seed."""
    import torch
    n, nb, seed = 98304, 3072, 1
    A = hpl.generate(seed, hpl.STREAM_A, n, n, hpl.GEN_DIAG_DOMINANT) if stored else None
    b = hpl.generate(seed, hpl.STREAM_B, n, 1)[:, 0].contiguous()
    x, info, ws = hpl.mxp_solve(A, b, nb=nb, prec=prec, seed=seed, storage=storage)
    torch.cuda.synchronize()
    rec = info.read()
    assert rec["status"] == 0 and rec["scaled_residual"] < 16, rec
    del ws, A
    torch.cuda.empty_cache()
    assert orc.scaled_residual_gen(seed, n, True, _np(x)[:, 0], _np(b)) < 16


@pytest.mark.parametrize("n,nrhs,nb,prec", [(1000, 7, 256, 0), (777, 70, 128, 1), (130, 2, 64, 0)])
def test_mxp_block_refinement(hpl, orc, n, nrhs, nb, prec):
    """Several right-hand sides with classic refinement: the columns are refined
    together (block residual, block preconditioner); every column meets the
    residual test (recomputed by the oracle) and the forward-error bound."""
    import torch
    A = hpl.generate(9, hpl.STREAM_A, n, n, hpl.GEN_DIAG_DOMINANT)
    B = hpl.generate(9, hpl.STREAM_B, n, nrhs)
    X, info, ws = hpl.mxp_solve(A, B, nb=nb, refine=hpl.REFINE_IR, prec=prec)
    torch.cuda.synchronize()
    rec = info.read()
    assert rec["status"] == 0 and rec["scaled_residual"] < 16, rec
    A0, B0, Xg = _np(A).copy(order="F"), _np(B), _np(X)
    kappa = np.linalg.cond(A0, np.inf)
    for c in range(nrhs):
        assert orc.scaled_residual(A0, Xg[:, c].copy(), B0[:, c].copy()) < 16, c
        x64, _ = orc.solve(A0, B0[:, c].copy())
        assert np.abs(Xg[:, c] - x64).max() / np.abs(x64).max() < 2 * 16 * n * EPS * kappa, c
    # the same columns refined one by one (GMRES) agree to the same bound
    Xs, info1, _ = hpl.mxp_solve(A, B, nb=nb, prec=prec)
    torch.cuda.synchronize()
    assert info1.read()["status"] == 0
    assert np.abs(_np(Xs) - Xg).max() / np.abs(Xg).max() < 4 * 16 * n * EPS * kappa


def test_mxp_regenerated_matrix_several_rhs(hpl, orc):
    """A = NULL with several right-hand sides and classic refinement: the
    block residual needs the stored matrix, so the columns are refined one by
    one against the regenerated matrix."""
    import torch
    n, nrhs, seed = 300, 3, 4
    B = hpl.generate(seed, hpl.STREAM_B, n, nrhs)
    X, info, _ = hpl.mxp_solve(None, B, nb=64, refine=hpl.REFINE_IR, seed=seed)
    torch.cuda.synchronize()
    assert info.read()["status"] == 0
    for c in range(nrhs):
        assert orc.scaled_residual_gen(seed, n, True, _np(X)[:, c].copy(), _np(B)[:, c].copy()) < 16


@pytest.mark.parametrize("n,nb,prec", [(1000, 256, 0), (777, 128, 1), (64, 64, 0), (1, 8, 0), (900, 128, 2)])
def test_mxp_regenerated_matrix(hpl, orc, n, nb, prec):
    """A = NULL: the library generates the FP32 working copy itself and
    regenerates A in every FP64 residual. The factor must be bit-identical to
    the one built from the stored FP64 matrix (same FP32 rounding of the same
    entries, same diagonal), and x must meet the same bounds."""
    import torch
    seed = 5
    A, b = _system(hpl, n, seed)
    x1, i1, ws1 = hpl.mxp_solve(A, b, nb=nb, prec=prec)
    x2, i2, ws2 = hpl.mxp_solve(None, b, nb=nb, prec=prec, seed=seed)
    torch.cuda.synchronize()
    F1, D1 = hpl.mxp_factor_views(ws1, n, nb)
    F2, D2 = hpl.mxp_factor_views(ws2, n, nb)
    assert torch.equal(F1, F2)
    r1, r2 = i1.read(), i2.read()
    assert r2["status"] == 0 and r2["scaled_residual"] < 16, r2
    assert abs(r2["iters"] - r1["iters"]) <= 1, (r1, r2)
    A0, b0 = _np(A).copy(order="F"), _np(b).copy()
    xg = _np(x2)[:, 0]
    assert orc.scaled_residual_gen(seed, n, True, xg, b0) < 16
    x64, _ = orc.solve(A0, b0)
    assert np.abs(xg - x64).max() / np.abs(x64).max() < 2 * 16 * n * EPS * np.linalg.cond(A0, np.inf)


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
    assert_blocks_close(Fg, Fo, nb, **TOL_FP8)
    _check_against_plain(orc, A0, Fg, nb, 1)
    emu = orc.mxp_solve(A0, b0, nb, prec=orc.PREC_FP8, refine=1)
    assert abs(rec["iters"] - emu["iters"]) <= 2
    plain = orc.mxp_solve_plain(A0, b0, nb, prec=orc.PREC_FP8, refine=1)
    assert abs(rec["iters"] - plain["iters"]) <= 2


@pytest.mark.parametrize("n,nb", [(512, 128), (1000, 256), (2560, 256), (300, 100)])
def test_mxp_fp16_variant(hpl, orc, n, nb):
    """FP16 operands (scaled per row / column) in the panel product and the
    trailing update: factor vs the oracle's FP16 emulation, about 8x less
    factorization error than BF16, FP64 solution, iteration counts."""
    import torch
    A, b = _system(hpl, n, 13)
    A0, b0 = _np(A).copy(order="F"), _np(b).copy()
    x, info, ws = hpl.mxp_solve(A, b, nb=nb, prec=hpl.PREC_FP16)
    torch.cuda.synchronize()
    rec = info.read()
    assert rec["status"] == 0, rec
    xg = _np(x)[:, 0]
    assert orc.scaled_residual(A0, xg, b0) < 16
    x64, _ = orc.solve(A0, b0)
    assert np.abs(xg - x64).max() / np.abs(x64).max() < 2 * 16 * n * EPS * np.linalg.cond(A0, np.inf)
    F, _ = hpl.mxp_factor_views(ws, n, nb)
    Fg = _np(F).astype(np.float64)
    Fo, _, _ = orc.mxp_factor(A0, nb, orc.PREC_FP16)
    assert_blocks_close(Fg, Fo, nb, **TOL_FP16)
    _check_against_plain(orc, A0, Fg, nb, 2)
    # backward error of the GPU factor against the BF16 factor's
    _, _, wsb = hpl.mxp_solve(A, b, nb=nb, prec=hpl.PREC_BF16)
    torch.cuda.synchronize()
    Fb, _ = hpl.mxp_factor_views(wsb, n, nb)

    def berr(Fx):
        L, U = orc.block_lu_parts(_np(Fx).astype(np.float32), nb)
        return np.abs(A0 - L @ U).max()
    assert berr(F) < berr(Fb) / 4
    emu = orc.mxp_solve(A0, b0, nb, prec=orc.PREC_FP16, refine=1)
    assert abs(rec["iters"] - emu["iters"]) <= 2


@pytest.mark.parametrize("n,nb", [(512, 128), (1000, 256), (2560, 256), (300, 100), (301, 64)])
def test_mxp_bf16_storage(hpl, orc, n, nb):
    """BF16 storage of the working matrix: the factor (BF16 values) against the
    oracle's BF16-storage emulation, the FP64 solution, iteration counts; the
    regenerated-A factor is bit-identical to the stored-A one."""
    import torch
    A, b = _system(hpl, n, 21)
    A0, b0 = _np(A).copy(order="F"), _np(b).copy()
    x, info, ws = hpl.mxp_solve(A, b, nb=nb, storage=hpl.STORAGE_BF16)
    torch.cuda.synchronize()
    rec = info.read()
    assert rec["status"] == 0, rec
    xg = _np(x)[:, 0]
    assert orc.scaled_residual(A0, xg, b0) < 16
    x64, _ = orc.solve(A0, b0)
    assert np.abs(xg - x64).max() / np.abs(x64).max() < 2 * 16 * n * EPS * np.linalg.cond(A0, np.inf)
    F, Dinv = hpl.mxp_factor_views(ws, n, nb, storage=hpl.STORAGE_BF16)
    assert F.dtype == torch.bfloat16
    Fg = F.float().cpu().numpy().astype(np.float64)
    Fo, Do, _ = orc.mxp_factor(A0, nb, orc.PREC_BF16, storage=orc.STORAGE_BF16)
    # BF16 rounding of values whose FP32 computations differ in their last bits
    assert_blocks_close(Fg, Fo, nb, **TOL_BF16_STORAGE)
    # the first block is the BF16 rounding of A itself (one rounding from FP64)
    k = min(nb, n)
    first = np.array([orc.round_bf16_d(v) for v in A0[:k, 0]])
    assert np.array_equal(Fg[:k, 0], first)
    emu = orc.mxp_solve(A0, b0, nb, prec=orc.PREC_BF16, refine=1, storage=orc.STORAGE_BF16)
    assert abs(rec["iters"] - emu["iters"]) <= 2
    # regenerated A, BF16 storage: the same factor bit for bit
    x2, i2, ws2 = hpl.mxp_solve(None, b, nb=nb, seed=21, storage=hpl.STORAGE_BF16)
    torch.cuda.synchronize()
    F2, D2 = hpl.mxp_factor_views(ws2, n, nb, storage=hpl.STORAGE_BF16)
    assert torch.equal(F2, F)
    for k0 in range(0, n, k):              # only the kb x kb part of each inverse slot is defined
        kb = min(k, n - k0)
        assert torch.equal(D2[k0:k0 + kb, :kb], Dinv[k0:k0 + kb, :kb])
    assert i2.read()["status"] == 0


def test_mxp_bf16_storage_adjoint_and_rejects(hpl, orc):
    """The adjoint from a BF16-stored factor against the oracle's FP64
    adjoint; BF16 storage with FP8 or FP16 operands is refused."""
    import ctypes
    import torch
    n, nb = 700, 128
    A, b = _system(hpl, n, 22)
    x, info, ws = hpl.mxp_solve(A, b, nb=nb, storage=hpl.STORAGE_BF16)
    g = torch.from_numpy(np.random.default_rng(3).standard_normal(n)).cuda()
    gB, gA, inf2 = hpl.lu_solve_backward(A, x, g, ws, nb=nb, storage=hpl.STORAGE_BF16)
    torch.cuda.synchronize()
    assert inf2.read()["status"] == 0
    want_b, want_a = orc.adjoint(_np(A), _np(x).reshape(n, 1), _np(g).reshape(n, 1))
    gb = _np(gB)[:, 0]
    assert np.abs(gb - want_b[:, 0]).max() <= 1e-9 * np.abs(want_b).max()
    lib = hpl.load()
    for prec in (hpl.PREC_FP8_E4M3, hpl.PREC_FP16):
        opts = hpl.make_opts(nb=nb, prec=prec, storage=hpl.STORAGE_BF16)
        X = hpl.colmajor(n, 1)
        st = lib.mxp_solve(n, 1, A.data_ptr(), n, 0, b.data_ptr(), n, X.data_ptr(), n, ctypes.byref(opts),
                           ws.data_ptr(), ws.numel(), hpl.Info().ptr(), torch.cuda.current_stream().cuda_stream)
        assert st == 1


def _a32_view(ws, n, need):
    """The FP32 copy of A that opts.inner = FP32 keeps at the end of the
    workspace (followed by 16 x n FP64 chunk sums), as an n x n view."""
    al = lambda x: (x + 255) // 256 * 256
    off = need - al(8 * 16 * n) - al(4 * n * n)
    return ws[off:off + 4 * n * n].view(__import__("torch").float32).view(n, n).t()


@pytest.mark.parametrize("n,nb,prec,stored,storage", [(1000, 256, 0, True, 0), (777, 128, 1, True, 0),
                                                      (900, 128, 2, True, 0), (1000, 256, 0, False, 0),
                                                      (1000, 256, 0, True, 1), (301, 64, 0, False, 1),
                                                      (2048, 512, 0, True, 0)])
def test_mxp_inner_fp32(hpl, orc, n, nb, prec, stored, storage):
    """GMRES's inner products on the FP32 copy of A (opts.inner = FP32): the
    copy is the FP32 rounding of A (stored or regenerated), the factor is the
    same as with FP64 inner products, x meets the FP64 bounds recomputed by the
    oracle, and the iteration counts are within 2 of the oracle's emulation of
    the same option."""
    import ctypes
    import torch
    seed = 31
    A, b = _system(hpl, n, seed)
    A0, b0 = _np(A).copy(order="F"), _np(b).copy()
    x1, i1, ws1 = hpl.mxp_solve(A if stored else None, b, nb=nb, prec=prec, seed=seed, storage=storage,
                                inner=hpl.INNER_FP32)
    x0, i0, ws0 = hpl.mxp_solve(A if stored else None, b, nb=nb, prec=prec, seed=seed, storage=storage)
    torch.cuda.synchronize()
    r1 = i1.read()
    assert r1["status"] == 0 and r1["scaled_residual"] < 16, r1
    opts = hpl.make_opts(nb=nb, prec=prec, storage=storage, inner=hpl.INNER_FP32)
    need = hpl.load().mxp_workspace_size(n, 1, ctypes.byref(opts))
    assert torch.equal(_a32_view(ws1, n, need), A.float())
    F1, _ = hpl.mxp_factor_views(ws1, n, nb, storage=storage)
    F0, _ = hpl.mxp_factor_views(ws0, n, nb, storage=storage)
    assert torch.equal(F1, F0)
    xg = _np(x1)[:, 0]
    assert orc.scaled_residual(A0, xg, b0) < 16
    x64, _ = orc.solve(A0, b0)
    assert np.abs(xg - x64).max() / np.abs(x64).max() < 2 * 16 * n * EPS * np.linalg.cond(A0, np.inf)
    emu = orc.mxp_solve(A0, b0, nb, prec=prec, refine=1, storage=storage, inner=orc.INNER_FP32)
    assert emu["status"] == 0
    assert abs(r1["iters"] - emu["iters"]) <= 2, (r1, emu["iters"])


def test_mxp_inner_rejects_unknown(hpl):
    import ctypes
    import torch
    lib = hpl.load()
    n = 64
    A, b = _system(hpl, n, 2)
    x = hpl.colmajor(n, 1)
    info = hpl.Info()
    opts = hpl.make_opts(nb=64)
    need = lib.mxp_workspace_size(n, 1, ctypes.byref(opts))
    ws = hpl.workspace(need + 512, A.device)
    bad = hpl.make_opts(nb=64, inner=2)
    st = lib.mxp_solve(n, 1, A.data_ptr(), n, 0, b.data_ptr(), n, x.data_ptr(), n, ctypes.byref(bad), ws.data_ptr(),
                       need, info.ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 1


@pytest.mark.parametrize("n,nb", [(512, 128), (1000, 256), (2560, 256), (300, 100)])
def test_mxp_tf32_variant(hpl, orc, n, nb):
    """TF32 operands (no scales) in the panel product and the trailing update:
    factor parts against the oracle's TF32 emulation, backward error against
    the plain emulation, the FP64 solution and iteration counts."""
    import torch
    A, b = _system(hpl, n, 14)
    A0, b0 = _np(A).copy(order="F"), _np(b).copy()
    x, info, ws = hpl.mxp_solve(A, b, nb=nb, prec=hpl.PREC_TF32)
    torch.cuda.synchronize()
    rec = info.read()
    assert rec["status"] == 0, rec
    xg = _np(x)[:, 0]
    assert orc.scaled_residual(A0, xg, b0) < 16
    x64, _ = orc.solve(A0, b0)
    assert np.abs(xg - x64).max() / np.abs(x64).max() < 2 * 16 * n * EPS * np.linalg.cond(A0, np.inf)
    F, _ = hpl.mxp_factor_views(ws, n, nb)
    Fg = _np(F).astype(np.float64)
    Fo, _, _ = orc.mxp_factor(A0, nb, orc.PREC_TF32)
    assert_blocks_close(Fg, Fo, nb, **TOL_TF32)
    _check_against_plain(orc, A0, Fg, nb, orc.PREC_TF32)
    emu = orc.mxp_solve(A0, b0, nb, prec=orc.PREC_TF32, refine=1)
    assert abs(rec["iters"] - emu["iters"]) <= 2
    plain = orc.mxp_solve_plain(A0, b0, nb, prec=orc.PREC_TF32, refine=1)
    assert abs(rec["iters"] - plain["iters"]) <= 2


def test_mxp_tf32_rejects_bf16_storage(hpl):
    import ctypes
    import torch
    lib = hpl.load()
    n = 64
    A, b = _system(hpl, n, 2)
    x = hpl.colmajor(n, 1)
    opts = hpl.make_opts(nb=64, prec=hpl.PREC_TF32, storage=hpl.STORAGE_BF16)
    ws = hpl.workspace(lib.mxp_workspace_size(n, 1, ctypes.byref(opts)) + 512, A.device)
    st = lib.mxp_solve(n, 1, A.data_ptr(), n, 0, b.data_ptr(), n, x.data_ptr(), n, ctypes.byref(opts), ws.data_ptr(),
                       ws.numel(), hpl.Info().ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 1


@pytest.mark.parametrize("n,nb", [(1000, 256), (2600, 512), (777, 128), (5000, 1024)])
def test_mxp_l21_copy_from_the_product_epilogue(hpl, n, nb):
    """With the bulk-tensor epilogue the L21 product also writes L21's BF16
    operand copy for the trailing update (no separate transposing pass); with
    the per-thread epilogue that copy is made by the conversion kernel. Both
    factorizations must be bit-identical (ragged last blocks included: the
    copy's padding columns are zeros)."""
    import torch
    A, b = _system(hpl, n, 7)
    x0, i0, ws0 = hpl.mxp_solve(A, b, nb=nb, prec=0)
    hpl.gemm_config(hpl.GEMM_EPILOGUE, 1)
    try:
        x1, i1, ws1 = hpl.mxp_solve(A, b, nb=nb, prec=0)
    finally:
        hpl.gemm_config(hpl.GEMM_EPILOGUE, 0)
    torch.cuda.synchronize()
    F0, D0 = hpl.mxp_factor_views(ws0, n, nb)
    F1, D1 = hpl.mxp_factor_views(ws1, n, nb)
    assert torch.equal(F0, F1) and torch.equal(D0, D1)
    assert torch.equal(x0, x1)
    assert i0.read()["status"] == 0


@pytest.mark.parametrize("storage", [0, 1])
def test_mxp_factor_same_bits_with_one_or_two_atom_stages(hpl, storage):
    """The pair kernel's pipeline stages of one or two swizzle atoms issue the
    same MMAs in the same order: the factor must not change, for an FP32
    working matrix (bulk-tensor epilogue) and a BF16 one (per-thread epilogue
    on a BF16 C)."""
    import torch
    n, nb = 5000, 512
    A, b = _system(hpl, n, 11)
    F = []
    try:
        for atoms in (1, 2):
            hpl.gemm_config(hpl.GEMM_PAIR_ATOMS, atoms)
            x, i, ws = hpl.mxp_solve(A, b, nb=nb, prec=0, storage=storage)
            torch.cuda.synchronize()
            assert i.read()["status"] == 0
            F.append(hpl.mxp_factor_views(ws, n, nb, storage=storage)[0].clone())
    finally:
        hpl.gemm_config(hpl.GEMM_PAIR_ATOMS, 2)
    assert torch.equal(F[0], F[1])
