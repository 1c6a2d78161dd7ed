"""GPU parity of the FP64 HPL path (generator, lu_factor, lu_solve, residual)
against the CPU oracle, through the C ABI."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


def _to_np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("m,ncols,ld,kind", [(1, 1, 1, 0), (7, 3, 9, 0), (300, 7, 300, 0), (257, 257, 260, 1),
                                              (1000, 1000, 1000, 1), (1, 1, 1, 1)])
def test_generate_bit_exact(hpl, orc, m, ncols, ld, kind):
    import torch
    A = hpl.colmajor(m, ncols, ld=ld)
    hpl.generate(5, hpl.STREAM_A, m, ncols, kind, out=A)
    torch.cuda.synchronize()
    want = orc.generate(5, orc.STREAM_A, m, ncols, dominant=bool(kind))
    assert np.array_equal(_to_np(A), want)


def test_generate_large_sampled(hpl, orc):
    import torch
    n = 8192
    A = hpl.generate(1, hpl.STREAM_A, n, n, hpl.GEN_DIAG_DOMINANT)
    torch.cuda.synchronize()
    want = orc.generate(1, orc.STREAM_A, n, n, dominant=True)
    assert np.array_equal(_to_np(A), want)


def _factor_and_check(hpl, orc, n, nb, lookahead, seed=1, emu=0):
    import torch
    A = hpl.generate(seed, hpl.STREAM_A, n, n)
    A0 = _to_np(A).copy(order="F")
    ipiv, info = hpl.lu_factor(A, nb=nb, lookahead=lookahead, fp64_emulation=emu)
    torch.cuda.synchronize()
    rec = info.read()
    assert rec["status"] == 0 and rec["info"] == 0, rec
    LU = _to_np(A)
    LUo, ipo, info_o, gap = orc.getrf(A0)
    gp = _to_np(ipiv)
    if gap > 1e-12:
        assert np.array_equal(gp, ipo), np.nonzero(gp != ipo)[0][:10]
    # backward error of the GPU factors
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    rowmap = orc.perm_from_ipiv(gp)
    err = np.abs(A0[rowmap, :] - L @ U).sum(axis=1).max()
    assert err / (n * EPS * np.abs(A0).sum(axis=1).max()) < 10
    assert np.abs(np.tril(LU, -1)).max() <= 1.0
    return A0, A, ipiv, LUo, ipo


@pytest.mark.parametrize("n,nb,la", [(1, 64, 0), (2, 64, 1), (3, 64, 1), (7, 64, 1), (33, 32, 1), (64, 64, 0),
                                      (65, 64, 1), (127, 64, 1), (300, 48, 1), (1000, 64, 1), (1024, 64, 0),
                                      (1024, 64, 1), (1500, 256, 1), (2048, 512, 1)])
def test_lu_factor_matches_oracle(hpl, orc, n, nb, la):
    _factor_and_check(hpl, orc, n, nb, la)


@pytest.mark.parametrize("n,nb,la", [(1000, 64, 1), (777, 128, 0), (2048, 256, 1), (3000, 256, 1)])
def test_lu_fp64_emulation_matches_oracle(hpl, orc, n, nb, la):
    """The trailing update on the BF16 tensor cores with FP64 accuracy (sliced
    products): pivots equal the oracle's, the backward error is at the FP64
    level, and the factors agree with the DFMA factorization to rounding."""
    import torch
    A0, A, ipiv, LUo, ipo = _factor_and_check(hpl, orc, n, nb, la, seed=3, emu=1)
    An = hpl.generate(3, hpl.STREAM_A, n, n)
    ipn, infon = hpl.lu_factor(An, nb=nb, lookahead=la)
    torch.cuda.synchronize()
    assert torch.equal(ipiv, ipn)
    # two FP64-accurate factorizations in different rounding orders: the
    # emulated factors differ from the DFMA ones no more than the DFMA ones
    # differ from the oracle's (the differences grow with the conditioning)
    LU, LUn = _to_np(A), _to_np(An)
    d_ref = max(np.abs(LUn - LUo).max(), 1e-14 * np.abs(LUn).max())
    assert np.abs(LU - LUn).max() <= 10 * d_ref, (np.abs(LU - LUn).max(), d_ref)


def test_lu_fp64_emulation_rejects_wide_panels(hpl):
    """The exactness argument needs panels of at most 256 columns."""
    import ctypes
    import torch
    lib = hpl.load()
    n = 600
    A = hpl.generate(1, hpl.STREAM_A, n, n)
    ipiv = torch.empty(n, dtype=torch.int32, device="cuda")
    info = hpl.Info()
    opts = hpl.make_opts(nb=512, fp64_emulation=1)
    ws = hpl.workspace(lib.lu_factor_workspace_size(n, ctypes.byref(opts)))
    assert lib.lu_factor(n, A.data_ptr(), n, ipiv.data_ptr(), ctypes.byref(opts), ws.data_ptr(), ws.numel(),
                         info.ptr(), torch.cuda.current_stream().cuda_stream) == 1


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6, 7, 8])
def test_lu_1024_nb64_seeds(hpl, orc, seed):
    """The small HPL configuration (n=1024, NB=64, no look-ahead), seeds 1..8:
    exact pivots, solution within the conditioning bound, residual < 16."""
    import torch
    n = 1024
    A0, A, ipiv, LUo, ipo = _factor_and_check(hpl, orc, n, 64, 0, seed=seed)
    b = hpl.generate(seed, hpl.STREAM_B, n, 1)[:, 0].contiguous()
    b0 = _to_np(b).copy()
    hpl.lu_solve(A, ipiv, b)
    torch.cuda.synchronize()
    x = _to_np(b)
    xo = orc.getrs(LUo, ipo, b0)
    kappa = np.linalg.cond(A0, np.inf)
    assert np.abs(x - xo).max() / np.abs(xo).max() <= 100 * n * EPS * kappa
    assert orc.scaled_residual(A0, x, b0) < 16
    Ag = hpl.generate(seed, hpl.STREAM_A, n, n)
    bg = torch.from_numpy(b0).cuda()
    r_gpu = float(hpl.scaled_residual(Ag, b, bg))
    assert r_gpu < 16


def test_lookahead_is_bit_identical(hpl):
    import torch
    n = 1500
    A1 = hpl.generate(3, hpl.STREAM_A, n, n)
    A2 = hpl.generate(3, hpl.STREAM_A, n, n)
    p1, _ = hpl.lu_factor(A1, nb=128, lookahead=0)
    p2, _ = hpl.lu_factor(A2, nb=128, lookahead=1)
    A3 = hpl.generate(3, hpl.STREAM_A, n, n)
    p3, _ = hpl.lu_factor(A3, nb=128, lookahead=1)
    torch.cuda.synchronize()
    assert torch.equal(A1, A2) and torch.equal(p1, p2)
    assert torch.equal(A2, A3) and torch.equal(p2, p3)


@pytest.mark.parametrize("trans", [0, 1])
@pytest.mark.parametrize("n,nrhs", [(1, 1), (65, 3), (700, 1), (1024, 7)])
def test_lu_solve_matches_oracle(hpl, orc, n, nrhs, trans):
    import torch
    A = hpl.generate(9, hpl.STREAM_A, n, n)
    A0 = _to_np(A).copy(order="F")
    ipiv, _ = hpl.lu_factor(A, nb=64)
    B = hpl.generate(9, hpl.STREAM_B, n, nrhs)
    B0 = _to_np(B).copy(order="F")
    hpl.lu_solve(A, ipiv, B, trans=trans)
    torch.cuda.synchronize()
    X = _to_np(B)
    M = A0.T if trans else A0
    Xo, _ = orc.solve(M, B0)
    kappa = np.linalg.cond(A0, np.inf)
    assert np.abs(X - Xo).max() / np.abs(Xo).max() <= 100 * n * EPS * max(kappa, 1.0)


def test_residual_matches_oracle_when_dominated_by_perturbation(hpl, orc):
    import torch
    for kind in (0, 1):
        n = 777
        A = hpl.generate(4, hpl.STREAM_A, n, n, kind)
        A0 = _to_np(A)
        b0 = orc.generate(4, orc.STREAM_B, n, 1)[:, 0]
        x0 = np.linalg.solve(A0, b0)
        x0[11] += 1e-3          # residual dominated by the perturbation, not by rounding
        x = torch.from_numpy(x0).cuda()
        b = torch.from_numpy(b0).cuda()
        want = orc.scaled_residual(A0, x0, b0)
        got_stored = float(hpl.scaled_residual(A, x, b))
        got_regen = float(hpl.scaled_residual(None, x, b, seed=4, kind=kind))
        assert got_stored == pytest.approx(want, rel=1e-7)
        assert got_regen == pytest.approx(want, rel=1e-7)
        assert orc.scaled_residual_gen(4, n, bool(kind), x0, b0) == pytest.approx(want, rel=1e-12)


def test_singular_matrix_reports_first_zero_pivot(hpl):
    import torch
    n = 200
    A = hpl.generate(2, hpl.STREAM_A, n, n)
    A[:, 37] = 0.0
    A[:, 90] = 0.0
    _, info = hpl.lu_factor(A, nb=64)
    torch.cuda.synchronize()
    rec = info.read()
    assert rec["status"] == 2 and rec["info"] == 38


def test_nan_input_does_not_hang(hpl):
    import torch
    n = 100
    A = hpl.generate(2, hpl.STREAM_A, n, n)
    A[:, 5] = float("nan")
    ipiv, info = hpl.lu_factor(A, nb=32)
    torch.cuda.synchronize()
    p = ipiv.cpu().numpy()
    assert p.min() >= 0 and p.max() < n


def test_invalid_arguments(hpl):
    import torch
    A = hpl.colmajor(10, 10)
    with pytest.raises(hpl.HplError):
        hpl.lu_factor(A, nb=1024)
    import ctypes
    n = 64
    A = hpl.generate(1, 0, n, n)
    lib = hpl.load()
    ipiv = torch.empty(n, dtype=torch.int32, device="cuda")
    info = hpl.Info()
    opts = hpl.make_opts(nb=64)
    # a workspace of the full size, declared as 16 bytes: were the size check
    # missing, the launch would still stay inside memory the test owns
    small = hpl.workspace(lib.lu_factor_workspace_size(n, ctypes.byref(opts)))
    st = lib.lu_factor(n, A.data_ptr(), n, ipiv.data_ptr(), ctypes.byref(opts), small.data_ptr(), 16,
                       info.ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 6                                   # HPL_ERR_NOMEM, nothing launched
    assert lib.lu_factor(n, A.data_ptr(), n - 1, ipiv.data_ptr(), None, small.data_ptr(), 16, info.ptr(),
                         None) == 1                  # lda < n
    # empty system: nothing to do
    A0 = hpl.colmajor(0, 0)
    ipiv, info = hpl.lu_factor(A0)
    torch.cuda.synchronize()
    assert info.read()["status"] == 0


@pytest.mark.slow
def test_full_size_n32768_sampled(hpl, orc):
    """n = 32768, NB = 256, look-ahead: the launch configuration of the
    benchmark. The oracle cannot refactor this size, so it checks sampled
    entries of PA - LU (A regenerated on the CPU), |L| <= 1 and the scaled
    residual of the GPU solution computed independently on the CPU."""
    import torch
    n, nb, seed = 32768, 256, 1
    A = hpl.generate(seed, hpl.STREAM_A, n, n)
    ipiv, info = hpl.lu_factor(A, nb=nb, lookahead=1)
    b = hpl.generate(seed, hpl.STREAM_B, n, 1)[:, 0].contiguous()
    b0 = _to_np(b).copy()
    hpl.lu_solve(A, ipiv, b)
    torch.cuda.synchronize()
    assert info.read()["status"] == 0
    assert float(torch.tril(A, -1).abs().max()) <= 1.0
    gp = _to_np(ipiv)
    assert gp.min() >= 0 and gp.max() < n and np.all(gp >= np.arange(n))
    rng = np.random.default_rng(0)
    si = np.concatenate([rng.integers(0, n, 1500), np.arange(0, n, 4096), [n - 1]])
    sj = np.concatenate([rng.integers(0, n, 1500), np.arange(0, n, 4096), [n - 1]])
    rows, cols = np.unique(si), np.unique(sj)
    Lrows = A[torch.from_numpy(rows).cuda()].cpu().numpy()       # rows of L\U
    Ucols = A[:, torch.from_numpy(cols).cuda()].cpu().numpy()    # columns of L\U
    ridx = {r: k for k, r in enumerate(rows)}
    cidx = {c: k for k, c in enumerate(cols)}
    lu = np.empty(si.shape[0])
    for t, (i, j) in enumerate(zip(si, sj)):
        li, uj = Lrows[ridx[i]], Ucols[:, cidx[j]]
        kmax = min(i, j)
        lu[t] = float(np.dot(li[:kmax], uj[:kmax])) + (li[j] if i <= j else li[j] * uj[j])
    rowmap = orc.perm_from_ipiv(gp)
    pa = orc.generate_at(seed, orc.STREAM_A, n, rowmap[si], sj)
    assert np.abs(pa - lu).max() < 1e-9
    x = _to_np(b)
    assert orc.scaled_residual_gen(seed, n, False, x, b0) < 16
