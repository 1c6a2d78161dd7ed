"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test checks one oracle function against an external fact: a published
value, exact rational arithmetic, Cramer's rule, a library routine (LAPACK
through scipy, PyTorch casts and autograd), a closed form or an invariant.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = 2.0 ** -53


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line)
    return rows


# --- generator ---------------------------------------------------------------

def test_splitmix64_published_outputs(orc):
    want = [int(v, 16) for v in _read_golden("splitmix64_state0.txt")]
    got = [orc.sm64_next(0, c) for c in (1, 2, 3)]
    assert got == want


def test_uniform_entries_on_53bit_grid(orc):
    A = orc.generate(7, orc.STREAM_A, 300, 200)
    assert A.min() >= -0.5 and A.max() < 0.5
    units = (A + 0.5) * 2.0 ** 53
    assert np.all(units == np.floor(units))
    # the entry is the top 53 bits of the raw draw (stream key, then draw j*m+i)
    key = orc.stream_key(7, orc.STREAM_A)
    for (i, j) in [(0, 0), (5, 3), (299, 199)]:
        assert A[i, j] == (orc.raw(key, j * 300 + i) >> 11) * 2.0 ** -53 - 0.5


def test_uniform_moments(orc):
    A = orc.generate(11, orc.STREAM_A, 1000, 1000)
    N = A.size
    assert abs(A.mean()) < 5 * math.sqrt(1 / 12 / N)
    assert abs(A.var() - 1 / 12) < 5 * math.sqrt(1 / 180 / N)
    # different streams / seeds are different draws
    B = orc.generate(11, orc.STREAM_B, 1000, 1)
    assert not np.array_equal(A[:, 0], B[:, 0])
    assert abs(np.corrcoef(A[:, 0], B[:, 0])[0, 1]) < 0.15


def test_dominant_diagonal_is_exact_row_sum(orc):
    n = 9
    G = orc.generate(3, orc.STREAM_A, n, n, dominant=False)
    D = orc.generate(3, orc.STREAM_A, n, n, dominant=True)
    off = ~np.eye(n, dtype=bool)
    assert np.array_equal(D[off], G[off])
    for i in range(n):
        s = sum(abs(Fraction(float(v))) for v in G[i, :])   # exact dyadic sum
        assert D[i, i] == float(s)                           # one correct rounding
        assert D[i, i] > sum(abs(G[i, j]) for j in range(n) if j != i)


def test_generate_at_matches_full_matrix(orc):
    n = 40
    for dom in (False, True):
        A = orc.generate(6, orc.STREAM_A, n, n, dominant=dom)
        rng = np.random.default_rng(1)
        r, c = rng.integers(0, n, 300), rng.integers(0, n, 300)
        r[:5] = c[:5]
        assert np.array_equal(orc.generate_at(6, orc.STREAM_A, n, r, c, dominant=dom), A[r, c])


def test_batch_sizes_range(orc):
    s = orc.batch_sizes(5, 4096)
    assert s.min() >= 32 and s.max() <= 512
    assert abs(s.mean() - 272) < 10
    assert len(np.unique(s)) > 400


# --- getrf / getrs -------------------------------------------------------------

def _exact_lu(A):
    """Gaussian elimination with partial pivoting in exact rationals."""
    n = len(A)
    M = [[Fraction(float(A[i, j])) for j in range(n)] for i in range(n)]
    ipiv = []
    for k in range(n):
        p = max(range(k, n), key=lambda i: (abs(M[i][k]), -i))
        ipiv.append(p)
        M[k], M[p] = M[p], M[k]
        if M[k][k] != 0:
            for i in range(k + 1, n):
                M[i][k] = M[i][k] / M[k][k]
                for j in range(k + 1, n):
                    M[i][j] -= M[i][k] * M[k][j]
    return M, ipiv


def _det(M):
    n = len(M)
    if n == 1:
        return M[0][0]
    return sum((-1) ** j * M[0][j] * _det([row[:j] + row[j + 1:] for row in M[1:]]) for j in range(n))


@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (3, 3), (4, 4), (5, 5), (6, 6)])
def test_getrf_matches_exact_rational_elimination(orc, n, seed):
    A = orc.generate(seed, orc.STREAM_A, n, n)
    LU, ipiv, info, gap = orc.getrf(A)
    M, ipiv_exact = _exact_lu(A)
    assert info == 0
    assert list(ipiv) == ipiv_exact
    exact = np.array([[float(v) for v in row] for row in M])
    assert np.allclose(LU, exact, rtol=0, atol=1e-13 * max(1.0, np.abs(exact).max()))


@pytest.mark.parametrize("n,seed", [(2, 1), (3, 2), (4, 3), (5, 4)])
def test_getrs_matches_cramer(orc, n, seed):
    A = orc.generate(seed, orc.STREAM_A, n, n)
    b = orc.generate(seed, orc.STREAM_B, n, 1)[:, 0]
    LU, ipiv, info, _ = orc.getrf(A)
    x = orc.getrs(LU, ipiv, b)
    Mq = [[Fraction(float(A[i, j])) for j in range(n)] for i in range(n)]
    bq = [Fraction(float(v)) for v in b]
    d = _det(Mq)
    xq = []
    for c in range(n):
        Mc = [row[:] for row in Mq]
        for i in range(n):
            Mc[i][c] = bq[i]
        xq.append(_det(Mc) / d)
    xe = np.array([float(v) for v in xq])
    kappa = np.linalg.cond(A, np.inf)
    assert np.max(np.abs(x - xe)) / np.max(np.abs(xe)) <= 4 * n * kappa * EPS


def test_lu_2x2_by_hand(orc):
    rows = dict((r.split()[0], r.split()[1:]) for r in _read_golden("lu_2x2_by_hand.txt"))
    A = np.array([float(Fraction(v)) for v in rows["A"]]).reshape(2, 2)
    LU, ipiv, info, _ = orc.getrf(A)
    assert list(ipiv) == [int(v) for v in rows["ipiv"]]
    assert LU[1, 0] == float(Fraction(rows["L10"][0]))
    U = [float(Fraction(v)) for v in rows["U"]]
    assert LU[0, 0] == U[0] and LU[0, 1] == U[1]
    assert abs(LU[1, 1] - U[2]) <= 2 * EPS
    b = np.array([float(Fraction(v)) for v in rows["b"]])
    x = orc.getrs(LU, ipiv, b)
    xe = np.array([float(Fraction(v)) for v in rows["x"]])
    assert np.allclose(x, xe, rtol=0, atol=1e-14)


@pytest.mark.parametrize("n,seed", [(64, 1), (257, 2), (1024, 3)])
def test_getrf_pivots_match_lapack(orc, n, seed):
    sl = pytest.importorskip("scipy.linalg")
    A = orc.generate(seed, orc.STREAM_A, n, n)
    LU, ipiv, info, gap = orc.getrf(A)
    lu, piv = sl.lu_factor(A)
    assert info == 0
    assert gap > 1e-12, ("near-tie pivot column: pick another seed", gap)
    assert np.array_equal(ipiv, piv.astype(np.int32))
    assert np.max(np.abs(LU - lu)) < 1e-9 * n


@pytest.mark.parametrize("n", [100, 512])
def test_getrf_backward_error_invariant(orc, n):
    A = orc.generate(n, orc.STREAM_A, n, n)
    LU, ipiv, info, _ = orc.getrf(A)
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    rowmap = orc.perm_from_ipiv(ipiv)
    PA = A[rowmap, :]
    err = np.abs(PA - L @ U).sum(axis=1).max()
    assert err / (n * EPS * np.abs(A).sum(axis=1).max()) < 10
    assert np.abs(np.tril(LU, -1)).max() <= 1.0
    b = orc.generate(n, orc.STREAM_B, n, 1)[:, 0]
    x = orc.getrs(LU, ipiv, b)
    assert orc.scaled_residual(A, x, b) < 16


def test_getrf_closed_forms(orc):
    n = 6
    LU, ipiv, info, _ = orc.getrf(np.eye(n))
    assert np.array_equal(LU, np.eye(n)) and list(ipiv) == list(range(n)) and info == 0
    perm = [3, 0, 5, 1, 4, 2]
    P = np.zeros((n, n))
    for i, p in enumerate(perm):
        P[i, p] = 1.0
    LU, ipiv, info, _ = orc.getrf(P)
    rowmap = orc.perm_from_ipiv(ipiv)
    assert np.array_equal(P[rowmap, :], np.eye(n)) and np.array_equal(LU, np.eye(n))
    U = np.triu(orc.generate(4, orc.STREAM_A, n, n)) + 4 * np.eye(n)
    LU, ipiv, info, _ = orc.getrf(U)
    assert np.array_equal(LU, U) and list(ipiv) == list(range(n))
    d = np.array([2.0, -4.0, 0.5, 8.0, -1.0, 16.0])
    b = np.array([1.0, 3.0, -2.0, 5.0, 7.0, -9.0])
    LU, ipiv, info, _ = orc.getrf(np.diag(d))
    x = orc.getrs(LU, ipiv, b)
    assert np.array_equal(x, b / d)


def test_getrf_singular_reports_first_zero_pivot(orc):
    n = 8
    A = orc.generate(9, orc.STREAM_A, n, n)
    A[:, 2] = 0.0
    A[:, 5] = 0.0
    _, _, info, _ = orc.getrf(A)
    assert info == 3
    _, _, info, _ = orc.getrf(np.zeros((3, 3)))
    assert info == 1


@pytest.mark.parametrize("n", [37, 200])
def test_getrs_transpose_and_multi_rhs(orc, n):
    A = orc.generate(n, orc.STREAM_A, n, n)
    B = orc.generate(n, orc.STREAM_B, n, 3)
    LU, ipiv, _, _ = orc.getrf(A)
    X = orc.getrs(LU, ipiv, B, trans=0)
    XT = orc.getrs(LU, ipiv, B, trans=1)
    assert np.allclose(X, np.linalg.solve(A, B), rtol=0, atol=1e-10)
    assert np.allclose(XT, np.linalg.solve(A.T, B), rtol=0, atol=1e-10)


# --- residual --------------------------------------------------------------------

def test_scaled_residual_closed_form(orc):
    n = 4
    A = np.eye(n)
    b = np.array([1.0, -2.0, 0.5, 0.25])
    assert orc.scaled_residual(A, b, b) == 0.0
    delta = 2.0 ** -40
    x = b.copy()
    x[0] += delta
    want = delta / (EPS * (1.0 * np.abs(x).max() + np.abs(b).max()) * n)
    assert orc.scaled_residual(A, x, b) == pytest.approx(want, rel=1e-15)
    # ||A||_inf is the maximum absolute row sum
    A2 = np.array([[1.0, -3.0], [2.0, 0.5]])
    x2 = np.array([1.0, 1.0])
    b2 = A2 @ x2 + np.array([0.0, 1e-12])
    want2 = 1e-12 / (EPS * (4.0 * 1.0 + np.abs(b2).max()) * 2)
    assert orc.scaled_residual(A2, x2, b2) == pytest.approx(want2, rel=1e-3)


@pytest.mark.parametrize("dominant", [False, True])
def test_scaled_residual_regenerated_matches_stored(orc, dominant):
    n = 150
    A = orc.generate(21, orc.STREAM_A, n, n, dominant=dominant)
    b = orc.generate(21, orc.STREAM_B, n, 1)[:, 0]
    x = np.linalg.solve(A, b)
    x[3] += 1e-9
    assert orc.scaled_residual_gen(21, n, dominant, x, b) == orc.scaled_residual(A, x, b)


def test_lu_sample_diff(orc):
    n = 80
    A = orc.generate(2, orc.STREAM_A, n, n)
    LU, ipiv, _, _ = orc.getrf(A)
    rng = np.random.default_rng(0)
    si, sj = rng.integers(0, n, 200), rng.integers(0, n, 200)
    d = orc.lu_sample_diff(2, n, False, LU, ipiv, si, sj)
    assert np.abs(d).max() < 1e-13
    LU2 = LU.copy()
    LU2[10, 20] += 1e-6       # a planted error in the factor must show
    d2 = orc.lu_sample_diff(2, n, False, LU2, ipiv, np.array([10]), np.array([20]))
    assert abs(d2[0]) > 1e-7


# --- low precision rounding ------------------------------------------------------

def _tie_cases_bf16():
    base = np.array([1.0, 1.5, -3.25, 1e-30, 7e20, 0.1], dtype=np.float32).view(np.uint32)
    out = []
    for b in base:
        hi = b & 0xFFFF0000
        for low in (0x8000, 0x7FFF, 0x8001, 0x0001, 0xFFFF):
            out.append(np.uint32(hi | low))
        out.append(np.uint32(hi | 0x18000))
    return np.array(out, dtype=np.uint32).view(np.float32)


def _subnormal_cases_bf16():
    """FP32 values at and below BF16's smallest normal 2^-126, where the BF16
    grid is the fixed spacing 2^-133: every FP32 subnormal bit pattern class
    (smallest, ties at 2^-134 multiples, just off ties, the normal boundary)."""
    bits = [0x00000001, 0x00000002, 0x0000FFFF, 0x00008000, 0x00018000, 0x00010000, 0x00007FFF,
            0x00008001, 0x007FFFFF, 0x007F8000, 0x007F7FFF, 0x00800000, 0x00808000, 0x00818000,
            0x0017F3E0, 0x00123456, 0x00400000, 0x003FFFFF]
    out = []
    for b in bits:
        out.append(np.uint32(b))
        out.append(np.uint32(b | 0x80000000))
    rng = np.random.default_rng(11)
    out.extend(rng.integers(1, 0x00800000, 3000, dtype=np.uint32))
    return np.array(out, dtype=np.uint32).view(np.float32)


def _overflow_cases_bf16():
    """Around the largest finite BF16, 0x7F7F: below, at and past the midpoint
    to 2^128 (which rounds to infinity)."""
    bits = [0x7F7F0000, 0x7F7F7FFF, 0x7F7F8000, 0x7F7F8001, 0x7F7FFFFF, 0x7F7E8000, 0x7F7F4000]
    return np.array(bits + [b | 0x80000000 for b in bits], dtype=np.uint32).view(np.float32)


def test_round_bf16_matches_torch(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    vals = np.concatenate([rng.standard_normal(2000).astype(np.float32) * 10.0 ** rng.integers(-20, 20, 2000),
                           _tie_cases_bf16(), _subnormal_cases_bf16(), _overflow_cases_bf16(),
                           np.array([2.0 ** -149, 3 * 2.0 ** -140, 1.7e-39], dtype=np.float32)]).astype(np.float32)
    want = torch.from_numpy(vals).to(torch.bfloat16).float().numpy()
    got = np.array([orc.round_bf16(v) for v in vals], dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_round_bf16_subnormal_grid(orc):
    """Below 2^-126 every result is a multiple of 2^-133 (BF16's subnormal
    spacing) and the nearest one, ties to an even multiple; 2^-149 (FP32's
    smallest subnormal) rounds to zero."""
    for k in (0, 1, 2, 3, 5, 127):
        for frac in (0.25, 0.5, 0.75):
            x = np.float32((k + frac) * 2.0 ** -133)
            got = orc.round_bf16(float(x))
            q = k + (1 if frac > 0.5 or (frac == 0.5 and k % 2 == 1) else 0)
            assert got == q * 2.0 ** -133, (k, frac, got)
    assert orc.round_bf16(2.0 ** -149) == 0.0


def test_round_e4m3_matches_torch(orc):
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8 in this torch")
    rng = np.random.default_rng(2)
    vals = rng.uniform(-448, 448, 3000).astype(np.float32)
    small = (rng.standard_normal(2000) * 2.0 ** rng.integers(-12, 4, 2000)).astype(np.float32)
    grid = np.array([k * 2.0 ** -10 for k in range(-40, 41)], dtype=np.float32)  # subnormal ties
    vals = np.concatenate([vals, small, grid, np.float32([448.0, -448.0, 0.0, 1.0625, 1.1875])])
    want = torch.from_numpy(vals).to(torch.float8_e4m3fn).float().numpy()
    got = np.array([orc.round_e4m3(v) for v in vals], dtype=np.float32)
    assert np.array_equal(got, want)
    assert orc.round_e4m3(1000.0) == 448.0 and orc.round_e4m3(-500.0) == -448.0


def test_round_fp16_matches_numpy(orc):
    """IEEE binary16 round-to-nearest-even against NumPy's float16 cast:
    normals, subnormals (spacing 2^-24), exact ties, the overflow threshold."""
    rng = np.random.default_rng(3)
    vals = (rng.standard_normal(4000) * 2.0 ** rng.integers(-30, 17, 4000)).astype(np.float32)
    ties = np.array([(2 * k + 1) * 2.0 ** (e - 11) for e in range(-13, 16) for k in (1024, 1500, 2047)],
                    dtype=np.float32)                                  # halfway between two binary16 values
    sub = np.array([(k + 0.5) * 2.0 ** -24 for k in range(-40, 40)], dtype=np.float32)
    edge = np.float32([65504.0, 65519.0, 65520.0, -65520.0, 2.0 ** -14, 2.0 ** -25, 2.0 ** -26, 0.0, -0.0])
    vals = np.concatenate([vals, ties, -ties, sub, edge])
    with np.errstate(over="ignore"):
        want = vals.astype(np.float16).astype(np.float32)
    got = np.array([orc.round_fp16(v) for v in vals], dtype=np.float32)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("prec,bound,rnd", [(1, 448.0, "round_e4m3"), (2, 65504.0, "round_fp16")])
def test_scaled_operand_rounding(orc, prec, bound, rnd):
    """FP8 / FP16 operands: per A-operand row (per B-operand column) the scale
    is the smallest power of two 2^e with max|x| 2^-e <= bound (found here by
    brute force over e), and every entry is 2^e round(x 2^-e)."""
    rng = np.random.default_rng(prec)
    X = (rng.standard_normal((37, 23)) * 10.0 ** rng.integers(-9, 6, (37, 1))).astype(np.float32)
    X[5, :] = 0.0                                       # an all-zero row keeps scale 1
    f = getattr(orc, rnd)
    for kdim_is_rows, Y in ((False, X), (True, X.T.copy())):
        Q = orc.round_operand(prec, Y, kdim_is_rows)
        lines = range(Y.shape[1]) if kdim_is_rows else range(Y.shape[0])
        for t in lines:
            y = Y[:, t] if kdim_is_rows else Y[t, :]
            q = Q[:, t] if kdim_is_rows else Q[t, :]
            amax = float(np.abs(y.astype(np.float64)).max())
            e = 0 if amax == 0.0 else min(e for e in range(-160, 160) if amax * 2.0 ** -e <= bound)
            want = np.array([np.ldexp(f(float(np.ldexp(np.float64(v), -e))), e) for v in y], dtype=np.float32)
            assert np.array_equal(q, want), (kdim_is_rows, t)


# --- HPL-MxP emulation ---------------------------------------------------------------

def test_mxp_factor_fp32_mode_is_block_lu(orc):
    """FP32 reference mode: L U reproduces A, and every D_k equals L_kk U_kk of
    the scalar unpivoted LU (computed independently by getrf, which makes no
    interchange on a diagonally dominant matrix)."""
    n, nb = 96, 32
    A = orc.generate(4, orc.STREAM_A, n, n, dominant=True)
    # at n = 96 the matrix is only weakly dominant (diagonal ~24 against
    # off-diagonal block row sums ~8): a third Newton-Schulz step brings the
    # inverse to FP32 accuracy
    F, Dinv, info = orc.mxp_factor(A, nb, orc.PREC_FP32, ns_iters=3)
    assert info == 0
    L, U = orc.block_lu_parts(F, nb)
    assert np.abs(A - L @ U).max() / np.abs(A).max() < 1e-6
    LU, ipiv, _, _ = orc.getrf(A)
    assert list(ipiv) == list(range(n))
    Ls, Us = np.tril(LU, -1) + np.eye(n), np.triu(LU)
    for k0 in range(0, n, nb):
        s = slice(k0, k0 + nb)
        Dk = Ls[s, s] @ Us[s, s]
        assert np.abs(F[s, s] - Dk).max() / np.abs(Dk).max() < 1e-6
        assert np.abs(Dinv[s, :] @ Dk - np.eye(nb)).max() < 1e-5


def test_newton_schulz_inverse_accuracy(orc):
    n, nb = 512, 256
    A = orc.generate(14, orc.STREAM_A, n, n, dominant=True)
    for prec, tol in ((orc.PREC_BF16, 2e-5), (orc.PREC_FP8, 2e-5), (orc.PREC_FP16, 2e-5), (orc.PREC_FP32, 5e-6)):
        F, Dinv, _ = orc.mxp_factor(A, nb, prec)
        for k0 in range(0, n, nb):
            s = slice(k0, k0 + nb)
            resid = np.abs(F[s, s].astype(np.float64) @ Dinv[s, :].astype(np.float64) - np.eye(nb)).max()
            assert resid < tol, (prec, k0, resid)
    # fewer iterations give a worse inverse (the iteration is really applied)
    F1, D1, _ = orc.mxp_factor(A, nb, orc.PREC_BF16, ns_iters=1)
    r1 = np.abs(F1[:nb, :nb].astype(np.float64) @ D1[:nb, :].astype(np.float64) - np.eye(nb)).max()
    assert r1 > 1e-5


def test_mxp_factor_lowprec_error_levels(orc):
    n, nb = 192, 64
    A = orc.generate(5, orc.STREAM_A, n, n, dominant=True)

    def err(prec):
        F, _, _ = orc.mxp_factor(A, nb, prec)
        L, U = orc.block_lu_parts(F, nb)
        return np.abs(A - L @ U).max() / np.abs(A[~np.eye(n, dtype=bool)]).max()

    e32, e16, e8, eh = err(orc.PREC_FP32), err(orc.PREC_BF16), err(orc.PREC_FP8), err(orc.PREC_FP16)
    assert e32 < 1e-4
    assert e32 < e16 < 2.0 ** -6
    assert e16 < e8 < 2.0 ** -2
    # FP16 keeps 11 significant bits against BF16's 8 (and its scale keeps L21
    # out of the subnormal range)
    assert e32 < eh < e16 / 4


def test_mxp_factor_diagonal_matrix_exact(orc):
    d = np.array([2.0, 4.0, 0.25, 8.0, 0.5, 1.0])
    F, Dinv, info = orc.mxp_factor(np.diag(d), 4, orc.PREC_BF16)
    assert np.array_equal(F, np.diag(d).astype(np.float32))
    assert np.array_equal(Dinv[:4, :4], np.diag(1 / d[:4]).astype(np.float32))
    assert np.array_equal(Dinv[4:, :2], np.diag(1 / d[4:]).astype(np.float32))


@pytest.mark.parametrize("refine", [0, 1])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_mxp_solve_reaches_fp64_solution(orc, refine, prec):
    n, nb = 256, 64
    A = orc.generate(6, orc.STREAM_A, n, n, dominant=True)
    b = orc.generate(6, orc.STREAM_B, n, 1)[:, 0]
    out = orc.mxp_solve(A, b, nb, prec=prec, refine=refine)
    assert out["status"] == 0 and out["sr"] < 16
    x64, _ = orc.solve(A, b)
    # a scaled residual below 16 bounds the forward error by ~ kappa * 16 * n * eps
    bound = 2 * 16 * n * EPS * np.linalg.cond(A, np.inf)
    assert np.abs(out["x"] - x64).max() / np.abs(x64).max() < bound
    assert 1 <= out["iters"] <= 20


def test_mxp_preconditioner_is_block_lu_inverse(orc):
    """With the FP32 factor, one preconditioner application solves L U x = b
    (checked against numpy's solve of the assembled L U)."""
    n, nb = 128, 32
    A = orc.generate(15, orc.STREAM_A, n, n, dominant=True)
    b = orc.generate(15, orc.STREAM_B, n, 1)[:, 0].astype(np.float32).astype(np.float64)
    # weakly dominant at n = 128: three Newton-Schulz steps for an FP32-accurate D^-1
    F, Dinv, _ = orc.mxp_factor(A, nb, orc.PREC_FP32, ns_iters=3)
    out = orc.mxp_refine(A, F, Dinv, nb, b, refine=0, max_iter=0)
    L, U = orc.block_lu_parts(F, nb)
    x_ref = np.linalg.solve(L @ U, b)
    assert np.abs(out["x"] - x_ref).max() / np.abs(x_ref).max() < 1e-5


def test_mxp_identity_needs_no_correction(orc):
    n = 16
    b = np.array([float(np.float32(v)) for v in np.linspace(-1, 1, n)])
    out = orc.mxp_solve(np.eye(n), b, 8)
    assert out["iters"] == 0 and out["sr"] == 0.0 and np.array_equal(out["x"], b)


def test_mxp_gmres_not_worse_than_classic_ir(orc):
    n, nb = 256, 64
    A = orc.generate(8, orc.STREAM_A, n, n, dominant=True)
    b = orc.generate(8, orc.STREAM_B, n, 1)[:, 0]
    ir = orc.mxp_solve(A, b, nb, prec=orc.PREC_FP8, refine=0)
    gm = orc.mxp_solve(A, b, nb, prec=orc.PREC_FP8, refine=1)
    assert gm["iters"] <= ir["iters"]


def test_mxp_refine_not_converged_status(orc):
    n = 64
    A = orc.generate(9, orc.STREAM_A, n, n)          # general matrix, useless preconditioner
    b = orc.generate(9, orc.STREAM_B, n, 1)[:, 0]
    F = np.asfortranarray(np.eye(n, dtype=np.float32))
    Dinv = np.asfortranarray(np.eye(n, 32, dtype=np.float32))
    Dinv[32:, :] = np.eye(32, dtype=np.float32)
    out = orc.mxp_refine(A, F, Dinv, 32, b, refine=0, max_iter=2)
    assert out["status"] == 4 and out["iters"] == 2


# --- HPL-MxP plain LU emulation (paper order, independent of the block design) -------

def _golden_kv(name):
    out = {}
    for line in _read_golden(name):
        k, *v = line.split()
        out[k] = v
    return out


def _frac_matrix(vals, n):
    return np.array([float(Fraction(v)) for v in vals]).reshape(n, n)


def test_mxp_lu_plain_by_hand(orc):
    """Two panel steps of a 4 x 4 case worked by hand in exact rationals, for
    every operand precision: the BF16 rounding of one U12 entry (up), the FP8
    rounding of the same entry (down), FP16 and FP32 exact."""
    g = _golden_kv("mxp_2step_by_hand.txt")
    nb = int(g["nb"][0])
    A = _frac_matrix(g["A"], 4)
    for prec in (3, 0, 2, 1):
        F, info = orc.mxp_lu_plain(A, nb, prec)
        assert info == 0
        want = _frac_matrix(g[f"F_prec{prec}"], 4)
        assert np.array_equal(F.astype(np.float64), want), (prec, F)
    for prec in (3, 0, 2, 1):
        F, _ = orc.mxp_lu_plain(A, 4, prec)
        assert np.array_equal(F.astype(np.float64), _frac_matrix(g["F_nb4"], 4)), prec


def _exact_unpivoted_lu(A):
    n = A.shape[0]
    M = [[Fraction(float(A[i, j])) for j in range(n)] for i in range(n)]
    for k in range(n):
        for i in range(k + 1, n):
            M[i][k] = M[i][k] / M[k][k]
            for j in range(k + 1, n):
                M[i][j] -= M[i][k] * M[k][j]
    return M


def test_mxp_lu_plain_fp32_within_error_bound_of_exact(orc):
    """FP32 mode on a ragged panel split (n = 10, NB = 3): the computed L, U
    satisfy the componentwise backward-error bound of Gaussian elimination,
    |A - L U| <= gamma_n |L| |U| with gamma_n = n u / (1 - n u), u = 2^-24
    (evaluated in exact rationals), and are close to the exact unpivoted LU
    of the same (FP32) matrix."""
    n, nb = 10, 3
    A = orc.generate(41, orc.STREAM_A, n, n, dominant=True).astype(np.float32).astype(np.float64)
    F, info = orc.mxp_lu_plain(A, nb, orc.PREC_FP32)
    assert info == 0
    Fq = [[Fraction(float(F[i, j])) for j in range(n)] for i in range(n)]
    u = Fraction(1, 2 ** 24)
    gamma = n * u / (1 - n * u)
    for i in range(n):
        for j in range(n):
            lu = sum((Fq[i][k] if k < i else Fraction(1)) * Fq[k][j] for k in range(min(i, j) + 1) if k <= j)
            absl = sum(abs(Fq[i][k] if k < i else Fraction(1)) * abs(Fq[k][j]) for k in range(min(i, j) + 1))
            assert abs(Fraction(float(A[i, j])) - lu) <= gamma * absl, (i, j)
    E = _exact_unpivoted_lu(A)
    scale = np.abs(A).max()
    err = max(abs(float(Fq[i][j] - E[i][j])) for i in range(n) for j in range(n))
    assert err <= 8 * n * 2.0 ** -24 * scale


def test_mxp_lu_plain_fp32_matches_lapack(orc):
    """FP32 mode against LAPACK's LU of the same matrix (scipy): on a
    diagonally dominant matrix partial pivoting makes no interchange, so the
    two are the same factorization, FP32 against FP64 arithmetic."""
    sl = pytest.importorskip("scipy.linalg")
    n, nb = 300, 64
    A = orc.generate(42, orc.STREAM_A, n, n, dominant=True)
    P, L, U = sl.lu(A.astype(np.float32).astype(np.float64))
    assert np.array_equal(P, np.eye(n))
    F, _ = orc.mxp_lu_plain(A, nb, orc.PREC_FP32)
    F = F.astype(np.float64)
    assert np.abs(np.tril(F, -1) - np.tril(L, -1)).max() <= 1e-5 * np.abs(np.tril(L, -1)).max()
    assert np.abs(np.triu(F) - U).max() <= 1e-5 * np.abs(U).max()


def test_mxp_lu_plain_panel_width_independent_in_fp32(orc):
    """Without operand rounding the panel width only reorders FP32 operations:
    every NB gives the factor of the unblocked elimination to FP32 accuracy;
    with BF16 operands the width matters (the updates are rounded)."""
    n = 200
    A = orc.generate(43, orc.STREAM_A, n, n, dominant=True)
    ref, _ = orc.mxp_lu_plain(A, n, orc.PREC_FP32)
    for nb in (1, 7, 64, 199):
        F, _ = orc.mxp_lu_plain(A, nb, orc.PREC_FP32)
        assert np.abs(F.astype(np.float64) - ref).max() <= 1e-5 * np.abs(ref).max(), nb
    Fb, _ = orc.mxp_lu_plain(A, 64, orc.PREC_BF16)
    assert np.abs(Fb.astype(np.float64) - ref).max() > 1e-6 * np.abs(ref).max()


def test_mxp_lu_plain_error_levels(orc):
    """Backward error ||A - LU||_inf / ||A||_inf by operand precision: FP32 <
    FP16 < BF16 < FP8 (BF16 keeps 8 significant bits, FP16 11, E4M3 4): the
    rounded operands really enter the update, and FP16 is at least 4x better
    than BF16."""
    from _parity import plain_lu_backward_error
    n, nb = 384, 128
    A = orc.generate(44, orc.STREAM_A, n, n, dominant=True)
    e = {p: plain_lu_backward_error(A, orc.mxp_lu_plain(A, nb, p)[0]) for p in (3, 2, 0, 1)}
    assert e[3] < 1e-6
    assert e[3] < e[2] < e[0] < e[1]
    assert 16 * e[3] < e[0] < 2.0 ** -9
    assert e[2] < e[0] / 4
    assert e[1] < 2.0 ** -6


@pytest.mark.parametrize("refine", [0, 1])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_mxp_solve_plain_reaches_fp64_solution(orc, refine, prec):
    n, nb = 256, 64
    A = orc.generate(6, orc.STREAM_A, n, n, dominant=True)
    b = orc.generate(6, orc.STREAM_B, n, 1)[:, 0]
    out = orc.mxp_solve_plain(A, b, nb, prec=prec, refine=refine)
    assert out["status"] == 0 and out["sr"] < 16
    x64, _ = orc.solve(A, b)
    bound = 2 * 16 * n * EPS * np.linalg.cond(A, np.inf)
    assert np.abs(out["x"] - x64).max() / np.abs(x64).max() < bound
    assert 1 <= out["iters"] <= 20


def test_mxp_plain_preconditioner_solves_lu(orc):
    """One application of the plain preconditioner solves L U x = b (numpy's
    solve of the assembled FP32 factors) to FP32 accuracy."""
    n, nb = 128, 32
    A = orc.generate(15, orc.STREAM_A, n, n, dominant=True)
    b = orc.generate(15, orc.STREAM_B, n, 1)[:, 0].astype(np.float32).astype(np.float64)
    F, _ = orc.mxp_lu_plain(A, nb, orc.PREC_BF16)
    out = orc.mxp_refine_plain(A, F, b, refine=0, max_iter=0)
    Fd = F.astype(np.float64)
    x_ref = np.linalg.solve((np.tril(Fd, -1) + np.eye(n)) @ np.triu(Fd), b)
    assert np.abs(out["x"] - x_ref).max() / np.abs(x_ref).max() < 1e-5


def test_block_and_plain_emulations_agree_on_iterations(orc):
    """The two readings of the low-precision factorization (the block LU with a
    Newton-Schulz diagonal inverse, and the plain LU in the paper's order)
    need the same number of GMRES-IR corrections on the same system, and the
    block factor's backward error stays within the factor stated for the GPU
    parity tests (the block LU rounds A21 itself to BF16 inside L21 = A21 D^-1;
    the plain LU rounds only the update operands L21 ~ 1/n and U12)."""
    from _parity import block_lu_backward_error, plain_lu_backward_error, BLOCK_VS_PLAIN_BERR
    for n, nb, prec in ((512, 128, 0), (300, 100, 0), (512, 128, 1), (512, 128, 2)):
        A = orc.generate(3, orc.STREAM_A, n, n, dominant=True)
        b = orc.generate(3, orc.STREAM_B, n, 1)[:, 0]
        Fp, _ = orc.mxp_lu_plain(A, nb, prec)
        Fb, Db, _ = orc.mxp_factor(A, nb, prec)
        ep, eb = plain_lu_backward_error(A, Fp), block_lu_backward_error(A, Fb, nb)
        assert ep / 4 <= eb <= BLOCK_VS_PLAIN_BERR[prec] * ep, (n, nb, prec, ep, eb)
        sp, sb = orc.mxp_refine_plain(A, Fp, b), orc.mxp_refine(A, Fb, Db, nb, b)
        assert abs(sp["iters"] - sb["iters"]) <= 2


def test_block_tolerances_catch_planted_mistakes(orc):
    """The per-part tolerances of the GPU factor tests fail on a CPU copy of the
    oracle's factor with one mistake planted (L21 of one step scaled by 2, one
    U12 entry's sign flipped, a diagonal of D perturbed), and pass on the
    unmodified copy. A single tolerance over all off-diagonal entries relative
    to their overall maximum (an entry of U, ~1/2) would let the scaled L21
    (entries ~2/n) through."""
    from _parity import assert_blocks_close
    n, nb = 1000, 256
    A = orc.generate(3, orc.STREAM_A, n, n, dominant=True)
    Fo, _, _ = orc.mxp_factor(A, nb, orc.PREC_BF16)
    Fo = Fo.astype(np.float64)
    tol = dict(l21=2.0 ** -7, u12=2.0 ** -7, doff=2.0 ** -7, ddiag=1e-5)
    assert_blocks_close(Fo.copy(), Fo, nb, **tol)
    bad = Fo.copy()
    bad[512:, 256:512] *= 2.0
    off = ~np.eye(n, dtype=bool)
    assert np.abs(bad - Fo)[off].max() <= 2.0 ** -7 * np.abs(Fo[off]).max()   # the old global test passes it
    with pytest.raises(AssertionError):
        assert_blocks_close(bad, Fo, nb, **tol)
    bad = Fo.copy()
    bad[300, 700] = -bad[300, 700]
    with pytest.raises(AssertionError):
        assert_blocks_close(bad, Fo, nb, **tol)
    bad = Fo.copy()
    bad[600, 600] *= 1 + 1e-4
    with pytest.raises(AssertionError):
        assert_blocks_close(bad, Fo, nb, **tol)


# --- adjoint ---------------------------------------------------------------------

def test_adjoint_matches_finite_differences(orc):
    """The differentiable-solve check at n = 64: every entry of grad_A and
    grad_B against central differences of sum(G * A^-1 B) in FP64, within
    1e-6 relative per entry (no absolute floor)."""
    from _parity import fd_gradients, max_rel_err
    n, nrhs = 64, 3
    A = orc.generate(21, orc.STREAM_A, n, n, dominant=True)
    B = orc.generate(21, orc.STREAM_B, n, nrhs)
    G = np.random.default_rng(5).standard_normal((n, nrhs))
    X = np.linalg.solve(A, B)
    gB, gA = orc.adjoint(A, X, G)
    fdA, fdB = fd_gradients(A, B, G)
    assert max_rel_err(gA, fdA) <= 1e-6
    assert max_rel_err(gB, fdB) <= 1e-6


def test_fd_yardstick_catches_wrong_gradients(orc):
    """The finite-difference yardstick flags a gradient with one wrong sign or
    a transposed grad_A (planted in a CPU copy of the oracle's result)."""
    from _parity import fd_gradients, max_rel_err
    n, nrhs = 12, 2
    A = orc.generate(31, orc.STREAM_A, n, n, dominant=True)
    B = orc.generate(31, orc.STREAM_B, n, nrhs)
    G = np.random.default_rng(9).standard_normal((n, nrhs))
    gB, gA = orc.adjoint(A, np.linalg.solve(A, B), G)
    fdA, fdB = fd_gradients(A, B, G)
    assert max_rel_err(gA, fdA) <= 1e-6 and max_rel_err(gB, fdB) <= 1e-6
    bad = gA.copy()
    bad[3, 7] = -bad[3, 7]
    assert max_rel_err(bad, fdA) > 1e-6
    assert max_rel_err(gA.T, fdA) > 1e-6
    assert max_rel_err(gB * (1 + 1e-5), fdB) > 1e-6


def test_adjoint_matches_torch_autograd(orc):
    torch = pytest.importorskip("torch")
    n, nrhs = 24, 3
    A = orc.generate(13, orc.STREAM_A, n, n)
    B = orc.generate(13, orc.STREAM_B, n, nrhs)
    G = np.random.default_rng(4).standard_normal((n, nrhs))
    At = torch.tensor(A, requires_grad=True)
    Bt = torch.tensor(B, requires_grad=True)
    Xt = torch.linalg.solve(At, Bt)
    (Xt * torch.tensor(G)).sum().backward()
    gB, gA = orc.adjoint(A, Xt.detach().numpy(), G)
    assert np.abs(gB - Bt.grad.numpy()).max() <= 1e-10 * np.abs(gB).max()
    assert np.abs(gA - At.grad.numpy()).max() <= 1e-10 * np.abs(gA).max()


def test_adjoint_closed_forms(orc):
    n, nrhs = 5, 2
    G = np.arange(10, dtype=np.float64).reshape(n, nrhs)
    X = np.ones((n, nrhs))
    gB, gA = orc.adjoint(np.eye(n), X, G)
    assert np.array_equal(gB, G) and np.array_equal(gA, -G @ X.T)
    d = np.array([2.0, 4.0, 8.0, 0.5, 0.25])
    gB, _ = orc.adjoint(np.diag(d), X, G)
    assert np.allclose(gB, G / d[:, None], rtol=1e-15)


def test_flop_count(orc):
    assert orc.flops(1024) == 2 * 1024 ** 3 / 3 + 2 * 1024 ** 2


def _nearest_bf16_bruteforce(x: float) -> float:
    """The BF16 value nearest to the double x (ties to an even last fraction
    bit), by exact comparison of the candidates around x."""
    from fractions import Fraction
    if x == 0.0:
        return 0.0
    m, e = np.frexp(abs(x))                      # |x| = m 2^e, 0.5 <= m < 1
    e = int(e)
    cands = set()
    for ee in (e - 1, e, e + 1):
        base = int(np.floor(abs(x) / 2.0 ** (ee - 8)))
        for k in range(base - 2, base + 3):
            if 128 <= k < 256:                   # 8 significant bits
                cands.add((k, int(ee - 8)))
    X = Fraction(abs(x))
    best = min(cands, key=lambda c: (abs(Fraction(c[0]) * Fraction(2) ** c[1] - X), c[0] & 1))
    return float(np.copysign(best[0] * 2.0 ** best[1], x))


def test_round_bf16_double_single_rounding(orc):
    """FP64 -> BF16 in one rounding against a brute-force nearest search,
    including doubles just off a BF16 midpoint, where rounding through FP32
    first would land on the other neighbour."""
    rng = np.random.default_rng(11)
    vals = list(rng.standard_normal(3000) * 2.0 ** rng.integers(-30, 30, 3000))
    for k in range(128, 256, 7):
        for e in (-20, -3, 0, 5):
            mid = (k + 0.5) * 2.0 ** e                # exact BF16 midpoint
            vals += [mid, -mid, mid * (1 + 2.0 ** -40), mid * (1 - 2.0 ** -40)]
    for v in vals:
        assert orc.round_bf16_d(v) == _nearest_bf16_bruteforce(float(v)), v
    # a double just above a midpoint whose FP32 rounding is the midpoint itself
    x = (129 + 0.5) * 2.0 ** -7 * (1 + 2.0 ** -30)
    assert np.float32(x) == np.float32((129 + 0.5) * 2.0 ** -7)
    assert orc.round_bf16_d(x) == 130 * 2.0 ** -7


def test_mxp_factor_bf16_storage(orc):
    """BF16 storage of the working matrix: every stored value is a BF16 value;
    one block is the FP32-storage factor of the BF16-rounded matrix (rounding
    pinned above); the factorization error sits between the FP32-storage
    error and the BF16 unit roundoff; the refinement still reaches the HPL
    tolerance with an FP64-accurate solution."""
    n, nb = 192, 64
    A = orc.generate(5, orc.STREAM_A, n, n, dominant=True)
    F, Dinv, info = orc.mxp_factor(A, nb, orc.PREC_BF16, storage=orc.STORAGE_BF16)
    assert info == 0
    assert all(orc.round_bf16(float(v)) == float(v) for v in F.ravel()[::7])
    # one block: only the storage rounding of the input differs
    A1 = A[:48, :48]
    F1, D1, _ = orc.mxp_factor(A1, 64, orc.PREC_BF16, storage=orc.STORAGE_BF16)
    Ar = np.vectorize(_nearest_bf16_bruteforce)(A1)
    F2, D2, _ = orc.mxp_factor(Ar, 64, orc.PREC_BF16, storage=orc.STORAGE_FP32)
    assert np.array_equal(F1, F2) and np.array_equal(D1, D2)

    def err(storage):
        Fx, _, _ = orc.mxp_factor(A, nb, orc.PREC_BF16, storage=storage)
        L, U = orc.block_lu_parts(Fx, nb)
        return np.abs(A - L @ U).max() / np.abs(A).max()
    e32, e16 = err(orc.STORAGE_FP32), err(orc.STORAGE_BF16)
    assert e32 < e16 < 2.0 ** -7
    b = orc.generate(5, orc.STREAM_B, n, 1)[:, 0]
    out = orc.mxp_solve(A, b, nb, refine=1, storage=orc.STORAGE_BF16)
    assert out["status"] == 0 and orc.scaled_residual(A, out["x"], b) < 16
    x64, _ = orc.solve(A, b)
    assert np.abs(out["x"] - x64).max() / np.abs(x64).max() < 2 * 16 * n * 2.0 ** -53 * np.linalg.cond(A, np.inf)


def test_fp16_factor_needs_no_more_corrections_than_bf16(orc):
    """Classic refinement contracts the error by about the factorization's
    relative accuracy per step, so the more accurate FP16 factor (8x smaller
    error, pinned above) never needs more corrections than the BF16 one."""
    n, nb = 384, 64
    A = orc.generate(8, orc.STREAM_A, n, n, dominant=True)
    b = orc.generate(8, orc.STREAM_B, n, 1)[:, 0]
    it16 = orc.mxp_solve(A, b, nb, prec=orc.PREC_FP16, refine=0)
    itbf = orc.mxp_solve(A, b, nb, prec=orc.PREC_BF16, refine=0)
    assert it16["status"] == 0 and itbf["status"] == 0
    assert it16["iters"] <= itbf["iters"]


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_mxp_inner_fp32_reaches_fp64_solution(orc, prec):
    """GMRES with inner products from the FP32 rounding of A and the vector
    still reaches the FP64 solution (the residual of each outer step is FP64),
    in at most a few more outer steps than with FP64 inner products; with FP32
    operands the inner products really differ (a correction is less exact)."""
    n, nb = 512, 128
    A = orc.generate(7, orc.STREAM_A, n, n, dominant=True)
    b = orc.generate(7, orc.STREAM_B, n, 1)[:, 0]
    r64 = orc.mxp_solve(A, b, nb, prec=prec, inner=orc.INNER_FP64)
    r32 = orc.mxp_solve(A, b, nb, prec=prec, inner=orc.INNER_FP32)
    assert r32["status"] == 0 and r32["sr"] < 16
    x64, _ = orc.solve(A, b)
    bound = 2 * 16 * n * EPS * np.linalg.cond(A, np.inf)
    assert np.abs(r32["x"] - x64).max() / np.abs(x64).max() < bound
    assert r64["iters"] <= r32["iters"] <= r64["iters"] + 3
    # after the first correction the FP32 inner products leave a larger residual
    assert r32["hist"][1] > r64["hist"][1]



def test_newton_schulz_first_step_closed_form(orc):
    """One Newton-Schulz step from X0 = diag(D)^-1 is X1 = 2 X0 - X0 D X0 (the
    two products of a diagonal X0 are scalings): the oracle's one-step inverse
    equals that closed form, evaluated in FP64 from the same FP32 diagonal
    blocks, to within three FP32 roundings per entry; a second step moves it
    (the later steps really are products)."""
    n, nb = 300, 100
    A = orc.generate(16, orc.STREAM_A, n, n, dominant=True)
    F1, D1, _ = orc.mxp_factor(A, nb, orc.PREC_BF16, ns_iters=1)
    F2, D2, _ = orc.mxp_factor(A, nb, orc.PREC_BF16, ns_iters=2)
    for k0 in range(0, n, nb):
        D = F1[k0:k0 + nb, k0:k0 + nb].astype(np.float64)
        x0 = np.diag(1.0 / np.diag(D).astype(np.float32).astype(np.float64))
        want = 2 * x0 - x0 @ D @ x0
        got = D1[k0:k0 + nb, :].astype(np.float64)
        assert np.all(np.abs(got - want) <= 4 * 2.0 ** -24 * (np.abs(x0) @ (np.abs(D) @ np.abs(x0)) + 2 * np.abs(x0)))
    assert not np.array_equal(D1[:nb], D2[:nb])


def _nearest_tf32_bruteforce(x: float) -> float:
    """The TF32 value nearest to x (FP32's exponent range, 11 significant bits
    for normals, the fixed spacing 2^-136 below 2^-126; ties to an even last
    fraction bit), by exact comparison of every grid point around x."""
    if x == 0.0:
        return 0.0
    X = Fraction(abs(x))
    cands = set()
    # normal grid points k 2^(ee-10), 2^10 <= k < 2^11, around x
    e = int(np.frexp(abs(x))[1]) - 1             # 2^e <= |x| < 2^(e+1)
    for ee in (e - 1, e, e + 1):
        if ee < -126:
            continue
        q = Fraction(2) ** (ee - 10)
        base = int(X / q)
        for k in range(base - 2, base + 3):
            if 1024 <= k < 2048:
                cands.add((Fraction(k) * q, k))
        if ee == 127:
            cands.add((Fraction(2) ** 128, 2))  # the overflow point (even)
    # subnormal grid points k 2^-136, 0 <= k < 2^10
    q = Fraction(2) ** -136
    base = int(X / q)
    for k in range(base - 2, base + 3):
        if 0 <= k < 1024:
            cands.add((Fraction(k) * q, k))
    best = min(cands, key=lambda c: (abs(c[0] - X), c[1] & 1))
    v = float(best[0]) if best[0] < Fraction(2) ** 128 else float("inf")
    return float(np.copysign(v, x))


def test_round_tf32_matches_bruteforce(orc):
    """TF32 rounding against the nearest-grid-point search: random values over
    the whole exponent range, exact ties and values one FP32 unit off a tie,
    subnormals, and the overflow threshold."""
    rng = np.random.default_rng(21)
    vals = list((rng.standard_normal(1500) * 10.0 ** rng.integers(-35, 35, 1500)).astype(np.float32))
    bits = rng.integers(0x00800000, 0x7f000000, 300, dtype=np.uint32)
    for b in bits:                                 # ties (low 13 bits 0x1000) and their neighbours
        hi = int(b) & ~0x1FFF
        for low in (0x1000, 0x0FFF, 0x1001, 0x0000, 0x1FFF):
            vals.append(np.array([hi | low], dtype=np.uint32).view(np.float32)[0])
    vals += list(np.array([0x00000001, 0x00001000, 0x00003000, 0x007FFFFF, 0x007FF000, 0x00800000,
                           0x7F7FF000, 0x7F7FEFFF, 0x7F7FF001, 0x7F7FFFFF], dtype=np.uint32).view(np.float32))
    for v in vals:
        for sgn in (1.0, -1.0):
            x = float(np.float32(sgn * v))
            got = orc.round_tf32(x)
            want = _nearest_tf32_bruteforce(x)
            assert got == want or (np.isinf(got) and np.isinf(want) and np.sign(got) == np.sign(want)), (x, got, want)
            assert np.isinf(got) or (np.array([got], dtype=np.float32).view(np.uint32)[0] & 0x1FFF) == 0


def test_mxp_tf32_operands(orc):
    """TF32 operands (no scales) in the panel product and the update: the
    factor's backward error sits between FP32 and BF16 and near FP16's (the
    same 11 significant bits), for both readings of the factorization, and
    the refinement reaches the FP64 solution."""
    from _parity import block_lu_backward_error, plain_lu_backward_error
    n, nb = 384, 128
    A = orc.generate(44, orc.STREAM_A, n, n, dominant=True)
    b = orc.generate(44, orc.STREAM_B, n, 1)[:, 0]
    eb = {p: block_lu_backward_error(A, orc.mxp_factor(A, nb, p)[0], nb) for p in (3, 4, 2, 0)}
    ep = {p: plain_lu_backward_error(A, orc.mxp_lu_plain(A, nb, p)[0]) for p in (3, 4, 2, 0)}
    for e in (eb, ep):
        assert e[3] < e[4] < e[0]
        assert e[4] < 4 * e[2] and e[2] < 4 * e[4]
    out = orc.mxp_solve(A, b, nb, prec=orc.PREC_TF32)
    assert out["status"] == 0 and out["sr"] < 16
    x64, _ = orc.solve(A, b)
    assert np.abs(out["x"] - x64).max() / np.abs(x64).max() < 2 * 16 * n * EPS * np.linalg.cond(A, np.inf)


def _block_prec(F, Dinv, nb):
    """M^-1 of the block factor, restated in numpy from its definition: block
    forward substitution with the block unit lower L (the blocks of F below
    the diagonal), then block backward substitution with U (the blocks of F on
    and above it), each diagonal block D_k applied through its approximate
    inverse Dinv_k. Computed in FP64 on the factor's values so that it is
    linear to rounding (scipy's GMRES forms M^-1 of a combination of basis
    vectors, the oracle the combination of M^-1 of each)."""
    F64 = np.asarray(F, dtype=np.float64)
    D64 = np.asarray(Dinv, dtype=np.float64)
    n = F64.shape[0]
    blocks = [(k0, min(n, k0 + nb)) for k0 in range(0, n, nb)]

    def apply(v):
        y = np.array(v, dtype=np.float64)
        for k0, k1 in blocks:
            for j0, j1 in blocks:
                if j0 >= k0:
                    break
                y[k0:k1] -= F64[k0:k1, j0:j1] @ y[j0:j1]
        x = np.zeros(n)
        for k0, k1 in reversed(blocks):
            x[k0:k1] = D64[k0:k1, :k1 - k0] @ (y[k0:k1] - F64[k0:k1, k1:] @ x[k1:])
        return x
    return apply


def _plain_prec(F):
    """M^-1 of the plain factor (L unit lower, U upper, both in F): two
    triangular solves (LAPACK through scipy), in FP64 on the factor's values
    for the same reason."""
    from scipy.linalg import solve_triangular
    F64 = np.asarray(F, dtype=np.float64)

    def apply(v):
        y = solve_triangular(F64, np.asarray(v, dtype=np.float64), lower=True, unit_diagonal=True)
        return solve_triangular(F64, y, lower=False)
    return apply


def _gmres_ir_scipy(A, b, apply_minv, m=30, tol=16.0, max_iter=50):
    """GMRES-based iterative refinement (Sec. II-B) around scipy's GMRES: x0 =
    M^-1 b; while the HPL scaled residual of the FP64 residual r = b - A x is
    16 or more, one restart cycle of GMRES on A M^-1 u = r (at most m steps,
    stopping at a residual of 1e-10 |r|) and x += M^-1 u. Returns (outer
    corrections, GMRES steps, final scaled residual)."""
    from scipy.sparse.linalg import LinearOperator, gmres
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    anorm = np.abs(A).sum(axis=1).max()
    bnorm = np.abs(b).max()
    B = LinearOperator((n, n), matvec=lambda u: A @ apply_minv(np.ravel(u)), dtype=np.float64)
    x = apply_minv(b)
    outer = steps = 0
    while True:
        r = b - A @ x
        sr = np.abs(r).max() / (EPS * (anorm * np.abs(x).max() + bnorm) * n)
        if sr < tol or outer >= max_iter:
            return outer, steps, sr
        seen = []
        u, _ = gmres(B, r, rtol=1e-10, atol=0.0, restart=m, maxiter=1, callback=seen.append,
                     callback_type="pr_norm")
        steps += len(seen)
        x = x + apply_minv(u)
        outer += 1


@pytest.mark.parametrize("prec", ["PREC_BF16", "PREC_FP16", "PREC_FP8"])
@pytest.mark.parametrize("case", ["dominant", "weak"])
def test_mxp_refinement_counts_match_scipy_gmres(orc, prec, case):
    """The oracle's GMRES-IR iteration counts (outer corrections and GMRES
    steps), for the block factor and for the plain factor, against the same
    refinement written around scipy's GMRES with each preconditioner restated
    in numpy (in FP64 where the oracle applies it in FP32, a 1e-7 difference
    against the factor's own 2^-8 .. 2^-4): the same outcome and number of
    corrections and at most one GMRES step apart per restart cycle (rounding
    can move the 1e-10 crossing by one step). Cases: the HPL-MxP matrix with
    restarts of 30, and a weakly dominant one (diagonal 0.1 of the absolute
    row sum) with restarts of 3, several cycles. This pins the FP8 counts,
    which no closed form gives."""
    pytest.importorskip("scipy")
    p = getattr(orc, prec)
    n, nb = 384, 64
    b = orc.generate(12, orc.STREAM_B, n, 1)[:, 0]
    if case == "dominant":
        A, m = orc.generate(12, orc.STREAM_A, n, n, dominant=True), 30
    else:
        R = orc.generate(12, orc.STREAM_A, n, n)
        A, m = R + 0.1 * np.diag(np.abs(R).sum(axis=1)), 3
    F, Dinv, info = orc.mxp_factor(A, nb, p)
    assert info == 0
    Fp, info = orc.mxp_lu_plain(A, nb, p)
    assert info == 0
    for out, minv in ((orc.mxp_refine(A, F, Dinv, nb, b, refine=1, gmres_m=m), _block_prec(F, Dinv, nb)),
                      (orc.mxp_refine_plain(A, Fp, b, refine=1, gmres_m=m), _plain_prec(Fp))):
        outer, steps, sr = _gmres_ir_scipy(A, b, minv, m=m)
        assert out["status"] == 0 and sr < 16
        assert out["iters"] == outer, (out["iters"], outer)
        assert abs(out["inner"] - steps) <= outer, (out["inner"], steps)


def test_scaled_residual_is_nan_for_nonfinite_solution(orc):
    """A NaN in x (or a NaN residual entry) is no pass of the acceptance test:
    the scaled residual is NaN, never below 16."""
    n = 64
    A = orc.generate(3, orc.STREAM_A, n, n)
    b = orc.generate(3, orc.STREAM_B, n, 1)[:, 0]
    x, _ = orc.solve(A, b)
    assert orc.scaled_residual(A, x, b) < 16
    for bad in (np.nan, np.inf):
        y = x.copy()
        y[17] = bad
        assert np.isnan(orc.scaled_residual(A, y, b))
        assert np.isnan(orc.scaled_residual_gen(3, n, False, y, b))


def test_mxp_refinement_reports_nonfinite(orc):
    """Where the unpivoted low-precision factor is a useless preconditioner
    (a matrix far from diagonal dominance), refinement ends with status 3
    (non-finite) once its iterate overflows, instead of reading the NaN
    residual as a pass."""
    n, nb = 384, 64
    R = orc.generate(12, orc.STREAM_A, n, n)
    b = orc.generate(12, orc.STREAM_B, n, 1)[:, 0]
    F, Dinv, _ = orc.mxp_factor(R, nb, orc.PREC_FP8)
    out = orc.mxp_refine(R, F, Dinv, nb, b, refine=0)
    assert out["status"] == 3 and not np.isfinite(out["x"]).all()
    A = R + 0.05 * np.diag(np.abs(R).sum(axis=1))     # I - M^-1 A has spectral radius ~ 10: IR diverges
    F, Dinv, _ = orc.mxp_factor(A, nb, orc.PREC_FP8)
    assert orc.mxp_refine(A, F, Dinv, nb, b, refine=0)["status"] == 3
    assert orc.mxp_refine(A, F, Dinv, nb, b, refine=1)["status"] == 4     # GMRES: no blow-up, no convergence
