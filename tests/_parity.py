"""Comparison helpers shared by the parity tests (CPU and GPU).

Nothing here computes the method: these are the yardsticks the tests apply
to a result and its reference (the oracle's output, or finite differences
taken with numpy's LAPACK solve).
"""
from __future__ import annotations

import numpy as np


# --- block factor of the mixed-precision solve -----------------------------------------

def factor_blocks(n: int, nb: int):
    """(k0, k1) of every block step of an n x n block factor with panel nb."""
    return [(k0, min(n, k0 + nb)) for k0 in range(0, n, nb)]


def block_errors(Fg, Fo, nb: int) -> list[dict]:
    """Per step k of the block factor F (L21 below the diagonal block, the
    block row of U right of it, the Schur-complemented diagonal block D_k on
    it), the largest |Fg - Fo| of each part relative to the largest |Fo| of
    the same part: L21, U12, the off-diagonal of D_k and its diagonal. A part
    with no entries, or whose reference is all zero, reports 0 (and the
    difference must then be exactly zero: reported as inf otherwise)."""
    Fg = np.asarray(Fg, dtype=np.float64)
    Fo = np.asarray(Fo, dtype=np.float64)
    n = Fo.shape[0]
    out = []

    def rel(g, o):
        if o.size == 0:
            return 0.0
        d = np.abs(g - o).max()
        s = np.abs(o).max()
        if s == 0.0:
            return 0.0 if d == 0.0 else np.inf
        return float(d / s)

    for k0, k1 in factor_blocks(n, nb):
        D_g, D_o = Fg[k0:k1, k0:k1], Fo[k0:k1, k0:k1]
        off = ~np.eye(k1 - k0, dtype=bool)
        out.append(dict(k0=k0,
                        L21=rel(Fg[k1:, k0:k1], Fo[k1:, k0:k1]),
                        U12=rel(Fg[k0:k1, k1:], Fo[k0:k1, k1:]),
                        Doff=rel(D_g[off], D_o[off]),
                        Ddiag=rel(np.diag(D_g), np.diag(D_o))))
    return out


def assert_blocks_close(Fg, Fo, nb: int, l21: float, u12: float, doff: float, ddiag: float):
    """Every part of every step within its own relative tolerance."""
    for e in block_errors(Fg, Fo, nb):
        assert e["L21"] <= l21, e
        assert e["U12"] <= u12, e
        assert e["Doff"] <= doff, e
        assert e["Ddiag"] <= ddiag, e


# Largest ratio of the block factor's backward error to the plain LU's, by
# operand precision (0 BF16, 1 FP8, 2 FP16, 4 TF32). The block LU forms L21 = A21 D^-1
# with A21 itself rounded to the operand precision, an error of one rounding
# of |A21| (~1/2); the plain LU rounds only the update's operands L21 (~2/n)
# and U12. Measured on the oracle's two emulations at n <= 2560: 18-55x for
# BF16, FP16 and TF32 (growing with n), 1.8-4x for FP8, whose rounding of the
# update dominates both.
BLOCK_VS_PLAIN_BERR = {0: 100.0, 1: 8.0, 2: 100.0, 4: 100.0}


def block_lu_backward_error(A, F, nb: int) -> float:
    """||A - L U||_inf / ||A||_inf of a block factor (L block unit lower with
    the L21 blocks, U block upper with the D_k and U12 blocks)."""
    A = np.asarray(A, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    n = A.shape[0]
    L = np.eye(n)
    U = np.zeros((n, n))
    for k0, k1 in factor_blocks(n, nb):
        L[k1:, k0:k1] = F[k1:, k0:k1]
        U[k0:k1, k0:] = F[k0:k1, k0:]
    return float(np.abs(A - L @ U).sum(axis=1).max() / np.abs(A).sum(axis=1).max())


def plain_lu_backward_error(A, F) -> float:
    """||A - L U||_inf / ||A||_inf of a conventional LU (L unit lower strictly
    below the diagonal of F, U upper on and above it)."""
    A = np.asarray(A, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    n = A.shape[0]
    L = np.tril(F, -1) + np.eye(n)
    U = np.triu(F)
    return float(np.abs(A - L @ U).sum(axis=1).max() / np.abs(A).sum(axis=1).max())


# --- finite differences of the solve -------------------------------------------------------

FD_STEP = 2.0 ** -10


def fd_gradients(A, B, G, h: float = FD_STEP):
    """Central differences of f(A, B) = sum(G * A^-1 B) in FP64 for every
    entry of A and of B (numpy's LAPACK solve). The step is absolute: for a
    perturbation of a_ij by +-h the central difference equals the gradient
    times 1 / (1 - (h (A^-1)_ji)^2) exactly (Sherman-Morrison), so the
    truncation error is relative to the entry itself; f is linear in B, so
    there the difference has rounding error only. The actual step (the
    difference of the two perturbed values as stored) is the divisor."""
    A = np.array(A, dtype=np.float64)
    B = np.array(B, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    n, nrhs = B.shape

    def f(Am, Bm):
        return float(np.sum(G * np.linalg.solve(Am, Bm)))

    fdA = np.empty((n, n))
    for i in range(n):
        for j in range(n):
            a = A[i, j]
            A[i, j] = a + h
            fp = f(A, B)
            up = A[i, j]
            A[i, j] = a - h
            fm = f(A, B)
            dn = A[i, j]
            A[i, j] = a
            fdA[i, j] = (fp - fm) / (up - dn)
    fdB = np.empty((n, nrhs))
    for i in range(n):
        for c in range(nrhs):
            v = B[i, c]
            B[i, c] = v + h
            fp = f(A, B)
            up = B[i, c]
            B[i, c] = v - h
            fm = f(A, B)
            dn = B[i, c]
            B[i, c] = v
            fdB[i, c] = (fp - fm) / (up - dn)
    return fdA, fdB


def max_rel_err(got, want) -> float:
    """Largest |got - want| / |want| over all entries; an entry whose
    reference is exactly zero must be exactly zero (inf otherwise)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    nz = want != 0.0
    if np.any(got[~nz] != 0.0):
        return float("inf")
    if not np.any(nz):
        return 0.0
    return float(np.max(np.abs(got[nz] - want[nz]) / np.abs(want[nz])))
