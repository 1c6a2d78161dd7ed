"""CPU oracle for the HPL / HPL-MxP dense LU solve (test infrastructure).

This package is the plain, slow, FP64 statement of what the GPU library
computes, written from the paper (arXiv 2604.09517, Sec. III-A.1 for HPL,
Sec. III-A.2 for HPL-MxP, Sec. II-B for GMRES-based refinement) and from the
published methods it names. Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it. The GPU library never
calls it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, OpenMP); this module builds it
with gcc and exposes thin numpy wrappers. All matrices are numpy arrays in
Fortran (column-major) order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

# Stream tags of the generator (see oracle.c).
STREAM_A = 0
STREAM_B = 1
STREAM_BATCH_SIZES = 2


def batch_stream_a(s: int) -> int:
    return 16 + 2 * s


def batch_stream_b(s: int) -> int:
    return 17 + 2 * s


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, -O3, OpenMP).

    FMA contraction is off so the oracle gives the same bits on x86 and Arm.
    """
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, u64, dp, fp, ip = (ctypes.c_int64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32))
        i64p = ctypes.POINTER(ctypes.c_int64)
        intp = ctypes.POINTER(ctypes.c_int)
        sig = {
            "orc_sm64_next": (u64, [u64, u64]),
            "orc_stream_key": (u64, [u64, u64]),
            "orc_raw": (u64, [u64, u64]),
            "orc_uniform": (ctypes.c_double, [u64, u64]),
            "orc_generate": (None, [u64, u64, i64, i64, ctypes.c_int, dp, i64]),
            "orc_generate_at": (None, [u64, u64, i64, ctypes.c_int, i64, i64p, i64p, dp]),
            "orc_getrf": (i64, [i64, dp, i64, ip, dp]),
            "orc_getrs": (None, [i64, i64, dp, i64, ip, ctypes.c_int, dp, i64]),
            "orc_scaled_residual": (ctypes.c_double, [i64, dp, i64, dp, dp]),
            "orc_scaled_residual_gen": (ctypes.c_double, [u64, i64, ctypes.c_int, dp, dp]),
            "orc_perm_from_ipiv": (None, [i64, ip, i64p]),
            "orc_lu_sample_diff": (None, [u64, i64, ctypes.c_int, dp, i64, i64p, i64, i64p, i64p, dp]),
            "orc_round_bf16": (ctypes.c_float, [ctypes.c_float]),
            "orc_round_e4m3": (ctypes.c_float, [ctypes.c_float]),
            "orc_round_fp16": (ctypes.c_float, [ctypes.c_float]),
            "orc_round_tf32": (ctypes.c_float, [ctypes.c_float]),
            "orc_round_operand_ext": (None, [ctypes.c_int, fp, i64, i64, i64, ctypes.c_int]),
            "orc_mxp_factor": (i64, [i64, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, fp, i64, fp]),
            "orc_to_bf16_storage": (None, [i64, i64, dp, i64, fp, i64]),
            "orc_round_bf16_d": (ctypes.c_float, [ctypes.c_double]),
            "orc_mxp_refine": (ctypes.c_int, [i64, dp, i64, i64, fp, i64, fp, dp, dp, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_int, ctypes.c_double, intp, intp, dp, dp]),
            "orc_mxp_lu_plain": (i64, [i64, i64, ctypes.c_int, fp, i64]),
            "orc_mxp_refine_plain": (ctypes.c_int, [i64, dp, i64, fp, i64, dp, dp, ctypes.c_int, ctypes.c_int,
                                                    ctypes.c_int, ctypes.c_int, ctypes.c_double, intp, intp, dp,
                                                    dp]),
            "orc_adjoint": (i64, [i64, i64, dp, i64, dp, i64, dp, i64, dp, i64, dp, i64]),
            "orc_batch_sizes": (None, [u64, i64, i64p]),
            "orc_num_threads": (ctypes.c_int, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _i64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _fortran(a, dtype):
    a = np.asarray(a, dtype=dtype)
    return np.asfortranarray(a)


def num_threads() -> int:
    return int(_load().orc_num_threads())


# --- generator -------------------------------------------------------------

def sm64_next(state: int, c: int) -> int:
    """c-th SplitMix64 output (c >= 1) from initial state ``state``."""
    return int(_load().orc_sm64_next(state & (2**64 - 1), c & (2**64 - 1)))


def stream_key(seed: int, stream: int) -> int:
    return int(_load().orc_stream_key(seed, stream))


def raw(key: int, idx: int) -> int:
    return int(_load().orc_raw(key, idx))


def generate(seed: int, stream: int, m: int, ncols: int, dominant: bool = False) -> np.ndarray:
    """m x ncols matrix of stream ``stream`` (Fortran order)."""
    A = np.empty((m, ncols), dtype=np.float64, order="F")
    _load().orc_generate(seed, stream, m, ncols, int(bool(dominant)), _dp(A), max(m, 1))
    return A


def generate_at(seed: int, stream: int, m: int, rows, cols, dominant: bool = False) -> np.ndarray:
    """Entries (rows[t], cols[t]) of the m-row matrix of a stream."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    out = np.empty(rows.shape[0], dtype=np.float64)
    _load().orc_generate_at(seed, stream, m, int(bool(dominant)), rows.shape[0], _i64p(rows), _i64p(cols), _dp(out))
    return out


def batch_sizes(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.int64)
    _load().orc_batch_sizes(seed, count, _i64p(out))
    return out


# --- HPL ---------------------------------------------------------------------

def getrf(A):
    """LU with partial pivoting. Returns (LU, ipiv, info, min_gap)."""
    LU = _fortran(A, np.float64).copy(order="F")
    n = LU.shape[0]
    assert LU.shape == (n, n)
    ipiv = np.zeros(n, dtype=np.int32)
    gap = ctypes.c_double(0.0)
    info = _load().orc_getrf(n, _dp(LU), max(n, 1), _ip(ipiv), ctypes.byref(gap))
    return LU, ipiv, int(info), float(gap.value)


def getrs(LU, ipiv, B, trans: int = 0):
    LU = _fortran(LU, np.float64)
    X = _fortran(B, np.float64).copy(order="F")
    vec = X.ndim == 1
    if vec:
        X = X.reshape(-1, 1, order="F")
    n, nrhs = X.shape
    ipiv = np.ascontiguousarray(ipiv, dtype=np.int32)
    _load().orc_getrs(n, nrhs, _dp(LU), max(n, 1), _ip(ipiv), int(trans), _dp(X), max(n, 1))
    return X[:, 0].copy() if vec else X


def solve(A, B):
    LU, ipiv, info, _ = getrf(A)
    return getrs(LU, ipiv, B), info


def scaled_residual(A, x, b) -> float:
    A = _fortran(A, np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = A.shape[0]
    return float(_load().orc_scaled_residual(n, _dp(A), max(n, 1), _dp(x), _dp(b)))


def scaled_residual_gen(seed: int, n: int, dominant: bool, x, b) -> float:
    """Scaled residual with A regenerated from (seed, stream 0)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return float(_load().orc_scaled_residual_gen(seed, n, int(bool(dominant)), _dp(x), _dp(b)))


def perm_from_ipiv(ipiv) -> np.ndarray:
    ipiv = np.ascontiguousarray(ipiv, dtype=np.int32)
    out = np.empty(ipiv.shape[0], dtype=np.int64)
    _load().orc_perm_from_ipiv(ipiv.shape[0], _ip(ipiv), _i64p(out))
    return out


def lu_sample_diff(seed: int, n: int, dominant: bool, LU, ipiv, si, sj) -> np.ndarray:
    """(PA - LU)_ij at sampled (i,j), A regenerated, for factors too big to redo."""
    LU = _fortran(LU, np.float64)
    rowmap = perm_from_ipiv(ipiv)
    si = np.ascontiguousarray(si, dtype=np.int64)
    sj = np.ascontiguousarray(sj, dtype=np.int64)
    out = np.empty(si.shape[0], dtype=np.float64)
    _load().orc_lu_sample_diff(seed, n, int(bool(dominant)), _dp(LU), LU.shape[0], _i64p(rowmap),
                               si.shape[0], _i64p(si), _i64p(sj), _dp(out))
    return out


# --- HPL-MxP ------------------------------------------------------------------

PREC_BF16 = 0
PREC_FP8 = 1
PREC_FP16 = 2
PREC_FP32 = 3
PREC_TF32 = 4


def round_bf16_d(x: float) -> float:
    """A double rounded once to BF16 (round to nearest even)."""
    return float(_load().orc_round_bf16_d(float(x)))


def round_bf16(x: float) -> float:
    return float(_load().orc_round_bf16(float(x)))


def round_e4m3(x: float) -> float:
    return float(_load().orc_round_e4m3(float(x)))


def round_fp16(x: float) -> float:
    return float(_load().orc_round_fp16(float(x)))


def round_tf32(x: float) -> float:
    return float(_load().orc_round_tf32(float(x)))


def round_operand(prec: int, X, kdim_is_rows: bool) -> np.ndarray:
    """An FP32 operand rounded as the factorization rounds it (dequantised):
    kdim_is_rows for a B operand (K x cols), else an A operand (rows x K)."""
    X = np.asfortranarray(np.asarray(X, dtype=np.float32)).copy(order="F")
    r, c = X.shape
    _load().orc_round_operand_ext(prec, _fp(X), r, c, max(r, 1), int(bool(kdim_is_rows)))
    return X


NS_ITERS = 2


STORAGE_FP32 = 0
STORAGE_BF16 = 1


def mxp_factor(A, nb: int, prec: int = PREC_BF16, ns_iters: int = NS_ITERS, storage: int = STORAGE_FP32):
    """Block LU without pivoting of the FP32 (storage 0) or BF16 (storage 1)
    working copy of A (see oracle.c). Returns (F, Dinv, info).

    F holds L21 blocks below the diagonal, the block rows A12 above it and the
    Schur-complemented diagonal blocks D_k on it; Dinv (n x nb) holds D_k^-1
    in rows k0..k0+kb.
    """
    A64 = _fortran(A, np.float64)
    n = A64.shape[0]
    if storage == STORAGE_BF16:
        F = np.zeros((n, n), dtype=np.float32, order="F")
        _load().orc_to_bf16_storage(n, n, _dp(A64), max(n, 1), _fp(F), max(n, 1))
    else:
        F = np.asfortranarray(A64.astype(np.float32))
    Dinv = np.zeros((n, nb), dtype=np.float32, order="F")
    info = _load().orc_mxp_factor(n, nb, prec, ns_iters, storage, _fp(F), max(n, 1), _fp(Dinv))
    return F, Dinv, int(info)


def block_lu_parts(F, nb: int):
    """(L, U) of the block factor as dense FP64 matrices: L block unit lower,
    U block upper with the D_k on its diagonal."""
    F = np.asarray(F, dtype=np.float64)
    n = F.shape[0]
    L = np.eye(n)
    U = np.zeros((n, n))
    for k0 in range(0, n, nb):
        k1 = min(n, k0 + nb)
        L[k1:, k0:k1] = F[k1:, k0:k1]
        U[k0:k1, k0:] = F[k0:k1, k0:]
    return L, U


INNER_FP64 = 0
INNER_FP32 = 1


def mxp_refine(A, F, Dinv, nb: int, b, refine: int = 1, max_iter: int = 50, gmres_m: int = 30,
               tol: float = 16.0, inner: int = INNER_FP64):
    """Refine with the block factor (F, Dinv). inner = INNER_FP32 takes GMRES's
    inner products from the FP32 rounding of A and of the vector. Returns
    dict(x, status, iters, inner, sr, hist)."""
    A = _fortran(A, np.float64)
    F = np.asfortranarray(F, dtype=np.float32)
    Dinv = np.asfortranarray(Dinv, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = A.shape[0]
    x = np.zeros(n, dtype=np.float64)
    it, inn = ctypes.c_int(0), ctypes.c_int(0)
    sr = ctypes.c_double(0.0)
    hist = np.full(max_iter + 1, np.nan)
    st = _load().orc_mxp_refine(n, _dp(A), max(n, 1), nb, _fp(F), max(n, 1), _fp(Dinv), _dp(b), _dp(x),
                                int(refine), int(max_iter), int(gmres_m), int(inner), float(tol), ctypes.byref(it),
                                ctypes.byref(inn), ctypes.byref(sr), _dp(hist))
    return dict(x=x, status=int(st), iters=int(it.value), inner=int(inn.value), sr=float(sr.value),
                hist=hist[: it.value + 1])


def mxp_solve(A, b, nb: int, prec: int = PREC_BF16, refine: int = 1, max_iter: int = 50,
              gmres_m: int = 30, tol: float = 16.0, ns_iters: int = NS_ITERS, storage: int = STORAGE_FP32,
              inner: int = INNER_FP64):
    F, Dinv, info = mxp_factor(A, nb, prec, ns_iters, storage)
    out = mxp_refine(A, F, Dinv, nb, b, refine, max_iter, gmres_m, tol, inner)
    out["F"] = F
    out["Dinv"] = Dinv
    out["info"] = info
    return out


def mxp_lu_plain(A, nb: int, prec: int = PREC_BF16):
    """The paper-order HPL-MxP factor: plain right-looking LU without
    pivoting of the FP32 working copy of A, FP32 panel and U12 solve, trailing
    update with operands rounded to ``prec`` and FP32 accumulation (see
    oracle.c). Returns (F, info): L strictly below the diagonal, U on and
    above it, as float32."""
    F = np.asfortranarray(_fortran(A, np.float64).astype(np.float32))
    n = F.shape[0]
    info = _load().orc_mxp_lu_plain(n, nb, prec, _fp(F), max(n, 1))
    return F, int(info)


def mxp_refine_plain(A, F, b, refine: int = 1, max_iter: int = 50, gmres_m: int = 30, tol: float = 16.0,
                     inner: int = INNER_FP64):
    """Refinement (classic or GMRES-IR) with the plain factor F as M = L U,
    applied in FP32. Returns dict(x, status, iters, inner, sr, hist)."""
    A = _fortran(A, np.float64)
    F = np.asfortranarray(F, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = A.shape[0]
    x = np.zeros(n, dtype=np.float64)
    it, inn = ctypes.c_int(0), ctypes.c_int(0)
    sr = ctypes.c_double(0.0)
    hist = np.full(max_iter + 1, np.nan)
    st = _load().orc_mxp_refine_plain(n, _dp(A), max(n, 1), _fp(F), max(n, 1), _dp(b), _dp(x), int(refine),
                                      int(max_iter), int(gmres_m), int(inner), float(tol), ctypes.byref(it),
                                      ctypes.byref(inn), ctypes.byref(sr), _dp(hist))
    return dict(x=x, status=int(st), iters=int(it.value), inner=int(inn.value), sr=float(sr.value),
                hist=hist[: it.value + 1])


def mxp_solve_plain(A, b, nb: int, prec: int = PREC_BF16, refine: int = 1, max_iter: int = 50,
                    gmres_m: int = 30, tol: float = 16.0, inner: int = INNER_FP64):
    F, info = mxp_lu_plain(A, nb, prec)
    out = mxp_refine_plain(A, F, b, refine, max_iter, gmres_m, tol, inner)
    out["F"] = F
    out["info"] = info
    return out


# --- adjoint -------------------------------------------------------------------

def adjoint(A, X, G, want_grad_a: bool = True):
    """grad_B = A^-T G, grad_A = -grad_B X^T (FP64 LU of A)."""
    A = _fortran(A, np.float64)
    X = _fortran(X, np.float64)
    G = _fortran(G, np.float64)
    n, nrhs = G.shape
    gB = np.empty((n, nrhs), dtype=np.float64, order="F")
    gA = np.empty((n, n), dtype=np.float64, order="F") if want_grad_a else None
    _load().orc_adjoint(n, nrhs, _dp(A), n, _dp(X), n, _dp(G), n, _dp(gB), n,
                        _dp(gA) if gA is not None else None, n)
    return gB, gA


def flops(n: int) -> float:
    """Operation count credited to one solve: 2n^3/3 + 2n^2."""
    return 2.0 * n ** 3 / 3.0 + 2.0 * n ** 2
