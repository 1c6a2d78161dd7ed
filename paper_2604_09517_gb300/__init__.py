"""hplgb: dense LU solve of HPL and HPL-MxP on one GB300 (sm_103a).

Thin ctypes binding over the C ABI in ``include/hplgb.h`` (libhplgb.so, built
in-tree from ``csrc/``). Every step of the computation runs in the library's
CUDA kernels; this module only marshals arguments. PyTorch provides device
memory and the current stream. There is no CPU fallback: if the library is
missing or no GPU is present, the calls raise.

Matrices are column-major: an m x n matrix is a torch tensor of shape (m, n)
with strides (1, ld). ``colmajor(m, n)`` allocates one.
"""
from __future__ import annotations

import ctypes
import os
import struct
import threading

import torch

from . import _build

__all__ = [
    "HplError", "load", "build", "colmajor", "Info", "Opts", "generate", "lu_factor", "lu_solve",
    "scaled_residual", "STATUS", "GEN_GENERAL", "GEN_DIAG_DOMINANT", "STREAM_A", "STREAM_B",
]

GEN_GENERAL = 0
GEN_DIAG_DOMINANT = 1
PREC_BF16 = 0
PREC_FP8_E4M3 = 1
PREC_FP16 = 2
PREC_TF32 = 3
STORAGE_FP32 = 0
STORAGE_BF16 = 1
INNER_FP64 = 0          # GMRES inner matrix-vector products with the FP64 A
INNER_FP32 = 1          # ... with an FP32 copy of A kept in the workspace
REFINE_IR = 0
REFINE_GMRES = 1
STREAM_A = 0
STREAM_B = 1

STATUS = {0: "HPL_OK", 1: "HPL_ERR_INVALID", 2: "HPL_ERR_SINGULAR", 3: "HPL_ERR_NONFINITE",
          4: "HPL_ERR_NOT_CONVERGED", 5: "HPL_ERR_TIMEOUT", 6: "HPL_ERR_NOMEM", 7: "HPL_ERR_CUDA"}

_lock = threading.Lock()
_lib = None


class HplError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        msg = f"{where}: {STATUS.get(status, status)}"
        if status == 7 and _lib is not None:
            msg += " (" + _lib.hplgb_last_error().decode(errors="replace") + ")"
        super().__init__(msg)


class Opts(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int64), ("lookahead", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("refine", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("gmres_m", ctypes.c_int32),
                ("ns_iters", ctypes.c_int32), ("tol", ctypes.c_double), ("timeout_ns", ctypes.c_int64),
                ("fp64_emulation", ctypes.c_int32), ("pfact", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("inner", ctypes.c_int32)]


def library_path() -> str:
    return _build.LIB


def build(force: bool = False) -> str:
    return _build.build(force=force)


def load():
    """Load libhplgb.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libhplgb.so missing at {path}; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        i64, u64, vp, i32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
        sz = ctypes.c_size_t
        op = ctypes.POINTER(Opts)
        sig = {
            "hpl_default_opts": (None, [op]),
            "hpl_status_string": (ctypes.c_char_p, [i32]),
            "hplgb_last_error": (ctypes.c_char_p, []),
            "hpl_generate": (i32, [u64, u64, i64, i64, i32, vp, i64, vp]),
            "lu_factor_workspace_size": (sz, [i64, op]),
            "lu_factor": (i32, [i64, vp, i64, vp, op, vp, sz, vp, vp]),
            "lu_solve_workspace_size": (sz, [i64, i64]),
            "lu_solve": (i32, [i64, i64, vp, i64, vp, i32, vp, i64, vp, sz, vp, vp]),
            "hpl_residual_workspace_size": (sz, [i64]),
            "hpl_scaled_residual": (i32, [i64, vp, i64, u64, i32, vp, vp, vp, vp, sz, vp]),
            "hplgb_gemm_bf16": (i32, [i64, i64, i64, vp, i64, vp, i64, vp, i64, i32, vp, vp]),
            "hplgb_gemm_fp8": (i32, [i64, i64, i64, vp, i64, vp, i64, vp, vp, vp, i64, i32, vp, vp]),
            "hplgb_gemm_f16": (i32, [i64, i64, i64, vp, i64, vp, i64, vp, vp, vp, i64, i32, vp, vp]),
            "hplgb_gemm_tf32": (i32, [i64, i64, i64, vp, i64, vp, i64, vp, i64, i32, vp, vp]),
            "mxp_workspace_size": (sz, [i64, i64, op]),
            "lu_solve_backward": (i32, [i64, i64, vp, i64, vp, i64, vp, i64, vp, i64, vp, i64, op, vp, sz, vp, vp]),
            "hpl_batch_sizes": (i32, [u64, i64, vp]),
            "hpl_batch_shard": (i32, [i64, vp, vp, i32, vp]),
            "solve_batched_workspace_size": (sz, [i64, vp, vp]),
            "solve_batched_plan": (i32, [i64, vp, vp, vp, vp, vp, vp, vp, op, vp, sz]),
            "solve_batched_run": (i32, [vp, vp, i32, vp]),
            "mxp_solve": (i32, [i64, i64, vp, i64, u64, vp, i64, vp, i64, op, vp, sz, vp, vp]),
            "hplgb_launch_count": (ctypes.c_longlong, []),
            "hplgb_set_phase_timing": (None, [i32]),
            "hplgb_gemm_config": (i32, [i32, ctypes.c_longlong]),
            "hpl_upload": (i32, [i64, i64, vp, i64, vp, i64, vp]),
            "hpl_download": (i32, [i64, i64, vp, i64, vp, i64, vp]),
            "hplgb_lu_config": (i32, [i32, ctypes.c_longlong]),
            "hplgb_batched_config": (i32, [i32, ctypes.c_longlong]),
            "hplgb_phase_times": (i32, [vp, vp, vp]),
            "hplgb_phase_records": (i32, [vp, vp, vp, vp, vp, ctypes.c_longlong, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(st: int, where: str):
    if st != 0:
        raise HplError(st, where)


def _stream(device=None) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _ld(t: torch.Tensor) -> int:
    """Leading dimension of a column-major matrix view (or a vector)."""
    if t.dim() == 1:
        assert t.stride(0) == 1
        return max(t.shape[0], 1)
    assert t.stride(0) == 1, "matrices must be column-major (stride(0) == 1)"
    return max(t.stride(1), t.shape[0], 1) if t.shape[1] > 1 else max(t.shape[0], 1)


def colmajor(m: int, n: int, dtype=torch.float64, device="cuda", ld: int | None = None) -> torch.Tensor:
    ld = max(m, 1) if ld is None else ld
    return torch.empty((n, ld), dtype=dtype, device=device).t()[:m, :]


def make_opts(nb: int = 0, lookahead: int = 1, prec: int = PREC_BF16, refine: int = REFINE_GMRES,
              max_iter: int = 50, gmres_m: int = 30, tol: float = 16.0, timeout_ns: int = 0,
              fp64_emulation: int = 0, pfact: int = 0, storage: int = STORAGE_FP32, ns_iters: int = 0,
              inner: int = 0) -> Opts:
    o = Opts()
    load().hpl_default_opts(ctypes.byref(o))
    if ns_iters:
        o.ns_iters = ns_iters
    o.nb, o.lookahead, o.prec, o.refine = nb, lookahead, prec, refine
    o.fp64_emulation, o.pfact, o.storage, o.inner = fp64_emulation, pfact, storage, inner
    o.max_iter, o.gmres_m, o.tol = max_iter, gmres_m, tol
    if timeout_ns:
        o.timeout_ns = timeout_ns
    return o


class Info:
    """Device-resident hpl_info record (32 bytes)."""

    def __init__(self, device="cuda"):
        self.buf = torch.zeros(4, dtype=torch.int64, device=device)

    def ptr(self):
        return ctypes.c_void_p(self.buf.data_ptr())

    def read(self) -> dict:
        raw = self.buf.cpu().numpy().tobytes()
        status, iters, info, sr, inner, _ = struct.unpack("<iiqdii", raw)
        return dict(status=status, status_name=STATUS.get(status, str(status)), iters=iters, info=info,
                    scaled_residual=sr, inner_iters=inner)


def workspace(nbytes: int, device="cuda") -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def generate(seed: int, stream_id: int, m: int, ncols: int, kind: int = GEN_GENERAL, out: torch.Tensor | None = None,
             device="cuda") -> torch.Tensor:
    """Seeded matrix of hpl_generate (column-major m x ncols, FP64)."""
    lib = load()
    if out is None:
        out = colmajor(m, ncols, device=device)
    _check(lib.hpl_generate(seed, stream_id, m, ncols, kind, _ptr(out), _ld(out), _stream(out.device)),
           "hpl_generate")
    return out


def lu_factor(A: torch.Tensor, nb: int = 256, lookahead: int = 1, ipiv: torch.Tensor | None = None,
              ws: torch.Tensor | None = None, info: Info | None = None, fp64_emulation: int = 0,
              pfact: int = 0):
    """In-place LU with partial pivoting. Returns (ipiv, info). fp64_emulation=1
    runs the trailing update on the BF16 tensor cores with FP64 accuracy;
    pfact=1 keeps every panel leaf on the grid-cooperative kernel."""
    lib = load()
    n = A.shape[0]
    assert A.shape == (n, n) and A.dtype == torch.float64 and A.is_cuda
    opts = make_opts(nb=nb, lookahead=lookahead, fp64_emulation=fp64_emulation, pfact=pfact)
    if ipiv is None:
        ipiv = torch.empty(max(n, 1), dtype=torch.int32, device=A.device)
    need = lib.lu_factor_workspace_size(n, ctypes.byref(opts))
    if ws is None or ws.numel() < need:
        ws = workspace(need, A.device)
    if info is None:
        info = Info(A.device)
    _check(lib.lu_factor(n, _ptr(A), _ld(A), _ptr(ipiv), ctypes.byref(opts), _ptr(ws), ws.numel(), info.ptr(),
                         _stream(A.device)), "lu_factor")
    return ipiv[:n], info


def lu_solve(LU: torch.Tensor, ipiv: torch.Tensor, B: torch.Tensor, trans: int = 0, ws: torch.Tensor | None = None,
             info: Info | None = None) -> torch.Tensor:
    """Solve A X = B (trans=0) or A^T X = B (trans=1) in place on B."""
    lib = load()
    n = LU.shape[0]
    nrhs = 1 if B.dim() == 1 else B.shape[1]
    need = lib.lu_solve_workspace_size(n, nrhs)
    if ws is None or ws.numel() < need:
        ws = workspace(need, B.device)
    _check(lib.lu_solve(n, nrhs, _ptr(LU), _ld(LU), _ptr(ipiv), trans, _ptr(B), _ld(B), _ptr(ws), ws.numel(),
                        info.ptr() if info is not None else None, _stream(B.device)), "lu_solve")
    return B


def scaled_residual(A: torch.Tensor | None, x: torch.Tensor, b: torch.Tensor, seed: int = 0,
                    kind: int = GEN_GENERAL, ws: torch.Tensor | None = None) -> torch.Tensor:
    """HPL scaled residual as a 0-dim device tensor (A=None: regenerate A from seed)."""
    lib = load()
    n = x.shape[0]
    out = torch.empty((), dtype=torch.float64, device=x.device)
    need = lib.hpl_residual_workspace_size(n)
    if ws is None or ws.numel() < need:
        ws = workspace(need, x.device)
    _check(lib.hpl_scaled_residual(n, _ptr(A), _ld(A) if A is not None else n, seed, kind, _ptr(x), _ptr(b),
                                   _ptr(out), _ptr(ws), ws.numel(), _stream(x.device)), "hpl_scaled_residual")
    return out


def mxp_solve(A: torch.Tensor | None, B: torch.Tensor, nb: int = 3072, refine: int = REFINE_GMRES, max_iter: int = 50,
              gmres_m: int = 30, tol: float = 16.0, X: torch.Tensor | None = None, ws: torch.Tensor | None = None,
              info: Info | None = None, prec: int = PREC_BF16, seed: int = 0, storage: int = STORAGE_FP32,
              ns_iters: int = 0, inner: int = INNER_FP64):
    """Mixed-precision solve of A X = B (A FP64 n x n column-major, diagonally dominant).

    A = None solves with the dominant generated matrix of `seed` without storing
    it (the library regenerates its entries). storage = STORAGE_BF16 keeps the
    working matrix in BF16. inner = INNER_FP32 runs GMRES's inner
    matrix-vector products on an FP32 copy of A. Returns (X, info, ws); ws
    holds the block factor afterwards (see mxp_factor_views).
    """
    lib = load()
    n = B.shape[0]
    dev = B.device
    vec = B.dim() == 1
    Bm = B.reshape(n, 1) if vec else B
    if Bm.stride(0) != 1:
        Bc = colmajor(n, Bm.shape[1], device=dev)
        Bc.copy_(Bm)
        Bm = Bc
    nrhs = Bm.shape[1]
    opts = make_opts(nb=nb, refine=refine, max_iter=max_iter, gmres_m=gmres_m, tol=tol, prec=prec, storage=storage,
                     ns_iters=ns_iters, inner=inner)
    if X is None:
        X = colmajor(n, nrhs, device=dev)
    Xm = X.view(n, 1) if X.dim() == 1 else X
    need = lib.mxp_workspace_size(n, nrhs, ctypes.byref(opts))
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    if info is None:
        info = Info(dev)
    a_ptr, a_ld = (None, n) if A is None else (_ptr(A), _ld(A))
    _check(lib.mxp_solve(n, nrhs, a_ptr, a_ld, seed, _ptr(Bm), _ld(Bm) if nrhs > 1 else n, _ptr(Xm),
                         _ld(Xm) if nrhs > 1 else n, ctypes.byref(opts), _ptr(ws), ws.numel(), info.ptr(),
                         _stream(dev)), "mxp_solve")
    return X, info, ws


def lu_solve_backward(A: torch.Tensor, X: torch.Tensor, G: torch.Tensor, ws: torch.Tensor, nb: int = 3072,
                      want_grad_a: bool = True, refine: int = REFINE_GMRES, max_iter: int = 50, gmres_m: int = 30,
                      tol: float = 16.0, storage: int = STORAGE_FP32):
    """Adjoint of X = A^-1 B from the factor mxp_solve left in ws (factored with
    the same storage): (grad_B, grad_A, info)."""
    lib = load()
    n = A.shape[0]
    Gm = G.reshape(n, -1) if G.dim() == 1 else G
    Xm = X.reshape(n, -1) if X.dim() == 1 else X
    nrhs = Gm.shape[1]
    Gc = colmajor(n, nrhs, device=A.device)
    Gc.copy_(Gm)
    Xc = colmajor(n, nrhs, device=A.device)
    Xc.copy_(Xm)
    gB = colmajor(n, nrhs, device=A.device)
    gA = colmajor(n, n, device=A.device) if want_grad_a else None
    opts = make_opts(nb=nb, refine=refine, max_iter=max_iter, gmres_m=gmres_m, tol=tol, storage=storage)
    info = Info(A.device)
    _check(lib.lu_solve_backward(n, nrhs, _ptr(A), _ld(A), _ptr(Xc), n, _ptr(Gc), n, _ptr(gB), n, _ptr(gA), n,
                                 ctypes.byref(opts), _ptr(ws), ws.numel(), info.ptr(), _stream(A.device)),
           "lu_solve_backward")
    return gB, gA, info


class SolveFn(torch.autograd.Function):
    """X = A^-1 B with the mixed-precision forward (BF16 block LU + FP64
    refinement) and the hand-written adjoint backward on the saved factor.
    A must be FP64, square, column-major and diagonally dominant. Several
    right-hand sides are refined together (classic refinement on the block);
    one right-hand side uses GMRES-based refinement."""

    @staticmethod
    def forward(ctx, A, B, nb=3072):
        Ac = A if A.stride(0) == 1 else A.t().contiguous().t()
        Bm = B.reshape(B.shape[0], -1) if B.dim() == 1 else B
        Bc = colmajor(Bm.shape[0], Bm.shape[1], device=A.device)
        Bc.copy_(Bm)
        refine = REFINE_IR if Bc.shape[1] > 1 else REFINE_GMRES
        X, info, ws = mxp_solve(Ac.detach(), Bc, nb=nb, refine=refine)
        rec = info.read()
        if rec["status"] != 0:
            raise HplError(rec["status"], "SolveFn.forward")
        ctx.save_for_backward(Ac.detach(), X)
        ctx.ws, ctx.nb, ctx.vec, ctx.refine = ws, nb, B.dim() == 1, refine
        out = X.clone()
        return out[:, 0] if ctx.vec else out

    @staticmethod
    def backward(ctx, G):
        A, X = ctx.saved_tensors
        gB, gA, info = lu_solve_backward(A, X, G, ctx.ws, nb=ctx.nb, want_grad_a=ctx.needs_input_grad[0],
                                         refine=ctx.refine)
        rec = info.read()
        if rec["status"] != 0:
            raise HplError(rec["status"], "SolveFn.backward")
        if ctx.vec:
            gB = gB[:, 0]
        return gA, gB, None


def solve(A: torch.Tensor, B: torch.Tensor, nb: int = 3072) -> torch.Tensor:
    """Differentiable mixed-precision solve X = A^-1 B (see SolveFn)."""
    return SolveFn.apply(A, B, nb)


def batch_sizes(seed: int, count: int):
    """Sizes of the batched workload (generator stream 2), as a numpy int64 array."""
    import numpy as np
    out = np.empty(count, dtype=np.int64)
    _check(load().hpl_batch_sizes(seed, count, out.ctypes.data), "hpl_batch_sizes")
    return out


def batch_shard(n, kind, world: int):
    """Rank (0..world-1) that solves each system when a batch is split over
    world GPUs (host only; every rank computes the same split)."""
    import numpy as np
    n = np.ascontiguousarray(n, dtype=np.int64)
    kind = np.ascontiguousarray(kind, dtype=np.uint8)
    owner = np.empty(n.shape[0], dtype=np.int32)
    _check(load().hpl_batch_shard(n.shape[0], n.ctypes.data, kind.ctypes.data, world, owner.ctypes.data),
           "hpl_batch_shard")
    return owner


class Batch:
    """Device buffers and the plan of a batched solve.

    System s has size n[s] and kind[s] (0: general, pivoted FP64; 1: diagonally
    dominant, BF16 factor + FP64 refinement); its matrix (column-major, ld n[s])
    and right-hand side live in two flat FP64 buffers at offsets a_off[s] and
    b_off[s]; generate() fills them from generator streams 16+2g and 17+2g,
    g = ids[s] the system's index in the whole batch (default s; a rank that
    solves a share of a batch passes the ids of its systems).
    """

    def __init__(self, n, kind, device="cuda", ids=None):
        import numpy as np
        self.n = np.ascontiguousarray(n, dtype=np.int64)
        self.kind = np.ascontiguousarray(kind, dtype=np.uint8)
        self.count = len(self.n)
        self.ids = np.arange(self.count, dtype=np.int64) if ids is None else np.ascontiguousarray(ids, dtype=np.int64)
        self.device = device
        sq = self.n * self.n
        self.a_off = np.concatenate([[0], np.cumsum(sq)[:-1]]).astype(np.int64)
        self.b_off = np.concatenate([[0], np.cumsum(self.n)[:-1]]).astype(np.int64)
        self.A = torch.empty(int(sq.sum()), dtype=torch.float64, device=device)
        self.B = torch.empty(int(self.n.sum()), dtype=torch.float64, device=device)
        self.ipiv = torch.zeros(int(self.n.sum()), dtype=torch.int32, device=device)
        self.infos = torch.zeros(self.count * 4, dtype=torch.int64, device=device)
        ea, eb, ei = self.A.element_size(), self.B.element_size(), self.ipiv.element_size()
        self.pA = (ctypes.c_void_p * self.count)(*[self.A.data_ptr() + int(o) * ea for o in self.a_off])
        self.pB = (ctypes.c_void_p * self.count)(*[self.B.data_ptr() + int(o) * eb for o in self.b_off])
        self.pP = (ctypes.c_void_p * self.count)(*[self.ipiv.data_ptr() + int(o) * ei for o in self.b_off])
        self.lda = np.ascontiguousarray(self.n, dtype=np.int64)
        self.ws = None

    def matrix(self, s):
        n, o = int(self.n[s]), int(self.a_off[s])
        return self.A[o:o + n * n].view(n, n).t()

    def rhs(self, s):
        n, o = int(self.n[s]), int(self.b_off[s])
        return self.B[o:o + n]

    def pivots(self, s):
        n, o = int(self.n[s]), int(self.b_off[s])
        return self.ipiv[o:o + n]

    def generate(self, seed: int):
        for s in range(self.count):
            n, g = int(self.n[s]), int(self.ids[s])
            generate(seed, 16 + 2 * g, n, n, int(self.kind[s]), out=self.matrix(s), device=self.device)
            generate(seed, 17 + 2 * g, n, 1, GEN_GENERAL, out=self.rhs(s).view(n, 1), device=self.device)

    def plan(self, max_iter: int = 50, tol: float = 16.0, variant=None):
        """Write the work table. variant: per-system tile shape (0: panel 32,
        1: panel 16); None takes it from the autotuner's table."""
        import numpy as np
        from . import autotune
        lib = load()
        need = lib.solve_batched_workspace_size(self.count, self.n.ctypes.data, self.kind.ctypes.data)
        if self.ws is None or self.ws.numel() < need:
            self.ws = workspace(need, self.device)
        if variant is None:
            variant = autotune.variants(self.n, self.kind)
        self.variant = np.ascontiguousarray(np.broadcast_to(variant, (self.count,)), dtype=np.uint8)
        opts = make_opts(max_iter=max_iter, tol=tol)
        torch.cuda.synchronize(self.device)
        _check(lib.solve_batched_plan(self.count, self.n.ctypes.data, self.pA, self.lda.ctypes.data, self.pB,
                                      self.pP, self.kind.ctypes.data, self.variant.ctypes.data, ctypes.byref(opts),
                                      _ptr(self.ws), self.ws.numel()), "solve_batched_plan")

    def run(self, max_ctas: int = 0):
        _check(load().solve_batched_run(_ptr(self.ws), _ptr(self.infos), max_ctas, _stream(self.device)),
               "solve_batched_run")

    def info(self, s=None):
        raw = self.infos.cpu().numpy()
        recs = []
        for q in range(self.count) if s is None else [s]:
            st, it, inf, sr, inner, _ = struct.unpack("<iiqdii", raw[4 * q:4 * q + 4].tobytes())
            recs.append(dict(status=st, iters=it, info=inf, scaled_residual=sr, inner_iters=inner))
        return recs if s is None else recs[0]


def mxp_factor_views(ws: torch.Tensor, n: int, nb: int = 3072, storage: int = STORAGE_FP32):
    """(F, Dinv) views of the block factor that mxp_solve leaves in its workspace
    (F is bfloat16 for BF16 storage, else float32)."""
    nb = min(nb, n)
    esz, dt = (2, torch.bfloat16) if storage == STORAGE_BF16 else (4, torch.float32)
    f_bytes = esz * n * n
    d_off = (f_bytes + 255) // 256 * 256
    F = ws[:f_bytes].view(dt).view(n, n).t()
    Dinv = ws[d_off:d_off + 4 * n * nb].view(torch.float32).view(nb, n).t()
    return F, Dinv


def gemm_bf16(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, sub: bool = True) -> torch.Tensor:
    """C = C - A B^T (sub) or A B^T on the tcgen05 tensor cores.

    A (M x K) and B (N x K) are bfloat16 with K contiguous; C is FP32 column-major.
    """
    lib = load()
    assert A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16 and C.dtype == torch.float32
    assert A.stride(1) == 1 and B.stride(1) == 1 and C.stride(0) == 1
    M, K = A.shape
    N = B.shape[0]
    err = torch.zeros(1, dtype=torch.int32, device=C.device)
    _check(lib.hplgb_gemm_bf16(M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(C), _ld(C), int(sub),
                               _ptr(err), _stream(C.device)), "hplgb_gemm_bf16")
    torch.cuda.current_stream(C.device).synchronize()
    e = int(err.item())
    if e:
        raise HplError(e, "hplgb_gemm_bf16 (device)")
    return C


def gemm_fp8(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, sa=None, sb=None, sub: bool = True) -> torch.Tensor:
    """C = C - (A B^T) * sa sb^T (sub) or the product, A and B float8_e4m3fn with K contiguous."""
    lib = load()
    assert A.dtype == torch.float8_e4m3fn and B.dtype == torch.float8_e4m3fn and C.dtype == torch.float32
    assert A.stride(1) == 1 and B.stride(1) == 1 and C.stride(0) == 1
    M, K = A.shape
    N = B.shape[0]
    err = torch.zeros(1, dtype=torch.int32, device=C.device)
    _check(lib.hplgb_gemm_fp8(M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(sa), _ptr(sb), _ptr(C),
                              _ld(C), int(sub), _ptr(err), _stream(C.device)), "hplgb_gemm_fp8")
    torch.cuda.current_stream(C.device).synchronize()
    e = int(err.item())
    if e:
        raise HplError(e, "hplgb_gemm_fp8 (device)")
    return C


def gemm_f16(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, sa=None, sb=None, sub: bool = True) -> torch.Tensor:
    """C = C - (A B^T) * sa sb^T (sub) or the product, A and B float16 with K contiguous."""
    lib = load()
    assert A.dtype == torch.float16 and B.dtype == torch.float16 and C.dtype == torch.float32
    assert A.stride(1) == 1 and B.stride(1) == 1 and C.stride(0) == 1
    M, K = A.shape
    N = B.shape[0]
    err = torch.zeros(1, dtype=torch.int32, device=C.device)
    _check(lib.hplgb_gemm_f16(M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(sa), _ptr(sb), _ptr(C),
                              _ld(C), int(sub), _ptr(err), _stream(C.device)), "hplgb_gemm_f16")
    torch.cuda.current_stream(C.device).synchronize()
    e = int(err.item())
    if e:
        raise HplError(e, "hplgb_gemm_f16 (device)")
    return C


def upload(dst: torch.Tensor, src: torch.Tensor) -> torch.Tensor:
    """Copy the host FP64 matrix src (page-locked, or any host memory where the
    GPU can address pageable memory) into the device matrix dst (both
    column-major, stride(0) == 1) with the library's kernel copy (hpl_upload)."""
    assert src.dtype == torch.float64 and dst.dtype == torch.float64 and dst.is_cuda and not src.is_cuda
    if src.dim() == 1:
        src, dst = src.view(-1, 1), dst.view(-1, 1)
    assert src.shape == dst.shape and src.stride(0) == 1 and dst.stride(0) == 1
    m, n = src.shape
    _check(load().hpl_upload(m, n, _ptr(src), _ld(src), _ptr(dst), _ld(dst), _stream(dst.device)), "hpl_upload")
    return dst


def download(dst: torch.Tensor, src: torch.Tensor) -> torch.Tensor:
    """Copy the device FP64 matrix src into the host matrix dst (page-locked,
    or any host memory the GPU can address; both column-major, stride(0) == 1)
    with the library's kernel copy (hpl_download); asynchronous on the current
    stream: synchronize before reading dst."""
    assert src.dtype == torch.float64 and dst.dtype == torch.float64 and src.is_cuda and not dst.is_cuda
    if src.dim() == 1:
        src, dst = src.view(-1, 1), dst.view(-1, 1)
    assert src.shape == dst.shape and src.stride(0) == 1 and dst.stride(0) == 1
    m, n = src.shape
    _check(load().hpl_download(m, n, _ptr(src), _ld(src), _ptr(dst), _ld(dst), _stream(src.device)),
           "hpl_download")
    return dst


def gemm_tf32(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, sub: bool = True) -> torch.Tensor:
    """C = C - A B^T (sub) or A B^T, A and B float32 words already rounded to
    TF32 (K contiguous), on the tensor cores' TF32 path."""
    lib = load()
    assert A.dtype == torch.float32 and B.dtype == torch.float32 and C.dtype == torch.float32
    assert A.stride(1) == 1 and B.stride(1) == 1 and C.stride(0) == 1
    M, K = A.shape
    N = B.shape[0]
    err = torch.zeros(1, dtype=torch.int32, device=C.device)
    _check(lib.hplgb_gemm_tf32(M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(C), _ld(C), int(sub),
                               _ptr(err), _stream(C.device)), "hplgb_gemm_tf32")
    torch.cuda.current_stream(C.device).synchronize()
    e = int(err.item())
    if e:
        raise HplError(e, "hplgb_gemm_tf32 (device)")
    return C


PHASES = ("pfact", "swap", "trsm", "update", "other", "convert", "resid", "refine", "opconv")


def launch_count() -> int:
    return int(load().hplgb_launch_count())


GEMM_EPILOGUE = 0        # hplgb_gemm_config switches
GEMM_GROUP_M = 1
GEMM_PAIR_MAX_MN = 2
GEMM_PAIR_ATOMS = 3


def gemm_config(what: int, value: int) -> None:
    """Tuning switch of the tensor-core product (see include/hplgb.h)."""
    _check(load().hplgb_gemm_config(int(what), int(value)), "hplgb_gemm_config")


LU_TRSM_BLOCKED = 0       # hplgb_lu_config switches
LU_SOLVE_WAVE = 1
LU_SOLVE_WAVE_GRID = 2


def lu_config(what: int, value: int) -> None:
    """Measurement switch of the FP64 LU and its solve (see include/hplgb.h)."""
    _check(load().hplgb_lu_config(int(what), int(value)), "hplgb_lu_config")


def batched_config(what: int, value: int) -> None:
    """Residency switch of the batched solver (see include/hplgb.h)."""
    _check(load().hplgb_batched_config(int(what), int(value)), "hplgb_batched_config")


def set_phase_timing(on: bool) -> None:
    load().hplgb_set_phase_timing(int(bool(on)))


def phase_times() -> dict:
    """Per-phase {name: (ms, work, intervals)} since timing was switched on."""
    import numpy as np
    ms = np.zeros(len(PHASES))
    work = np.zeros(len(PHASES))
    cnt = np.zeros(len(PHASES), dtype=np.int64)
    _check(load().hplgb_phase_times(ms.ctypes.data, work.ctypes.data, cnt.ctypes.data), "hplgb_phase_times")
    return {name: (float(ms[i]), float(work[i]), int(cnt[i])) for i, name in enumerate(PHASES)}


def phase_records(cap: int = 1 << 16) -> dict:
    """The timed intervals one by one (call before phase_times, which clears
    them): numpy arrays phase, step, start_ms, ms, work."""
    import numpy as np
    ph = np.zeros(cap, dtype=np.int32)
    st = np.zeros(cap, dtype=np.int32)
    t0 = np.zeros(cap)
    ms = np.zeros(cap)
    wk = np.zeros(cap)
    cnt = ctypes.c_longlong(0)
    _check(load().hplgb_phase_records(ph.ctypes.data, st.ctypes.data, t0.ctypes.data, ms.ctypes.data, wk.ctypes.data,
                                      cap, ctypes.byref(cnt)), "hplgb_phase_records")
    k = min(cnt.value, cap)
    return {"phase": ph[:k], "step": st[:k], "start_ms": t0[:k], "ms": ms[:k], "work": wk[:k]}


def flops(n: int) -> float:
    """Operation count credited to one solve: 2n^3/3 + 2n^2."""
    return 2.0 * n ** 3 / 3.0 + 2.0 * n ** 2
