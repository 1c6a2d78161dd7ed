"""lu_factor_noalloc: the factorization for callers that cannot allocate.

Callers that run under an allocator they do not own, or with a device-memory
budget fixed at start-up, cannot cudaMalloc a workspace where they factor.
lu_factor_noalloc takes none: its scratch is a fixed device array inside the
library. This checks, through the C ABI, that it gives the same factors and
pivots as lu_factor (bit for bit: same kernels, only the scratch differs) on
two calls in a row for each panel-leaf kind and look-ahead setting (the
grid-cooperative leaf, pfact = 1, is the one that uses the array's barrier and
candidate slots, so two calls in a row show they are cleared between calls),
and that options the array cannot serve are refused with the right status.
This file is collected last on purpose.
"""
import ctypes

import pytest

pytestmark = pytest.mark.gpu

HPL_ERR_INVALID = 1
HPL_ERR_NOMEM = 6


def _noalloc(lib):
    f = lib.lu_factor_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    g = lib.lu_factor_noalloc_max_scratch
    g.restype = ctypes.c_size_t
    g.argtypes = []
    return f, g


def _call(hpl, f, A, nb, lookahead, pfact, stream=None):
    import torch
    n = A.shape[0]
    ipiv = torch.empty(n, dtype=torch.int32, device="cuda")
    info = hpl.Info()
    opts = hpl.make_opts(nb=nb, lookahead=lookahead, pfact=pfact)
    st = f(n, A.data_ptr(), n, ipiv.data_ptr(), ctypes.byref(opts), info.ptr(),
           torch.cuda.current_stream().cuda_stream if stream is None else stream)
    return st, ipiv, info


@pytest.mark.parametrize("lookahead,pfact", [(1, 0), (1, 1), (0, 0), (0, 1)])
def test_noalloc_matches_lu_factor_twice(hpl, lookahead, pfact):
    import torch
    lib = hpl.load()
    f, max_scratch = _noalloc(lib)
    assert max_scratch() == 320 * 1024
    for n, nb, seed in [(700, 64, 11), (1024, 256, 12)]:      # two calls in a row share the array
        A_ref = hpl.generate(seed, hpl.STREAM_A, n, n)
        A = hpl.generate(seed, hpl.STREAM_A, n, n)
        p_ref, info_ref = hpl.lu_factor(A_ref, nb=nb, lookahead=lookahead, pfact=pfact)
        st, ipiv, info = _call(hpl, f, A, nb, lookahead, pfact)
        assert st == 0, hpl.STATUS.get(st)
        torch.cuda.synchronize()
        assert info.read()["status"] == 0 and info_ref.read()["status"] == 0
        assert torch.equal(ipiv, p_ref)
        assert torch.equal(A, A_ref)


def test_noalloc_refusals(hpl):
    import torch
    lib = hpl.load()
    f, _ = _noalloc(lib)
    lib.hplgb_last_error.restype = ctypes.c_char_p
    n = 64
    A = hpl.generate(1, hpl.STREAM_A, n, n)
    before = A.clone()
    ipiv = torch.empty(n, dtype=torch.int32, device="cuda")
    info = hpl.Info()
    # a panel width lu_factor itself refuses: HPL_ERR_INVALID, not a size error
    for nb in (513, 4096):
        opts = hpl.make_opts(nb=nb)
        st = f(n, A.data_ptr(), n, ipiv.data_ptr(), ctypes.byref(opts), info.ptr(), None)
        assert st == HPL_ERR_INVALID
    # the FP64-emulated update needs scratch that grows with n: refused by name
    opts = hpl.make_opts(nb=256, fp64_emulation=1)
    st = f(n, A.data_ptr(), n, ipiv.data_ptr(), ctypes.byref(opts), info.ptr(), None)
    assert st == HPL_ERR_INVALID
    assert b"fp64_emulation" in lib.hplgb_last_error()
    torch.cuda.synchronize()
    assert torch.equal(A, before)                  # nothing was launched
