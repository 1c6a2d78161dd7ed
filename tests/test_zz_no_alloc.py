"""lu_factor_noalloc: the factorization for callers that cannot allocate.

Callers that run under an allocator they do not own, or with a device-memory
budget fixed at start-up, cannot cudaMalloc a workspace where they factor.
lu_factor_noalloc takes none: its scratch is a fixed device array inside the
library. This checks, through the C ABI, that it gives the same factors and
pivots as lu_factor (bit for bit: same kernels, only the scratch differs) on
two calls in a row, and that a panel width beyond the array is refused.
This file is collected last on purpose.
"""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


def _noalloc(lib):
    f = lib.lu_factor_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    g = lib.lu_factor_noalloc_max_scratch
    g.restype = ctypes.c_size_t
    g.argtypes = []
    return f, g


@pytest.mark.parametrize("calls", [[(700, 64, 11), (1024, 256, 12)]])
def test_noalloc_matches_lu_factor_twice(hpl, calls):
    import torch
    lib = hpl.load()
    f, max_scratch = _noalloc(lib)
    assert max_scratch() == 320 * 1024
    for n, nb, seed in calls:                       # two calls in a row share the scratch array
        A_ref = hpl.generate(seed, hpl.STREAM_A, n, n)
        A = hpl.generate(seed, hpl.STREAM_A, n, n)
        p_ref, info_ref = hpl.lu_factor(A_ref, nb=nb, lookahead=1)
        ipiv = torch.empty(n, dtype=torch.int32, device="cuda")
        info = hpl.Info()
        opts = hpl.make_opts(nb=nb, lookahead=1)
        st = f(n, A.data_ptr(), n, ipiv.data_ptr(), ctypes.byref(opts), info.ptr(),
               torch.cuda.current_stream().cuda_stream)
        assert st == 0, hpl.STATUS.get(st)
        torch.cuda.synchronize()
        assert info.read()["status"] == 0 and info_ref.read()["status"] == 0
        assert torch.equal(ipiv, p_ref)
        assert torch.equal(A, A_ref)


def test_noalloc_rejects_panel_beyond_scratch(hpl):
    import torch
    lib = hpl.load()
    f, _ = _noalloc(lib)
    n = 64
    A = hpl.generate(1, hpl.STREAM_A, n, n)
    ipiv = torch.empty(n, dtype=torch.int32, device="cuda")
    info = hpl.Info()
    opts = hpl.make_opts(nb=4096)
    st = f(n, A.data_ptr(), n, ipiv.data_ptr(), ctypes.byref(opts), info.ptr(), None)
    assert st == 6                                   # HPL_ERR_NOMEM, nothing launched
    lib.hplgb_last_error.restype = ctypes.c_char_p
    assert b"scratch" in lib.hplgb_last_error()
