"""hpl_upload / hpl_download: FP64 column-major matrices between page-locked
host memory and device memory by the library's copy kernel (the end-to-end
path's data staging and result read-back), through the C ABI."""
import pytest

pytestmark = pytest.mark.gpu


def test_upload_contiguous_and_strided(hpl):
    import torch
    g = torch.Generator().manual_seed(5)
    # contiguous (the 16-byte flat path)
    n = 1024
    src = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
    src.copy_(torch.randn(n, n, generator=g, dtype=torch.float64))
    dst = hpl.colmajor(n, n)
    hpl.upload(dst, src)
    torch.cuda.synchronize()
    assert torch.equal(dst.cpu(), src)
    # leading dimensions larger than the rows, odd rows (the column path)
    m, k, lds, ldd = 777, 301, 800, 779
    big = torch.empty((k, lds), dtype=torch.float64, pin_memory=True)
    big.copy_(torch.randn(k, lds, generator=g, dtype=torch.float64))
    src = big.t()[:m]                               # m x k view, stride(1) = lds
    dbuf = torch.full((k, ldd), -7.0, dtype=torch.float64, device="cuda")
    dst = dbuf.t()[:m]
    hpl.upload(dst, src)
    torch.cuda.synchronize()
    assert torch.equal(dst.cpu(), src)
    assert bool((dbuf.t()[m:] == -7.0).all())        # rows beyond m untouched
    # a vector
    v = torch.randn(333, generator=g, dtype=torch.float64).pin_memory()
    dv = torch.empty(333, dtype=torch.float64, device="cuda")
    hpl.upload(dv, v)
    torch.cuda.synchronize()
    assert torch.equal(dv.cpu(), v)


def test_upload_pageable_memory_copied_or_refused(hpl):
    """Pageable host memory: where the platform lets the GPU address it (Grace:
    the runtime maps every host address) the copy must be exact; elsewhere it
    is refused with HPL_ERR_INVALID and nothing is written."""
    import torch
    src = torch.randn(64, 64, dtype=torch.float64).t()    # not page-locked
    dst = hpl.colmajor(64, 64)
    dst.zero_()
    try:
        hpl.upload(dst, src)
        refused = False
    except hpl.HplError as e:
        refused = True
        assert e.status == 1
    torch.cuda.synchronize()
    if refused:
        assert bool((dst == 0).all())
    else:
        assert torch.equal(dst.cpu(), src)


def test_download_contiguous_strided_and_vector(hpl):
    """The reverse copy writes the host buffer through its mapped address:
    exact values, only the m rows of each column, visible after a sync."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(9)
    n = 1000
    src = hpl.colmajor(n, n)
    src.copy_(torch.randn(n, n, generator=g, dtype=torch.float64, device="cuda"))
    dst = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
    hpl.download(dst, src)
    torch.cuda.synchronize()
    assert torch.equal(dst, src.cpu())
    m, k, lds, ldd = 513, 77, 520, 600
    sbuf = torch.randn(k, lds, generator=g, dtype=torch.float64, device="cuda")
    src = sbuf.t()[:m]
    hbuf = torch.full((k, ldd), -3.0, dtype=torch.float64).pin_memory()
    dst = hbuf.t()[:m]
    hpl.download(dst, src)
    torch.cuda.synchronize()
    assert torch.equal(dst, src.cpu())
    assert bool((hbuf.t()[m:] == -3.0).all())
    v = torch.randn(4097, generator=g, dtype=torch.float64, device="cuda")
    hv = torch.zeros(4097, dtype=torch.float64).pin_memory()
    hpl.download(hv, v)
    torch.cuda.synchronize()
    assert torch.equal(hv, v.cpu())


def test_download_rejects_bad_sizes(hpl):
    import ctypes
    import torch
    lib = hpl.load()
    d = torch.zeros(16, dtype=torch.float64, device="cuda")
    h = torch.zeros(16, dtype=torch.float64).pin_memory()
    assert lib.hpl_download(16, 1, d.data_ptr(), 8, h.data_ptr(), 16, None) == 1      # lds < m
    assert lib.hpl_download(-1, 1, d.data_ptr(), 16, h.data_ptr(), 16, None) == 1
    assert lib.hpl_download(0, 5, d.data_ptr(), 1, h.data_ptr(), 1, None) == 0        # empty: nothing to do
    torch.cuda.synchronize()
    assert bool((h == 0).all())


def test_download_pageable_memory_copied_or_refused(hpl):
    """Pageable host memory as the destination: copied exactly where the
    platform lets the GPU address it, else refused with HPL_ERR_INVALID and
    the host buffer left as it was."""
    import torch
    src = torch.randn(64, 64, dtype=torch.float64, device="cuda").t()
    dst = torch.zeros(64, 64, dtype=torch.float64).t()     # not page-locked
    try:
        hpl.download(dst, src)
        refused = False
    except hpl.HplError as e:
        refused = True
        assert e.status == 1
    torch.cuda.synchronize()
    if refused:
        assert bool((dst == 0).all())
    else:
        assert torch.equal(dst, src.cpu())
