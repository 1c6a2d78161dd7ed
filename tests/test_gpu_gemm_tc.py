"""The tcgen05 BF16 GEMM (C = C - A B^T, FP32 accumulate in TMEM) against a
plain PyTorch FP64 product of the same BF16 operands, through the C ABI."""
import pytest

pytestmark = pytest.mark.gpu


def _case(hpl, M, N, K, sub, seed, ld_pad=0):
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    lda = ((K + 7) // 8) * 8 + ld_pad
    Abuf = torch.randn(M, lda, device="cuda", generator=g).to(torch.bfloat16)
    Bbuf = torch.randn(N, lda, device="cuda", generator=g).to(torch.bfloat16)
    A, B = Abuf[:, :K], Bbuf[:, :K]
    C = hpl.colmajor(M, N, dtype=torch.float32)
    C.copy_(torch.randn(M, N, device="cuda", generator=g))
    C0 = C.clone()
    hpl.gemm_bf16(A, B, C, sub=sub)
    prod = A.double() @ B.double().t()
    ref = (C0.double() - prod) if sub else prod
    bound = A.double().abs() @ B.double().abs().t()
    err = (C.double() - ref).abs()
    tol = (K * 2.0 ** -23 + 1e-6) * bound + 2.0 ** -23 * C0.double().abs()
    bad = (err > tol).sum().item()
    assert bad == 0, f"{bad} entries out of tolerance, max err {err.max().item():.3g}"


@pytest.mark.parametrize("M,N,K,sub", [(128, 256, 64, True), (128, 256, 128, False), (1, 1, 8, True),
                                       (300, 500, 200, True), (257, 513, 72, False), (129, 255, 64, True),
                                       (1536, 1536, 1536, True), (2048, 4096, 1536, True),
                                       (4000, 300, 1024, False),
                                       # >= 76 tiles of 256 x 256: the two-SM pair kernel, ragged edges,
                                       # K tails, and a last tile row whose second half lies beyond M
                                       (2304, 2304, 704, True), (2500, 2100, 200, True), (2404, 2300, 136, False)])
def test_gemm_bf16_matches_fp64(hpl, M, N, K, sub):
    _case(hpl, M, N, K, sub, seed=M + N + K)


def test_gemm_bf16_padded_leading_dimension(hpl):
    _case(hpl, 640, 384, 256, True, seed=3, ld_pad=64)


def test_gemm_bf16_rejects_bad_strides(hpl):
    import torch
    A = torch.zeros(16, 12, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(16, 12, dtype=torch.bfloat16, device="cuda")
    C = hpl.colmajor(16, 16, dtype=torch.float32)
    with pytest.raises(hpl.HplError):
        hpl.gemm_bf16(A, B, C)          # row stride 12 is not a multiple of 8 elements


@pytest.mark.parametrize("M,N,K,sub,scaled", [(128, 256, 128, True, False), (300, 500, 208, True, True),
                                              (1536, 2048, 1536, True, True), (257, 129, 64, False, True),
                                              (2304, 2560, 256, True, True), (2404, 2100, 208, True, True)])
def test_gemm_fp8_matches_fp64(hpl, M, N, K, sub, scaled):
    import torch
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    ld = (K + 15) // 16 * 16
    A = (torch.randn(M, ld, device="cuda", generator=g) * 8).to(torch.float8_e4m3fn)[:, :K]
    B = (torch.randn(N, ld, device="cuda", generator=g) * 8).to(torch.float8_e4m3fn)[:, :K]
    sa = torch.pow(2.0, torch.randint(-4, 4, (M,), device="cuda", generator=g).float()) if scaled else None
    sb = torch.pow(2.0, torch.randint(-4, 4, (N,), device="cuda", generator=g).float()) if scaled else None
    C = hpl.colmajor(M, N, dtype=torch.float32)
    C.copy_(torch.randn(M, N, device="cuda", generator=g))
    C0 = C.clone()
    hpl.gemm_fp8(A, B, C, sa, sb, sub=sub)
    Ad, Bd = A.double(), B.double()
    if scaled:
        Ad = Ad * sa.double()[:, None]
        Bd = Bd * sb.double()[:, None]
    prod = Ad @ Bd.t()
    ref = C0.double() - prod if sub else prod
    bound = Ad.abs() @ Bd.abs().t()
    err = (C.double() - ref).abs()
    tol = (K * 2.0 ** -23 + 1e-6) * bound + 2.0 ** -23 * C0.double().abs()
    assert (err > tol).sum().item() == 0, err.max().item()


@pytest.mark.parametrize("M,N,K,sub,scaled", [(128, 256, 128, True, False), (300, 500, 200, True, True),
                                              (1536, 2048, 1536, True, True), (257, 129, 64, False, True),
                                              (2304, 2560, 256, True, True), (2404, 2100, 200, True, True)])
def test_gemm_f16_matches_fp64(hpl, M, N, K, sub, scaled):
    """FP16 operands (kind::f16 with F16 inputs), optional power-of-two row and
    column scales, against the FP64 product of the same FP16 values."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(M + N + K + 1)
    ld = (K + 7) // 8 * 8
    A = (torch.randn(M, ld, device="cuda", generator=g) * 1000).to(torch.float16)[:, :K]
    B = (torch.randn(N, ld, device="cuda", generator=g) * 1000).to(torch.float16)[:, :K]
    sa = torch.pow(2.0, torch.randint(-20, 4, (M,), device="cuda", generator=g).float()) if scaled else None
    sb = torch.pow(2.0, torch.randint(-4, 4, (N,), device="cuda", generator=g).float()) if scaled else None
    C = hpl.colmajor(M, N, dtype=torch.float32)
    C.copy_(torch.randn(M, N, device="cuda", generator=g))
    C0 = C.clone()
    hpl.gemm_f16(A, B, C, sa, sb, sub=sub)
    Ad, Bd = A.double(), B.double()
    if scaled:
        Ad = Ad * sa.double()[:, None]
        Bd = Bd * sb.double()[:, None]
    prod = Ad @ Bd.t()
    ref = C0.double() - prod if sub else prod
    bound = Ad.abs() @ Bd.abs().t()
    err = (C.double() - ref).abs()
    tol = (K * 2.0 ** -23 + 1e-6) * bound + 2.0 ** -23 * C0.double().abs()
    assert (err > tol).sum().item() == 0, err.max().item()


@pytest.mark.parametrize("M,N,K", [(256, 512, 2304), (2304, 2560, 1536), (130, 70, 264)])
def test_gemm_bf16_small_integer_products_are_exact(hpl, M, N, K):
    """Integer BF16 operands below 2^6 in magnitude: every product and every
    partial sum is an integer below 2^24, so the FP32 accumulation in tensor
    memory must return the exact integer dot products (the property the
    sliced FP64 emulation of the trailing update relies on)."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N + K)
    ld = (K + 7) // 8 * 8
    Ai = torch.randint(-63, 64, (M, ld), device="cuda", generator=g)
    Bi = torch.randint(-63, 64, (N, ld), device="cuda", generator=g)
    A, B = Ai.to(torch.bfloat16)[:, :K], Bi.to(torch.bfloat16)[:, :K]
    C = hpl.colmajor(M, N, dtype=torch.float32)
    C.zero_()
    hpl.gemm_bf16(A, B, C, sub=False)
    exact = Ai[:, :K].double() @ Bi[:, :K].double().t()     # integers below 2^53: exact in FP64
    assert exact.abs().max().item() < 2 ** 24
    assert torch.equal(C.double(), exact)


@pytest.mark.parametrize("kind", ["bf16", "fp8", "f16", "tf32"])
@pytest.mark.parametrize("M,N,K,sub", [(300, 500, 208, True), (2404, 2300, 208, True), (1540, 1030, 96, False),
                                       (2304, 2560, 256, True), (64, 4096, 128, True)])
def test_gemm_epilogues_bit_identical(hpl, kind, M, N, K, sub):
    """The bulk-tensor epilogue (C += -(A B^T) reduced in L2 from shared
    memory, or stored) against the per-thread one (each thread reads and
    writes its row of C): the same bits, for every operand kind, with scales,
    ragged tile edges and both kernels (sizes with >= 76 tiles of 256 x 256 go
    to the pair kernel)."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N + K)
    ld = (K + 15) // 16 * 16
    if kind == "bf16":
        A = torch.randn(M, ld, device="cuda", generator=g).to(torch.bfloat16)[:, :K]
        B = torch.randn(N, ld, device="cuda", generator=g).to(torch.bfloat16)[:, :K]
    elif kind == "fp8":
        A = (torch.randn(M, ld, device="cuda", generator=g) * 8).to(torch.float8_e4m3fn)[:, :K]
        B = (torch.randn(N, ld, device="cuda", generator=g) * 8).to(torch.float8_e4m3fn)[:, :K]
    elif kind == "f16":
        A = torch.randn(M, ld, device="cuda", generator=g).to(torch.float16)[:, :K]
        B = torch.randn(N, ld, device="cuda", generator=g).to(torch.float16)[:, :K]
    else:
        A = _tf32(torch.randn(M, ld, device="cuda", generator=g))[:, :K]
        B = _tf32(torch.randn(N, ld, device="cuda", generator=g))[:, :K]
    sa = torch.pow(2.0, torch.randint(-4, 4, (M,), device="cuda", generator=g).float())
    sb = torch.pow(2.0, torch.randint(-4, 4, (N,), device="cuda", generator=g).float())
    C0 = hpl.colmajor(M, N, dtype=torch.float32)
    C0.copy_(torch.randn(M, N, device="cuda", generator=g))
    out = []
    try:
        for mode in (0, 1):
            hpl.gemm_config(hpl.GEMM_EPILOGUE, mode)
            C = C0.clone()
            if kind == "bf16":
                hpl.gemm_bf16(A, B, C, sub=sub)
            elif kind == "fp8":
                hpl.gemm_fp8(A, B, C, sa, sb, sub=sub)
            elif kind == "f16":
                hpl.gemm_f16(A, B, C, sa, sb, sub=sub)
            else:
                hpl.gemm_tf32(A, B, C, sub=sub)
            torch.cuda.synchronize()
            out.append(C)
    finally:
        hpl.gemm_config(hpl.GEMM_EPILOGUE, 0)
    assert torch.equal(out[0], out[1])


@pytest.mark.parametrize("kind", ["bf16", "fp8", "f16", "tf32"])
@pytest.mark.parametrize("M,N,K,sub", [(2560, 2304, 4096, True), (2404, 2600, 200, True), (2560, 2560, 328, False)])
def test_gemm_pair_two_atom_stages_bit_identical(hpl, kind, M, N, K, sub):
    """The pair kernel with two 128-byte swizzle atoms of K per pipeline stage
    (switch 3) issues the same MMAs in the same K order as with one, so C must
    be bit-identical; a K that ends inside a stage (the second atom entirely
    past K, zero-filled) included."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(M + 3 * N + K)
    ld = (K + 15) // 16 * 16
    if kind == "bf16":
        A = torch.randn(M, ld, device="cuda", generator=g).to(torch.bfloat16)[:, :K]
        B = torch.randn(N, ld, device="cuda", generator=g).to(torch.bfloat16)[:, :K]
    elif kind == "fp8":
        A = (torch.randn(M, ld, device="cuda", generator=g) * 8).to(torch.float8_e4m3fn)[:, :K]
        B = (torch.randn(N, ld, device="cuda", generator=g) * 8).to(torch.float8_e4m3fn)[:, :K]
    elif kind == "f16":
        A = torch.randn(M, ld, device="cuda", generator=g).to(torch.float16)[:, :K]
        B = torch.randn(N, ld, device="cuda", generator=g).to(torch.float16)[:, :K]
    else:
        A = _tf32(torch.randn(M, ld, device="cuda", generator=g))[:, :K]
        B = _tf32(torch.randn(N, ld, device="cuda", generator=g))[:, :K]
    sa = torch.pow(2.0, torch.randint(-4, 4, (M,), device="cuda", generator=g).float())
    sb = torch.pow(2.0, torch.randint(-4, 4, (N,), device="cuda", generator=g).float())
    C0 = hpl.colmajor(M, N, dtype=torch.float32)
    C0.copy_(torch.randn(M, N, device="cuda", generator=g))
    out = []
    try:
        for atoms in (1, 2):
            hpl.gemm_config(hpl.GEMM_PAIR_ATOMS, atoms)
            C = C0.clone()
            if kind == "bf16":
                hpl.gemm_bf16(A, B, C, sub=sub)
            elif kind == "fp8":
                hpl.gemm_fp8(A, B, C, sa, sb, sub=sub)
            elif kind == "f16":
                hpl.gemm_f16(A, B, C, sa, sb, sub=sub)
            else:
                hpl.gemm_tf32(A, B, C, sub=sub)
            torch.cuda.synchronize()
            out.append(C)
    finally:
        hpl.gemm_config(hpl.GEMM_PAIR_ATOMS, 2)
    assert torch.equal(out[0], out[1])


def test_gemm_config_rejects_unknown(hpl):
    with pytest.raises(hpl.HplError):
        hpl.gemm_config(9, 0)
    with pytest.raises(hpl.HplError):
        hpl.gemm_config(hpl.GEMM_EPILOGUE, 5)
    with pytest.raises(hpl.HplError):
        hpl.gemm_config(hpl.GEMM_PAIR_ATOMS, 3)


def _tf32(x):
    """Input preparation: round float32 values to TF32 (round to nearest even
    at fraction bit 13) so that the MMA, which reads only the top 19 bits,
    sees exactly these values."""
    import torch
    u = x.contiguous().view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    finite = (u & 0x7F800000) != 0x7F800000
    r = (u + 0x0FFF + ((u >> 13) & 1)) & 0xFFFFE000
    u = torch.where(finite, r, u)
    u = torch.where(u >= 2 ** 31, u - 2 ** 32, u).to(torch.int32)
    return u.view(torch.float32).view(x.shape)


@pytest.mark.parametrize("M,N,K,sub", [(128, 256, 64, True), (300, 500, 200, True), (257, 129, 72, False),
                                       (1536, 2048, 1536, True), (2304, 2560, 256, True), (2404, 2100, 200, True)])
def test_gemm_tf32_matches_fp64(hpl, M, N, K, sub):
    """kind::tf32 products of TF32-rounded FP32 operands against the FP64
    product of the same operands, FP32 accumulation bound; single-CTA and
    pair kernels, ragged edges and K tails."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(M + 3 * N + K)
    ld = (K + 7) // 8 * 8
    A = _tf32(torch.randn(M, ld, device="cuda", generator=g))[:, :K]
    B = _tf32(torch.randn(N, ld, device="cuda", generator=g))[:, :K]
    C = hpl.colmajor(M, N, dtype=torch.float32)
    C.copy_(torch.randn(M, N, device="cuda", generator=g))
    C0 = C.clone()
    hpl.gemm_tf32(A, B, C, sub=sub)
    prod = A.double() @ B.double().t()
    ref = C0.double() - prod if sub else prod
    bound = A.double().abs() @ B.double().abs().t()
    err = (C.double() - ref).abs()
    tol = (K * 2.0 ** -23 + 1e-6) * bound + 2.0 ** -23 * C0.double().abs()
    assert (err > tol).sum().item() == 0, err.max().item()
    # the operands really are TF32: a BF16 rounding of them would miss this bound
    assert torch.equal(_tf32(A), A)
