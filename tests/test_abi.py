"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/*.h declares (no compute call is made here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", text):
            name = m.group(1)
            start = text.rfind("\n", 0, m.start()) + 1
            prefix = text[start:m.start()]
            if name in ("if", "while", "for", "sizeof", "defined") or "#" in prefix:
                continue
            if re.search(r"\b(int|size_t|void|const char\s*\*|double|int64_t|uint64_t)\s*\*?\s*$", prefix):
                names.add(name)
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2604_09517_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_api():
    names = _declared_functions()
    for must in ["hpl_generate", "lu_factor", "lu_solve", "hpl_scaled_residual", "lu_factor_workspace_size"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(lib):
    lib.hpl_status_string.restype = ctypes.c_char_p
    assert lib.hpl_status_string(0) == b"HPL_OK"
    assert lib.hpl_status_string(2) == b"HPL_ERR_SINGULAR"
    assert lib.hpl_status_string(99) == b"HPL_ERR_UNKNOWN"


def test_invalid_arguments_rejected_before_any_launch(lib):
    """Argument checks run on the host and launch nothing. The pointers are
    placeholders, so this runs only where no GPU is visible (the GPU tests
    repeat such checks with real buffers)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("placeholder pointers are never passed where a GPU is visible")
    lib.hpl_generate.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                 ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    assert lib.hpl_generate(1, 0, 10, 10, 0, None, 10, None) == 1          # NULL A
    assert lib.hpl_generate(1, 0, 10, 10, 0, 8, 5, None) == 1              # lda < m
    assert lib.hpl_generate(1, 0, 10, 9, 1, 8, 10, None) == 1              # dominant, not square
    assert lib.hpl_generate(1, 0, 0, 10, 0, None, 1, None) == 0            # empty: nothing to do
    lib.lu_factor.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.lu_factor(-1, 8, 1, 8, None, 8, 1 << 20, 8, None) == 1
    assert lib.lu_factor(10, 8, 5, 8, None, 8, 1 << 20, 8, None) == 1
    assert lib.lu_factor(10, 8, 10, 8, None, 8, 16, 8, None) == 6          # workspace too small
    import paper_2604_09517_gb300 as hpl
    bad_pfact = hpl.make_opts(nb=64, pfact=2)
    assert lib.lu_factor(10, 8, 10, 8, ctypes.byref(bad_pfact), 8, 1 << 20, 8, None) == 1
    lib.mxp_solve.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                              ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p]
    for o in (hpl.make_opts(nb=64, storage=2), hpl.make_opts(nb=64, prec=hpl.PREC_FP8_E4M3, storage=1),
              hpl.make_opts(nb=64, prec=hpl.PREC_FP16, storage=1), hpl.make_opts(nb=64, prec=3)):
        assert lib.mxp_solve(10, 1, 8, 10, 0, 8, 10, 8, 10, ctypes.byref(o), 8, 1 << 30, 8, None) == 1


def test_batch_sizes_host_function_matches_oracle(lib, orc):
    """hpl_batch_sizes is host code (no GPU needed): same draws as the oracle."""
    import numpy as np
    out = np.empty(4096, dtype=np.int64)
    lib.hpl_batch_sizes.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
    assert lib.hpl_batch_sizes(1, 4096, out.ctypes.data) == 0
    assert np.array_equal(out, orc.batch_sizes(1, 4096))


def test_autotune_table_lookup():
    """The batched tile-shape table maps (kind, size bucket) to a variant."""
    import numpy as np
    from paper_2604_09517_gb300 import autotune
    assert list(autotune.bucket_of([32, 63, 64, 127, 128, 255, 256, 512])) == [0, 0, 1, 1, 2, 2, 3, 3]
    table = {"GPU-X": {"choice": {"0": [1, 0, 0, 0], "1": [0, 1, 1, 0]}}}
    got = autotune.variants([40, 100, 300, 40, 200], [0, 0, 0, 1, 1], table, "GPU-X")
    assert list(got) == [1, 0, 0, 0, 1]
    assert list(autotune.variants([40, 300], [0, 1], {}, "GPU-X")) == [0, 0]
    # the whole-batch policy "narrow" (16-wide panels everywhere, two CTAs per
    # SM) overrides the per-bucket widths; "per_bucket" keeps them
    table["GPU-X"]["policy"] = "narrow"
    assert list(autotune.variants([40, 100, 300], [0, 0, 1], table, "GPU-X")) == [1, 1, 1]
    table["GPU-X"]["policy"] = "per_bucket"
    assert list(autotune.variants([40, 100, 300], [0, 0, 1], table, "GPU-X")) == [1, 0, 0]


def test_workspace_sizes_follow_the_options():
    """Workspace queries are host code: BF16 storage halves the working matrix
    of the mixed-precision solve; the tensor-core FP64 emulation adds its
    slice buffers to the LU workspace; the pfact option does not change it."""
    import ctypes as C
    import paper_2604_09517_gb300 as hpl
    lib = hpl.load()
    n = 4096
    o32 = hpl.make_opts(nb=512)
    o16 = hpl.make_opts(nb=512, storage=hpl.STORAGE_BF16)
    s32 = lib.mxp_workspace_size(n, 1, C.byref(o32))
    s16 = lib.mxp_workspace_size(n, 1, C.byref(o16))
    assert s32 - s16 >= 2 * n * n - 256 and s32 - s16 <= 2 * n * n + 256
    base = lib.lu_factor_workspace_size(n, C.byref(hpl.make_opts(nb=256)))
    emu = lib.lu_factor_workspace_size(n, C.byref(hpl.make_opts(nb=256, fp64_emulation=1)))
    coop = lib.lu_factor_workspace_size(n, C.byref(hpl.make_opts(nb=256, pfact=1)))
    assert emu > base + 40 * n * n // 2 and coop == base
    # lu_solve: the interchange pairs (2 x 2 x 256 ints per 256 pivots) and the
    # one-launch solve's published blocks (y and x: 2 x 64 doubles per 64 rows)
    for m in (1, 63, 64, 65, 1000, 32768):
        blocks64, blocks256 = -(-m // 64), -(-m // 256)
        need = 2 * 8 * 64 * blocks64 + 2 * 2 * 4 * 256 * blocks256
        got = lib.lu_solve_workspace_size(m, 1)
        assert need <= got <= need + 4096 + 4 * blocks256, (m, got, need)
        assert lib.lu_solve_workspace_size(m, 7) == got


def test_profiles_are_short_text_with_their_command():
    """profiles/ holds short text summaries, each naming the command that made
    it and running only committed files (no scratch paths)."""
    names = sorted(glob.glob(os.path.join(ROOT, "profiles", "*")))
    assert names
    for p in names:
        assert p.endswith((".txt", ".md")), p
        text = open(p).read()
        assert len(text) < 16384, p
        assert "Command" in text and "ncu" in text, p
        assert "_work" not in text, p


def test_measurement_switches_accept_documented_values_only(lib):
    """hplgb_gemm_config, hplgb_lu_config and hplgb_batched_config take the
    values include/hplgb.h documents and refuse others with HPL_ERR_INVALID
    (1). They only set host state, so this runs without a GPU. The defaults
    are restored at the end."""
    ok = {
        "hplgb_gemm_config": [(0, 0), (0, 1), (1, 0), (1, 16), (1, 4096), (2, 0), (2, -1), (2, 1 << 30), (3, 1),
                              (3, 2)],
        "hplgb_lu_config": [(0, 0), (0, 1), (1, 0), (1, 1), (2, 0), (2, 1), (2, 4096)],
        "hplgb_batched_config": [(0, 0), (0, 1)],
    }
    bad = {
        "hplgb_gemm_config": [(0, 2), (0, -1), (1, -1), (1, 4097), (3, 0), (3, 3), (4, 0), (-1, 0)],
        "hplgb_lu_config": [(0, 2), (0, -1), (1, 2), (1, -1), (2, -1), (2, 4097), (3, 0), (-1, 0)],
        "hplgb_batched_config": [(0, 2), (0, -1), (1, 0)],
    }
    defaults = {
        "hplgb_gemm_config": [(0, 0), (1, 0), (2, 0), (3, 2)],
        "hplgb_lu_config": [(0, 1), (1, 1), (2, 0)],
        "hplgb_batched_config": [(0, 0)],
    }
    fn = {}
    for name in ok:
        f = getattr(lib, name)
        f.argtypes = [ctypes.c_int, ctypes.c_longlong]
        f.restype = ctypes.c_int
        fn[name] = f
    try:
        for name, cases in ok.items():
            for what, value in cases:
                assert fn[name](what, value) == 0, (name, what, value)
        for name, cases in bad.items():
            for what, value in cases:
                assert fn[name](what, value) == 1, (name, what, value)
    finally:
        for name, cases in defaults.items():
            for what, value in cases:
                assert fn[name](what, value) == 0
