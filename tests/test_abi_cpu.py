"""Host-side checks of the C-ABI library that need no GPU: it loads, it exports
every entry point include/*.h declares, its null-argument paths return
status codes, and the oracle and the product path stay independent."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1503_03806_gb300")


@pytest.fixture(scope="module")
def helk():
    from paper_1503_03806_gb300 import build
    build.build()
    from paper_1503_03806_gb300 import helk as h
    return h


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(helk_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol(helk):
    names = declared_functions()
    assert len(names) >= 9
    for n in names:
        assert hasattr(helk.lib, n), n
    bound = {s[0] for s in helk.SIGNATURES}
    assert names == bound, (names - bound, bound - names)


def test_null_arguments_are_rejected_without_a_gpu(helk):
    lib = helk.lib
    assert lib.helk_create(None, 0, None) == helk.HELK_ERR_INVALID_ARG
    assert lib.helk_sync(None) == helk.HELK_ERR_INVALID_ARG
    assert lib.helk_set_stream(None, None) == helk.HELK_ERR_INVALID_ARG
    s = helk.helk_lines()
    assert lib.helk_lines_upload(None, ctypes.byref(s), 0, 0) == helk.HELK_ERR_INVALID_ARG
    g = helk.helk_grid(0.0, 0.01, 10)
    c = helk.helk_cutoff(0, 1.0, 0.0)
    assert lib.helk_opacity(None, 1.0, 1.0, 1.0, ctypes.byref(c), ctypes.byref(g), None,
                            None) == helk.HELK_ERR_INVALID_ARG
    assert lib.helk_kdist(None, None, 10, 1, 1, 1e-250, None, None, 0, None) == helk.HELK_ERR_INVALID_ARG
    assert lib.helk_opacity_stats(None, None, None) == helk.HELK_ERR_INVALID_ARG
    assert helk.helk_last_error(None) == "null context"
    lib.helk_destroy(None)


def test_kernel_shapes_decode_without_a_gpu(helk):
    # the autotuner's dimensions: tile width (slots per warp), warps per CTA
    # and candidate lines per pipeline stage, each shape named by its code
    f32 = helk.helk_tile_candidates(helk.HELK_PREC_F32_KAHAN)
    shapes = [helk.helk_tile_shape(helk.HELK_PREC_F32_KAHAN, c) for c in f32]
    assert len(set(f32)) == len(f32) >= 10
    assert {s["warps"] for s in shapes} >= {4, 8, 12}
    assert {s["lines_per_stage"] for s in shapes} >= {64, 128, 256}
    assert len({s["points"] for s in shapes if s["warps"] == 8 and s["lines_per_stage"] == 128}) >= 8
    for s in shapes:
        assert s["points"] % (32 * s["warps"]) == 0
    f64 = helk.helk_tile_candidates(helk.HELK_PREC_F64)
    assert [helk.helk_tile_shape(helk.HELK_PREC_F64, c)["points"] for c in f64] == [256 * c for c in f64]
    for prec, bad in ((helk.HELK_PREC_F32_KAHAN, 0), (helk.HELK_PREC_F32_KAHAN, len(f32) + 1),
                      (helk.HELK_PREC_F64, 9), (7, 1)):
        with pytest.raises(helk.HelkError):
            helk.helk_tile_shape(prec, bad)


def test_create_without_gpu_returns_status():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1503_03806_gb300 import helk as h
    out = ctypes.c_void_p()
    assert h.lib.helk_create(ctypes.byref(out), 0, None) == h.HELK_ERR_CUDA


def _sources(path, exts):
    for dp, _, fs in os.walk(path):
        if "_build" in dp or "__pycache__" in dp:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(dp, f)


def test_oracle_and_product_share_nothing():
    # neither side imports, includes or loads the other
    for f in _sources(os.path.join(ROOT, "oracle"), (".py", ".c", ".h")):
        text = open(f).read()
        assert not re.search(r"^\s*(from|import)\s+paper_1503_03806_gb300", text, re.M), f
        assert "csrc" not in text and "helk_internal" not in text and "libhelk" not in text, f
    for f in _sources(PKG, (".py", ".cu", ".cuh", ".h")):
        text = open(f).read()
        assert not re.search(r"^\s*(from|import)\s+oracle\b", text, re.M), f
        assert "liboracle" not in text and "helk_oracle" not in text, f


def test_static_kdist_limits_are_checked_before_any_gpu_work(helk):
    # helk_kdist_static rejects what its fixed scratch cannot hold -- bins
    # above 12288 points, more than 32 coefficients -- and malformed sizes,
    # before it touches a device (the pointers are never dereferenced here)
    lib = helk.lib
    fake = ctypes.c_void_p(0x1000)
    bad = [
        (2 * 12289, 2, 20, 1e-250),   # 12289 points a bin: above the maximum
        (100, 1, 33, 1e-250),         # 33 coefficients
        (100, 1, 0, 1e-250),          # no coefficient
        (101, 2, 20, 1e-250),         # n not a multiple of nbins
        (100, 10, 20, 1e-250),        # ncheb > N_b
        (100, 1, 20, 0.0),            # floor must be > 0
        (100, 1, 20, float("nan")),
        (0, 1, 20, 1e-250),
    ]
    for n, nbins, ncheb, floor in bad:
        st = lib.helk_kdist_static(fake, n, nbins, ncheb, floor, fake, None, None, None)
        assert st == helk.HELK_ERR_INVALID_ARG, (n, nbins, ncheb, floor)
    assert lib.helk_kdist_static(None, 100, 1, 20, 1e-250, fake, None, None, None) == helk.HELK_ERR_INVALID_ARG
    assert lib.helk_kdist_static(fake, 100, 1, 20, 1e-250, None, None, None, None) == helk.HELK_ERR_INVALID_ARG
