"""The C-ABI library loads and exports every entry point include/mm.h declares,
and its host-side argument checks reject bad calls before touching a device.
No GPU is needed: nothing here enqueues work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(mm_[a-z0-9_]+)\s*\(", text):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def native():
    from paper_1106_1347_gb300 import build, _native

    build.build()
    return _native


def test_header_declares_the_paper_methods():
    names = declared_functions()
    for required in ("mm_naive", "mm_kahan", "mm_winograd", "mm_winograd_scaled", "mm_strassen",
                     "mm_strassen_winograd", "mm_norm_inf", "mm_emulated"):
        assert required in names


def test_every_declared_symbol_is_exported(native):
    lib = ctypes.CDLL(native.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(native):
    assert set(declared_functions()) <= set(native.SIGNATURES)


def test_host_side_queries_and_checks(native):
    lib = native.lib()
    assert lib.mm_version() >= 100
    assert lib.mm_emulated_slices(0, 0, 1e-14) == 8
    assert lib.mm_emulated_slices(0, 3, 1e-14) == 3
    assert lib.mm_emulated_slices(1, 0, 1e-14) < 0
    assert lib.mm_winograd_workspace_bytes(100, 50, 70) >= 8 * 170
    assert lib.mm_strassen_workspace_bytes(256, 256, 256, 128) == 0  # one fused level needs no workspace
    assert lib.mm_strassen_workspace_bytes(256, 256, 256, 64) > 0
    assert lib.mm_emulated_workspace_bytes(300, 200, 100, 0, 8, 1e-14) >= 8 * 2 * 200 * (300 + 100)
    fake = ctypes.c_void_p(0x10000)
    # negative size, short lda, NULL operands, overlapping C: rejected with MM_ERR_ARG (-1)
    assert lib.mm_naive(-1, 2, 2, fake, 2, fake, 2, fake, 2, None) == -1
    assert lib.mm_naive(2, 4, 2, fake, 3, fake, 2, ctypes.c_void_p(0x20000), 2, None) == -1
    assert lib.mm_kahan(2, 2, 2, None, 2, fake, 2, ctypes.c_void_p(0x20000), 2, None) == -1
    assert lib.mm_naive(4, 4, 4, fake, 4, ctypes.c_void_p(0x30000), 4, ctypes.c_void_p(0x10008), 4, None) == -1
    assert b"overlap" in lib.mm_last_error()
    # short workspace is reported as MM_ERR_WORKSPACE (-6)
    assert lib.mm_winograd(8, 8, 8, fake, 8, ctypes.c_void_p(0x30000), 8, ctypes.c_void_p(0x50000), 8,
                           ctypes.c_void_p(0x70000), 8, None) == -6
    # degenerate shapes are no-ops that return MM_OK without a device
    assert lib.mm_naive(0, 5, 5, None, 5, fake, 5, None, 5, None) == 0
    assert lib.mm_emulated(3, 3, 3, fake, 3, ctypes.c_void_p(0x30000), 3, ctypes.c_void_p(0x50000), 3, 1, 0, 1e-14,
                           None, 0, None) == -4  # 1e-14 needs 12 FP8-E4M3 slices, more than 8
    # the slice product's tile width: 64 (up to 8 slices) or 32, anything else is refused before any device work
    w = ctypes.c_void_p(0x30000), ctypes.c_void_p(0x50000)
    assert lib.mm_emulated_tiled(3, 3, 3, fake, 3, w[0], 3, w[1], 3, 0, 8, 1e-14, 48, None, 0, None) == -1
    assert lib.mm_emulated_tiled(3, 3, 3, fake, 3, w[0], 3, w[1], 3, 1, 10, 1e-14, 64, None, 0, None) == -1
    assert lib.mm_emulated_tiled(0, 3, 3, fake, 3, w[0], 3, w[1], 3, 0, 8, 1e-14, 32, None, 0, None) == 0
    assert lib.mm_emulated_slices(1, 0, 1e-6) == 6  # beta = 5: ceil((log2(1e6) + 9) / 5)
    assert lib.mm_emulated_slices(0, 0, 1e-6) == 5  # beta = 7
    assert lib.mm_emulated_slices(2, 0, 1e-6) < 0  # unknown format
    # FP8 slices take one byte per digit: about half the BF16 workspace
    bf = lib.mm_emulated_workspace_bytes(1024, 1024, 1024, 0, 6, 1e-14)
    f8 = lib.mm_emulated_workspace_bytes(1024, 1024, 1024, 1, 6, 1e-14)
    assert 0 < f8 < bf
    # Strassen levels over the emulated product: variant 0/1, levels 0..4
    assert lib.mm_strassen_emulated_workspace_bytes(512, 512, 512, 0, 1, 0, 8, 1e-14) > \
        lib.mm_emulated_workspace_bytes(256, 256, 256, 0, 8, 1e-14) * 7
    assert lib.mm_strassen_emulated_workspace_bytes(512, 512, 512, 2, 1, 0, 8, 1e-14) == 0
    assert lib.mm_strassen_emulated_workspace_bytes(512, 512, 512, 0, 5, 0, 8, 1e-14) == 0
    assert lib.mm_strassen_emulated_workspace_bytes(512, 512, 512, 0, -2, 0, 8, 1e-14) == 0
    # levels = -1: none below 5120, one up to 12288, two from there
    for n, lv in ((4096, 0), (8192, 1), (16384, 2)):
        assert lib.mm_strassen_emulated_workspace_bytes(n, n, n, 1, -1, 0, 8, 1e-14) == \
            lib.mm_strassen_emulated_workspace_bytes(n, n, n, 1, lv, 0, 8, 1e-14)
    assert lib.mm_strassen_emulated(8, 8, 8, fake, 8, ctypes.c_void_p(0x30000), 8, ctypes.c_void_p(0x50000), 8, 2, 1, 0,
                                    8, 1e-14, None, 0, None) == -1
    assert lib.mm_strassen_emulated(8, 8, 8, fake, 8, ctypes.c_void_p(0x30000), 8, ctypes.c_void_p(0x50000), 8, 0, 5, 0,
                                    8, 1e-14, None, 0, None) == -1
    assert lib.mm_strassen_emulated(8, 8, 8, fake, 8, ctypes.c_void_p(0x30000), 8, ctypes.c_void_p(0x50000), 8, 0, 1, 0,
                                    8, 1e-14, None, 0, None) == -6  # no workspace
    # the paper's Strassen rule at 4096 (depth 8) needs a workspace; depth 17 (X = 2^21) is refused
    assert lib.mm_strassen_workspace_bytes(4096, 4096, 4096, 0) > 0
    assert lib.mm_strassen(4096, 4096, 4096, fake, 4096, ctypes.c_void_p(0x30000), 4096, ctypes.c_void_p(0x10000000000),
                           4096, 0, None, 0, None) == -6
    assert lib.mm_strassen_workspace_bytes(1 << 21, 1, 1, 0) == 0
    assert lib.mm_strassen(1 << 21, 1, 1, fake, 1, ctypes.c_void_p(0x1000000000), 1, ctypes.c_void_p(0x2000000000),
                           1, 0, None, 0, None) == -4
