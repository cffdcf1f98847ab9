"""The autotuner's table on the host (no GPU): the model's choices without
entries, recorded choices after mm_tune_load, a save/load round trip, and
malformed lines skipped.  The choices decide what mm_emulated_auto,
cutoff = -1 Strassen and serving method 2 run."""
import ctypes
import math

import pytest


@pytest.fixture()
def lib():
    from paper_1106_1347_gb300 import _native, build

    build.build()
    L = _native.lib()
    L.mm_tune_clear()
    yield L
    L.mm_tune_clear()


def choice(L, n, p, m, tier, with_tile=False):
    k, s, lv, tl = ctypes.c_int32(-1), ctypes.c_int32(-1), ctypes.c_int32(-1), ctypes.c_int32(-1)
    rc = L.mm_tune_emulated_choice(n, p, m, tier, ctypes.byref(k), ctypes.byref(s), ctypes.byref(lv), ctypes.byref(tl))
    return (rc, (k.value, s.value, lv.value, tl.value)) if with_tile else (rc, (k.value, s.value, lv.value))


def test_model_choices_without_entries(lib):
    # 1e-14: only BF16 reaches it (8 slices); 4096 is below the first Strassen crossover.
    assert choice(lib, 4096, 4096, 4096, 1e-14) == (0, (0, 8, 0))
    # 1e-6: 6 FP8 slices (21 pairs at twice the rate) cost less than 5 BF16 slices (15 pairs).
    assert choice(lib, 8192, 8192, 8192, 1e-6) == (0, (1, 6, 1))
    assert choice(lib, 16384, 16384, 16384, 1e-14)[1][2] == 2
    # the slice counts are the tier formula's: ceil((log2(1/tier) + 9) / beta)
    for tier in (1e-3, 1e-9, 1e-12):
        rc, (k, s, lv) = choice(lib, 1000, 1000, 1000, tier)
        assert rc == 0 and s == math.ceil((-math.log2(tier) + 9) / (5 if k == 1 else 7))
    assert choice(lib, 100, 100, 100, 0.0)[0] < 0
    assert choice(lib, 100, 100, 100, -1.0)[0] < 0


def test_model_tile_width(lib):
    # 64-column tiles unless M is narrow enough that 32-column ones (at about 2/3
    # of the MMA rate) pad less by more than a third: M <= 32
    assert choice(lib, 4096, 4096, 32, 1e-14, True) == (0, (0, 8, 0, 32))
    assert choice(lib, 4096, 4096, 20, 1e-6, True)[1][3] == 32
    assert choice(lib, 4096, 4096, 33, 1e-14, True)[1][3] == 64
    assert choice(lib, 4096, 4096, 4096, 1e-14, True)[1][3] == 64
    # past 8 FP8 slices the tile is 32 columns whatever M is
    rc, (k, s, lv, tl) = choice(lib, 4096, 4096, 4096, 1e-12, True)
    assert (k == 1 and s > 8 and tl == 32) or (s <= 8 and tl == 64)


def test_recorded_choices_round_trip(lib, tmp_path):
    f = tmp_path / "tune.txt"
    f.write_text("strassen 0 12 5\n"
                 "emulated 12 12 12 6 0 5 1\n"     # no tile width (older files): the default
                 "emulated 9 9 9 14 0 8 0 32\n"
                 "emulated 1 2 3\n"            # short line: skipped
                 "strassen 5 3 3\n"            # no such variant: skipped
                 "emulated 9 9 9 9 7 8 0\n"    # no such format: skipped
                 "emulated 9 9 9 3 0 8 0 48\n"  # no such tile width: skipped
                 "comment line\n")
    assert lib.mm_tune_load(str(f).encode()) == 3
    assert choice(lib, 4096, 4096, 4096, 1e-6, True) == (1, (0, 5, 1, 64))
    assert choice(lib, 600, 700, 1000, 1e-14, True) == (1, (0, 8, 0, 32))  # bucket (9, 9, 9), tier decade 14
    assert choice(lib, 4096, 4096, 4096, 1e-14)[0] == 0          # other tier decade: the model
    # the loaded Strassen depth drives cutoff = -1: depth 5 at 4096 is cutoff 128's plan
    assert lib.mm_strassen_workspace_bytes(4096, 4096, 4096, -1) == lib.mm_strassen_workspace_bytes(4096, 4096, 4096,
                                                                                                   128)
    g = tmp_path / "saved.txt"
    assert lib.mm_tune_save(str(g).encode()) == 0
    lines = sorted(g.read_text().splitlines())
    assert lines == sorted(["strassen 0 12 5", "emulated 12 12 12 6 0 5 1 0", "emulated 9 9 9 14 0 8 0 32"])
    lib.mm_tune_clear()
    assert choice(lib, 4096, 4096, 4096, 1e-6)[0] == 0
    assert lib.mm_tune_load(str(g).encode()) == 3
    assert choice(lib, 4096, 4096, 4096, 1e-6) == (1, (0, 5, 1))


def test_untuned_strassen_default_is_the_papers_depth(lib):
    # no entry: depth floor(log2 min dim) - 4, each dimension padded to a multiple of 2^depth
    for n, depth in ((1024, 6), (4096, 8), (300, 4)):
        assert lib.mm_strassen_workspace_bytes(n, n, n, -1) == \
            lib.mm_strassen_workspace_bytes(n, n, n, -(-n // (1 << depth)))
    # Winograd's variant stops at 6 levels (its error about doubles per level)
    for n, depth in ((1024, 6), (8192, 6), (300, 4)):
        assert lib.mm_strassen_winograd_workspace_bytes(n, n, n, -1) == \
            lib.mm_strassen_winograd_workspace_bytes(n, n, n, -(-n // (1 << depth)))
