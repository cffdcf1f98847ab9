"""The emulated product's autotuner through the C ABI: mm_tune_emulated times
the candidates (slice format x Strassen-Winograd levels) and records one;
mm_emulated_auto then runs exactly that choice -- bit-identical to the
explicit call with the same format, slice count and levels -- and meets the
tier against the oracle's Dot2 product."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mm():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1106_1347_gb300 import build

    build.build()
    import paper_1106_1347_gb300 as mm

    mm.lib()
    return mm


def dev(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


@pytest.mark.parametrize("shape,tier", [((640, 700, 600), 1e-6), ((2048, 2048, 2048), 1e-14),
                                        ((1100, 3000, 1030), 1e-9), ((3000, 2000, 24), 1e-14)])
def test_tune_emulated_then_auto(mm, orc, tmp_path, shape, tier):
    mm.tune_clear()
    a = S.loguniform(shape[0], shape[1], S.stream_seed(3, 60))
    b = S.loguniform(shape[1], shape[2], S.stream_seed(3, 61))
    ta, tb = dev(a), dev(b)
    (k0, s0, l0, w0), tuned = mm.emulated_choice(*shape, tier)
    assert not tuned  # the model's choice before tuning
    kind, s, levels, ms, tile = mm.tune_emulated(ta, tb, tier=tier)
    assert ms > 0 and kind in (0, 1) and 1 <= s <= 8 and 0 <= levels <= 2 and tile in (32, 64)
    assert levels == 0 or tile == 64
    assert s == mm.emulated_slices(0, tier, kind)
    (k1, s1, l1, w1), tuned = mm.emulated_choice(*shape, tier)
    assert tuned and (k1, s1, l1, w1) == (kind, s, levels, tile)
    c, used = mm.emulated_auto(ta, tb, tier=tier, return_choice=True)
    assert used == (kind, s, levels, tile)
    if levels == 0:
        ref = mm.emulated_tiled(ta, tb, tile, nslices=s, kind=kind)
        assert np.array_equal(ref.cpu().numpy(), mm.emulated(ta, tb, nslices=s, kind=kind).cpu().numpy())
    else:
        ref = mm.strassen_emulated(ta, tb, variant=1, levels=levels, nslices=s, kind=kind)
    assert np.array_equal(c.cpu().numpy(), ref.cpu().numpy())
    rows = np.linspace(0, shape[0] - 1, 6).astype(np.int64)
    truth = orc.dot2_product(a[rows], b)
    na, nb = float(np.abs(a).sum(axis=1).max()), float(np.abs(b).sum(axis=1).max())
    err = float(np.abs(c.cpu().numpy()[rows] - truth).sum(axis=1).max() / (na * nb))
    assert err <= tier
    # the choice persists through save / load
    path = tmp_path / "tune.txt"
    mm.tune_save(path)
    mm.tune_clear()
    assert not mm.emulated_choice(*shape, tier)[1]
    assert mm.tune_load(path) == 1
    assert mm.emulated_choice(*shape, tier) == ((kind, s, levels, tile), True)
    mm.tune_clear()
