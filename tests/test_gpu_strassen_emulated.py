"""GPU parity of Strassen / Strassen-Winograd levels over the emulated product
(mm_strassen_emulated) against the oracle's restatement of the same
definition: bit-exact, since every step (operand sums, split products, H
combinations) is deterministic."""
import numpy as np
import pytest

import synthetic as S
from strassen_sampled import one_level_sampled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mm():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1106_1347_gb300 import build

    build.build()
    import paper_1106_1347_gb300 as m

    return m


def dev(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def pair(n, p, m, tag):
    return S.loguniform(n, p, S.stream_seed(3, 500 + 2 * tag)), S.loguniform(p, m, S.stream_seed(3, 501 + 2 * tag))


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("levels", [1, 2])
@pytest.mark.parametrize("shape", [(64, 64, 64), (97, 130, 71), (1, 1, 1), (3, 5, 2), (256, 200, 136)])
def test_bf16_bit_exact_vs_oracle(mm, orc, variant, levels, shape):
    a, b = pair(*shape, tag=levels + 3 * variant)
    got = mm.strassen_emulated(dev(a), dev(b), variant=variant, levels=levels, nslices=8).cpu().numpy()
    assert np.array_equal(got, orc.strassen_emulated(a, b, variant, levels, 7, 8))


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("levels,s", [(1, 6), (2, 3), (3, 8)])
def test_fp8_bit_exact_vs_oracle(mm, orc, variant, levels, s):
    a, b = pair(90, 150, 66, tag=20 + levels)
    got = mm.strassen_emulated(dev(a), dev(b), variant=variant, levels=levels, nslices=s,
                               kind=mm.SLICE_FP8E4M3).cpu().numpy()
    assert np.array_equal(got, orc.strassen_emulated(a, b, variant, levels, 5, s))


@pytest.mark.parametrize("variant", [0, 1])
def test_three_and_four_levels_bit_exact(mm, orc, variant):
    a, b = pair(80, 112, 48, tag=30)
    for levels in (3, 4):
        got = mm.strassen_emulated(dev(a), dev(b), variant=variant, levels=levels, nslices=4).cpu().numpy()
        assert np.array_equal(got, orc.strassen_emulated(a, b, variant, levels, 7, 4))


def test_automatic_levels_below_the_crossover_is_the_emulated_product(mm):
    a, b = pair(120, 90, 100, tag=41)
    ta, tb = dev(a), dev(b)
    got = mm.strassen_emulated(ta, tb, variant=1, levels=-1, nslices=8)
    assert bool((got == mm.emulated(ta, tb, nslices=8)).all())


def test_zero_levels_is_the_emulated_product(mm):
    a, b = pair(150, 97, 130, tag=40)
    ta, tb = dev(a), dev(b)
    for variant in (0, 1):
        got = mm.strassen_emulated(ta, tb, variant=variant, levels=0, nslices=8)
        assert bool((got == mm.emulated(ta, tb, nslices=8)).all())


@pytest.mark.parametrize("variant", [0, 1])
def test_integers_exact(mm, variant):
    a = S.integers(130, 77, S.stream_seed(0, 61))
    b = S.integers(77, 95, S.stream_seed(0, 62))
    got = mm.strassen_emulated(dev(a), dev(b), variant=variant, levels=2, nslices=3).cpu().numpy()
    assert np.array_equal(got, a @ b)


@pytest.mark.parametrize("variant", [0, 1])
def test_tier_accuracy(mm, orc, variant):
    a = S.uniform(200, 180, S.stream_seed(1, 71))
    b = S.uniform(180, 160, S.stream_seed(1, 72))
    truth = orc.dot2_product(a, b)
    for levels in (1, 2, 3):
        got = mm.strassen_emulated(dev(a), dev(b), variant=variant, levels=levels, tier=1e-14).cpu().numpy()
        assert orc.rel_inf_error(got, truth, a, b) <= 1e-14


def test_strided_operands_and_output(mm, orc):
    """Operands and result inside larger matrices (lda, ldb, ldc > the widths)."""
    import torch

    a, b = pair(66, 90, 50, tag=50)
    big_a = torch.zeros((66, 128), dtype=torch.float64, device="cuda")
    big_b = torch.zeros((90, 77), dtype=torch.float64, device="cuda")
    big_c = torch.full((66, 99), 7.0, dtype=torch.float64, device="cuda")
    big_a[:, :90] = dev(a)
    big_b[:, :50] = dev(b)
    mm.strassen_emulated(big_a[:, :90], big_b[:, :50], variant=1, levels=2, nslices=8, out=big_c[:, :50])
    assert np.array_equal(big_c[:, :50].cpu().numpy(), orc.strassen_emulated(a, b, 1, 2, 7, 8))
    assert bool((big_c[:, 50:] == 7.0).all())


@pytest.fixture(scope="module")
def big():
    return S.loguniform(8192, 8192, S.stream_seed(3, 0)), S.loguniform(8192, 8192, S.stream_seed(3, 1))


@pytest.mark.parametrize("variant", [0, 1])
def test_8192_cubed_one_level_sampled_bit_exact(mm, orc, big, variant):
    """The bench workload (8192^3, log-uniform): sampled entries in all four
    quadrants equal the definition bit for bit."""
    a, b = big
    c = mm.strassen_emulated(dev(a), dev(b), variant=variant, levels=1, nslices=8)
    rows = np.array([0, 1, 4095, 4096, 4097, 8191])
    cols = np.array([0, 63, 64, 4095, 4096, 5000, 8191])
    got = c[rows][:, cols].cpu().numpy()
    assert np.array_equal(got, one_level_sampled(orc, a, b, variant, rows, cols, 7, 8))
