"""GPU parity: every method through the C ABI against the CPU oracle, element by
element, on seeded inputs.  Bar: bit-exact for integer-valued inputs (every
method), for NormInf, Kahan, Winograd's y/z path ... and for the emulated
product (its definition is exact integer arithmetic plus one rounding); within
||C - C_ref||_inf / (||A||_inf ||B||_inf) <= 1e-14 for the FP64 methods whose
GPU evaluation order differs from the oracle's (FMA/MMA blocking)."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

TOL = 1e-14


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


def host(t):
    return t.cpu().numpy()


def pair(n, p, m, kind, tag):
    if kind == "int":
        return S.integers(n, p, S.stream_seed(0, 2 * tag)), S.integers(p, m, S.stream_seed(0, 2 * tag + 1))
    if kind == "uni":
        return S.uniform(n, p, S.stream_seed(0, 2 * tag)), S.uniform(p, m, S.stream_seed(0, 2 * tag + 1))
    if kind == "log":
        return S.loguniform(n, p, S.stream_seed(3, 2 * tag)), S.loguniform(p, m, S.stream_seed(3, 2 * tag + 1))
    raise ValueError(kind)


SHAPES = [(1, 1, 1), (3, 5, 2), (64, 64, 64), (65, 17, 33), (128, 129, 63), (256, 256, 256), (200, 333, 150)]


# ----------------------------------------------------------------- NormInf

@pytest.mark.parametrize("shape", [(1, 1), (31, 33), (64, 1000), (257, 129), (1000, 7)])
def test_norm_inf_bit_exact(mm, orc, shape):
    a = S.uniform(*shape, S.stream_seed(0, 900 + shape[0])) * 3.0
    assert float(host(mm.norm_inf(dev(a)))) == orc.norm_inf(a)
    g = np.array([[2.0 ** 53, 1.0, 1.0], [3.0, -4.0, 0.5]])
    assert float(host(mm.norm_inf(dev(g)))) == orc.norm_inf(g)


# ------------------------------------------------------------------ naive

@pytest.mark.parametrize("shape", SHAPES)
def test_naive_integer_bit_exact(mm, orc, shape):
    a, b = pair(*shape, "int", 1)
    assert np.array_equal(host(mm.naive(dev(a), dev(b))), orc.naiv_standard(a, b))


@pytest.mark.parametrize("shape", SHAPES)
def test_naive_uniform_within_tolerance(mm, orc, shape):
    a, b = pair(*shape, "uni", 2)
    got = host(mm.naive(dev(a), dev(b)))
    assert orc.rel_inf_error(got, orc.naiv_standard(a, b), a, b) <= TOL


# ------------------------------------------------------------------ Kahan

@pytest.mark.parametrize("shape", SHAPES)
def test_kahan_bit_exact_on_reals(mm, orc, shape):
    a, b = pair(*shape, "uni", 3)
    assert np.array_equal(host(mm.kahan(dev(a), dev(b))), orc.naiv_kahan(a, b))


def test_kahan_discriminator(mm):
    a = np.array([[2.0 ** 53, 1.0, -(2.0 ** 53)]])
    assert host(mm.kahan(dev(a), dev(np.ones((3, 1)))))[0, 0] == 1.0


# --------------------------------------------------------------- Winograd

@pytest.mark.parametrize("shape", SHAPES + [(33, 2047 % 97, 40)])
def test_winograd_integer_bit_exact(mm, orc, shape):
    a, b = pair(*shape, "int", 4)
    assert np.array_equal(host(mm.winograd(dev(a), dev(b))), orc.winograd_original(a, b))


@pytest.mark.parametrize("shape", SHAPES)
def test_winograd_uniform_within_tolerance(mm, orc, shape):
    a, b = pair(*shape, "uni", 5)
    got = host(mm.winograd(dev(a), dev(b)))
    assert orc.rel_inf_error(got, orc.winograd_original(a, b), a, b) <= TOL


@pytest.mark.parametrize("shape", SHAPES)
def test_winograd_scaled_lambda_and_result(mm, orc, shape):
    a, b = pair(*shape, "uni", 6)
    b = b * 1024.0
    c, lam = mm.winograd_scaled(dev(a), dev(b), return_lambda=True)
    ref, lam_ref = orc.winograd_scaled(a, b)
    assert int(host(lam)[0]) == lam_ref
    assert orc.rel_inf_error(host(c), ref, a, b) <= TOL


def test_winograd_scaled_paper_tie(mm, orc):
    a = S.uniform(40, 40, 77)
    c, lam = mm.winograd_scaled(dev(a), dev(8.0 * a), return_lambda=True)
    assert int(host(lam)[0]) == 1
    ai = S.integers(33, 21, 78)
    bi = S.integers(21, 19, 79) * 64.0
    assert np.array_equal(host(mm.winograd_scaled(dev(ai), dev(bi))), ai @ bi)


# ------------------------------------------- NaivOnArray, loop unrolling

@pytest.mark.parametrize("u", [1, 2, 3, 4])
@pytest.mark.parametrize("shape", SHAPES + [(70, 97, 45), (33, 1001, 65)])
def test_naive_unrolled_bit_exact_on_reals(mm, orc, shape, u):
    """Every product and sum rounded on its own, in the paper's grouping: the
    GPU result equals the sequential CPU one bit for bit (P mod u = 0..3)."""
    a, b = pair(*shape, "log", 30 + u)
    got = host(mm.naive_unrolled(dev(a), dev(b), unroll=u))
    assert np.array_equal(got, orc.naiv_unrolled(a, b, u))
    if u == 1:
        assert np.array_equal(got, orc.naiv_on_array(a, b))


def test_naive_unrolled_discriminator(mm):
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_pins.json")))
    for case in g["loop_unrolling_discriminator"]["cases"]:
        a = np.array([case["row"]])
        b = np.ones((a.shape[1], 1))
        assert host(mm.naive_unrolled(dev(a), dev(b), unroll=1))[0, 0] == case["naive"]
        for u in (2, 3, 4):
            assert host(mm.naive_unrolled(dev(a), dev(b), unroll=u))[0, 0] == case[f"u{u}"]


def test_naive_unrolled_rejects_bad_factor(mm):
    import torch

    a = torch.ones((4, 4), dtype=torch.float64, device="cuda")
    c = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    for u in (0, 5, -1):
        rc = mm.lib().mm_naive_unrolled(4, 4, 4, a.data_ptr(), 4, a.data_ptr(), 4, c.data_ptr(), 4, u, None)
        assert rc == -1


# ---------------------------------------- per-row/column scaled Winograd

@pytest.mark.parametrize("shape", SHAPES + [(33, 2047 % 97, 40)])
def test_winograd_rowcol_integer_bit_exact(mm, orc, shape):
    a, b = pair(*shape, "int", 21)
    got = host(mm.winograd_rowcol_scaled(dev(a), dev(b)))
    assert np.array_equal(got, orc.winograd_rowcol_scaled(a, b)[0])
    assert np.array_equal(got, a @ b)


@pytest.mark.parametrize("shape", SHAPES)
def test_winograd_rowcol_uniform_within_tolerance(mm, orc, shape):
    a, b = pair(*shape, "uni", 22)
    got = host(mm.winograd_rowcol_scaled(dev(a), dev(b)))
    assert orc.rel_inf_error(got, orc.winograd_rowcol_scaled(a, b)[0], a, b) <= TOL


@pytest.mark.parametrize("n", [64, 301])
def test_winograd_rowcol_badly_scaled(mm, orc, n):
    """Rows of A times 10^u, columns of B times 10^v: every element within the
    elementwise bound 8 gamma (gamma + 5) u 2^(e_i + f_k) of the exact product
    (the oracle's own pin), which plain Winograd misses by orders of magnitude."""
    a, b = S.badly_scaled(n, S.stream_seed(2, 20 + n), S.stream_seed(2, 21 + n))
    truth = orc.dot2_product(a, b)
    ref, e, f = orc.winograd_rowcol_scaled(a, b)
    got = host(mm.winograd_rowcol_scaled(dev(a), dev(b)))
    gamma = n // 2
    bound = 8 * gamma * (gamma + 5) * 2.0 ** -53 * np.ldexp(1.0, e[:, None] + f[None, :])
    assert (np.abs(got - truth) <= bound).all()
    assert (np.abs(got - ref) <= 2 * bound).all()


@pytest.mark.parametrize("sa,sb", [(-1045, 1023), (1000, -1030), (-1000, 990)])
def test_winograd_rowcol_extreme_exponents(mm, orc, sa, sb):
    """Rows of A or columns of B at the ends of the double range (subnormal
    entries, scalings past the normal exponents): every element within the
    elementwise bound of the exact product, as for the badly scaled inputs."""
    n = 96
    a = S.uniform(n, n, S.stream_seed(2, 40))
    b = S.uniform(n, n, S.stream_seed(2, 41))
    a[: n // 2] = np.ldexp(a[: n // 2], sa)
    b[:, : n // 2] = np.ldexp(b[:, : n // 2], sb)
    truth = orc.dot2_product(a, b)
    ref, e, f = orc.winograd_rowcol_scaled(a, b)
    got = host(mm.winograd_rowcol_scaled(dev(a), dev(b)))
    keep = np.isfinite(truth) & (np.abs(truth) > 2.0 ** -900)  # products inside the normal range
    assert keep[: n // 2, : n // 2].all()
    gamma = n // 2
    bound = 8 * gamma * (gamma + 5) * 2.0 ** -53 * np.ldexp(1.0, e[:, None] + f[None, :])
    assert (np.abs(got[keep] - truth[keep]) <= bound[keep]).all()
    assert (np.abs(got[keep] - ref[keep]) <= 2 * bound[keep]).all()


def test_winograd_rowcol_power_of_two_invariance(mm):
    """Prescaling rows of A and columns of B by powers of two leaves the scaled
    operands unchanged, so the GPU result scales by exactly 2^(r_i + c_k)."""
    a = S.uniform(70, 45, 23)
    b = S.uniform(45, 66, 24)
    rng = np.random.default_rng(12)
    r = rng.integers(-60, 61, size=70)
    c = rng.integers(-60, 61, size=66)
    c0 = host(mm.winograd_rowcol_scaled(dev(a), dev(b)))
    c1 = host(mm.winograd_rowcol_scaled(dev(np.ldexp(a, r[:, None])), dev(np.ldexp(b, c[None, :]))))
    assert np.array_equal(c1, np.ldexp(c0, r[:, None] + c[None, :]))


# --------------------------------------------------------------- Strassen

STRASSEN = [("strassen", "strassen_naiv"), ("strassen_winograd", "strassen_winograd")]


@pytest.mark.parametrize("gpu_name,orc_name", STRASSEN)
@pytest.mark.parametrize("shape", [(17, 33, 12), (100, 100, 100), (200, 200, 200), (129, 64, 77)])
def test_strassen_paper_rule(mm, orc, gpu_name, orc_name, shape):
    ai, bi = pair(*shape, "int", 7)
    assert np.array_equal(host(getattr(mm, gpu_name)(dev(ai), dev(bi), cutoff=0)), ai @ bi)
    a, b = pair(*shape, "uni", 8)
    got = host(getattr(mm, gpu_name)(dev(a), dev(b), cutoff=0))
    ref = getattr(orc, orc_name)(a, b)
    assert orc.rel_inf_error(got, ref, a, b) <= TOL


@pytest.mark.parametrize("gpu_name,orc_name", STRASSEN)
@pytest.mark.parametrize("shape,cutoff", [((256, 256, 256), 128), ((256, 256, 256), 64), ((300, 257, 190), 80),
                                          ((64, 512, 96), 130), ((1000, 600, 500), 300)])
def test_strassen_cutoff_depths(mm, orc, gpu_name, orc_name, shape, cutoff):
    n, p, m = shape
    X = max(shape)
    depth = 0
    while -(-X // (1 << depth)) > cutoff:
        depth += 1
    q = 1 << depth
    padded = tuple(-(-d // q) * q for d in shape)
    ai, bi = pair(*shape, "int", 9)
    assert np.array_equal(host(getattr(mm, gpu_name)(dev(ai), dev(bi), cutoff=cutoff)), ai @ bi)
    a, b = pair(*shape, "uni", 10)
    got = host(getattr(mm, gpu_name)(dev(a), dev(b), cutoff=cutoff))
    ref = getattr(orc, orc_name)(a, b, depth=depth, padded=padded)
    assert orc.rel_inf_error(got, ref, a, b) <= TOL


@pytest.mark.parametrize("gpu_name", ["strassen", "strassen_winograd"])
def test_strassen_tuned_default(mm, orc, gpu_name):
    a, b = pair(512, 384, 448, "uni", 11)
    got = host(getattr(mm, gpu_name)(dev(a), dev(b)))
    assert orc.rel_inf_error(got, orc.dot2_product(a, b), a, b) <= TOL


# ---------------------------------------------------------------- emulated

@pytest.mark.parametrize("kind,beta,s", [(0, 7, 8), (0, 7, 3), (1, 5, 6)])
def test_emulated_subnormal_and_overflowing_results(mm, orc, kind, beta, s):
    """The final rounding at the edges of the double range: results below
    2^-1022 land on the subnormal grid (rounded once more, ties to even) and
    results past the largest double are +-inf, bit for bit as the oracle's
    RN(W) followed by ldexp."""
    a, b = pair(130, 70, 90, "log", 40)
    for sa, sb in ((-600, -460), (600, 390)):
        a2, b2 = np.ldexp(a, sa), np.ldexp(b, sb)
        ref = orc.split_product(a2, b2, beta, s)
        if sa < 0:  # subnormal and normal results side by side
            assert ((ref != 0) & (np.abs(ref) < 2.0 ** -1022)).sum() > 100 and (np.abs(ref) >= 2.0 ** -1022).sum() > 100
        else:  # infinite and finite results side by side
            assert np.isinf(ref).sum() > 100 and np.isfinite(ref).sum() > 100
        got = host(mm.emulated(dev(a2), dev(b2), nslices=s, kind=kind))
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("kind,beta,s", [(0, 7, 8), (0, 7, 3), (1, 5, 10)])
def test_emulated_subnormal_operands(mm, orc, kind, beta, s):
    """Rows of A and columns of B whose largest entry is subnormal: the split
    scales them by up to 2^(beta s + 1021) (a left shift of the mantissa far
    past the normal case), bit for bit as the oracle's frexp and RN."""
    a, b = pair(140, 90, 75, "log", 41)
    a[:40] = np.ldexp(a[:40], -1050)              # whole rows subnormal (|a| < 2^-1030)
    a[40:45] = 0.0
    a[40:45, :3] = np.array([5e-324, 1.5e-323, -2e-323])  # rows of a few units in the last place
    a[45:60, ::2] = np.ldexp(a[45:60, ::2], -1070)  # subnormal beside normal in one row
    b = np.ldexp(b, 900)
    b[:, :20] = np.ldexp(b[:, :20], -1950)        # whole columns subnormal
    assert (np.abs(a[:40]) < 2.0 ** -1022).all() and (a[:40] != 0).all()
    assert (np.abs(b[:, :20]) < 2.0 ** -1022).all() and (b[:, :20] != 0).all()
    ref = orc.split_product(a, b, beta, s)
    assert np.isfinite(ref).all() and (ref[:40] != 0).sum() > 1000
    got = host(mm.emulated(dev(a), dev(b), nslices=s, kind=kind))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 3, 7), (128, 32, 64), (129, 33, 65), (200, 333, 150),
                                   (256, 1100, 130)])
@pytest.mark.parametrize("s", [8, 3])
def test_emulated_bit_exact_vs_oracle(mm, orc, shape, s):
    a, b = pair(*shape, "log", 12)
    got = host(mm.emulated(dev(a), dev(b), nslices=s))
    assert np.array_equal(got, orc.split_product(a, b, 7, s))


@pytest.mark.parametrize("kind,beta", [(0, 7), (1, 5)])
@pytest.mark.parametrize("s", [1, 3, 6, 8])
@pytest.mark.parametrize("shape", [(130, 200, 24), (257, 300, 97), (64, 65, 1)])
def test_emulated_narrow_tile_bit_exact(mm, orc, kind, beta, s, shape):
    """The 32-column tile gives the 64-column tile's result bit for bit (both
    are the oracle's definition), ragged widths included."""
    a, b = pair(*shape, "log", 90 + s)
    narrow = host(mm.emulated_tiled(dev(a), dev(b), 32, nslices=s, kind=kind))
    assert np.array_equal(narrow, orc.split_product(a, b, beta, s))
    assert np.array_equal(narrow, host(mm.emulated_tiled(dev(a), dev(b), 64, nslices=s, kind=kind)))


def test_emulated_tile_width_rejected(mm):
    import paper_1106_1347_gb300 as pkg

    a, b = pair(40, 30, 20, "uni", 95)
    with pytest.raises(pkg.MMError):
        mm.emulated_tiled(dev(a), dev(b), 48, nslices=8)
    with pytest.raises(pkg.MMError):  # 10 FP8 slices only fit 32-column tiles
        mm.emulated_tiled(dev(a), dev(b), 64, nslices=10, kind=1)


@pytest.mark.parametrize("s", [1, 2, 4, 5, 6, 7])
def test_emulated_other_slice_counts(mm, orc, s):
    a, b = pair(130, 200, 70, "uni", 13)
    assert np.array_equal(host(mm.emulated(dev(a), dev(b), nslices=s)), orc.split_product(a, b, 7, s))


def test_emulated_integers_exact(mm):
    a, b = pair(150, 520, 90, "int", 14)
    assert np.array_equal(host(mm.emulated(dev(a), dev(b), nslices=2)), a @ b)


def test_emulated_tier_accuracy(mm, orc):
    a, b = pair(192, 700, 160, "log", 15)
    truth = orc.dot2_product(a, b)
    got = host(mm.emulated(dev(a), dev(b), tier=1e-14))
    assert orc.rel_inf_error(got, truth, a, b) <= TOL
    got6 = host(mm.emulated(dev(a), dev(b), tier=1e-6))
    assert orc.rel_inf_error(got6, truth, a, b) <= 1e-6


def test_emulated_multi_chunk_exactness(mm, orc):
    """P spans several exact K-chunks of every diagonal (512 to 4096 K for 8 slices) and a ragged K tail."""
    a, b = pair(130, 9000, 66, "uni", 16)
    assert np.array_equal(host(mm.emulated(dev(a), dev(b), nslices=8)), orc.split_product(a, b, 7, 8))


def test_emulated_positive_worst_case_sums(mm, orc):
    """All-positive operands make every digit sum grow linearly: the chunk drains
    must keep the FP32 accumulation exact."""
    a = np.abs(S.uniform(128, 1500, 171)) + 0.5
    b = np.abs(S.uniform(1500, 64, 172)) + 0.5
    assert np.array_equal(host(mm.emulated(dev(a), dev(b), nslices=8)), orc.split_product(a, b, 7, 8))


def test_emulated_extreme_digit_sums(mm, orc):
    """Every digit of x = -(63 2^49 + 64 (2^42 + 2^35 + ... + 1)) 2^-55 is -64
    except the top one (-63), the largest magnitudes the balanced split allows,
    so every diagonal's per-k product sum sits within 128 of (d + 1) 2^12.  With
    rows of alternating sign and P beyond the longest exact chunk (4096 K for
    diagonal 0), each accumulator runs through whole chunks at the edge of
    FP32's exact integer range, positive and negative."""
    v = 63 * 2 ** 49 + 64 * sum(2 ** (7 * t) for t in range(7))
    x = -float(v) * 2.0 ** -55
    assert x * 2.0 ** 55 == -v  # exactly representable
    n, p, m = 130, 4500, 70
    sign = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)[:, None]
    a = np.full((n, p), x) * sign
    b = np.full((p, m), x)
    got = host(mm.emulated(dev(a), dev(b), nslices=8))
    assert np.array_equal(got, orc.split_product(a, b, 7, 8))


# ------------------------------------------------------- FP8-E4M3 slices

@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 3, 7), (128, 64, 64), (129, 65, 65), (200, 333, 150),
                                   (256, 1100, 130)])
@pytest.mark.parametrize("s", [10, 9, 8, 6, 3, 1])
def test_emulated_fp8_bit_exact_vs_oracle(mm, orc, shape, s):
    """FP8-E4M3 slices hold balanced base-2^5 digits: the same definition with
    beta = 5 (9 and 10 slices run on 32-column tiles and accumulators)."""
    a, b = pair(*shape, "log", 40 + s)
    got = host(mm.emulated(dev(a), dev(b), nslices=s, kind=mm.SLICE_FP8E4M3))
    assert np.array_equal(got, orc.split_product(a, b, 5, s))


@pytest.mark.parametrize("s", [2, 4, 5, 7])
def test_emulated_fp8_other_slice_counts(mm, orc, s):
    """Every E4M3 slice count (the split peels up to 5 digits from the low 25 bits, the rest from the high part)."""
    a, b = pair(130, 200, 70, "log", 60 + s)
    got = host(mm.emulated(dev(a), dev(b), nslices=s, kind=mm.SLICE_FP8E4M3))
    assert np.array_equal(got, orc.split_product(a, b, 5, s))


def test_emulated_fp8_tiers(mm, orc):
    a, b = pair(192, 700, 160, "log", 47)
    truth = orc.dot2_product(a, b)
    got = host(mm.emulated(dev(a), dev(b), tier=1e-6, kind=mm.SLICE_FP8E4M3))
    assert orc.rel_inf_error(got, truth, a, b) <= 1e-6
    assert mm.emulated_slices(tier=1e-6, kind=mm.SLICE_FP8E4M3) == 6
    # 1e-12 needs ceil((log2(1e12) + 9) / 5) = 10 slices, the most the FP8 kernel holds
    assert mm.emulated_slices(tier=1e-12, kind=mm.SLICE_FP8E4M3) == 10
    got = host(mm.emulated(dev(a), dev(b), tier=1e-12, kind=mm.SLICE_FP8E4M3))
    assert orc.rel_inf_error(got, truth, a, b) <= 1e-12
    with pytest.raises(mm.MMError):  # 1e-14 needs 12 FP8 slices: more than the 10 accumulators
        mm.emulated(dev(a), dev(b), tier=1e-14, kind=mm.SLICE_FP8E4M3)


@pytest.mark.parametrize("s", [8, 10])
def test_emulated_fp8_extreme_digit_sums(mm, orc, s):
    """Every base-2^5 digit at the split's extreme (-15 on top, -16 below), rows
    of alternating sign and P past the exact length of the last diagonal (8192 K
    for 8 slices, 6553 K for 10): the accumulators run whole chunks at FP32's
    exact-integer edge."""
    v = 15 * 2 ** (5 * (s - 1)) + 16 * sum(2 ** (5 * t) for t in range(s - 1))
    x = -float(v) * 2.0 ** -(5 * s - 1)
    assert x * 2.0 ** (5 * s - 1) == -v
    n, p, m = 130, 9000, 70
    sign = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)[:, None]
    a = np.full((n, p), x) * sign
    b = np.full((p, m), x)
    got = host(mm.emulated(dev(a), dev(b), nslices=s, kind=mm.SLICE_FP8E4M3))
    assert np.array_equal(got, orc.split_product(a, b, 5, s))


def test_emulated_fp8_group_matches_single_calls(mm, orc):
    shapes = [(37, 65, 129), (128, 64, 64), (300, 40, 17), (5, 1000, 3)]
    hostpairs = [(S.loguniform(n, p, S.stream_seed(6, 50 + i)), S.loguniform(p, m, S.stream_seed(6, 60 + i)))
                 for i, (n, p, m) in enumerate(shapes)]
    pairs = [(dev(a), dev(b)) for a, b in hostpairs]
    for s in (5, 10):
        outs = mm.emulated_group(pairs, nslices=s, kind=mm.SLICE_FP8E4M3)
        for (a, b), c in zip(hostpairs, outs):
            assert np.array_equal(host(c), orc.split_product(a, b, 5, s))


# ------------------------------------------------- host-operand pipeline

@pytest.mark.parametrize("shape", [(2500, 300, 190), (129, 65, 65), (1, 1, 1), (700, 1000, 64), (4100, 70, 2100),
                                   (4500, 60, 4097)])
@pytest.mark.parametrize("kind", [0, 1])
def test_emulated_host_matches_device_call(mm, shape, kind):
    """Blocks of C (row blocks, and from N = 4096, M = 2048 on two column blocks)
    copied up, multiplied and copied back on overlapping streams give the
    device call's result bit for bit (ragged last blocks included)."""
    a, b = pair(*shape, "log", 70 + kind)
    s = 8 if kind == 0 else 6
    ref = host(mm.emulated(dev(a), dev(b), nslices=s, kind=kind))
    assert np.array_equal(mm.emulated_host(a, b, nslices=s, kind=kind), ref)


def test_emulated_host_pinned_strided_views(mm, orc):
    import torch

    big_a = torch.from_numpy(S.loguniform(1100, 260, 73)).pin_memory()
    big_b = torch.from_numpy(S.loguniform(250, 90, 74)).pin_memory()
    big_c = torch.zeros((1200, 100), dtype=torch.float64).pin_memory()
    a, b, c = big_a[7:1037, 3:243], big_b[2:242, 5:85], big_c[11:1041, 7:87]
    mm.emulated_host(a, b, out=c, nslices=8)
    assert np.array_equal(c.numpy(), orc.split_product(a.numpy(), b.numpy(), 7, 8))
    mask = np.ones(big_c.shape, dtype=bool)
    mask[11:1041, 7:87] = False
    assert np.all(big_c.numpy()[mask] == 0.0)


def test_emulated_host_wide_strided_views(mm):
    """Two column blocks of B and C taken from views with leading dimensions
    larger than their widths, against the device call on the same values."""
    import torch

    big_a = torch.from_numpy(S.loguniform(4200, 90, 75)).pin_memory()
    big_b = torch.from_numpy(S.loguniform(80, 4300, 76)).pin_memory()
    big_c = torch.zeros((4220, 4310), dtype=torch.float64).pin_memory()
    a, b, c = big_a[5:4155, 9:77], big_b[3:71, 17:4250], big_c[13:4163, 41:4274]
    mm.emulated_host(a, b, out=c, nslices=8)
    ref = host(mm.emulated(dev(np.ascontiguousarray(a.numpy())), dev(np.ascontiguousarray(b.numpy())), nslices=8))
    assert np.array_equal(c.numpy(), ref)
    mask = np.ones(big_c.shape, dtype=bool)
    mask[13:4163, 41:4274] = False
    assert np.all(big_c.numpy()[mask] == 0.0)


# ---------------------------------------------------------- grouped launch

def test_emulated_group_matches_single_calls(mm, orc):
    import torch

    rng = np.random.default_rng(5)
    shapes = [(1, 1, 1), (37, 65, 129), (128, 64, 64), (300, 40, 17), (5, 1000, 3), (200, 333, 150), (64, 0, 9),
              (0, 5, 5), (129, 513, 250)]
    pairs, hostpairs = [], []
    for i, (n, p, m) in enumerate(shapes):
        a = S.loguniform(n, p, S.stream_seed(6, 2 * i)) if n * p else np.zeros((n, p))
        b = S.loguniform(p, m, S.stream_seed(6, 2 * i + 1)) if p * m else np.zeros((p, m))
        hostpairs.append((a, b))
        pairs.append((dev(a), dev(b)))
    for s in (8, 3):
        outs = mm.emulated_group(pairs, nslices=s)
        for (a, b), (ta, tb), c in zip(hostpairs, pairs, outs):
            single = host(mm.emulated(ta, tb, nslices=s))
            assert np.array_equal(host(c), single)
            if a.size and b.size and a.shape[0] <= 200:
                assert np.array_equal(single, orc.split_product(a, b, 7, s))


def test_emulated_group_rejects_overlapping_outputs(mm):
    import torch
    from paper_1106_1347_gb300._native import Problem

    a = torch.ones((8, 8), dtype=torch.float64, device="cuda")
    c = torch.zeros((16, 8), dtype=torch.float64, device="cuda")
    arr = (Problem * 2)(Problem(8, 8, 8, a.data_ptr(), 8, a.data_ptr(), 8, c.data_ptr(), 8),
                        Problem(8, 8, 8, a.data_ptr(), 8, a.data_ptr(), 8, c[4:].data_ptr(), 8))
    assert mm.lib().mm_emulated_group(arr, 2, 0, 3, 1e-6, None, 0, None) == -1


# ------------------------------------------------------------ edge cases

@pytest.mark.parametrize("name", ["naive", "naive_unrolled", "kahan", "winograd", "winograd_scaled",
                                  "winograd_rowcol_scaled", "strassen", "strassen_winograd", "emulated",
                                  "strassen_emulated"])
def test_degenerate_shapes(mm, name):
    import torch

    fn = getattr(mm, name)
    a = torch.zeros((4, 0), dtype=torch.float64, device="cuda")
    b = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    out = torch.full((4, 3), 7.0, dtype=torch.float64, device="cuda")
    fn(a, b, out=out)
    assert torch.count_nonzero(out).item() == 0
    a = torch.zeros((0, 5), dtype=torch.float64, device="cuda")
    b = torch.ones((5, 3), dtype=torch.float64, device="cuda")
    assert fn(a, b).shape == (0, 3)


@pytest.mark.parametrize("name", ["naive", "kahan", "winograd", "winograd_rowcol_scaled", "strassen", "emulated"])
def test_strided_views(mm, orc, name):
    """Leading dimensions larger than the column count (sub-matrix views)."""
    big_a = S.integers(90, 120, 181)
    big_b = S.integers(110, 100, 182)
    a, b = big_a[5:75, 7:100], big_b[3:96, 11:80]
    ta, tb = dev(big_a)[5:75, 7:100], dev(big_b)[3:96, 11:80]
    big_c = dev(np.zeros((80, 90)))
    out = big_c[4:74, 9:78]
    kw = {"nslices": 1} if name == "emulated" else {}
    getattr(mm, name)(ta, tb, out=out, **kw)
    got = host(big_c)
    assert np.array_equal(got[4:74, 9:78], a @ b)
    mask = np.ones_like(got, dtype=bool)
    mask[4:74, 9:78] = False
    assert np.all(got[mask] == 0.0)


def test_argument_errors(mm):
    import torch

    a = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(mm.MMError):
        mm.naive(a, a, out=a)  # C overlaps A
    with pytest.raises(ValueError):
        mm.naive(a, torch.zeros((5, 4), dtype=torch.float64, device="cuda"))


def test_bounded_wait_gives_up_and_context_survives(mm, orc):
    """A device wait on a barrier nothing completes gives up after its poll
    limit, raises the status word and returns; the context keeps working."""
    import ctypes

    import torch

    lib = mm.lib()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = ctypes.c_int32(0)
    lib.mm_device_status(st, ctypes.byref(code))  # clear anything earlier
    assert lib.mm_selftest_wait_timeout(st) == 0
    assert lib.mm_device_status(st, ctypes.byref(code)) == -5  # MM_ERR_TIMEOUT
    assert code.value == 8
    a, b = pair(70, 90, 50, "int", 60)
    assert np.array_equal(host(mm.naive(dev(a), dev(b))), a @ b)
    assert lib.mm_device_status(st, ctypes.byref(code)) == 0 and code.value == 0


def test_no_timeouts_raised(mm):
    assert mm.device_status() == 0


# -------------------------------------------------------------- autotuner

def test_tune_strassen_records_and_persists(mm, orc, tmp_path):
    import ctypes

    L = mm.lib()
    L.mm_tune_clear()
    a, b = pair(600, 520, 560, "uni", 21)
    depth, ms = mm.tune_strassen(dev(a), dev(b), variant=0)
    assert 0 <= depth <= 5 and ms > 0  # blocks of at least 16: 520 >> 5 = 16
    q = 1 << depth
    want = 0 if depth <= 1 else L.mm_strassen_workspace_bytes(600, 520, 560, max(1, -(-600 // q)))
    assert L.mm_strassen_workspace_bytes(600, 520, 560, -1) == want
    got = host(mm.strassen(dev(a), dev(b), cutoff=-1))
    assert orc.rel_inf_error(got, orc.dot2_product(a, b), a, b) <= TOL
    path = str(tmp_path / "tune.txt").encode()
    assert L.mm_tune_save(path) == 0
    L.mm_tune_clear()
    assert L.mm_tune_load(path) == 1
    assert L.mm_strassen_workspace_bytes(600, 520, 560, -1) == want
    L.mm_tune_clear()
