"""Pins for the CPU oracle (no GPU): each check ties the oracle to something other
than itself -- hand-derived values from the paper's definitions
(tests/golden/paper_pins.json), exact integer products, exact rational
arithmetic (fractions.Fraction), closed forms and published error bounds.
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import synthetic as S

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_pins.json")))
U = 2.0 ** -53

GEMMS = ["naiv_standard", "naiv_on_array", "naiv_unrolled_2", "naiv_unrolled_3", "naiv_unrolled_4", "naiv_kahan",
         "winograd_original", "winograd_scaled", "winograd_rowcol_scaled", "strassen_naiv", "strassen_winograd",
         "dot2_product"]


def run(orc, name, a, b, **kw):
    out = getattr(orc, name)(a, b, **kw)
    return out[0] if isinstance(out, tuple) else out


def exact_product(a, b):
    """Exact rational product of two small float matrices."""
    n, p = a.shape
    m = b.shape[1]
    fa = [[Fraction(float(x)) for x in row] for row in a]
    fb = [[Fraction(float(x)) for x in row] for row in b]
    return [[sum((fa[i][k] * fb[k][j] for k in range(p)), Fraction(0)) for j in range(m)] for i in range(n)]


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("name", GEMMS)
def test_all_sign_matrices_2x2_and_3x3(orc, name):
    """Every method equals the exact product on all {-1,0,1} 2x2 pairs and on sampled 3x3 pairs."""
    vals = (-1.0, 0.0, 1.0)
    mats2 = [np.array(v, dtype=np.float64).reshape(2, 2) for v in itertools.product(vals, repeat=4)]
    for a in mats2[::3]:
        for b in mats2:
            assert np.array_equal(run(orc, name, a, b), a @ b)
    rng = np.random.default_rng(7)
    for _ in range(60):
        a = rng.integers(-1, 2, size=(3, 3)).astype(np.float64)
        b = rng.integers(-1, 2, size=(3, 3)).astype(np.float64)
        assert np.array_equal(run(orc, name, a, b), a @ b)


@pytest.mark.parametrize("name", GEMMS)
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 5, 2), (7, 1, 4), (6, 9, 5), (17, 33, 12), (40, 31, 23)])
def test_integer_inputs_exact(orc, name, shape):
    """Integer entries in [-8, 8]: every intermediate is an integer below 2^53, so
    each method must reproduce the exact product (odd and even P included)."""
    n, p, m = shape
    a = S.integers(n, p, S.stream_seed(0, 100 + n))
    b = S.integers(p, m, S.stream_seed(0, 200 + m))
    ref = (a.astype(np.int64) @ b.astype(np.int64)).astype(np.float64)
    assert np.array_equal(run(orc, name, a, b), ref)


@pytest.mark.parametrize("name", ["strassen_naiv", "strassen_winograd"])
@pytest.mark.parametrize("depth,padded", [(1, (18, 34, 12)), (2, (20, 36, 16)), (3, (24, 40, 24)), (2, (40, 40, 40))])
def test_strassen_explicit_depths_exact(orc, name, depth, padded):
    a = S.integers(17, 33, S.stream_seed(0, 5))
    b = S.integers(33, 12, S.stream_seed(0, 6))
    got = getattr(orc, name)(a, b, depth=depth, padded=padded)
    assert np.array_equal(got, a @ b)


def test_closed_forms(orc):
    n = 9
    b = S.uniform(n, 7, S.stream_seed(0, 9))
    eye = np.eye(n)
    ones_a = np.ones((5, n))
    ones_b = np.ones((n, 6))
    bi = S.integers(n, 7, S.stream_seed(0, 10))
    for name in GEMMS:
        # I B = B: exact for the inner-product methods (every other term is an exact zero);
        # Winograd and Strassen round their operand sums, so they are held to it on integers.
        exact_on_reals = name in ("naiv_standard", "naiv_kahan", "dot2_product")
        bb = b if exact_on_reals else bi
        assert np.array_equal(run(orc, name, eye, bb), bb), name
        assert np.array_equal(run(orc, name, ones_a, ones_b), np.full((5, 6), float(n))), name
    u = S.integers(6, 1, 11)
    v = S.integers(1, 8, 12)
    for name in GEMMS:
        assert np.array_equal(run(orc, name, u, v), u * v), name         # rank one, P = 1


def test_empty_and_zero_inner(orc):
    a = np.zeros((3, 0))
    b = np.zeros((0, 4))
    for name in GEMMS:
        assert np.array_equal(run(orc, name, a, b), np.zeros((3, 4))), name


# -------------------------------------------------------- hand-derived goldens

def test_strassen_rule_golden(orc):
    for case in GOLD["strassen_rule"]["cases"]:
        assert orc.strassen_paper_rule(case["X"], 1, 1) == (case["k"], case["Y"]), case


def test_brent_lambda_tie_golden(orc):
    g = GOLD["brent_lambda_tie"]
    assert orc.brent_lambda(g["norm_a"], g["norm_b"]) == g["lambda"]
    a = S.uniform(6, 6, 3)
    _, lam = orc.winograd_scaled(a, 8.0 * a)
    assert lam == g["lambda"]


def test_kahan_discriminator_golden(orc):
    g = GOLD["kahan_discriminator"]
    a = np.array([g["row"]])
    b = np.ones((3, 1))
    assert orc.naiv_kahan(a, b)[0, 0] == g["kahan"]
    assert orc.naiv_standard(a, b)[0, 0] == g["naive"]


def test_norm_inf_order_golden(orc):
    g = GOLD["norm_inf_order"]
    assert orc.norm_inf(np.array(g["rows"])) == g["value"]


def test_split_example_golden(orc):
    g = GOLD["split_example"]
    a, b = np.array(g["A"]), np.array(g["B"])
    ea, da = orc.split_digits(a, False, g["beta"], g["s"])
    fb, db = orc.split_digits(b, True, g["beta"], g["s"])
    assert ea[0] == g["e"] and fb[0] == g["f"]
    assert da[0, 0, 0] == g["V"] and db[0, 0, 0] == g["U"]
    assert orc.split_product(a, b, g["beta"], g["s"])[0, 0] == g["C"]


# ------------------------------------------------------------ exact arithmetic

def test_norm_inf_against_exact(orc):
    a = S.uniform(13, 57, 21)
    exact = max(sum((Fraction(abs(float(x))) for x in row), Fraction(0)) for row in a)
    bound = (a.shape[1] - 1) * U * float(exact)  # recursive summation of non-negatives
    assert abs(orc.norm_inf(a) - float(exact)) <= bound
    ai = S.integers(9, 14, 22)
    assert orc.norm_inf(ai) == float(np.abs(ai.astype(np.int64)).sum(axis=1).max())
    assert orc.norm_inf(np.zeros((0, 3))) == 0.0


def test_dot2_is_nearly_correctly_rounded(orc):
    """Ogita-Rump-Oishi Dot2 bound: |res - x.y| <= u|x.y| + gamma_n^2 sum|x_i y_i|."""
    a = S.uniform(5, 40, 31) * 1e3
    b = S.uniform(40, 4, 32)
    b[::2] *= -1e-3  # mixed magnitudes and signs
    got = orc.dot2_product(a, b)
    ex = exact_product(a, b)
    n = a.shape[1]
    g2 = (n * U / (1 - n * U)) ** 2
    for i in range(a.shape[0]):
        for j in range(b.shape[1]):
            absdot = float(sum(abs(Fraction(float(a[i, k])) * Fraction(float(b[k, j]))) for k in range(n)))
            err = abs(Fraction(float(got[i, j])) - ex[i][j])
            assert err <= U * abs(ex[i][j]) + 2 * g2 * absdot


def test_kahan_error_bound_and_gain(orc):
    """Kahan's compensated sum: |S_hat - S| <= (2u + O(n u^2)) sum|x| (Higham, Accuracy and
    Stability of Numerical Algorithms, Thm 4.8).  On 1 followed by many terms below
    half an ulp of 1, the naive sum never moves while Kahan's recovers them."""
    n = 400
    x = S.uniform(1, n, 41)
    x = x * np.ldexp(1.0, (np.arange(n) % 40) - 20)  # spread magnitudes
    x = np.concatenate([x, -x[:, ::-1] * (1 + 2.0 ** -30)], axis=1)
    ones = np.ones((x.shape[1], 1))
    exact = sum((Fraction(float(v)) for v in x.ravel()), Fraction(0))
    absum = float(sum(abs(Fraction(float(v))) for v in x.ravel()))
    k = orc.naiv_kahan(x, ones)[0, 0]
    nn = x.shape[1]
    assert abs(Fraction(float(k)) - exact) <= (2 * U + 2 * nn * U * U) * absum

    tiny = np.concatenate([[1.0], np.full(1000, 2.0 ** -60)])[None, :]
    ones = np.ones((tiny.shape[1], 1))
    exact = Fraction(1) + 1000 * Fraction(2) ** -60
    assert orc.naiv_standard(tiny, ones)[0, 0] == 1.0
    k = orc.naiv_kahan(tiny, ones)[0, 0]
    assert abs(Fraction(float(k)) - exact) <= U * exact  # within half an ulp of 1


@pytest.mark.parametrize("name", ["naiv_standard", "naiv_unrolled_2", "naiv_unrolled_3", "naiv_unrolled_4",
                                  "winograd_original", "winograd_scaled", "winograd_rowcol_scaled",
                                  "strassen_naiv", "strassen_winograd"])
def test_real_inputs_near_exact(orc, name):
    """Random reals: normwise error against the exact product stays far below 1e-14."""
    a = S.uniform(12, 29, 51)
    b = S.uniform(29, 10, 52)
    ex = np.array([[float(v) for v in row] for row in exact_product(a, b)])
    got = run(orc, name, a, b)
    assert orc.rel_inf_error(got, ex, a, b) < 1e-15


def test_brent_bound_holds(orc):
    """Brent's bounds for Winograd (section 'WinogradScaled'), infinity norm, 2^-tau = 2^-52."""
    n = 48
    a = S.uniform(n, n, 61) * 100.0
    b = S.uniform(n, n, 62) * 0.01
    truth = orc.dot2_product(a, b)
    na, nb = orc.norm_inf(a), orc.norm_inf(b)
    e_orig = orc.norm_inf(orc.winograd_original(a, b) - truth)
    e_scaled = orc.norm_inf(orc.winograd_scaled(a, b)[0] - truth)
    c = (n * n + 12 * n - 8)
    assert e_orig <= 2.0 ** -52 * c / 4 * (na + nb) ** 2
    assert e_scaled <= 2.0 ** -52 * 9 / 8 * c * na * nb


def test_brent_lambda_is_smallest_valid(orc):
    rng = np.random.default_rng(3)
    for _ in range(300):
        na = float(np.ldexp(rng.uniform(0.5, 1.0), int(rng.integers(-60, 60))))
        nb = float(np.ldexp(rng.uniform(0.5, 1.0), int(rng.integers(-60, 60))))
        lam = orc.brent_lambda(na, nb)

        def ok(l):
            r = Fraction(na) * Fraction(4) ** l / Fraction(nb)
            return Fraction(1, 2) <= r <= 2

        assert ok(lam) and not ok(lam - 1)
    assert orc.brent_lambda(0.0, 3.0) == 0


def test_scaled_winograd_scaling_is_exact(orc):
    """2^lambda A times 2^-lambda B: with powers of two and no overflow, y and z
    scale by exactly 4^lambda and 4^-lambda (section 'WinogradScaled')."""
    a = S.uniform(8, 11, 71)
    b = S.uniform(11, 6, 72) * 64.0
    lam = orc.brent_lambda(orc.norm_inf(a), orc.norm_inf(b))
    assert lam != 0
    y, z = orc.winograd_terms(a, b)
    ys, zs = orc.winograd_terms(orc.multiply_with_scalar(2.0 ** lam, a), orc.multiply_with_scalar(2.0 ** -lam, b))
    assert np.array_equal(ys, y * 4.0 ** lam) and np.array_equal(zs, z * 4.0 ** -lam)


def test_winograd_identity_on_integers(orc):
    """sum_j (a+b)(a'+b') = (AB)_ik + y_i + z_k exactly (section 'WinogradOriginal')."""
    a = S.integers(7, 10, 81)
    b = S.integers(10, 5, 82)
    y, z = orc.winograd_terms(a, b)
    ai, bi = a.astype(np.int64), b.astype(np.int64)
    paired = np.zeros((7, 5), dtype=np.int64)
    for j in range(5):
        paired += np.outer(ai[:, 2 * j], np.ones(5, np.int64)) * 0 + \
            (ai[:, 2 * j][:, None] + bi[2 * j + 1][None, :]) * (ai[:, 2 * j + 1][:, None] + bi[2 * j][None, :])
    assert np.array_equal(paired, ai @ bi + y.astype(np.int64)[:, None] + z.astype(np.int64)[None, :])


# ---------------------------------------------------------- split decomposition

@pytest.mark.parametrize("beta,s", [(7, 8), (7, 3), (8, 7), (5, 11)])
def test_split_digits_reconstruct(orc, beta, s):
    """Balanced digits reconstruct RN(x 2^(beta s - 1 - e)) exactly, lie in range,
    and the scaled value is within half a unit of x."""
    x = S.loguniform(6, 9, 91)
    x[2] = 0.0
    exps, dig = orc.split_digits(x, False, beta, s)
    half = 1 << (beta - 1)
    assert np.all(np.abs(dig[1:]) <= half) and np.all(dig[1:] < half)
    assert np.all(np.abs(dig[0]) <= half)
    for i in range(x.shape[0]):
        mx = np.abs(x[i]).max()
        if mx == 0:
            assert np.all(dig[:, i] == 0)
            continue
        assert 2.0 ** (exps[i] - 1) <= mx < 2.0 ** exps[i]
        for j in range(x.shape[1]):
            V = sum(int(dig[t, i, j]) << (beta * (s - 1 - t)) for t in range(s))
            err = abs(Fraction(V) * Fraction(2) ** (int(exps[i]) - beta * s + 1) - Fraction(float(x[i, j])))
            assert err <= Fraction(2) ** (int(exps[i]) - beta * s)


def test_split_product_exact_on_integers(orc):
    a = S.integers(21, 37, 101)
    b = S.integers(37, 15, 102)
    for s in (1, 2, 8):
        assert np.array_equal(orc.split_product(a, b, 7, s), a @ b)


def test_split_product_single_rounding(orc):
    """With beta*s large enough to hold every input bit and no dropped pair able to
    matter, the result is the exact product rounded once."""
    a = S.uniform(4, 6, 111)
    b = S.uniform(6, 3, 112)
    got = orc.split_product(a, b, 9, 6)  # 53 significant bits fit in beta*s-1 = 53
    ex = exact_product(a, b)
    for i in range(4):
        for j in range(3):
            err = abs(Fraction(float(got[i, j])) - ex[i][j])
            # dropped pairs sigma+tau >= s carry weight <= 6 * 2^-54 relative to 2^(e+f)
            assert err <= U * abs(ex[i][j]) + Fraction(2) ** -50


@pytest.mark.parametrize("beta,s,tol", [(7, 8, 1e-15), (8, 7, 1e-15), (7, 7, 1e-13), (7, 3, 1e-5)])
def test_split_product_error_tiers(orc, beta, s, tol):
    a = S.loguniform(24, 40, 121)
    b = S.loguniform(40, 20, 122)
    truth = orc.dot2_product(a, b)
    assert orc.rel_inf_error(orc.split_product(a, b, beta, s), truth, a, b) <= tol


# ------------------------------------------- per-row/column scaled Winograd

def test_rowcol_exponents_follow_the_definition(orc):
    """e_i: 2^(e_i - 1) <= max_j |A_ij| < 2^e_i, 0 for a zero row; likewise f_k
    over the columns of B."""
    a = S.badly_scaled(24, S.stream_seed(2, 10), S.stream_seed(2, 11))[0][:, :17].copy()
    b = S.badly_scaled(24, S.stream_seed(2, 12), S.stream_seed(2, 13))[1][:17, :].copy()
    a[5, :] = 0.0
    b[:, 7] = 0.0
    _, e, f = orc.winograd_rowcol_scaled(a, b)
    for mx, ex in list(zip(np.abs(a).max(axis=1), e)) + list(zip(np.abs(b).max(axis=0), f)):
        if mx == 0.0:
            assert ex == 0
        else:
            assert np.ldexp(1.0, int(ex) - 1) <= mx < np.ldexp(1.0, int(ex))


def test_rowcol_power_of_two_invariance(orc):
    """Scaling row i of A by 2^r_i and column k of B by 2^c_k (exact) leaves A'
    and B' unchanged, so the result is the old one times 2^(r_i + c_k), bit for
    bit; a scale-back with a wrong exponent fails this."""
    a = S.uniform(13, 21, 91)
    b = S.uniform(21, 9, 92)
    rng = np.random.default_rng(11)
    r = rng.integers(-40, 41, size=13)
    c = rng.integers(-40, 41, size=9)
    c0 = orc.winograd_rowcol_scaled(a, b)[0]
    c1 = orc.winograd_rowcol_scaled(np.ldexp(a, r[:, None]), np.ldexp(b, c[None, :]))[0]
    assert np.array_equal(c1, np.ldexp(c0, r[:, None] + c[None, :]))


def test_rowcol_reduces_to_original_when_balanced(orc):
    """Every row maximum of A and column maximum of B in [1/2, 1): all exponents
    are 0 and the method is WinogradOriginal itself."""
    a = S.uniform(10, 15, 93) * 0.7
    b = S.uniform(15, 8, 94) * 0.7
    a[:, 3] = 0.75
    b[4, :] = -0.75
    c, e, f = orc.winograd_rowcol_scaled(a, b)
    assert not e.any() and not f.any()
    assert np.array_equal(c, orc.winograd_original(a, b))


def test_rowcol_elementwise_bound_on_badly_scaled(orc):
    """After scaling, |A'|, |B'| < 1: each paired factor is below 2 in magnitude,
    each product below 4, the paired sum below 4 gamma and y', z' below gamma,
    so a standard rounding-error count gives
    |C' - T'|_ik <= 8 gamma (gamma + 5) u (gamma = P/2, u = 2^-53), and the
    exact scale-back makes it |C - T|_ik <= 8 gamma (gamma + 5) u 2^(e_i + f_k)
    -- an elementwise form of the bound of section 'WinogradScaled'.  Plain
    Winograd breaks it on rows times 10^u and columns times 10^v."""
    n = 64
    a, b = S.badly_scaled(n, S.stream_seed(2, 14), S.stream_seed(2, 15))
    truth = orc.dot2_product(a, b)
    c, e, f = orc.winograd_rowcol_scaled(a, b)
    gamma = n // 2
    bound = 8 * gamma * (gamma + 5) * U * np.ldexp(1.0, e[:, None] + f[None, :])
    assert (np.abs(c - truth) <= bound).all()
    assert not (np.abs(orc.winograd_original(a, b) - truth) <= bound).all()


# ------------------------------------------------ NaivOnArray, loop unrolling

def test_loop_unrolling_discriminator_golden(orc):
    """Hand-derived sums where the grouping of the unrolled forms changes the
    rounded result (section 'Loop unrolling')."""
    g = GOLD["loop_unrolling_discriminator"]
    for case in g["cases"]:
        a = np.array([case["row"]])
        b = np.ones((a.shape[1], 1))
        assert orc.naiv_standard(a, b)[0, 0] == case["naive"]
        assert orc.naiv_on_array(a, b)[0, 0] == case["on_array"]
        for u in (2, 3, 4):
            assert orc.naiv_unrolled(a, b, u)[0, 0] == case[f"u{u}"], u


def test_unroll_one_and_on_array_are_naiv_standard(orc):
    """u = 1 is the plain sum, and accumulating in C rounds exactly as an auxiliary does."""
    a = S.loguniform(9, 37, 95)
    b = S.loguniform(37, 7, 96)
    ref = orc.naiv_standard(a, b)
    assert np.array_equal(orc.naiv_unrolled(a, b, 1), ref)
    assert np.array_equal(orc.naiv_on_array(a, b), ref)


@pytest.mark.parametrize("u", [2, 3, 4])
def test_unrolled_grouping_by_exact_rationals(orc, u):
    """Each unrolled result equals the same grouping evaluated with exact
    rational arithmetic and a rounding to double after every operation, for
    every P mod u (the correction terms included)."""
    rng = np.random.default_rng(40 + u)
    for p in range(1, 3 * u + 2):
        a = rng.uniform(-1, 1, size=(1, p)) * np.ldexp(1.0, rng.integers(-30, 30, size=(1, p)))
        b = rng.uniform(-1, 1, size=(p, 1))

        def rn(fr):
            return Fraction(float(fr))  # correctly rounded to double

        prods = [rn(Fraction(float(a[0, k])) * Fraction(float(b[k, 0]))) for k in range(p)]
        aux = Fraction(0)
        full = (p // u) * u
        for k in range(0, full, u):
            grp = prods[k]
            for t in range(1, u):
                grp = rn(grp + prods[k + t])
            aux = rn(aux + grp)
        for k in range(full, p):
            aux = rn(aux + prods[k])
        assert orc.naiv_unrolled(a, b, u)[0, 0] == float(aux)


# ------------------------------------- Strassen levels over the split product

@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("depth", [1, 2, 3])
@pytest.mark.parametrize("shape", [(17, 33, 12), (40, 31, 23), (8, 8, 8), (5, 3, 9)])
def test_strassen_emulated_exact_on_integers(orc, variant, depth, shape):
    """Integer entries in [-8, 8]: after at most 3 levels every operand sum is an
    integer below 2^7 * 8, which 3 BF16-width digits (beta = 7) hold exactly, and
    every H and C combination is an exact integer sum -- so the recursion must
    reproduce the exact product.  A dropped H, a wrong sign or a crossed
    quadrant changes some entry."""
    n, p, m = shape
    a = S.integers(n, p, S.stream_seed(0, 300 + n + depth))
    b = S.integers(p, m, S.stream_seed(0, 400 + m + depth))
    ref = (a.astype(np.int64) @ b.astype(np.int64)).astype(np.float64)
    assert np.array_equal(orc.strassen_emulated(a, b, variant, depth, 7, 3), ref)


@pytest.mark.parametrize("variant", [0, 1])
def test_strassen_emulated_depth_zero_is_the_split_product(orc, variant):
    a = S.loguniform(23, 41, 131)
    b = S.loguniform(41, 19, 132)
    for beta, s in ((7, 8), (5, 6)):
        assert np.array_equal(orc.strassen_emulated(a, b, variant, 0, beta, s), orc.split_product(a, b, beta, s))


@pytest.mark.parametrize("variant", [0, 1])
def test_strassen_emulated_one_level_structure(orc, variant):
    """On a 2x2 block matrix whose blocks are single entries, one level with a base
    that is exact for these integers gives the 2x2 product: each of the 8 sign
    patterns of a single nonzero in A against all-ones B isolates one quadrant term."""
    ones = np.ones((2, 2))
    for i in range(2):
        for k in range(2):
            a = np.zeros((2, 2))
            a[i, k] = 3.0
            got = orc.strassen_emulated(a, ones * 5.0, variant, 1, 7, 2)
            assert np.array_equal(got, a @ (ones * 5.0))
            got = orc.strassen_emulated(ones * 5.0, a, variant, 1, 7, 2)
            assert np.array_equal(got, (ones * 5.0) @ a)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("depth", [1, 2])
def test_strassen_emulated_error_tier(orc, variant, depth):
    """Reals: the FP64 operand sums and H combinations add a few ulps of
    ||A|| ||B|| per level, far inside the 1e-14 tier 8 BF16 slices serve."""
    a = S.uniform(48, 40, 141)
    b = S.uniform(40, 36, 142)
    truth = orc.dot2_product(a, b)
    err = orc.rel_inf_error(orc.strassen_emulated(a, b, variant, depth, 7, 8), truth, a, b)
    assert err <= 1e-14
    # and the recursion is not the base product under another name
    assert not np.array_equal(orc.strassen_emulated(a, b, variant, depth, 7, 8), orc.split_product(a, b, 7, 8))


@pytest.mark.parametrize("variant", [0, 1])
def test_sampled_one_level_helper_matches_the_oracle(orc, variant):
    """The sampled-entry helper the full-size GPU parity test uses agrees bit for
    bit with the oracle's full recursion (one level, log-uniform inputs)."""
    from strassen_sampled import one_level_sampled

    a = S.loguniform(36, 44, 151)
    b = S.loguniform(44, 30, 152)
    full = orc.strassen_emulated(a, b, variant, 1, 7, 8)
    rows, cols = [0, 5, 17, 18, 35], [0, 3, 14, 15, 29]
    assert np.array_equal(one_level_sampled(orc, a, b, variant, rows, cols, 7, 8), full[np.ix_(rows, cols)])
