"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times, on sampled outputs the oracle computes one by one.

The emulated product's definition is elementwise once the row exponent e_i
and the column exponent f_j are fixed, and e_i depends on row i of A only and
f_j on column j of B only: the oracle run on the sampled rows of A and the
sampled columns of B gives exactly those entries of the full product.  The
FP64 methods are checked on sampled rows (each row of C depends on one row of
A and all of B)."""
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
    import paper_1106_1347_gb300 as m

    return m


def _dev(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


ROWS = np.array([0, 1, 127, 128, 4095, 5000, 8190, 8191])
COLS = np.concatenate([np.arange(0, 64), np.arange(4032, 4160), np.arange(8128, 8192)])


@pytest.mark.parametrize("kind,s", [(0, 8), (1, 6), (1, 10)])
def test_emulated_8192_cubed_sampled_bit_exact(mm, orc, kind, s):
    """8192^3, log-uniform entries (the bench workload): sampled entries equal
    the oracle's definition bit for bit (BF16 8 slices; FP8-E4M3 6 and 10)."""
    a = S.loguniform(8192, 8192, S.stream_seed(3, 0))
    b = S.loguniform(8192, 8192, S.stream_seed(3, 1))
    c = mm.emulated(_dev(a), _dev(b), nslices=s, kind=kind)
    got = c[ROWS][:, COLS].cpu().numpy()
    beta = 5 if kind == 1 else 7
    assert np.array_equal(got, orc.split_product(a[ROWS], b[:, COLS], beta, s))


def test_emulated_4096_16384_4096_sampled_bit_exact(mm, orc):
    a = S.loguniform(4096, 16384, S.stream_seed(3, 2))
    b = S.loguniform(16384, 4096, S.stream_seed(3, 3))
    c = mm.emulated(_dev(a), _dev(b), nslices=8)
    rows, cols = np.array([0, 2047, 2048, 4095]), np.arange(1000, 1160)
    got = c[rows][:, cols].cpu().numpy()
    assert np.array_equal(got, orc.split_product(a[rows], b[:, cols], 7, 8))


@pytest.mark.parametrize("n", [2047, 4095, 8192])
def test_fp64_methods_full_size_sampled_rows(mm, orc, n):
    """Uniform entries at the sweep's largest and odd sizes: Kahan and the
    rounding-order naive sum are bit-exact on sampled rows; the FMA/MMA methods
    stay within 1e-14 normwise of the oracle's own method on those rows."""
    a = S.uniform(n, n, S.stream_seed(1, 0))
    b = S.uniform(n, n, S.stream_seed(1, 1))
    ta, tb = _dev(a), _dev(b)
    rows = np.array([0, 1, n // 2, n - 1])
    ar = a[rows]
    na, nb = float(np.abs(a).sum(axis=1).max()), float(np.abs(b).sum(axis=1).max())

    def rows_of(c):
        return c[rows].cpu().numpy()

    assert np.array_equal(rows_of(mm.kahan(ta, tb)), orc.naiv_kahan(ar, b))
    assert np.array_equal(rows_of(mm.naive_unrolled(ta, tb, unroll=1)), orc.naiv_standard(ar, b))
    assert np.array_equal(rows_of(mm.naive_unrolled(ta, tb, unroll=3)), orc.naiv_unrolled(ar, b, 3))

    def normwise(got, ref):
        return float(np.abs(got - ref).sum(axis=1).max() / (na * nb))

    assert normwise(rows_of(mm.naive(ta, tb)), orc.naiv_standard(ar, b)) <= 1e-14
    assert normwise(rows_of(mm.winograd(ta, tb)), orc.winograd_original(ar, b)) <= 1e-14
    truth = orc.dot2_product(ar, b)
    for name in ("winograd_scaled", "winograd_rowcol_scaled", "strassen", "strassen_winograd"):
        assert normwise(rows_of(getattr(mm, name)(ta, tb)), truth) <= 1e-14, name
    # The paper's own depth rule: 8 levels (Y = 4352) at 4095, 9 (Y = 8704) at 8192.
    for name in ("strassen", "strassen_winograd"):
        assert normwise(rows_of(getattr(mm, name)(ta, tb, cutoff=0)), truth) <= 1e-14, name
