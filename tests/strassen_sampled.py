"""Sampled entries of one Strassen level over the split product, for parity at
sizes where the oracle's full recursion would take too long.

One level of sections "StrassenNaiv" / "StrassenWinograd" with the split
product as the base: entry (i, j) of quadrant (qi, qj) combines H_k(i', j')
with i' = i mod N/2, j' = j mod M/2, and H_k(i', j') depends only on row i' of
H_k's A-side operand and column j' of its B-side operand (the split's
exponents are per row and per column).  So the operand rows and columns are
formed with the section's FP64 additions in the printed order, the oracle's
split product gives those entries of every H_k, and the C quadrants are the
printed sums.  A CPU test checks this against the oracle's full recursion."""
import numpy as np


def one_level_sampled(orc, a, b, variant, rows, cols, beta, s):
    n, p = a.shape
    m = b.shape[1]
    assert n % 2 == 0 and p % 2 == 0 and m % 2 == 0
    h, q, w = n // 2, p // 2, m // 2
    rows, cols = np.asarray(rows), np.asarray(cols)
    lr, lc = np.unique(rows % h), np.unique(cols % w)
    A11, A12, A21, A22 = a[lr, :q], a[lr, q:], a[lr + h, :q], a[lr + h, q:]
    B11, B12, B21, B22 = b[:q, lc], b[:q, lc + w], b[q:, lc], b[q:, lc + w]
    if variant == 0:
        ops = [(A11 + A22, B11 + B22), (A21 + A22, B11), (A11, B12 - B22), (A22, B21 - B11),
               (A11 + A12, B22), (A21 - A11, B11 + B12), (A12 - A22, B21 + B22)]
    else:
        A1 = A11 - A21
        A2 = A22 - A1
        B1 = B22 - B12
        B2 = B1 + B11
        ops = [(A11, B11), (A12, B21), (A2, B2), (A21 + A22, B12 - B11), (A1, B1), (A12 - A2, B22),
               (A22, B21 - B2)]
    H = [orc.split_product(x, y, beta, s) for x, y in ops]
    if variant == 0:
        C11 = ((H[0] + H[3]) - H[4]) + H[6]
        C12 = H[2] + H[4]
        C21 = H[1] + H[3]
        C22 = ((H[0] + H[2]) - H[1]) + H[5]
    else:
        H8 = H[0] + H[2]
        H9 = H8 + H[3]
        C11 = H[0] + H[1]
        C12 = H9 + H[5]
        C21 = (H8 + H[4]) + H[6]
        C22 = H9 + H[4]
    quads = {(0, 0): C11, (0, 1): C12, (1, 0): C21, (1, 1): C22}
    ri = {v: k for k, v in enumerate(lr)}
    ci = {v: k for k, v in enumerate(lc)}
    out = np.empty((len(rows), len(cols)))
    for x, i in enumerate(rows):
        for y, j in enumerate(cols):
            out[x, y] = quads[(int(i >= h), int(j >= w))][ri[int(i % h)], ci[int(j % w)]]
    return out
