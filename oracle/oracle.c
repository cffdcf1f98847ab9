/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, sequential CPU restatement of Hedtke, "Methods of Matrix
 * Multiplication" (arXiv:1106.1347), written from the paper's definitions.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it; the library never does, and this file shares no code, header
 * or constant with the GPU implementation.
 *
 * Conventions: A is N x P, B is P x M, C is N x M, all row-major double with
 * leading dimensions (section "Methods of Matrix Multiplication", opening
 * paragraph).  Every sum runs sequentially in index order, exactly as the
 * paper writes it, and nothing is fused: build with
 * -O2 -ffp-contract=off -fno-fast-math (GCC contracts a*b+c into an FMA by
 * default on aarch64, which would change the naive and Kahan results).
 *
 * Readings of the paper taken here (the printed C listings are not part of
 * the text, so loop orders follow the formulas):
 *  - Winograd: C_ik = (sum_j (A_i,2j-1 + B_2j,k)(A_i,2j + B_2j-1,k) - y_i) - z_k,
 *    then + A_i,P * B_P,k when P is odd (the printed "B_{B,k}" is read as B_{P,k}).
 *  - Scaled Winograd: lambda is the smallest integer with
 *    1/2 <= 4^lambda ||A|| / ||B|| <= 2 (two integers qualify when
 *    log2(||B||/||A||) is odd, as for the paper's own test B = 8A).
 *  - Strassen: X = max{N,P,M}, k = max(0, floor(log2 X) - 4), m = floor(X/2^k) + 1,
 *    Y = m 2^k; sums of several terms are evaluated left to right.  The same
 *    recursion also runs over the split product as its base (not in the paper:
 *    its Strassen levels above the emulated product), padded to multiples of
 *    2^depth.
 *  - Kahan: the paper's update is used as printed and the final err is not
 *    folded back into the sum.
 *  - Per-row/column scaled Winograd (not in the paper; its scaling taken from
 *    one pair of norms to every row of A and column of B): e_i and f_k are the
 *    frexp exponents of the row and column maxima, so every scaled row and
 *    column has its largest magnitude in [1/2, 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define AT(X, ld, i, j) ((X)[(int64_t)(i) * (ld) + (j)])

/* ---------------------------------------------------------------- auxiliaries */

/* Section "Plus": (A+B)_ij = A_ij + B_ij. */
static void plus(int64_t n, int64_t m, const double *X, int64_t ldx, const double *Y, int64_t ldy,
                 double *Z, int64_t ldz) {
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < m; ++j) AT(Z, ldz, i, j) = AT(X, ldx, i, j) + AT(Y, ldy, i, j);
}

/* Section "Minus": (A-B)_ij = A_ij - B_ij. */
static void minus(int64_t n, int64_t m, const double *X, int64_t ldx, const double *Y, int64_t ldy,
                  double *Z, int64_t ldz) {
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < m; ++j) AT(Z, ldz, i, j) = AT(X, ldx, i, j) - AT(Y, ldy, i, j);
}

/* Section "max": x if x >= y, else y. */
static double dmax(double x, double y) { return x >= y ? x : y; }
static int64_t imax(int64_t x, int64_t y) { return x >= y ? x : y; }

/* Section "NormInf": ||A||_inf = max_i sum_j |A_ij|, each row summed in order. */
double oracle_norm_inf(int64_t N, int64_t P, const double *A, int64_t lda) {
    double best = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < P; ++j) s = s + fabs(AT(A, lda, i, j));
        best = (i == 0) ? s : dmax(best, s);
    }
    return best;
}

/* Section "MultiplyWithScalar": (alpha A)_ij = alpha * A_ij. */
void oracle_multiply_with_scalar(int64_t N, int64_t P, double alpha, const double *A, int64_t lda,
                                 double *Z, int64_t ldz) {
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < P; ++j) AT(Z, ldz, i, j) = alpha * AT(A, lda, i, j);
}

/* -------------------------------------------------------------- naive method */

/* Section "NaivStandard": (AB)_ij = sum_k A_ik B_kj, accumulated in a local aux,
 * each product rounded before it is added. */
void oracle_naiv_standard(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                          int64_t ldb, double *C, int64_t ldc) {
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < M; ++j) {
            double aux = 0.0;
            for (int64_t k = 0; k < P; ++k) {
                double prod = AT(A, lda, i, k) * AT(B, ldb, k, j);
                aux = aux + prod;
            }
            AT(C, ldc, i, j) = aux;
        }
}

/* Section "NaivOnArray": the naive sum accumulated in C itself rather than in
 * an auxiliary variable (C_ij = 0, then C_ij = C_ij + A_ik B_kj for k in
 * order).  Each step still rounds to double, so the value equals NaivStandard's. */
void oracle_naiv_on_array(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                          int64_t ldb, double *C, int64_t ldc) {
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < M; ++j) {
            AT(C, ldc, i, j) = 0.0;
            for (int64_t k = 0; k < P; ++k) AT(C, ldc, i, j) = AT(C, ldc, i, j) + AT(A, lda, i, k) * AT(B, ldb, k, j);
        }
}

/* Section "Loop unrolling" (NaivLoopUnrollingTwo, -Three, -Four): the naive
 * sum taken u terms at a time, each group summed left to right before it is
 * added to the running sum,
 *   aux = aux + ((A_i,uk-u+1 B_uk-u+1,j + A_i,uk-u+2 B_uk-u+2,j) + ...),
 * for k = 1 .. floor(P/u), then the P mod u leftover terms added one by one in
 * index order (the "correction terms").  The printed A_i,2k B_2k,j of the
 * three-term formula is read as A_i,3k B_3k,j; the four-term form prints no
 * formula and follows the same pattern.  u = 1 is NaivStandard. */
int oracle_naiv_unrolled(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                         double *C, int64_t ldc, int u) {
    if (u < 1) return -1;
    const int64_t full = (P / u) * u;
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < M; ++j) {
            double aux = 0.0;
            for (int64_t k = 0; k < full; k += u) {
                double grp = AT(A, lda, i, k) * AT(B, ldb, k, j);
                for (int t = 1; t < u; ++t) {
                    double prod = AT(A, lda, i, k + t) * AT(B, ldb, k + t, j);
                    grp = grp + prod;
                }
                aux = aux + grp;
            }
            for (int64_t k = full; k < P; ++k) {
                double prod = AT(A, lda, i, k) * AT(B, ldb, k, j);
                aux = aux + prod;
            }
            AT(C, ldc, i, j) = aux;
        }
    return 0;
}

/* Section "NaivKahan": the naive sum with the compensated update
 *   err = err + x; t = sum + err; err = (sum - t) + err; sum = t
 * applied to x = A_ik * B_kj (rounded).  The result is sum. */
void oracle_naiv_kahan(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                       int64_t ldb, double *C, int64_t ldc) {
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < M; ++j) {
            double sum = 0.0, err = 0.0, t;
            for (int64_t k = 0; k < P; ++k) {
                double x = AT(A, lda, i, k) * AT(B, ldb, k, j);
                err = err + x;
                t = sum + err;
                err = (sum - t) + err;
                sum = t;
            }
            AT(C, ldc, i, j) = sum;
        }
}

/* ----------------------------------------------------------- Winograd's form */

/* Section "WinogradOriginal": y_i = sum_{j<=gamma} A_i,2j-1 A_i,2j and
 * z_k = sum_{j<=gamma} B_2j-1,k B_2j,k with gamma = floor(P/2) (1-based indices). */
void oracle_winograd_terms(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                           int64_t ldb, double *y, double *z) {
    int64_t gamma = P / 2;
    for (int64_t i = 0; i < N; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < gamma; ++j) {
            double prod = AT(A, lda, i, 2 * j) * AT(A, lda, i, 2 * j + 1);
            s = s + prod;
        }
        y[i] = s;
    }
    for (int64_t k = 0; k < M; ++k) {
        double s = 0.0;
        for (int64_t j = 0; j < gamma; ++j) {
            double prod = AT(B, ldb, 2 * j, k) * AT(B, ldb, 2 * j + 1, k);
            s = s + prod;
        }
        z[k] = s;
    }
}

/* Section "WinogradOriginal": C_ik = sum_j (A_i,2j-1 + B_2j,k)(A_i,2j + B_2j-1,k) - y_i - z_k,
 * plus A_i,P B_P,k when P is odd (upsilon = P mod 2). */
void oracle_winograd_original(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                              int64_t ldb, double *C, int64_t ldc) {
    int64_t gamma = P / 2, upsilon = P % 2;
    double *y = (double *)malloc(sizeof(double) * (size_t)imax(N, 1));
    double *z = (double *)malloc(sizeof(double) * (size_t)imax(M, 1));
    oracle_winograd_terms(N, P, M, A, lda, B, ldb, y, z);
    for (int64_t i = 0; i < N; ++i)
        for (int64_t k = 0; k < M; ++k) {
            double aux = 0.0;
            for (int64_t j = 0; j < gamma; ++j) {
                double s1 = AT(A, lda, i, 2 * j) + AT(B, ldb, 2 * j + 1, k);
                double s2 = AT(A, lda, i, 2 * j + 1) + AT(B, ldb, 2 * j, k);
                double prod = s1 * s2;
                aux = aux + prod;
            }
            double c = (aux - y[i]) - z[k];
            if (upsilon) {
                double prod = AT(A, lda, i, P - 1) * AT(B, ldb, P - 1, k);
                c = c + prod;
            }
            AT(C, ldc, i, k) = c;
        }
    free(y);
    free(z);
}

/* Section "WinogradScaled": the smallest integer lambda with
 * 1/2 <= 2^lambda a / (2^-lambda b) <= 2 for a = ||A||, b = ||B|| > 0.
 * ldexp is exact here because both sides are scaled by powers of two and the
 * comparison a*2^(2 lambda + 1) >= b is carried out on (fraction, exponent)
 * pairs, which never overflows.  Returns 0 when a or b is 0 or not finite. */
int oracle_brent_lambda(double a, double b) {
    if (!(a > 0.0) || !(b > 0.0) || !isfinite(a) || !isfinite(b)) return 0;
    int ea, eb;
    double fa = frexp(a, &ea), fb = frexp(b, &eb); /* a = fa 2^ea, fa in [1/2, 1) */
    /* lower bound holds at lambda  <=>  fa 2^(ea + 2 lambda + 1) >= fb 2^eb */
    int lam = (eb - ea - 1) / 2 - 2; /* safely below the answer */
    for (;;) {
        int ex = ea + 2 * lam + 1;
        int ok = (ex > eb) || (ex == eb && fa >= fb);
        if (ok) break;
        ++lam;
    }
    return lam;
}

/* Section "WinogradScaled": multiply 2^lambda A by 2^-lambda B with Winograd's
 * form.  The scalings are MultiplyWithScalar with exact powers of two. */
int oracle_winograd_scaled(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                           int64_t ldb, double *C, int64_t ldc) {
    double na = oracle_norm_inf(N, P, A, lda);
    double nb = oracle_norm_inf(P, M, B, ldb);
    int lam = oracle_brent_lambda(na, nb);
    double *As = (double *)malloc(sizeof(double) * (size_t)imax(N * P, 1));
    double *Bs = (double *)malloc(sizeof(double) * (size_t)imax(P * M, 1));
    oracle_multiply_with_scalar(N, P, ldexp(1.0, lam), A, lda, As, P);
    oracle_multiply_with_scalar(P, M, ldexp(1.0, -lam), B, ldb, Bs, M);
    oracle_winograd_original(N, P, M, As, P, Bs, M, C, ldc);
    free(As);
    free(Bs);
    return lam;
}

/* Per-row/column power-of-two scaling of Winograd's form: the exact scaling of
 * section "WinogradScaled" (MultiplyWithScalar by 2^lambda and 2^-lambda, Eq.
 * for lambda) taken from one global pair of norms down to each row of A and
 * each column of B.  e_i is the frexp exponent of max_j |A_ij| and f_k that of
 * max_j |B_jk| (0 for a zero row or column), so every row of A' = 2^-e_i A_i,:
 * and every column of B' = 2^-f_k B_:,k has its largest entry in [1/2, 1) and
 * each paired sum (A'_i,2j-1 + B'_2j,k) adds terms of like size.  Then
 * C_ik = 2^(e_i + f_k) C'_ik with C' = WinogradOriginal(A', B').  All scalings
 * are by ldexp, exact unless a scaled entry leaves the normal range.
 * e (N entries) and f (M entries) receive the exponents when not NULL. */
void oracle_winograd_rowcol_scaled(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                                   int64_t ldb, double *C, int64_t ldc, int *e, int *f) {
    int *ea = (int *)malloc(sizeof(int) * (size_t)imax(N, 1));
    int *fb = (int *)malloc(sizeof(int) * (size_t)imax(M, 1));
    double *As = (double *)malloc(sizeof(double) * (size_t)imax(N * P, 1));
    double *Bs = (double *)malloc(sizeof(double) * (size_t)imax(P * M, 1));
    double *Cs = (double *)malloc(sizeof(double) * (size_t)imax(N * M, 1));
    for (int64_t i = 0; i < N; ++i) {
        double mx = 0.0;
        for (int64_t j = 0; j < P; ++j) mx = fmax(mx, fabs(AT(A, lda, i, j)));
        int ex = 0;
        if (mx > 0.0) (void)frexp(mx, &ex);
        ea[i] = ex;
        for (int64_t j = 0; j < P; ++j) AT(As, P, i, j) = ldexp(AT(A, lda, i, j), -ex);
    }
    for (int64_t k = 0; k < M; ++k) {
        double mx = 0.0;
        for (int64_t j = 0; j < P; ++j) mx = fmax(mx, fabs(AT(B, ldb, j, k)));
        int ex = 0;
        if (mx > 0.0) (void)frexp(mx, &ex);
        fb[k] = ex;
        for (int64_t j = 0; j < P; ++j) AT(Bs, M, j, k) = ldexp(AT(B, ldb, j, k), -ex);
    }
    oracle_winograd_original(N, P, M, As, P, Bs, M, Cs, M);
    for (int64_t i = 0; i < N; ++i)
        for (int64_t k = 0; k < M; ++k) AT(C, ldc, i, k) = ldexp(AT(Cs, M, i, k), ea[i] + fb[k]);
    if (e)
        for (int64_t i = 0; i < N; ++i) e[i] = ea[i];
    if (f)
        for (int64_t k = 0; k < M; ++k) f[k] = fb[k];
    free(ea);
    free(fb);
    free(As);
    free(Bs);
    free(Cs);
}

/* --------------------------------------------------------------- Strassen */

/* Section "StrassenNaiv": X = max{N,P,M}, k = floor(log2 X) - 4 (taken as 0 when
 * negative), m = floor(X 2^-k) + 1, Y = m 2^k.  Writes k and Y. */
void oracle_strassen_paper_rule(int64_t N, int64_t P, int64_t M, int *k_out, int64_t *Y_out) {
    int64_t X = imax(imax(N, P), M);
    int lg = -1;
    for (int64_t t = X; t > 0; t >>= 1) ++lg; /* floor(log2 X) by bit length */
    int k = lg - 4;
    if (k < 0) k = 0;
    int64_t m = (X >> k) + 1;
    *k_out = k;
    *Y_out = m << k;
}

static double *zalloc(int64_t n) { return (double *)calloc((size_t)imax(n, 1), sizeof(double)); }

/* The product at the bottom of the recursion: the paper's NaivStandard
 * (beta == 0), or the split product of the given beta and slice count. */
struct strassen_base {
    int beta, s;
};
static const struct strassen_base naive_base = {0, 0};

int oracle_split_product(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                         int64_t ldb, double *C, int64_t ldc, int beta, int s);

static void base_product(const struct strassen_base *base, int64_t n, int64_t p, int64_t m, const double *A,
                         int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc) {
    if (base->beta == 0)
        oracle_naiv_standard(n, p, m, A, lda, B, ldb, C, ldc);
    else
        (void)oracle_split_product(n, p, m, A, lda, B, ldb, C, ldc, base->beta, base->s);
}

/* alpha_{m,k}: one level of the recursion on an n x p times p x m product whose
 * dimensions are all divisible by 2^depth. */
static void strassen_rec(int64_t n, int64_t p, int64_t m, const double *A, int64_t lda, const double *B,
                         int64_t ldb, double *C, int64_t ldc, int depth, const struct strassen_base *base) {
    if (depth == 0) {
        base_product(base, n, p, m, A, lda, B, ldb, C, ldc);
        return;
    }
    int64_t n2 = n / 2, p2 = p / 2, m2 = m / 2;
    const double *A11 = A, *A12 = A + p2, *A21 = A + n2 * lda, *A22 = A + n2 * lda + p2;
    const double *B11 = B, *B12 = B + m2, *B21 = B + p2 * ldb, *B22 = B + p2 * ldb + m2;
    double *C11 = C, *C12 = C + m2, *C21 = C + n2 * ldc, *C22 = C + n2 * ldc + m2;
    double *S = zalloc(n2 * p2), *T = zalloc(p2 * m2);
    double *H[8];
    for (int h = 1; h <= 7; ++h) H[h] = zalloc(n2 * m2);
    /* H1 = (A11 + A22)(B11 + B22) */
    plus(n2, p2, A11, lda, A22, lda, S, p2);
    plus(p2, m2, B11, ldb, B22, ldb, T, m2);
    strassen_rec(n2, p2, m2, S, p2, T, m2, H[1], m2, depth - 1, base);
    /* H2 = (A21 + A22) B11 */
    plus(n2, p2, A21, lda, A22, lda, S, p2);
    strassen_rec(n2, p2, m2, S, p2, B11, ldb, H[2], m2, depth - 1, base);
    /* H3 = A11 (B12 - B22) */
    minus(p2, m2, B12, ldb, B22, ldb, T, m2);
    strassen_rec(n2, p2, m2, A11, lda, T, m2, H[3], m2, depth - 1, base);
    /* H4 = A22 (B21 - B11) */
    minus(p2, m2, B21, ldb, B11, ldb, T, m2);
    strassen_rec(n2, p2, m2, A22, lda, T, m2, H[4], m2, depth - 1, base);
    /* H5 = (A11 + A12) B22 */
    plus(n2, p2, A11, lda, A12, lda, S, p2);
    strassen_rec(n2, p2, m2, S, p2, B22, ldb, H[5], m2, depth - 1, base);
    /* H6 = (A21 - A11)(B11 + B12) */
    minus(n2, p2, A21, lda, A11, lda, S, p2);
    plus(p2, m2, B11, ldb, B12, ldb, T, m2);
    strassen_rec(n2, p2, m2, S, p2, T, m2, H[6], m2, depth - 1, base);
    /* H7 = (A12 - A22)(B21 + B22) */
    minus(n2, p2, A12, lda, A22, lda, S, p2);
    plus(p2, m2, B21, ldb, B22, ldb, T, m2);
    strassen_rec(n2, p2, m2, S, p2, T, m2, H[7], m2, depth - 1, base);
    /* C11 = H1 + H4 - H5 + H7, C12 = H3 + H5, C21 = H2 + H4, C22 = H1 + H3 - H2 + H6 (left to right) */
    plus(n2, m2, H[1], m2, H[4], m2, C11, ldc);
    minus(n2, m2, C11, ldc, H[5], m2, C11, ldc);
    plus(n2, m2, C11, ldc, H[7], m2, C11, ldc);
    plus(n2, m2, H[3], m2, H[5], m2, C12, ldc);
    plus(n2, m2, H[2], m2, H[4], m2, C21, ldc);
    plus(n2, m2, H[1], m2, H[3], m2, C22, ldc);
    minus(n2, m2, C22, ldc, H[2], m2, C22, ldc);
    plus(n2, m2, C22, ldc, H[6], m2, C22, ldc);
    for (int h = 1; h <= 7; ++h) free(H[h]);
    free(S);
    free(T);
}

/* Section "StrassenWinograd": the Winograd variant (after Fischer and Probert)
 * with 15 additions, in the printed order. */
static void strassen_winograd_rec(int64_t n, int64_t p, int64_t m, const double *A, int64_t lda, const double *B,
                                  int64_t ldb, double *C, int64_t ldc, int depth,
                                  const struct strassen_base *base) {
    if (depth == 0) {
        base_product(base, n, p, m, A, lda, B, ldb, C, ldc);
        return;
    }
    int64_t n2 = n / 2, p2 = p / 2, m2 = m / 2;
    const double *A11 = A, *A12 = A + p2, *A21 = A + n2 * lda, *A22 = A + n2 * lda + p2;
    const double *B11 = B, *B12 = B + m2, *B21 = B + p2 * ldb, *B22 = B + p2 * ldb + m2;
    double *C11 = C, *C12 = C + m2, *C21 = C + n2 * ldc, *C22 = C + n2 * ldc + m2;
    double *A1 = zalloc(n2 * p2), *A2 = zalloc(n2 * p2), *B1 = zalloc(p2 * m2), *B2 = zalloc(p2 * m2);
    double *S = zalloc(n2 * p2), *T = zalloc(p2 * m2);
    double *H[10];
    for (int h = 1; h <= 9; ++h) H[h] = zalloc(n2 * m2);
    /* A1 = A11 - A21, A2 = A22 - A1, B1 = B22 - B12, B2 = B1 + B11 */
    minus(n2, p2, A11, lda, A21, lda, A1, p2);
    minus(n2, p2, A22, lda, A1, p2, A2, p2);
    minus(p2, m2, B22, ldb, B12, ldb, B1, m2);
    plus(p2, m2, B1, m2, B11, ldb, B2, m2);
    /* H1 = A11 B11, H2 = A12 B21, H3 = A2 B2, H4 = (A21 + A22)(B12 - B11) */
    strassen_winograd_rec(n2, p2, m2, A11, lda, B11, ldb, H[1], m2, depth - 1, base);
    strassen_winograd_rec(n2, p2, m2, A12, lda, B21, ldb, H[2], m2, depth - 1, base);
    strassen_winograd_rec(n2, p2, m2, A2, p2, B2, m2, H[3], m2, depth - 1, base);
    plus(n2, p2, A21, lda, A22, lda, S, p2);
    minus(p2, m2, B12, ldb, B11, ldb, T, m2);
    strassen_winograd_rec(n2, p2, m2, S, p2, T, m2, H[4], m2, depth - 1, base);
    /* H5 = A1 B1, H6 = (A12 - A2) B22, H7 = A22 (B21 - B2) */
    strassen_winograd_rec(n2, p2, m2, A1, p2, B1, m2, H[5], m2, depth - 1, base);
    minus(n2, p2, A12, lda, A2, p2, S, p2);
    strassen_winograd_rec(n2, p2, m2, S, p2, B22, ldb, H[6], m2, depth - 1, base);
    minus(p2, m2, B21, ldb, B2, m2, T, m2);
    strassen_winograd_rec(n2, p2, m2, A22, lda, T, m2, H[7], m2, depth - 1, base);
    /* H8 = H1 + H3, H9 = H8 + H4 */
    plus(n2, m2, H[1], m2, H[3], m2, H[8], m2);
    plus(n2, m2, H[8], m2, H[4], m2, H[9], m2);
    /* C11 = H1 + H2, C12 = H9 + H6, C21 = H8 + H5 + H7, C22 = H9 + H5 */
    plus(n2, m2, H[1], m2, H[2], m2, C11, ldc);
    plus(n2, m2, H[9], m2, H[6], m2, C12, ldc);
    plus(n2, m2, H[8], m2, H[5], m2, C21, ldc);
    plus(n2, m2, C21, ldc, H[7], m2, C21, ldc);
    plus(n2, m2, H[9], m2, H[5], m2, C22, ldc);
    for (int h = 1; h <= 9; ++h) free(H[h]);
    free(A1);
    free(A2);
    free(B1);
    free(B2);
    free(S);
    free(T);
}

/* Embed A and B into zero matrices of Np x Pp and Pp x Mp (each divisible by
 * 2^depth), run the recursion and extract the N x M result (section
 * "StrassenNaiv", last paragraph).  variant 0 = StrassenNaiv, 1 = StrassenWinograd. */
static int strassen_embedded(int variant, int64_t N, int64_t P, int64_t M, const double *A, int64_t lda,
                             const double *B, int64_t ldb, double *C, int64_t ldc, int depth, int64_t Np,
                             int64_t Pp, int64_t Mp, const struct strassen_base *base) {
    if (N == 0 || M == 0) return 0;
    if (depth < 0 || Np < N || Pp < P || Mp < M) return -1;
    int64_t q = (int64_t)1 << depth;
    if (Np % q || Pp % q || Mp % q) return -1;
    double *At = zalloc(Np * Pp), *Bt = zalloc(Pp * Mp), *Ct = zalloc(Np * Mp);
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < P; ++j) AT(At, Pp, i, j) = AT(A, lda, i, j);
    for (int64_t i = 0; i < P; ++i)
        for (int64_t j = 0; j < M; ++j) AT(Bt, Mp, i, j) = AT(B, ldb, i, j);
    if (variant == 0)
        strassen_rec(Np, Pp, Mp, At, Pp, Bt, Mp, Ct, Mp, depth, base);
    else
        strassen_winograd_rec(Np, Pp, Mp, At, Pp, Bt, Mp, Ct, Mp, depth, base);
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < M; ++j) AT(C, ldc, i, j) = AT(Ct, Mp, i, j);
    free(At);
    free(Bt);
    free(Ct);
    return 0;
}

/* depth < 0 selects the paper's rule (square embedding Y x Y); otherwise the
 * caller's depth and padded sizes are used. */
int oracle_strassen_naiv(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                         int64_t ldb, double *C, int64_t ldc, int depth, int64_t Np, int64_t Pp, int64_t Mp) {
    if (depth < 0) {
        int64_t Y;
        oracle_strassen_paper_rule(N, P, M, &depth, &Y);
        Np = Pp = Mp = Y;
    }
    return strassen_embedded(0, N, P, M, A, lda, B, ldb, C, ldc, depth, Np, Pp, Mp, &naive_base);
}

int oracle_strassen_winograd(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                             int64_t ldb, double *C, int64_t ldc, int depth, int64_t Np, int64_t Pp, int64_t Mp) {
    if (depth < 0) {
        int64_t Y;
        oracle_strassen_paper_rule(N, P, M, &depth, &Y);
        Np = Pp = Mp = Y;
    }
    return strassen_embedded(1, N, P, M, A, lda, B, ldb, C, ldc, depth, Np, Pp, Mp, &naive_base);
}

/* Strassen (variant 0, section "StrassenNaiv") or Strassen-Winograd (variant 1,
 * section "StrassenWinograd") recursion of `depth` levels whose base product is
 * the split product (beta, s) instead of NaivStandard: the operand sums and the
 * combinations of H1..H7 are the same FP64 additions, in the printed order.  A
 * and B are embedded in zero matrices whose sizes are the smallest multiples of
 * 2^depth >= N, P, M. */
int oracle_strassen_emulated(int variant, int64_t N, int64_t P, int64_t M, const double *A, int64_t lda,
                             const double *B, int64_t ldb, double *C, int64_t ldc, int depth, int beta, int s) {
    if (variant < 0 || variant > 1 || depth < 0 || depth > 6) return -1;
    if (beta < 2 || beta > 12 || s < 1 || beta * s > 62) return -1;
    const struct strassen_base base = {beta, s};
    const int64_t q = (int64_t)1 << depth;
    const int64_t Np = (N + q - 1) / q * q, Pp = (P + q - 1) / q * q, Mp = (M + q - 1) / q * q;
    return strassen_embedded(variant, N, P, M, A, lda, B, ldb, C, ldc, depth, Np, Pp, Mp, &base);
}

/* ------------------------------------------------------------- the truth */

/* Reference product for error reports: each C_ij is the dot product
 * evaluated with the Dot2 algorithm of Ogita, Rump and Oishi ("Accurate sum
 * and dot product", SIAM J. Sci. Comput. 26, 2005): TwoProduct (through a
 * correctly rounded fma) and Knuth's TwoSum, as accurate as a doubled-precision
 * evaluation rounded once to double. */
void oracle_dot2_product(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                         int64_t ldb, double *C, int64_t ldc) {
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < M; ++j) {
            double p = 0.0, s = 0.0;
            for (int64_t k = 0; k < P; ++k) {
                double a = AT(A, lda, i, k), b = AT(B, ldb, k, j);
                double h = a * b;
                double r = fma(a, b, -h); /* TwoProduct: a*b = h + r exactly */
                double x = p + h;         /* TwoSum(p, h) = (x, q) */
                double z = x - p;
                double q = (p - (x - z)) + (h - z);
                p = x;
                s = s + (q + r);
            }
            AT(C, ldc, i, j) = p + s;
        }
}

/* ------------------------------------------- split-precision emulated product */

/* The FP64-accurate product emulated from small-integer slices (not in the
 * paper; its per-row/column power-of-two scaling follows the exact
 * power-of-two rescaling of section "WinogradScaled").  Definition:
 *
 *   e_i = frexp exponent of max_k |A_ik| (so |A_ik| < 2^e_i), 0 for a zero row;
 *   f_j likewise for column j of B;
 *   V_ik = RN(A_ik 2^(beta s - 1 - e_i)) and U_kj = RN(B_kj 2^(beta s - 1 - f_j)),
 *     integers with |V|, |U| <= 2^(beta s - 1);
 *   balanced base-2^beta digits: V = sum_{t<s} v_t 2^(beta t), the low s-1 digits
 *     in [-2^(beta-1), 2^(beta-1)) and the top digit taking the remainder;
 *   slice sigma = digit s-1-sigma (sigma = 0 is the most significant);
 *   W_ij = sum over slice pairs with sigma + tau <= s-1 of
 *          2^(beta (s-1-sigma-tau)) sum_k a^(sigma)_ik b^(tau)_kj   (exact integer);
 *   C_ij = RN(W_ij) * 2^(e_i + f_j + 2 - beta (s+1)).
 *
 * Only the rounding of V, U, the dropped pairs sigma + tau >= s and the single
 * final rounding separate C from A*B.  Integer arithmetic is exact (__int128). */
static int64_t round_scaled(double x, int shift) {
    double v = nearbyint(ldexp(x, shift)); /* ties to even in the default rounding mode */
    return (int64_t)v;
}

static int frexp_exp(double x) {
    int e;
    if (x == 0.0) return 0;
    (void)frexp(x, &e);
    return e;
}

static void balanced_digits(int64_t V, int beta, int s, int32_t *digits /* s entries, index = slice */) {
    int64_t base = (int64_t)1 << beta, half = base >> 1;
    for (int t = 0; t < s - 1; ++t) {
        int64_t d = V % base;
        if (d < 0) d += base;
        if (d >= half) d -= base;
        digits[s - 1 - t] = (int32_t)d;
        V = (V - d) / base;
    }
    digits[0] = (int32_t)V;
}

int oracle_split_digits(int64_t rows, int64_t cols, const double *X, int64_t ldx, int by_columns, int beta, int s,
                        int32_t *exps, int32_t *digits) {
    /* digits[(slice * rows + i) * cols + j]; exps per row (by_columns = 0) or per column (1). */
    if (beta < 2 || beta > 12 || s < 1 || beta * s > 62) return -1;
    int64_t nexp = by_columns ? cols : rows;
    for (int64_t r = 0; r < nexp; ++r) {
        double mx = 0.0;
        int64_t len = by_columns ? rows : cols;
        for (int64_t q = 0; q < len; ++q) {
            double v = by_columns ? fabs(AT(X, ldx, q, r)) : fabs(AT(X, ldx, r, q));
            mx = dmax(mx, v);
        }
        exps[r] = frexp_exp(mx);
    }
    int32_t dg[64];
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < cols; ++j) {
            int e = by_columns ? exps[j] : exps[i];
            int64_t V = round_scaled(AT(X, ldx, i, j), beta * s - 1 - e);
            balanced_digits(V, beta, s, dg);
            for (int t = 0; t < s; ++t) digits[((int64_t)t * rows + i) * cols + j] = dg[t];
        }
    return 0;
}

int oracle_split_product(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                         int64_t ldb, double *C, int64_t ldc, int beta, int s) {
    if (beta < 2 || beta > 12 || s < 1 || beta * s > 62) return -1;
    if (N == 0 || M == 0) return 0;
    int32_t *ea = (int32_t *)malloc(sizeof(int32_t) * (size_t)imax(N, 1));
    int32_t *fb = (int32_t *)malloc(sizeof(int32_t) * (size_t)imax(M, 1));
    int32_t *da = (int32_t *)malloc(sizeof(int32_t) * (size_t)imax((int64_t)s * N * P, 1));
    int32_t *db = (int32_t *)malloc(sizeof(int32_t) * (size_t)imax((int64_t)s * P * M, 1));
    oracle_split_digits(N, P, A, lda, 0, beta, s, ea, da);
    oracle_split_digits(P, M, B, ldb, 1, beta, s, fb, db);
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < M; ++j) {
            __int128 W = 0;
            for (int sg = 0; sg < s; ++sg)
                for (int tu = 0; sg + tu <= s - 1; ++tu) {
                    __int128 dot = 0;
                    for (int64_t k = 0; k < P; ++k)
                        dot += (__int128)da[((int64_t)sg * N + i) * P + k] * db[((int64_t)tu * P + k) * M + j];
                    W += dot * ((__int128)1 << (beta * (s - 1 - sg - tu)));
                }
            double w = (double)W; /* correctly rounded conversion */
            AT(C, ldc, i, j) = ldexp(w, ea[i] + fb[j] + 2 - beta * (s + 1));
        }
    free(ea);
    free(fb);
    free(da);
    free(db);
    return 0;
}
