// Sections "WinogradOriginal" and "WinogradScaled".
//
//  1. row pass over A: y_i = sum_{j<gamma} RN(A_i,2j A_i,2j+1) (0-based), each
//     row summed in order by one lane after a shared-memory transpose of
//     coalesced 32x32 tiles; the scaled form also sums |A_ij| in the same pass
//     and folds the row maximum into ||A||_inf (NormInf fused into the y pass).
//  2. column pass over B: z_k = sum_j RN(B_2j,k B_2j+1,k), one thread per
//     column, coalesced across the warp.  The scaled form runs the NormInf
//     kernel over B as well.
//  3. main kernel: C_ik = (sum_j (A_i,2j + B_2j+1,k)(A_i,2j+1 + B_2j,k) - y'_i) - z'_k
//     (+ RN(A_i,P-1 B_P-1,k) when P is odd).  For the scaled form every CTA
//     derives Brent's lambda from the two device-resident norms (no host
//     round trip), multiplies A by 2^lambda and B by 2^-lambda while staging
//     tiles (MultiplyWithScalar by exact powers of two), and uses
//     y' = 4^lambda y and z' = 4^-lambda z, which equal the terms of the
//     scaled matrices bit for bit when nothing over- or underflows.
//  4. per-row/column scaled form (Brent's exact power-of-two scaling taken to
//     each row of A and column of B): the row pass first finds e_i, the frexp
//     exponent of max_j |A_ij|, then sums y'_i over A'_i,: = 2^-e_i A_i,:; the
//     column pass does the same for f_k and z'_k; the main kernel scales the
//     staged tiles by 2^-e_i and 2^-f_k and the result by 2^(e_i + f_k).
// y and z are bit-identical to a sequential evaluation; the paired sum uses
// one FMA per pair (2 DADD + 1 DFMA per pair per output, the FP64 pipe bound).
#include <type_traits>

#include "common.cuh"

namespace {

constexpr int kRows = 32;

// x * 2^k with ldexp's result.  When x is normal and the scaled exponent stays
// in the normal range, the product is exact and is x's bit pattern with k added
// to the exponent field (integer work only, no FP64 pipe); zeros, subnormals,
// and results that would leave the normal range go to ldexp.
__device__ __forceinline__ double pow2_scale(double x, int k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    if (E != 0 && E != 0x7FF && E + k >= 1 && E + k <= 0x7FE)
        return __longlong_as_double((long long)(b + ((unsigned long long)(long long)k << 52)));
    return ldexp(x, k);
}

// Row group `blk` (rows 32 blk .. 32 blk + 31) of the y pass, one warp.
template <bool kNorm>
__device__ __forceinline__ void a_terms_rows(int64_t blk, int64_t N, int64_t P, const double *__restrict__ A,
                                             int64_t lda, double *__restrict__ y, unsigned long long *norm_bits) {
    __shared__ double tile[kRows][kRows + 1];
    const int lane = threadIdx.x;
    const int64_t row0 = blk * kRows;
    const int64_t nrows = min((int64_t)kRows, N - row0);
    const int64_t gamma2 = (P / 2) * 2;  // columns that form pairs
    double next[kRows];
    auto fetch = [&](int64_t c0) {
        const int64_t c = c0 + lane;
#pragma unroll
        for (int r = 0; r < kRows; ++r) next[r] = (r < nrows && c < P) ? A[(row0 + r) * lda + c] : 0.0;
    };
    double ys = 0.0, ns = 0.0;
    fetch(0);
    for (int64_t c0 = 0; c0 < P; c0 += kRows) {
#pragma unroll
        for (int r = 0; r < kRows; ++r) tile[r][lane] = next[r];
        __syncwarp();
        if (c0 + kRows < P) fetch(c0 + kRows);
        const int npair = (int)max((int64_t)0, min((int64_t)kRows, gamma2 - c0)) / 2;
        for (int j = 0; j < npair; ++j) ys = __dadd_rn(ys, __dmul_rn(tile[lane][2 * j], tile[lane][2 * j + 1]));
        if (kNorm) {
            const int ncols = (int)min((int64_t)kRows, P - c0);
            for (int j = 0; j < ncols; ++j) ns = __dadd_rn(ns, fabs(tile[lane][j]));
        }
        __syncwarp();
    }
    if (lane < nrows) {
        y[row0 + lane] = ys;
        if (kNorm) atomicMax(norm_bits, (unsigned long long)__double_as_longlong(ns));
    }
}

// Column k of the z pass, one thread.
__device__ __forceinline__ void b_terms_col(int64_t k, int64_t P, int64_t M, const double *__restrict__ B, int64_t ldb,
                                            double *__restrict__ z) {
    if (k >= M) return;
    const int64_t gamma = P / 2;
    double s = 0.0;
    int64_t j = 0;
    for (; j + 4 <= gamma; j += 4) {
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = B[(2 * j + q) * ldb + k];
#pragma unroll
        for (int q = 0; q < 4; ++q) s = __dadd_rn(s, __dmul_rn(v[2 * q], v[2 * q + 1]));
    }
    for (; j < gamma; ++j) s = __dadd_rn(s, __dmul_rn(B[(2 * j) * ldb + k], B[(2 * j + 1) * ldb + k]));
    z[k] = s;
}

// frexp exponent of the double with bit pattern `bits` (>= 0), 0 for zero.
__device__ __forceinline__ int exponent_of(unsigned long long bits) {
    if (bits == 0) return 0;
    int e;
    (void)frexp(__longlong_as_double((long long)bits), &e);
    return e;
}

// Row pass of the per-row/column scaled form for row group `blk`: e_i, then
// y'_i over 2^-e_i A_i,:.
__device__ __forceinline__ void a_terms_rowcol_rows(int64_t blk, int64_t N, int64_t P, const double *__restrict__ A,
                                                    int64_t lda, double *__restrict__ y, int32_t *__restrict__ ea) {
    __shared__ double tile[kRows][kRows + 1];
    const int lane = threadIdx.x;
    const int64_t row0 = blk * kRows;
    const int64_t nrows = min((int64_t)kRows, N - row0);
    const int64_t gamma2 = (P / 2) * 2;
    // Pass 1: the row maximum of |A_ij| on the bit patterns (lane r owns row r).
    unsigned long long mx = 0;
    for (int64_t c0 = 0; c0 < P; c0 += kRows) {
        const int64_t c = c0 + lane;
#pragma unroll 4
        for (int r = 0; r < kRows; ++r)
            tile[r][lane] = (r < nrows && c < P) ? A[(row0 + r) * lda + c] : 0.0;
        __syncwarp();
        const int ncols = (int)min((int64_t)kRows, P - c0);
        for (int j = 0; j < ncols; ++j) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(tile[lane][j]) & ~(1ull << 63);
            mx = b > mx ? b : mx;
        }
        __syncwarp();
    }
    const int e = exponent_of(mx);
    // Pass 2: y'_i = sum_j RN(A'_i,2j A'_i,2j+1) in order, A' = 2^-e_i A (exact).
    double ys = 0.0;
    for (int64_t c0 = 0; c0 < gamma2; c0 += kRows) {
        const int64_t c = c0 + lane;
#pragma unroll 4
        for (int r = 0; r < kRows; ++r)
            tile[r][lane] = (r < nrows && c < gamma2) ? A[(row0 + r) * lda + c] : 0.0;
        __syncwarp();
        const int npair = (int)min((int64_t)kRows, gamma2 - c0) / 2;
        for (int j = 0; j < npair; ++j)
            ys = __dadd_rn(ys, __dmul_rn(pow2_scale(tile[lane][2 * j], -e), pow2_scale(tile[lane][2 * j + 1], -e)));
        __syncwarp();
    }
    if (lane < nrows) {
        y[row0 + lane] = ys;
        ea[row0 + lane] = e;
    }
}

// Column pass of the per-row/column scaled form for column k: f_k, then z'_k
// over 2^-f_k B_:,k.
__device__ __forceinline__ void b_terms_rowcol_col(int64_t k, int64_t P, int64_t M, const double *__restrict__ B,
                                                   int64_t ldb, double *__restrict__ z, int32_t *__restrict__ fb) {
    if (k >= M) return;
    unsigned long long mx = 0;
    for (int64_t j = 0; j < P; ++j) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(B[j * ldb + k]) & ~(1ull << 63);
        mx = b > mx ? b : mx;
    }
    const int f = exponent_of(mx);
    const int64_t gamma = P / 2;
    double s = 0.0;
    for (int64_t j = 0; j < gamma; ++j)
        s = __dadd_rn(s, __dmul_rn(pow2_scale(B[(2 * j) * ldb + k], -f), pow2_scale(B[(2 * j + 1) * ldb + k], -f)));
    z[k] = s;
    fb[k] = f;
}

// The y and z passes in one launch of 32-thread blocks: blocks [0, nA) take
// row groups of A, the rest take 32 columns of B each (the two passes are
// independent, so they run side by side).  kMode as winograd_kernel's.
template <int kMode>
__global__ void __launch_bounds__(32) terms_kernel(int64_t N, int64_t P, int64_t M, const double *__restrict__ A,
                                                   int64_t lda, const double *__restrict__ B, int64_t ldb,
                                                   double *__restrict__ y, double *__restrict__ z,
                                                   unsigned long long *norm_bits, int32_t *__restrict__ ea,
                                                   int32_t *__restrict__ fb, int64_t nA) {
    const int64_t blk = blockIdx.x;
    if (blk < nA) {
        if constexpr (kMode == 2)
            a_terms_rowcol_rows(blk, N, P, A, lda, y, ea);
        else
            a_terms_rows<kMode == 1>(blk, N, P, A, lda, y, norm_bits);
        return;
    }
    const int64_t k = (blk - nA) * 32 + threadIdx.x;
    if constexpr (kMode == 2)
        b_terms_rowcol_col(k, P, M, B, ldb, z, fb);
    else
        b_terms_col(k, P, M, B, ldb, z);
}

// Smallest lambda with 1/2 <= 4^lambda a / b <= 2, from frexp pairs (exact).
__device__ int brent_lambda(double a, double b) {
    if (!(a > 0.0) || !(b > 0.0) || isinf(a) || isinf(b)) return 0;
    int ea, eb;
    const double fa = frexp(a, &ea), fb = frexp(b, &eb);
    int lam = (eb - ea - 1) / 2 - 2;
    for (int it = 0; it < 8; ++it) {
        const int ex = ea + 2 * lam + 1;
        if (ex > eb || (ex == eb && fa >= fb)) break;
        ++lam;
    }
    return lam;
}

constexpr int TK = 16;

// kMode: 0 WinogradOriginal, 1 Brent's global lambda, 2 per-row/column exponents.
// 256 threads in a 16 x 16 layout, each owning R x R outputs strided by 16 of a
// 16R x 16R tile (R = 4, 2 or 1 by the size of the grid).
template <int kMode, int R>
__global__ void __launch_bounds__(256) winograd_kernel(int64_t N, int64_t P, int64_t M, const double *__restrict__ A,
                                                       int64_t lda, const double *__restrict__ B, int64_t ldb,
                                                       double *__restrict__ C, int64_t ldc,
                                                       const double *__restrict__ y, const double *__restrict__ z,
                                                       const double *norms, int32_t *lambda_out,
                                                       const int32_t *__restrict__ ea, const int32_t *__restrict__ fb) {
    constexpr bool kScaled = kMode == 1, kRowCol = kMode == 2;
    constexpr int T = 16 * R;  // output tile side
    __shared__ double As[T][TK + 1];
    __shared__ double Bs[TK][T];
    __shared__ double s_scale[2];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t i0 = (int64_t)blockIdx.y * T, j0 = (int64_t)blockIdx.x * T;
    const int64_t K2 = (P / 2) * 2;
    if (tid == 0) {
        double sa = 1.0, sb = 1.0;
        if (kScaled) {
            const int lam = brent_lambda(norms[0], norms[1]);
            sa = ldexp(1.0, lam);
            sb = ldexp(1.0, -lam);
            if (lambda_out && blockIdx.x == 0 && blockIdx.y == 0) *lambda_out = lam;
        }
        s_scale[0] = sa;
        s_scale[1] = sb;
    }
    __syncthreads();
    const double sa = s_scale[0], sb = s_scale[1];
    double acc[R][R];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c) acc[r][c] = 0.0;
    double ra[R], rb[R];
    // Per-row/column form: this thread stages rows (tid >> 4) + 16 q of A and
    // column tid mod T of B in every K-step (256 q is a multiple of T).
    int erow[R], fcol = 0;
    if (kRowCol) {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int64_t gi = i0 + ((tid + 256 * q) >> 4);
            erow[q] = gi < N ? ea[gi] : 0;
        }
        const int64_t bj = j0 + (tid % T);
        fcol = bj < M ? fb[bj] : 0;
    }
    auto fetch = [&](int64_t k0) {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int e = tid + 256 * q;
            const int64_t gi = i0 + (e >> 4), gk = k0 + (e & 15);
            double av = (gi < N && gk < K2) ? A[gi * lda + gk] : 0.0;
            const int64_t bk = k0 + e / T, bj = j0 + e % T;
            double bv = (bk < K2 && bj < M) ? B[bk * ldb + bj] : 0.0;
            if (kScaled) {
                av *= sa;
                bv *= sb;
            }
            if (kRowCol) {  // exponent-field scaling: measured faster here than ldexp or a multiplication
                av = pow2_scale(av, -erow[q]);
                bv = pow2_scale(bv, -fcol);
            }
            ra[q] = av;
            rb[q] = bv;
        }
    };
    if (K2 > 0) fetch(0);
    for (int64_t k0 = 0; k0 < K2; k0 += TK) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int e = tid + 256 * q;
            As[e >> 4][e & 15] = ra[q];
            Bs[e / T][e % T] = rb[q];
        }
        __syncthreads();
        if (k0 + TK < K2) fetch(k0 + TK);
        const int np = (int)min((int64_t)TK, K2 - k0) / 2;
        for (int jj = 0; jj < np; ++jj) {
            double ae[R], ao[R], be[R], bo[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                ae[r] = As[ty + 16 * r][2 * jj];
                ao[r] = As[ty + 16 * r][2 * jj + 1];
            }
#pragma unroll
            for (int c = 0; c < R; ++c) {
                be[c] = Bs[2 * jj][tx + 16 * c];
                bo[c] = Bs[2 * jj + 1][tx + 16 * c];
            }
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < R; ++c) {
                    const double s1 = __dadd_rn(ae[r], bo[c]);
                    const double s2 = __dadd_rn(ao[r], be[c]);
                    acc[r][c] = fma(s1, s2, acc[r][c]);
                }
        }
    }
    const bool odd = (P & 1) != 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t i = i0 + ty + 16 * r;
        if (i >= N) continue;
        double yi = y[i];
        double alast = 0.0;
        const int ei = kRowCol ? ea[i] : 0;
        if (kScaled) yi = (yi * sa) * sa;
        if (odd) alast = kRowCol ? pow2_scale(A[i * lda + (P - 1)], -ei) : A[i * lda + (P - 1)] * sa;
#pragma unroll
        for (int c = 0; c < R; ++c) {
            const int64_t k = j0 + tx + 16 * c;
            if (k >= M) continue;
            double zk = z[k];
            if (kScaled) zk = (zk * sb) * sb;
            double v = __dsub_rn(__dsub_rn(acc[r][c], yi), zk);
            if (kRowCol) {
                const int fk = fb[k];
                if (odd) v = __dadd_rn(v, __dmul_rn(alast, pow2_scale(B[(P - 1) * ldb + k], -fk)));
                v = pow2_scale(v, ei + fk);
            } else if (odd) {
                v = __dadd_rn(v, __dmul_rn(alast, B[(P - 1) * ldb + k] * sb));
            }
            C[i * ldc + k] = v;
        }
    }
}

}  // namespace

namespace mm {

size_t winograd_ws_bytes(int64_t N, int64_t P, int64_t M, int mode) {
    (void)P;
    if (N < 0 || M < 0) return 0;
    const size_t yb = align_up((size_t)std::max<int64_t>(N, 1) * 8, 256);
    const size_t zb = align_up((size_t)std::max<int64_t>(M, 1) * 8, 256);
    size_t b = yb + zb;
    if (mode == 1) b += 256;  // the two norms
    if (mode == 2) b += align_up((size_t)std::max<int64_t>(N, 1) * 4, 256) + align_up((size_t)std::max<int64_t>(M, 1) * 4, 256);
    return b;
}

int run_winograd(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                 double *C, int64_t ldc, int mode, int32_t *lambda_out, void *ws, cudaStream_t st) {
    char *w = (char *)ws;
    const size_t yb = align_up((size_t)std::max<int64_t>(N, 1) * 8, 256);
    const size_t zb = align_up((size_t)std::max<int64_t>(M, 1) * 8, 256);
    double *y = (double *)w;
    double *z = (double *)(w + yb);
    double *norms = mode == 1 ? (double *)(w + yb + zb) : nullptr;
    int32_t *ea = mode == 2 ? (int32_t *)(w + yb + zb) : nullptr;
    int32_t *fb = mode == 2 ? (int32_t *)(w + yb + zb + align_up((size_t)std::max<int64_t>(N, 1) * 4, 256)) : nullptr;
    int rc;
    if (mode == 1) {
        cudaError_t e = cudaMemsetAsync(norms, 0, 2 * sizeof(double), st);
        if (e != cudaSuccess) return cuda_fail(e, "mm_winograd_scaled");
        if (P > 0) {
            // ||B||_inf into norms[1] (NormInf over the rows of B).
            rc = run_norm_inf(P, M, B, ldb, norms + 1, st);
            if (rc) return rc;
        }
    }
    {
        const int64_t nA = ceil_div(N, (int64_t)kRows), nB = ceil_div(M, (int64_t)32);
        const unsigned g = (unsigned)(nA + nB);
        unsigned long long *nb = mode == 1 ? (unsigned long long *)norms : nullptr;
        rc = launch(mode == 2 ? "winograd_terms_rowcol" : mode == 1 ? "winograd_terms_norm" : "winograd_terms", st,
                    [&] {
                        if (mode == 2)
                            terms_kernel<2><<<g, 32, 0, st>>>(N, P, M, A, lda, B, ldb, y, z, nb, ea, fb, nA);
                        else if (mode == 1)
                            terms_kernel<1><<<g, 32, 0, st>>>(N, P, M, A, lda, B, ldb, y, z, nb, ea, fb, nA);
                        else
                            terms_kernel<0><<<g, 32, 0, st>>>(N, P, M, A, lda, B, ldb, y, z, nb, ea, fb, nA);
                    });
        if (rc) return rc;
    }
    static const int sides[3] = {64, 32, 16};
    const int T = pick_tile(N, M, sides, 3);
    dim3 grid((unsigned)ceil_div(M, T), (unsigned)ceil_div(N, T));
    if (grid.y > 65535) return fail(MM_ERR_UNSUPPORTED, "mm_winograd: N too large for one launch");
    auto go = [&](auto mode) {
        constexpr int kM = decltype(mode)::value;
        const double *nm = kM == 1 ? norms : nullptr;
        int32_t *lo = kM == 1 ? lambda_out : nullptr;
        const int32_t *e1 = kM == 2 ? ea : nullptr, *f1 = kM == 2 ? fb : nullptr;
        if (T == 64)
            winograd_kernel<kM, 4><<<grid, 256, 0, st>>>(N, P, M, A, lda, B, ldb, C, ldc, y, z, nm, lo, e1, f1);
        else if (T == 32)
            winograd_kernel<kM, 2><<<grid, 256, 0, st>>>(N, P, M, A, lda, B, ldb, C, ldc, y, z, nm, lo, e1, f1);
        else
            winograd_kernel<kM, 1><<<grid, 256, 0, st>>>(N, P, M, A, lda, B, ldb, C, ldc, y, z, nm, lo, e1, f1);
    };
    if (mode == 1) return launch("winograd_scaled_f64", st, [&] { go(std::integral_constant<int, 1>{}); });
    if (mode == 2) return launch("winograd_rowcol_scaled_f64", st, [&] { go(std::integral_constant<int, 2>{}); });
    return launch("winograd_f64", st, [&] { go(std::integral_constant<int, 0>{}); });
}

}  // namespace mm
