// Section "NaivKahan": every C_ij is the sum over k = 0..P-1, in order, of
// x = RN(A_ik B_kj) with the paper's compensated update
//   err = err + x;  t = sum + err;  err = (sum - t) + err;  sum = t.
// Written with __dmul_rn/__dadd_rn/__dsub_rn so nothing is contracted: the
// result is bit-identical to the sequential CPU evaluation.  The sequence
// stops at k = P-1 exactly (an extra zero term would fold err into sum).
//
// Warp-tiled CUDA-core kernel: 256 threads in a 16 x 16 layout, each owning
// R x R outputs strided by 16 (so shared-memory reads of B are conflict-free,
// A reads are broadcasts and stores are coalesced), with the (sum, err) pairs
// in registers; the output tile is 16R x 16R with R = 4, 2 or 1, the largest
// whose grid still fills the SMs (small products take small tiles).  Bound by
// the FP64 pipe: 1 DMUL + 4 DADD per k per output.
#include "common.cuh"

namespace {

constexpr int TK = 16;

template <int R>
__global__ void __launch_bounds__(256) kahan_kernel(int64_t N, int64_t P, int64_t M, const double *__restrict__ A,
                                                    int64_t lda, const double *__restrict__ B, int64_t ldb,
                                                    double *__restrict__ C, int64_t ldc) {
    constexpr int T = 16 * R;  // output tile side
    __shared__ double As[T][TK + 1];
    __shared__ double Bs[TK][T];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t i0 = (int64_t)blockIdx.y * T, j0 = (int64_t)blockIdx.x * T;
    double sum[R][R], err[R][R];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c) sum[r][c] = err[r][c] = 0.0;
    double ra[R], rb[R];
    auto fetch = [&](int64_t k0) {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int e = tid + 256 * q;
            const int64_t gi = i0 + (e >> 4), gk = k0 + (e & 15);
            ra[q] = (gi < N && gk < P) ? A[gi * lda + gk] : 0.0;
            const int64_t bk = k0 + e / T, bj = j0 + e % T;
            rb[q] = (bk < P && bj < M) ? B[bk * ldb + bj] : 0.0;
        }
    };
    fetch(0);
    for (int64_t k0 = 0; k0 < P; k0 += TK) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int e = tid + 256 * q;
            As[e >> 4][e & 15] = ra[q];
            Bs[e / T][e % T] = rb[q];
        }
        __syncthreads();
        if (k0 + TK < P) fetch(k0 + TK);
        const int kn = (int)min((int64_t)TK, P - k0);
        for (int kk = 0; kk < kn; ++kk) {
            double a[R], b[R];
#pragma unroll
            for (int r = 0; r < R; ++r) a[r] = As[ty + 16 * r][kk];
#pragma unroll
            for (int c = 0; c < R; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < R; ++c) {
                    const double x = __dmul_rn(a[r], b[c]);
                    double e = __dadd_rn(err[r][c], x);
                    const double t = __dadd_rn(sum[r][c], e);
                    err[r][c] = __dadd_rn(__dsub_rn(sum[r][c], t), e);
                    sum[r][c] = t;
                }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t i = i0 + ty + 16 * r;
        if (i >= N) continue;
#pragma unroll
        for (int c = 0; c < R; ++c) {
            const int64_t j = j0 + tx + 16 * c;
            if (j < M) C[i * ldc + j] = sum[r][c];
        }
    }
}

}  // namespace

namespace mm {

int run_kahan(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
              int64_t ldc, cudaStream_t st) {
    static const int sides[3] = {64, 32, 16};
    const int T = pick_tile(N, M, sides, 3);
    dim3 grid((unsigned)ceil_div(M, T), (unsigned)ceil_div(N, T));
    if (grid.y > 65535) return fail(MM_ERR_UNSUPPORTED, "mm_kahan: N too large for one launch");
    return launch("kahan_f64", st, [&] {
        if (T == 64)
            kahan_kernel<4><<<grid, 256, 0, st>>>(N, P, M, A, lda, B, ldb, C, ldc);
        else if (T == 32)
            kahan_kernel<2><<<grid, 256, 0, st>>>(N, P, M, A, lda, B, ldb, C, ldc);
        else
            kahan_kernel<1><<<grid, 256, 0, st>>>(N, P, M, A, lda, B, ldb, C, ldc);
    });
}

}  // namespace mm
