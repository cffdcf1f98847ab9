// Section "NaivKahan": every C_ij is the sum over k = 0..P-1, in order, of
// x = RN(A_ik B_kj) with the paper's compensated update
//   err = err + x;  t = sum + err;  err = (sum - t) + err;  sum = t.
// Written with __dmul_rn/__dadd_rn/__dsub_rn so nothing is contracted: the
// result is bit-identical to the sequential CPU evaluation.  The sequence
// stops at k = P-1 exactly (an extra zero term would fold err into sum).
//
// Warp-tiled CUDA-core kernel: 64x64 output tile, 256 threads, each owning a
// 4x4 set of outputs strided by 16 (so shared-memory reads of B are
// conflict-free and A reads are broadcasts, and stores are coalesced), with
// the (sum, err) pairs in registers.  Bound by the FP64 pipe: 1 DMUL + 4 DADD
// per k per output.
#include "common.cuh"

namespace {

constexpr int TM = 64, TN = 64, TK = 16;

__global__ void __launch_bounds__(256) kahan_kernel(int64_t N, int64_t P, int64_t M, const double *__restrict__ A,
                                                    int64_t lda, const double *__restrict__ B, int64_t ldb,
                                                    double *__restrict__ C, int64_t ldc) {
    __shared__ double As[TM][TK + 1];
    __shared__ double Bs[TK][TN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t i0 = (int64_t)blockIdx.y * TM, j0 = (int64_t)blockIdx.x * TN;
    double sum[4][4], err[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) sum[r][c] = err[r][c] = 0.0;
    double ra[4], rb[4];
    auto fetch = [&](int64_t k0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            const int64_t gi = i0 + (e >> 4), gk = k0 + (e & 15);
            ra[q] = (gi < N && gk < P) ? A[gi * lda + gk] : 0.0;
            const int64_t bk = k0 + (e >> 6), bj = j0 + (e & 63);
            rb[q] = (bk < P && bj < M) ? B[bk * ldb + bj] : 0.0;
        }
    };
    fetch(0);
    for (int64_t k0 = 0; k0 < P; k0 += TK) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            As[e >> 4][e & 15] = ra[q];
            Bs[e >> 6][e & 63] = rb[q];
        }
        __syncthreads();
        if (k0 + TK < P) fetch(k0 + TK);
        const int kn = (int)min((int64_t)TK, P - k0);
        for (int kk = 0; kk < kn; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[ty + 16 * r][kk];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const double x = __dmul_rn(a[r], b[c]);
                    double e = __dadd_rn(err[r][c], x);
                    const double t = __dadd_rn(sum[r][c], e);
                    err[r][c] = __dadd_rn(__dsub_rn(sum[r][c], t), e);
                    sum[r][c] = t;
                }
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t i = i0 + ty + 16 * r;
        if (i >= N) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t j = j0 + tx + 16 * c;
            if (j < M) C[i * ldc + j] = sum[r][c];
        }
    }
}

}  // namespace

namespace mm {

int run_kahan(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
              int64_t ldc, cudaStream_t st) {
    dim3 grid((unsigned)ceil_div(M, TN), (unsigned)ceil_div(N, TM));
    if (grid.y > 65535) return fail(MM_ERR_UNSUPPORTED, "mm_kahan: N too large for one launch");
    return launch("kahan_f64", st, [&] { kahan_kernel<<<grid, 256, 0, st>>>(N, P, M, A, lda, B, ldb, C, ldc); });
}

}  // namespace mm
