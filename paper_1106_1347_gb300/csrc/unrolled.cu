// Sections "NaivStandard", "NaivOnArray" and "Loop unrolling": the naive sum
// C_ij = sum_k RN(A_ik B_kj) in the paper's own evaluation orders.
//   u = 1: aux = aux + x_k for k in order (NaivStandard; NaivOnArray
//          accumulates in C itself and rounds identically);
//   u = 2, 3, 4: aux = aux + ((x_uk-u+1 + x_uk-u+2) + ...), the u products of
//          a group summed left to right first, then the P mod u leftover
//          products added one by one (NaivLoopUnrollingTwo/Three/Four).
// __dmul_rn/__dadd_rn keep every product and sum rounded on its own (no
// contraction), so the result is bit-identical to the sequential CPU
// evaluation.  The grouping exists in the paper to cut loop overhead on a CPU;
// here it only fixes the rounding order, and the plain FP64 product
// (mm_naive, DMMA) is the fast path.
//
// Same tiling as the Kahan kernel: 64x64 output tile, 256 threads, each owning
// 4x4 outputs strided by 16, (aux, group) pairs in registers; FP64-pipe bound at
// 1 DMUL + 1 DADD per k per output plus 1 DADD per group.
#include <type_traits>

#include "common.cuh"

namespace {

constexpr int TM = 64, TN = 64, TK = 16;

template <int U>
__global__ void __launch_bounds__(256) unrolled_kernel(int64_t N, int64_t P, int64_t M, const double *__restrict__ A,
                                                       int64_t lda, const double *__restrict__ B, int64_t ldb,
                                                       double *__restrict__ C, int64_t ldc) {
    __shared__ double As[TM][TK + 1];
    __shared__ double Bs[TK][TN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t i0 = (int64_t)blockIdx.y * TM, j0 = (int64_t)blockIdx.x * TN;
    const int64_t full = (P / U) * U;  // products that fall in complete groups
    double aux[4][4], grp[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) aux[r][c] = grp[r][c] = 0.0;
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
    int t = 0;  // position of k inside its group (k mod U), the same in every thread
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
        if (k0 + TK <= full) {
            // A whole tile inside the complete groups: the position of each k in
            // its group is (t + kk) mod U with t the tile's starting phase, fixed
            // per phase at compile time, so no selects are issued.
            auto tile = [&](auto phase) {
                constexpr int T0 = decltype(phase)::value;
#pragma unroll
                for (int kk = 0; kk < TK; ++kk) {
                    double a[4], b[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) a[r] = As[ty + 16 * r][kk];
#pragma unroll
                    for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
                    const int pos = (T0 + kk) % U;
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const double x = __dmul_rn(a[r], b[c]);
                            if (U == 1) {
                                aux[r][c] = __dadd_rn(aux[r][c], x);
                            } else {
                                grp[r][c] = pos == 0 ? x : __dadd_rn(grp[r][c], x);
                                if (pos == U - 1) aux[r][c] = __dadd_rn(aux[r][c], grp[r][c]);
                            }
                        }
                }
            };
            if (U == 3 && t == 1)
                tile(std::integral_constant<int, 1>{});
            else if (U == 3 && t == 2)
                tile(std::integral_constant<int, 2>{});
            else
                tile(std::integral_constant<int, 0>{});
            t = (t + TK) % U;
            continue;
        }
        for (int kk = 0; kk < kn; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[ty + 16 * r][kk];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
            const bool grouped = k0 + kk < full;
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const double x = __dmul_rn(a[r], b[c]);
                    if (U == 1 || !grouped) {
                        aux[r][c] = __dadd_rn(aux[r][c], x);
                    } else {
                        grp[r][c] = t == 0 ? x : __dadd_rn(grp[r][c], x);
                        if (t == U - 1) aux[r][c] = __dadd_rn(aux[r][c], grp[r][c]);
                    }
                }
            if (U > 1) t = t + 1 == U ? 0 : t + 1;
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t i = i0 + ty + 16 * r;
        if (i >= N) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t j = j0 + tx + 16 * c;
            if (j < M) C[i * ldc + j] = aux[r][c];
        }
    }
}

}  // namespace

namespace mm {

int run_unrolled(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                 double *C, int64_t ldc, int unroll, cudaStream_t st) {
    dim3 grid((unsigned)ceil_div(M, TN), (unsigned)ceil_div(N, TM));
    if (grid.y > 65535) return fail(MM_ERR_UNSUPPORTED, "mm_naive_unrolled: N too large for one launch");
    switch (unroll) {
    case 1:
        return launch("naive_ordered_f64", st,
                      [&] { unrolled_kernel<1><<<grid, 256, 0, st>>>(N, P, M, A, lda, B, ldb, C, ldc); });
    case 2:
        return launch("naive_unrolled2_f64", st,
                      [&] { unrolled_kernel<2><<<grid, 256, 0, st>>>(N, P, M, A, lda, B, ldb, C, ldc); });
    case 3:
        return launch("naive_unrolled3_f64", st,
                      [&] { unrolled_kernel<3><<<grid, 256, 0, st>>>(N, P, M, A, lda, B, ldb, C, ldc); });
    case 4:
        return launch("naive_unrolled4_f64", st,
                      [&] { unrolled_kernel<4><<<grid, 256, 0, st>>>(N, P, M, A, lda, B, ldb, C, ldc); });
    default:
        return fail(MM_ERR_ARG, "mm_naive_unrolled: unroll must be 1, 2, 3 or 4 (got %d)", unroll);
    }
}

}  // namespace mm
