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
// Same tiling as the Kahan kernel: 256 threads, each owning R x R outputs
// strided by 16 in a 16R x 16R tile (R = 4, 2 or 1 by the size of the grid),
// (aux, group) pairs in registers; FP64-pipe bound at 1 DMUL + 1 DADD per k per
// output plus 1 DADD per group.
#include <type_traits>

#include "common.cuh"

namespace {

constexpr int TK = 16;

template <int U, int R>
__global__ void __launch_bounds__(256) unrolled_kernel(int64_t N, int64_t P, int64_t M, const double *__restrict__ A,
                                                       int64_t lda, const double *__restrict__ B, int64_t ldb,
                                                       double *__restrict__ C, int64_t ldc) {
    constexpr int T = 16 * R;  // output tile side
    __shared__ double As[T][TK + 1];
    __shared__ double Bs[TK][T];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t i0 = (int64_t)blockIdx.y * T, j0 = (int64_t)blockIdx.x * T;
    const int64_t full = (P / U) * U;  // products that fall in complete groups
    double aux[R][R], grp[R][R];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c) aux[r][c] = grp[r][c] = 0.0;
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
    int t = 0;  // position of k inside its group (k mod U), the same in every thread
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
        if (k0 + TK <= full) {
            // A whole tile inside the complete groups: the position of each k in
            // its group is (t + kk) mod U with t the tile's starting phase, fixed
            // per phase at compile time, so no selects are issued.
            auto tile = [&](auto phase) {
                constexpr int T0 = decltype(phase)::value;
#pragma unroll
                for (int kk = 0; kk < TK; ++kk) {
                    double a[R], b[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) a[r] = As[ty + 16 * r][kk];
#pragma unroll
                    for (int c = 0; c < R; ++c) b[c] = Bs[kk][tx + 16 * c];
                    const int pos = (T0 + kk) % U;
#pragma unroll
                    for (int r = 0; r < R; ++r)
#pragma unroll
                        for (int c = 0; c < R; ++c) {
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
            double a[R], b[R];
#pragma unroll
            for (int r = 0; r < R; ++r) a[r] = As[ty + 16 * r][kk];
#pragma unroll
            for (int c = 0; c < R; ++c) b[c] = Bs[kk][tx + 16 * c];
            const bool grouped = k0 + kk < full;
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < R; ++c) {
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
    for (int r = 0; r < R; ++r) {
        const int64_t i = i0 + ty + 16 * r;
        if (i >= N) continue;
#pragma unroll
        for (int c = 0; c < R; ++c) {
            const int64_t j = j0 + tx + 16 * c;
            if (j < M) C[i * ldc + j] = aux[r][c];
        }
    }
}

}  // namespace

namespace mm {

template <int U>
int launch_unrolled(const char *name, int T, dim3 grid, int64_t N, int64_t P, int64_t M, const double *A, int64_t lda,
                    const double *B, int64_t ldb, double *C, int64_t ldc, cudaStream_t st) {
    return launch(name, st, [&] {
        if (T == 64)
            unrolled_kernel<U, 4><<<grid, 256, 0, st>>>(N, P, M, A, lda, B, ldb, C, ldc);
        else if (T == 32)
            unrolled_kernel<U, 2><<<grid, 256, 0, st>>>(N, P, M, A, lda, B, ldb, C, ldc);
        else
            unrolled_kernel<U, 1><<<grid, 256, 0, st>>>(N, P, M, A, lda, B, ldb, C, ldc);
    });
}

int run_unrolled(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                 double *C, int64_t ldc, int unroll, cudaStream_t st) {
    static const int sides[3] = {64, 32, 16};
    const int T = pick_tile(N, M, sides, 3);
    dim3 grid((unsigned)ceil_div(M, T), (unsigned)ceil_div(N, T));
    if (grid.y > 65535) return fail(MM_ERR_UNSUPPORTED, "mm_naive_unrolled: N too large for one launch");
    switch (unroll) {
    case 1:
        return launch_unrolled<1>("naive_ordered_f64", T, grid, N, P, M, A, lda, B, ldb, C, ldc, st);
    case 2:
        return launch_unrolled<2>("naive_unrolled2_f64", T, grid, N, P, M, A, lda, B, ldb, C, ldc, st);
    case 3:
        return launch_unrolled<3>("naive_unrolled3_f64", T, grid, N, P, M, A, lda, B, ldb, C, ldc, st);
    case 4:
        return launch_unrolled<4>("naive_unrolled4_f64", T, grid, N, P, M, A, lda, B, ldb, C, ldc, st);
    default:
        return fail(MM_ERR_ARG, "mm_naive_unrolled: unroll must be 1, 2, 3 or 4 (got %d)", unroll);
    }
}

}  // namespace mm
