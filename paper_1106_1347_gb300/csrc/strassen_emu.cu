// Strassen and Strassen-Winograd levels over the emulated FP64-accurate
// product (not in the paper: its recursion of sections "StrassenNaiv" and
// "StrassenWinograd" with the split product of emulated.cu as the base case).
//
// Definition (identical to the CPU oracle's): A and B are embedded in zero
// matrices whose sizes are the smallest multiples of 2^L >= N, P, M; each level
// forms the operands of H1..H7 with the FP64 additions of the paper's formulas
// and in their printed order, the 7^L products at the bottom are emulated
// products, and each level's C blocks are the printed sums of its H's, left to
// right.  Every step is deterministic, so the result is bit-identical to the
// oracle's.
//
// GB300 layout of the work: one elementwise kernel per node and operand side
// reads the node's four quadrants once and writes all of that side's operand
// sums (HBM-bound, one pass at about 0.8 of the copy bandwidth; forming the
// sums inside the split kernels instead measured slower, since the column
// split reads every operand twice and sums of up to four views cut the split
// kernels' memory parallelism); all 7^L base products run as ONE grouped
// emulated launch (persistent slice kernel over every leaf's tiles, so the
// tensor pipe sees 7^L x tiles of work at once rather than 7^L small
// launches); one elementwise kernel per internal node reads its seven H
// blocks once and writes its four C quadrants.  Operands that are plain quadrants are passed as views (the
// parent's leading dimension), never copied.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace {

// ---------------------------------------------------------------- kernels

// The operand sums of one level for one side (kSideA: the A side, else the B
// side) of one node whose operand X is 2h x 2w (leading dimension ldx).  Output
// k is the h x w matrix out + k * h * w (dense, leading dimension w).
//   Strassen, A side: S1 = A11 + A22, S2 = A21 + A22, S5 = A11 + A12, S6 = A21 - A11, S7 = A12 - A22.
//   Strassen, B side: T1 = B11 + B22, T3 = B12 - B22, T4 = B21 - B11, T6 = B11 + B12, T7 = B21 + B22.
//   Winograd, A side: A1 = A11 - A21, A2 = A22 - A1, S4 = A21 + A22, S6 = A12 - A2.
//   Winograd, B side: B1 = B22 - B12, B2 = B1 + B11, T4 = B12 - B11, T7 = B21 - B2.
template <int kVariant, bool kSideA>
__global__ void __launch_bounds__(256) operand_sums_kernel(const double *__restrict__ X, int64_t ldx, int64_t h,
                                                           int64_t w, double *__restrict__ out) {
    const int64_t hw = h * w;
    for (int64_t i = blockIdx.y; i < h; i += gridDim.y)
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < w; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i * w + j;
        const double x11 = X[i * ldx + j], x12 = X[i * ldx + w + j];
        const double x21 = X[(i + h) * ldx + j], x22 = X[(i + h) * ldx + w + j];
        if (kVariant == 0) {
            if (kSideA) {
                out[t] = __dadd_rn(x11, x22);
                out[hw + t] = __dadd_rn(x21, x22);
                out[2 * hw + t] = __dadd_rn(x11, x12);
                out[3 * hw + t] = __dsub_rn(x21, x11);
                out[4 * hw + t] = __dsub_rn(x12, x22);
            } else {
                out[t] = __dadd_rn(x11, x22);
                out[hw + t] = __dsub_rn(x12, x22);
                out[2 * hw + t] = __dsub_rn(x21, x11);
                out[3 * hw + t] = __dadd_rn(x11, x12);
                out[4 * hw + t] = __dadd_rn(x21, x22);
            }
        } else {
            if (kSideA) {
                const double a1 = __dsub_rn(x11, x21);
                const double a2 = __dsub_rn(x22, a1);
                out[t] = a1;
                out[hw + t] = a2;
                out[2 * hw + t] = __dadd_rn(x21, x22);
                out[3 * hw + t] = __dsub_rn(x12, a2);
            } else {
                const double b1 = __dsub_rn(x22, x12);
                const double b2 = __dadd_rn(b1, x11);
                out[t] = b1;
                out[hw + t] = b2;
                out[2 * hw + t] = __dsub_rn(x12, x11);
                out[3 * hw + t] = __dsub_rn(x21, b2);
            }
        }
    }
}

// C quadrants of one node from its seven h x w products H1..H7 (H_k at
// H + (k - 1) h w, dense):
//   Strassen: C11 = H1 + H4 - H5 + H7, C12 = H3 + H5, C21 = H2 + H4, C22 = H1 + H3 - H2 + H6;
//   Winograd: H8 = H1 + H3, H9 = H8 + H4; C11 = H1 + H2, C12 = H9 + H6, C21 = H8 + H5 + H7, C22 = H9 + H5.
template <int kVariant>
__global__ void __launch_bounds__(256) combine_kernel(const double *__restrict__ H, int64_t h, int64_t w,
                                                      double *__restrict__ C, int64_t ldc) {
    const int64_t hw = h * w;
    for (int64_t i = blockIdx.y; i < h; i += gridDim.y)
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < w; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i * w + j;
        const double h1 = H[t], h2 = H[hw + t], h3 = H[2 * hw + t], h4 = H[3 * hw + t], h5 = H[4 * hw + t],
                     h6 = H[5 * hw + t], h7 = H[6 * hw + t];
        double c11, c12, c21, c22;
        if (kVariant == 0) {
            c11 = __dadd_rn(__dsub_rn(__dadd_rn(h1, h4), h5), h7);
            c12 = __dadd_rn(h3, h5);
            c21 = __dadd_rn(h2, h4);
            c22 = __dadd_rn(__dsub_rn(__dadd_rn(h1, h3), h2), h6);
        } else {
            const double h8 = __dadd_rn(h1, h3), h9 = __dadd_rn(h8, h4);
            c11 = __dadd_rn(h1, h2);
            c12 = __dadd_rn(h9, h6);
            c21 = __dadd_rn(__dadd_rn(h8, h5), h7);
            c22 = __dadd_rn(h9, h5);
        }
        C[i * ldc + j] = c11;
        C[i * ldc + w + j] = c12;
        C[(i + h) * ldc + j] = c21;
        C[(i + h) * ldc + w + j] = c22;
    }
}

// ---------------------------------------------------------------- host plan

// Bump allocator over the workspace; with a null base it only counts bytes, so
// the size query and the run walk the same code.
struct Arena {
    char *base;
    size_t used = 0;
    char *take(size_t bytes) {
        used = mm::align_up(used, 4096);
        char *p = base ? base + used : nullptr;
        used += bytes;
        return p;
    }
};

struct View {
    const double *p;
    int64_t ld;
};

// One product of the recursion: out (leading dimension ldo) = a * b, at the
// level's size.  `kids` is where its children's H1..H7 live once expanded.
struct Node {
    View a, b;
    double *out;
    int64_t ldo;
    double *kids;
};

// Grid of an elementwise kernel over an h x w block: 256 columns per CTA in x,
// rows in y, about 16 CTAs per SM in all (the kernels stride over the rest).
dim3 elementwise_grid(int64_t h, int64_t w) {
    const int64_t gx = std::min<int64_t>(mm::ceil_div(std::max<int64_t>(w, 1), 256), 64);
    const int64_t gy = std::min<int64_t>(std::max<int64_t>(h, 1), std::max<int64_t>(1, 16 * mm::sm_count() / gx));
    return dim3((unsigned)gx, (unsigned)std::min<int64_t>(gy, 65535));
}

// Walks the plan; with dry == true nothing is launched and only `ar` grows.
int strassen_emulated_walk(bool dry, int variant, int levels, int64_t N, int64_t P, int64_t M, const double *A,
                           int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc, int s, int kind,
                           Arena &ar, cudaStream_t st) {
    const int64_t q = (int64_t)1 << levels;
    const int64_t Np = mm::ceil_div(N, q) * q, Pp = mm::ceil_div(P, q) * q, Mp = mm::ceil_div(M, q) * q;
    const bool pad = Np != N || Pp != P || Mp != M;
    View A0{A, lda}, B0{B, ldb};
    double *C0 = C;
    int64_t ldc0 = ldc;
    if (pad) {  // the zero embedding, as the definition states
        double *ap = (double *)ar.take((size_t)Np * Pp * 8);
        double *bp = (double *)ar.take((size_t)Pp * Mp * 8);
        C0 = (double *)ar.take((size_t)Np * Mp * 8);
        ldc0 = Mp;
        if (!dry) {
            cudaError_t e = cudaMemsetAsync(ap, 0, (size_t)Np * Pp * 8, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(bp, 0, (size_t)Pp * Mp * 8, st);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(ap, Pp * 8, A, lda * 8, P * 8, N, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(bp, Mp * 8, B, ldb * 8, M * 8, P, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return mm::cuda_fail(e, "mm_strassen_emulated: padding");
        }
        A0 = View{ap, Pp};
        B0 = View{bp, Mp};
    }
    const int nsa = variant == 0 ? 5 : 4, nsb = variant == 0 ? 5 : 4;
    std::vector<std::vector<Node>> tree(1, std::vector<Node>{Node{A0, B0, C0, ldc0, nullptr}});
    for (int j = 0; j < levels; ++j) {
        const int64_t h = (Np >> j) / 2, p2 = (Pp >> j) / 2, w = (Mp >> j) / 2;
        std::vector<Node> next;
        next.reserve(tree[j].size() * 7);
        for (Node &nd : tree[j]) {
            double *sa = (double *)ar.take((size_t)nsa * h * p2 * 8);
            double *sb = (double *)ar.take((size_t)nsb * p2 * w * 8);
            nd.kids = (double *)ar.take((size_t)7 * h * w * 8);
            if (!dry) {
                int rc = mm::launch("strassen_emu_operand_sums", st, [&] {
                    const dim3 ga = elementwise_grid(h, p2), gb = elementwise_grid(p2, w);
                    if (variant == 0) {
                        operand_sums_kernel<0, true><<<ga, 256, 0, st>>>(nd.a.p, nd.a.ld, h, p2, sa);
                        operand_sums_kernel<0, false><<<gb, 256, 0, st>>>(nd.b.p, nd.b.ld, p2, w, sb);
                    } else {
                        operand_sums_kernel<1, true><<<ga, 256, 0, st>>>(nd.a.p, nd.a.ld, h, p2, sa);
                        operand_sums_kernel<1, false><<<gb, 256, 0, st>>>(nd.b.p, nd.b.ld, p2, w, sb);
                    }
                });
                if (rc) return rc;
            }
            const View a11{nd.a.p, nd.a.ld}, a12{nd.a.p + p2, nd.a.ld}, a22{nd.a.p + h * nd.a.ld + p2, nd.a.ld};
            const View b11{nd.b.p, nd.b.ld}, b21{nd.b.p + p2 * nd.b.ld, nd.b.ld},
                b22{nd.b.p + p2 * nd.b.ld + w, nd.b.ld};
            auto S = [&](int k) { return View{sa + (size_t)k * h * p2, p2}; };
            auto T = [&](int k) { return View{sb + (size_t)k * p2 * w, w}; };
            View ao[7], bo[7];
            if (variant == 0) {  // H1..H7 of section "StrassenNaiv"
                ao[0] = S(0), bo[0] = T(0);
                ao[1] = S(1), bo[1] = b11;
                ao[2] = a11, bo[2] = T(1);
                ao[3] = a22, bo[3] = T(2);
                ao[4] = S(2), bo[4] = b22;
                ao[5] = S(3), bo[5] = T(3);
                ao[6] = S(4), bo[6] = T(4);
            } else {  // H1..H7 of section "StrassenWinograd"
                ao[0] = a11, bo[0] = b11;
                ao[1] = a12, bo[1] = b21;
                ao[2] = S(1), bo[2] = T(1);
                ao[3] = S(2), bo[3] = T(2);
                ao[4] = S(0), bo[4] = T(0);
                ao[5] = S(3), bo[5] = b22;
                ao[6] = a22, bo[6] = T(3);
            }
            for (int k = 0; k < 7; ++k) next.push_back(Node{ao[k], bo[k], nd.kids + (size_t)k * h * w, w, nullptr});
        }
        tree.push_back(std::move(next));
    }
    // Every base product in one grouped launch.
    const int64_t nl = Np >> levels, pl = Pp >> levels, ml = Mp >> levels;
    std::vector<mm_problem> probs;
    probs.reserve(tree[levels].size());
    for (const Node &nd : tree[levels])
        probs.push_back(mm_problem{nl, pl, ml, nd.a.p, nd.a.ld, nd.b.p, nd.b.ld, nd.out, nd.ldo});
    char *gws = ar.take(mm::emulated_group_ws_bytes(probs.data(), (int)probs.size(), s, kind));
    if (!dry) {
        int rc = mm::run_emulated_group(probs.data(), (int)probs.size(), s, kind, gws, st);
        if (rc) return rc;
        // Combine bottom-up: each internal node's C quadrants from its H1..H7.
        for (int j = levels - 1; j >= 0; --j) {
            const int64_t h = (Np >> j) / 2, w = (Mp >> j) / 2;
            for (const Node &nd : tree[j]) {
                rc = mm::launch("strassen_emu_combine", st, [&] {
                    const dim3 g = elementwise_grid(h, w);
                    if (variant == 0)
                        combine_kernel<0><<<g, 256, 0, st>>>(nd.kids, h, w, nd.out, nd.ldo);
                    else
                        combine_kernel<1><<<g, 256, 0, st>>>(nd.kids, h, w, nd.out, nd.ldo);
                });
                if (rc) return rc;
            }
        }
        if (pad) {
            cudaError_t e = cudaMemcpy2DAsync(C, ldc * 8, C0, ldc0 * 8, M * 8, N, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return mm::cuda_fail(e, "mm_strassen_emulated: result copy");
        }
    }
    return MM_OK;
}

}  // namespace

namespace mm {

// levels == -1: the level count that measured fastest on GB300 for 8 BF16
// slices, by the smallest dimension: none below 5120 (at 4096 one level ties),
// one up to 12288, two from there (5% faster than one at 16384).
int strassen_emulated_levels(int levels, int64_t N, int64_t P, int64_t M) {
    if (levels != -1) return levels;
    const int64_t n = std::min(N, std::min(P, M));
    return n < 5120 ? 0 : n < 12288 ? 1 : 2;
}

size_t strassen_emulated_ws_bytes(int variant, int levels, int64_t N, int64_t P, int64_t M, int s, int kind) {
    Arena ar{nullptr};
    if (strassen_emulated_walk(true, variant, levels, N, P, M, nullptr, 1, nullptr, 1, nullptr, 1, s, kind, ar,
                               nullptr) != MM_OK)
        return 0;
    return ar.used + 4096;  // the caller's pointer is aligned up to 4096 bytes first
}

int run_strassen_emulated(int variant, int levels, int64_t N, int64_t P, int64_t M, const double *A, int64_t lda,
                          const double *B, int64_t ldb, double *C, int64_t ldc, int s, int kind, void *ws,
                          cudaStream_t st) {
    char *base = (char *)align_up((size_t)(uintptr_t)ws, 4096);
    Arena ar{base};
    return strassen_emulated_walk(false, variant, levels, N, P, M, A, lda, B, ldb, C, ldc, s, kind, ar, st);
}

}  // namespace mm
