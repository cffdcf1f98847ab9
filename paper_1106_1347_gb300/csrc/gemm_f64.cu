// FP64 base product on the FP64 tensor-core MMA (mma.sync m8n8k4 f64), and
// the Strassen / Strassen-Winograd recursion built on it.
//
// One kernel, `level_kernel`, computes a list of products
//   H_h = (expression over quadrants of A) x (expression over quadrants of B)
// and folds each into up to four C quadrants, C_q := +-H_h (first touch) or
// C_q := C_q +- H_h, in list order.  With one product and no quadrants it is
// the naive method (section "The naive method"); with the seven products of
// section "StrassenNaiv" or "StrassenWinograd" it is one recursion level whose
// Plus/Minus operand sums are formed while tiles are staged into shared
// memory and whose C-block sums are formed in the epilogue -- no separate
// elementwise pass touches HBM.  Each CTA owns the same output tile of all
// four C quadrants and walks the products in an order that reproduces the
// paper's left-to-right sums:
//   Strassen:  H1 H3 H2 H4 H5 H6 H7 gives C11 = ((H1+H4)-H5)+H7, C12 = H3+H5,
//              C21 = H2+H4, C22 = ((H1+H3)-H2)+H6;
//   Winograd:  H1..H7 gives C11 = H1+H2, C12 = ((H1+H3)+H4)+H6 = H9+H6,
//              C21 = ((H1+H3)+H5)+H7 = (H8+H5)+H7, C22 = ((H1+H3)+H4)+H5 = H9+H5.
// Padding to the recursion's sizes is virtual: reads outside an operand's
// valid region return zero, writes outside C's region are dropped.  Grid z
// walks a batch of equal-size nodes laid out at fixed strides, so one launch
// runs the fused level of every node of a recursion level (strassen.cu drives
// the levels above it).
//
// Tiling: 64x64 output tile (32x32 or 16x16 when that leaves SMs idle), K-step 16,
// 4 warps each owning a quarter as 8x8x4 MMA tiles.  The kernel is bound by the FP64 pipe: on GB300 the
// m8n8k4 f64 MMA and DFMA both measure ~1.06 TFLOP/s, and the MMA needs 16x
// fewer instructions.  At that rate the loads do not matter, so operand tiles
// are staged with plain coalesced loads into padded, bank-conflict-free shared
// memory (the expression evaluation happens in those loads), prefetched one
// K-step ahead.
#include <vector>

#include "common.cuh"

namespace {

constexpr int BK = 16;
constexpr int AST = BK + 4;  // A tile row stride (doubles): conflict-free fragment reads

enum : uint8_t { T11 = 0, T12 = 1, T21 = 2, T22 = 3 };

// An operand sum as one of the seven tree shapes the paper's schedules use,
// with op[i] = +1 (Plus) or -1 (Minus); each node is rounded as the paper's
// Plus/Minus matrices are:
//   S1: t0                        S2: t0 o0 t1
//   S3: t0 o0 (t1 o1 t2)          S4: (t0 o0 t1) o1 t2
//   S5: t0 o0 (t1 o1 (t2 o2 t3))  S6: t0 o0 ((t1 o1 t2) o2 t3)
//   S7: ((t0 o0 t1) o1 t2) o2 t3
// Fixed shapes keep the evaluation in registers (no indexed stack).
struct Expr {
    uint8_t shape;
    uint8_t term[4];
    int8_t op[3];
};
struct Target {
    uint8_t quad;
    int8_t sign;
    uint8_t first;
};
struct Product {
    Expr a, b;
    uint8_t ntgt;
    Target tgt[4];
};
struct View {
    const double *p;
    int64_t ld, rows, cols;
};
struct LevelArgs {
    View A, B;
    double *C;
    int64_t ldc, crows, ccols;
    int64_t n, p, m;  // product size: H is n x m with inner dimension p (quadrant size for a level)
    int64_t za, zb, zc;  // element offsets from one node to the next (grid z walks nodes)
    int nprod;
    Product prod[7];
};

__device__ __forceinline__ double view_at(const View &v, int64_t r, int64_t c) {
    return (r < v.rows && c < v.cols) ? v.p[r * v.ld + c] : 0.0;
}

__device__ __forceinline__ double pm(double x, int8_t op, double y) {
    return op > 0 ? __dadd_rn(x, y) : __dsub_rn(x, y);
}

// Evaluates the shape on already loaded terms v[0..3].
__device__ __forceinline__ double eval_shape(const Expr &e, const double (&v)[4]) {
    switch (e.shape) {
        case 1: return v[0];
        case 2: return pm(v[0], e.op[0], v[1]);
        case 3: return pm(v[0], e.op[0], pm(v[1], e.op[1], v[2]));
        case 4: return pm(pm(v[0], e.op[0], v[1]), e.op[1], v[2]);
        case 5: return pm(v[0], e.op[0], pm(v[1], e.op[1], pm(v[2], e.op[2], v[3])));
        case 6: return pm(v[0], e.op[0], pm(pm(v[1], e.op[1], v[2]), e.op[2], v[3]));
        default: return pm(pm(pm(v[0], e.op[0], v[1]), e.op[1], v[2]), e.op[2], v[3]);
    }
}

__device__ __forceinline__ int expr_terms(const Expr &e) {
    return e.shape == 1 ? 1 : e.shape == 2 ? 2 : (e.shape == 3 || e.shape == 4) ? 3 : 4;
}

// Operand element (r, c) of the expression over quadrants of v; quadrant t
// sits at row offset (t >> 1) * rstep and column offset (t & 1) * cstep.
__device__ __forceinline__ double eval_expr(const Expr &e, const View &v, int64_t r, int64_t c, int64_t rstep,
                                            int64_t cstep) {
    double x[4] = {0.0, 0.0, 0.0, 0.0};
    const int nt = expr_terms(e);
#pragma unroll
    for (int t = 0; t < 4; ++t)
        if (t < nt) x[t] = view_at(v, r + (e.term[t] >> 1) * rstep, c + (e.term[t] & 1) * cstep);
    return eval_shape(e, x);
}

__device__ __forceinline__ void dmma_8x8x4(double (&c)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(c[0]), "+d"(c[1])
                 : "d"(a), "d"(b));
}

// BM x BN output tile per CTA of 4 warps (2 x 2), each warp owning
// (BM/2) x (BN/2) as MI x NI MMA tiles of 8 x 8: 64 x 64 for large grids,
// 32 x 32 or 16 x 16 when a larger tile's grid would leave SMs idle.
template <bool kSingle, int BM, int BN>
__global__ void __launch_bounds__(128) level_kernel(const __grid_constant__ LevelArgs args) {
    constexpr int BST = BN + 4;  // B tile row stride
    constexpr int MI = BM / 16, NI = BN / 16, RA = BM * BK / 128, RB = BK * BN / 128;
    __shared__ __align__(16) double As[BM][AST];
    __shared__ __align__(16) double Bs[BK][BST];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int g = lane >> 2, t4 = lane & 3;
    const int64_t i0 = (int64_t)blockIdx.y * BM, j0 = (int64_t)blockIdx.x * BN;
    const int64_t n = args.n, p = args.p, m = args.m;
    View Av = args.A, Bv = args.B;
    Av.p += (int64_t)blockIdx.z * args.za;
    Bv.p += (int64_t)blockIdx.z * args.zb;
    double *const Cz = args.C + (int64_t)blockIdx.z * args.zc;

    for (int pi = 0; pi < args.nprod; ++pi) {
        const Product &pr = args.prod[pi];
        double acc[MI][NI][2];
#pragma unroll
        for (int a = 0; a < MI; ++a)
#pragma unroll
            for (int b = 0; b < NI; ++b) acc[a][b][0] = acc[a][b][1] = 0.0;
        double ra[RA], rb[RB];
        auto fetch = [&](int64_t k0) {
#pragma unroll
            for (int r = 0; r < RA; ++r) {
                const int e = tid + 128 * r;
                const int64_t gi = i0 + (e >> 4), gk = k0 + (e & 15);
                double v = 0.0;
                if (gi < n && gk < p) {
                    if (kSingle)
                        v = view_at(Av, gi, gk);
                    else
                        v = eval_expr(pr.a, Av, gi, gk, n, p);
                }
                ra[r] = v;
            }
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                const int e = tid + 128 * r;
                const int64_t gk = k0 + e / BN, gj = j0 + e % BN;
                double v = 0.0;
                if (gk < p && gj < m) {
                    if (kSingle)
                        v = view_at(Bv, gk, gj);
                    else
                        v = eval_expr(pr.b, Bv, gk, gj, p, m);
                }
                rb[r] = v;
            }
        };
        fetch(0);
        for (int64_t k0 = 0; k0 < p; k0 += BK) {
            __syncthreads();
#pragma unroll
            for (int r = 0; r < RA; ++r) {
                const int e = tid + 128 * r;
                As[e >> 4][e & 15] = ra[r];
            }
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                const int e = tid + 128 * r;
                Bs[e / BN][e % BN] = rb[r];
            }
            __syncthreads();
            if (k0 + BK < p) fetch(k0 + BK);
#pragma unroll
            for (int kk = 0; kk < BK; kk += 4) {
                double af[MI], bf[NI];
#pragma unroll
                for (int mi = 0; mi < MI; ++mi) af[mi] = As[wm * (BM / 2) + mi * 8 + g][kk + t4];
#pragma unroll
                for (int ni = 0; ni < NI; ++ni) bf[ni] = Bs[kk + t4][wn * (BN / 2) + ni * 8 + g];
#pragma unroll
                for (int mi = 0; mi < MI; ++mi)
#pragma unroll
                    for (int ni = 0; ni < NI; ++ni) dmma_8x8x4(acc[mi][ni], af[mi], bf[ni]);
            }
        }
        // Epilogue: fold +-H into each target quadrant (vectorised when aligned).
        for (int ti = 0; ti < pr.ntgt; ++ti) {
            const Target tg = pr.tgt[ti];
            const int64_t roff = (tg.quad >> 1) * n, coff = (tg.quad & 1) * m;
            const double sgn = (double)tg.sign;
#pragma unroll
            for (int mi = 0; mi < MI; ++mi) {
                const int64_t row = i0 + wm * (BM / 2) + mi * 8 + g;
                const int64_t crow = row + roff;
                if (row >= n || crow >= args.crows) continue;
#pragma unroll
                for (int ni = 0; ni < NI; ++ni) {
                    const int64_t col = j0 + wn * (BN / 2) + ni * 8 + 2 * t4;
                    const int64_t ccol = col + coff;
                    double *dst = Cz + crow * args.ldc + ccol;
                    const double v0 = sgn * acc[mi][ni][0], v1 = sgn * acc[mi][ni][1];
                    const bool ok0 = col < m && ccol < args.ccols;
                    const bool ok1 = col + 1 < m && ccol + 1 < args.ccols;
                    if (ok0 && ok1 && (((uintptr_t)dst & 15) == 0)) {
                        double2 o;
                        if (tg.first) {
                            o = make_double2(v0, v1);
                        } else {
                            const double2 c = *reinterpret_cast<const double2 *>(dst);
                            o = make_double2(__dadd_rn(c.x, v0), __dadd_rn(c.y, v1));
                        }
                        *reinterpret_cast<double2 *>(dst) = o;
                    } else {
                        if (ok0) dst[0] = tg.first ? v0 : __dadd_rn(dst[0], v0);
                        if (ok1) dst[1] = tg.first ? v1 : __dadd_rn(dst[1], v1);
                    }
                }
            }
        }
    }
}

constexpr int8_t P_ = 1, M_ = -1;  // Plus, Minus
Expr E1(uint8_t t0) { return Expr{1, {t0, 0, 0, 0}, {0, 0, 0}}; }
Expr E2(uint8_t t0, int8_t o0, uint8_t t1) { return Expr{2, {t0, t1, 0, 0}, {o0, 0, 0}}; }
Expr E3(uint8_t t0, int8_t o0, uint8_t t1, int8_t o1, uint8_t t2) {  // t0 o0 (t1 o1 t2)
    return Expr{3, {t0, t1, t2, 0}, {o0, o1, 0}};
}
Expr E4(uint8_t t0, int8_t o0, uint8_t t1, int8_t o1, uint8_t t2) {  // (t0 o0 t1) o1 t2
    return Expr{4, {t0, t1, t2, 0}, {o0, o1, 0}};
}
Expr E5(uint8_t t0, int8_t o0, uint8_t t1, int8_t o1, uint8_t t2, int8_t o2, uint8_t t3) {
    return Expr{5, {t0, t1, t2, t3}, {o0, o1, o2}};  // t0 o0 (t1 o1 (t2 o2 t3))
}
Expr E6(uint8_t t0, int8_t o0, uint8_t t1, int8_t o1, uint8_t t2, int8_t o2, uint8_t t3) {
    return Expr{6, {t0, t1, t2, t3}, {o0, o1, o2}};  // t0 o0 ((t1 o1 t2) o2 t3)
}
Expr E7(uint8_t t0, int8_t o0, uint8_t t1, int8_t o1, uint8_t t2, int8_t o2, uint8_t t3) {
    return Expr{7, {t0, t1, t2, t3}, {o0, o1, o2}};  // ((t0 o0 t1) o1 t2) o2 t3
}
Target tgt(uint8_t q, int s, bool first) { return Target{q, (int8_t)s, (uint8_t)(first ? 1 : 0)}; }

// One recursion level of section "StrassenNaiv", in the order H1 H3 H2 H4 H5 H6 H7.
void strassen_products(Product (&pr)[7]) {
    pr[0] = Product{E2(T11, P_, T22), E2(T11, P_, T22), 2, {tgt(T11, 1, true), tgt(T22, 1, true)}};
    pr[1] = Product{E1(T11), E2(T12, M_, T22), 2, {tgt(T12, 1, true), tgt(T22, 1, false)}};
    pr[2] = Product{E2(T21, P_, T22), E1(T11), 2, {tgt(T21, 1, true), tgt(T22, -1, false)}};
    pr[3] = Product{E1(T22), E2(T21, M_, T11), 2, {tgt(T11, 1, false), tgt(T21, 1, false)}};
    pr[4] = Product{E2(T11, P_, T12), E1(T22), 2, {tgt(T11, -1, false), tgt(T12, 1, false)}};
    pr[5] = Product{E2(T21, M_, T11), E2(T11, P_, T12), 1, {tgt(T22, 1, false)}};
    pr[6] = Product{E2(T12, M_, T22), E2(T21, P_, T22), 1, {tgt(T11, 1, false)}};
}

// One recursion level of section "StrassenWinograd", H1..H7, with
// A1 = A11-A21, A2 = A22-A1, B1 = B22-B12, B2 = B1+B11 written out per use.
void strassen_winograd_products(Product (&pr)[7]) {
    pr[0] = Product{E1(T11), E1(T11), 4,
                    {tgt(T11, 1, true), tgt(T12, 1, true), tgt(T21, 1, true), tgt(T22, 1, true)}};
    pr[1] = Product{E1(T12), E1(T21), 1, {tgt(T11, 1, false)}};
    // A2 = A22 - (A11 - A21), B2 = (B22 - B12) + B11
    pr[2] = Product{E3(T22, M_, T11, M_, T21), E4(T22, M_, T12, P_, T11), 3,
                    {tgt(T12, 1, false), tgt(T21, 1, false), tgt(T22, 1, false)}};
    pr[3] = Product{E2(T21, P_, T22), E2(T12, M_, T11), 2, {tgt(T12, 1, false), tgt(T22, 1, false)}};
    pr[4] = Product{E2(T11, M_, T21), E2(T22, M_, T12), 2, {tgt(T21, 1, false), tgt(T22, 1, false)}};
    // A12 - A2 = A12 - (A22 - (A11 - A21))
    pr[5] = Product{E5(T12, M_, T22, M_, T11, M_, T21), E1(T22), 1, {tgt(T12, 1, false)}};
    // B21 - B2 = B21 - ((B22 - B12) + B11)
    pr[6] = Product{E1(T22), E6(T21, M_, T22, M_, T12, P_, T11), 1, {tgt(T21, 1, false)}};
}

int launch_level(const LevelArgs &a, bool single, cudaStream_t st, int64_t nodes = 1) {
    if (a.m <= 0 || a.n <= 0 || nodes <= 0) return MM_OK;
    // 64 x 64, 32 x 32 or 16 x 16 tiles: the side whose grid fills the SMs best.
    static const int sides[3] = {64, 32, 16};
    const int tile = mm::pick_tile(a.n, a.m, sides, 3, nodes);
    dim3 grid((unsigned)mm::ceil_div(a.m, tile), (unsigned)mm::ceil_div(a.n, tile), (unsigned)nodes);
    if (grid.y > 65535 || nodes > 65535) return mm::fail(MM_ERR_UNSUPPORTED, "product too tall for one launch");
    if (single)
        return mm::launch("gemm_f64_dmma", st, [&] {
            if (tile == 64)
                level_kernel<true, 64, 64><<<grid, 128, 0, st>>>(a);
            else if (tile == 32)
                level_kernel<true, 32, 32><<<grid, 128, 0, st>>>(a);
            else
                level_kernel<true, 16, 16><<<grid, 128, 0, st>>>(a);
        });
    return mm::launch("strassen_level_dmma", st, [&] {
        if (tile == 64)
            level_kernel<false, 64, 64><<<grid, 128, 0, st>>>(a);
        else if (tile == 32)
            level_kernel<false, 32, 32><<<grid, 128, 0, st>>>(a);
        else
            level_kernel<false, 16, 16><<<grid, 128, 0, st>>>(a);
    });
}

}  // namespace

namespace mm {

int run_naive(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
              int64_t ldc, cudaStream_t st) {
    LevelArgs a{};
    a.A = View{A, lda, N, P};
    a.B = View{B, ldb, P, M};
    a.C = C;
    a.ldc = ldc;
    a.crows = N;
    a.ccols = M;
    a.n = N;
    a.p = P;
    a.m = M;
    a.nprod = 1;
    a.prod[0] = Product{E1(T11), E1(T11), 1, {tgt(T11, 1, true)}};
    return launch_level(a, true, st);
}

// One fused recursion level for `nodes` equal-size nodes: node z's A operand
// (2n x 2p, leading dimension lda, reads at or past arows x acols return 0) sits
// at A + z za, its B operand (2p x 2m) at B + z zb, and its C (2n x 2m, writes
// at or past crows x ccols dropped) at C + z zc.
int run_strassen_level(int variant, int64_t nodes, int64_t n, int64_t p, int64_t m, const double *A, int64_t lda,
                       int64_t arows, int64_t acols, int64_t za, const double *B, int64_t ldb, int64_t brows,
                       int64_t bcols, int64_t zb, double *C, int64_t ldc, int64_t crows, int64_t ccols, int64_t zc,
                       cudaStream_t st) {
    LevelArgs a{};
    a.A = View{A, lda, arows, acols};
    a.B = View{B, ldb, brows, bcols};
    a.C = C;
    a.ldc = ldc;
    a.crows = crows;
    a.ccols = ccols;
    a.n = n;
    a.p = p;
    a.m = m;
    a.za = za;
    a.zb = zb;
    a.zc = zc;
    a.nprod = 7;
    if (variant == 0)
        strassen_products(a.prod);
    else
        strassen_winograd_products(a.prod);
    for (int64_t z0 = 0; z0 < nodes; z0 += 65535) {  // grid z holds at most 65535 nodes per launch
        LevelArgs b = a;
        b.A.p = A + z0 * za;
        b.B.p = B + z0 * zb;
        b.C = C + z0 * zc;
        const int rc = launch_level(b, false, st, std::min<int64_t>(65535, nodes - z0));
        if (rc) return rc;
    }
    return MM_OK;
}

}  // namespace mm
