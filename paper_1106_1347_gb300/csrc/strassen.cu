// Sections "StrassenNaiv" and "StrassenWinograd": the recursion driver.
//
// A plan has a depth d and padded sizes Np, Pp, Mp (multiples of 2^d; the
// paper's rule embeds everything in one Y x Y square).  Its levels run
// breadth-first: every node of a level is processed by the same launch, so a
// recursion of depth 9 (the paper's rule at 8192) is a few dozen launches and
// not 7^8 of them.
//
//   expand   -- the operand sums of one or two levels at once, for every node
//               of a level: a thread owns one position of the children's
//               blocks, reads the 4 (one level) or 16 (two levels) quadrant
//               values there and writes the 7 or 49 children's operands, each
//               sum rounded as the paper's Plus/Minus matrices are, in the
//               printed order.  The level in between never touches memory.
//   leaf     -- the bottom of the recursion, by the size of its blocks:
//               blocks <= 32: one CTA per node of the level above the
//                 bottom runs that last level in shared memory -- the seven
//                 operand sums, the seven naive block products (FMA, k in
//                 order) and the C-block sums in the paper's left-to-right
//                 order;
//               blocks <= 64: one CTA per bottom block, a naive product in
//                 shared memory;
//               larger blocks: the fused level of gemm_f64.cu (FP64 MMA,
//                 operand sums in staging, C-block sums in the epilogue) over
//                 every node of the level above the bottom in one launch.
//   combine  -- the C blocks of one or two levels at once from the children's
//               products, in the paper's left-to-right order, for every node of
//               a level.
//
// Operands past the caller's N x P (P x M) read as zero and results past N x M
// are dropped, so padding is virtual.  The breadth-first arrays of the deepest
// levels grow as (7/4)^level; when a whole plan would need more than
// breadth_cap() bytes of them, its top levels run depth-first instead: the
// children of a node are solved one after another (their operand sums
// materialised one child at a time, like the paper's Aux matrices), each
// child's subtree breadth-first.  The result does not depend on the split:
// every element sees the same operations in the same order.
#include <stdlib.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace {

// Bytes of breadth-first arrays one subtree may use (8 GiB; the environment
// variable MM_STRASSEN_BREADTH_CAP, read at every plan, overrides it).
size_t breadth_cap() {
    const char *v = getenv("MM_STRASSEN_BREADTH_CAP");
    if (v && *v) return (size_t)strtoull(v, nullptr, 10);
    return size_t(8) << 30;
}

// Operand access: node z's element (r, c) is p[z zs + r ld + c] when r < rows
// and c < cols, else 0.
struct Mat {
    const double *p;
    int64_t ld, rows, cols, zs;
};
// Result access: node z's element (r, c) goes to p[z zs + r ld + c] when
// r < rows and c < cols, else nowhere.
struct Out {
    double *p;
    int64_t ld, rows, cols, zs;
};

__device__ __forceinline__ double at(const Mat &m, int64_t z, int64_t r, int64_t c) {
    return (r < m.rows && c < m.cols) ? m.p[z * m.zs + r * m.ld + c] : 0.0;
}
__device__ __forceinline__ void put(const Out &m, int64_t z, int64_t r, int64_t c, double v) {
    if (r < m.rows && c < m.cols) m.p[z * m.zs + r * m.ld + c] = v;
}
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }

// The operands of H1..H7 at one position from the four quadrant values there.
//   StrassenNaiv, A: A11+A22, A21+A22, A11, A22, A11+A12, A21-A11, A12-A22
//                 B: B11+B22, B11, B12-B22, B21-B11, B22, B11+B12, B21+B22
//   StrassenWinograd (A1 = A11-A21, A2 = A22-A1, B1 = B22-B12, B2 = B1+B11),
//                 A: A11, A12, A2, A21+A22, A1, A12-A2, A22
//                 B: B11, B21, B2, B12-B11, B1, B22, B21-B2
template <int V, bool kA>
__device__ __forceinline__ void children(double x11, double x12, double x21, double x22, double (&o)[7]) {
    if (V == 0) {
        if (kA) {
            o[0] = add(x11, x22), o[1] = add(x21, x22), o[2] = x11, o[3] = x22;
            o[4] = add(x11, x12), o[5] = sub(x21, x11), o[6] = sub(x12, x22);
        } else {
            o[0] = add(x11, x22), o[1] = x11, o[2] = sub(x12, x22), o[3] = sub(x21, x11);
            o[4] = x22, o[5] = add(x11, x12), o[6] = add(x21, x22);
        }
    } else {
        if (kA) {
            const double a1 = sub(x11, x21), a2 = sub(x22, a1);
            o[0] = x11, o[1] = x12, o[2] = a2, o[3] = add(x21, x22), o[4] = a1, o[5] = sub(x12, a2), o[6] = x22;
        } else {
            const double b1 = sub(x22, x12), b2 = add(b1, x11);
            o[0] = x11, o[1] = x21, o[2] = b2, o[3] = sub(x12, x11), o[4] = b1, o[5] = x22, o[6] = sub(x21, b2);
        }
    }
}

// The C blocks at one position from H1..H7 there, left to right:
//   StrassenNaiv:     C11 = ((H1+H4)-H5)+H7, C12 = H3+H5, C21 = H2+H4, C22 = ((H1+H3)-H2)+H6;
//   StrassenWinograd: H8 = H1+H3, H9 = H8+H4; C11 = H1+H2, C12 = H9+H6, C21 = (H8+H5)+H7, C22 = H9+H5.
template <int V>
__device__ __forceinline__ void blocks(const double (&h)[7], double (&c)[4]) {
    if (V == 0) {
        c[0] = add(sub(add(h[0], h[3]), h[4]), h[6]);
        c[1] = add(h[2], h[4]);
        c[2] = add(h[1], h[3]);
        c[3] = add(sub(add(h[0], h[2]), h[1]), h[5]);
    } else {
        const double h8 = add(h[0], h[2]), h9 = add(h8, h[3]);
        c[0] = add(h[0], h[1]);
        c[1] = add(h9, h[5]);
        c[2] = add(add(h8, h[4]), h[6]);
        c[3] = add(h9, h[4]);
    }
}

// Operand sums of L (1 or 2) levels for `nodes` nodes whose operand is R x Cc:
// child block size h x w = (R >> L) x (Cc >> L); the 7^L children of node z are
// written densely at dst + (7^L z + child) h w (child = 7 i1 + i2 for two
// levels).  With only >= 0 (one level) just child `only` is written, at
// dst + z h w.
template <int V, bool kA, int L>
__global__ void __launch_bounds__(256) expand_kernel(const Mat src, double *__restrict__ dst, int64_t nodes,
                                                     int64_t R, int64_t Cc, int only) {
    const int64_t h = R >> L, w = Cc >> L, hw = h * w, total = nodes * hw;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t z = t / hw, pos = t - z * hw, r = pos / w, c = pos - (pos / w) * w;
        if (L == 1) {
            const double x11 = at(src, z, r, c), x12 = at(src, z, r, c + w), x21 = at(src, z, r + h, c),
                         x22 = at(src, z, r + h, c + w);
            if (only >= 0) {
                double v = 0.0;
                switch (only) {  // one child: each case evaluates only its own operand
#define MM_CHILD(i)                             \
    case i: {                                   \
        double o[7];                            \
        children<V, kA>(x11, x12, x21, x22, o); \
        v = o[i];                               \
        break;                                  \
    }
                    MM_CHILD(0) MM_CHILD(1) MM_CHILD(2) MM_CHILD(3) MM_CHILD(4) MM_CHILD(5) MM_CHILD(6)
#undef MM_CHILD
                }
                dst[z * hw + pos] = v;
            } else {
                double o[7];
                children<V, kA>(x11, x12, x21, x22, o);
#pragma unroll
                for (int i = 0; i < 7; ++i) dst[(7 * z + i) * hw + pos] = o[i];
            }
        } else {
            const int64_t hh = R >> 1, ww = Cc >> 1;  // first-level child block
            double l1[2][2][7];                        // first-level children at the four sub-positions
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const int64_t rr = r + a * h, cc = c + b * w;
                    children<V, kA>(at(src, z, rr, cc), at(src, z, rr, cc + ww), at(src, z, rr + hh, cc),
                                    at(src, z, rr + hh, cc + ww), l1[a][b]);
                }
#pragma unroll
            for (int i = 0; i < 7; ++i) {
                double o[7];
                children<V, kA>(l1[0][0][i], l1[0][1][i], l1[1][0][i], l1[1][1][i], o);
#pragma unroll
                for (int j = 0; j < 7; ++j) dst[(49 * z + 7 * i + j) * hw + pos] = o[j];
            }
        }
    }
}

// C blocks of L (1 or 2) levels for `nodes` nodes whose result is R x Cc, from
// the 7^L children's products stored densely at H + (7^L z + child) h w,
// h x w = (R >> L) x (Cc >> L).
template <int V, int L>
__global__ void __launch_bounds__(256) combine_kernel(const double *__restrict__ H, const Out dst, int64_t nodes,
                                                      int64_t R, int64_t Cc) {
    const int64_t h = R >> L, w = Cc >> L, hw = h * w, total = nodes * hw;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t z = t / hw, pos = t - z * hw, r = pos / w, c = pos - (pos / w) * w;
        if (L == 1) {
            double hv[7], q[4];
#pragma unroll
            for (int i = 0; i < 7; ++i) hv[i] = H[(7 * z + i) * hw + pos];
            blocks<V>(hv, q);
            put(dst, z, r, c, q[0]);
            put(dst, z, r, c + w, q[1]);
            put(dst, z, r + h, c, q[2]);
            put(dst, z, r + h, c + w, q[3]);
        } else {
            const int64_t hh = R >> 1, ww = Cc >> 1;
            double l1[7][4];  // first-level child i's block values at its four sub-positions
#pragma unroll
            for (int i = 0; i < 7; ++i) {
                double hv[7];
#pragma unroll
                for (int j = 0; j < 7; ++j) hv[j] = H[(49 * z + 7 * i + j) * hw + pos];
                blocks<V>(hv, l1[i]);
            }
#pragma unroll
            for (int ab = 0; ab < 4; ++ab) {
                double hv[7], q[4];
#pragma unroll
                for (int i = 0; i < 7; ++i) hv[i] = l1[i][ab];
                blocks<V>(hv, q);
                const int64_t rr = r + (ab >> 1) * h, cc = c + (ab & 1) * w;
                put(dst, z, rr, cc, q[0]);
                put(dst, z, rr, cc + ww, q[1]);
                put(dst, z, rr + hh, cc, q[2]);
                put(dst, z, rr + hh, cc + ww, q[3]);
            }
        }
    }
}

// Naive block product into registers: thread t owns outputs o0 + t,
// o0 + t + T, ..., o0 + t + (PER - 1) T of the n x m block (T threads; an
// index past the block is clamped to its last output and not stored by the
// caller), each summing its k in order with FMA; the PER chains are
// independent, which keeps the FP64 pipe fed with few CTAs per SM.
template <int C>
__device__ __forceinline__ void dot_chains(const double *X, const double *Y, int p, int m, const int (&r)[4],
                                           const int (&c)[4], double (&acc)[4]) {
    for (int k = 0; k < p; ++k) {
#pragma unroll
        for (int i = 0; i < C; ++i) acc[i] = fma(X[r[i] * p + k], Y[k * m + c[i]], acc[i]);
    }
}

template <int PER>
__device__ __forceinline__ void block_dot(const double *X, const double *Y, int n, int p, int m, int o0,
                                          int (&r)[4], int (&c)[4], double (&acc)[4]) {
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int o = min(o0 + (int)threadIdx.x + i * (int)blockDim.x, n * m - 1);
        r[i] = o / m, c[i] = o - (o / m) * m, acc[i] = 0.0;
    }
    // Chains the warp needs (warp-uniform): a chain no lane of the warp owns is
    // skipped, so the clamped duplicates cost at most part of one warp's chain.
    const int first = o0 + (int)(threadIdx.x & ~31u);
    int need = 1;
#pragma unroll
    for (int i = 1; i < PER; ++i) need += first + i * (int)blockDim.x < n * m ? 1 : 0;
    if (PER >= 4 && need >= 4) dot_chains<(PER >= 4 ? 4 : 1)>(X, Y, p, m, r, c, acc);
    else if (PER >= 3 && need == 3) dot_chains<(PER >= 3 ? 3 : 1)>(X, Y, p, m, r, c, acc);
    else if (PER >= 2 && need == 2) dot_chains<(PER >= 2 ? 2 : 1)>(X, Y, p, m, r, c, acc);
    else dot_chains<1>(X, Y, p, m, r, c, acc);
}

// Outputs o0 .. o0 + 4 T - 1 (or to the block's end): PER = the chains a
// thread needs for them, 1..4.  Returns PER.
__device__ __forceinline__ int block_dot_any(const double *X, const double *Y, int n, int p, int m, int o0,
                                            int (&r)[4], int (&c)[4], double (&acc)[4]) {
    const int per = min(4, (n * m - o0 + (int)blockDim.x - 1) / (int)blockDim.x);
    if (per <= 1) block_dot<1>(X, Y, n, p, m, o0, r, c, acc);
    else if (per == 2) block_dot<2>(X, Y, n, p, m, o0, r, c, acc);
    else if (per == 3) block_dot<3>(X, Y, n, p, m, o0, r, c, acc);
    else block_dot<4>(X, Y, n, p, m, o0, r, c, acc);
    return per;
}

// Naive block products (blocks of at most 64): node z's n x p and p x m blocks
// are staged in shared memory, each output sums its k in order with FMA.
__global__ void __launch_bounds__(256) leaf_naive_kernel(const Mat A, const Mat B, const Out C, int64_t nodes, int n,
                                                         int p, int m) {
    extern __shared__ double sm[];
    double *As = sm, *Bs = sm + n * p;
    for (int64_t z = blockIdx.x; z < nodes; z += gridDim.x) {
        for (int e = threadIdx.x; e < n * p; e += blockDim.x) As[e] = at(A, z, e / p, e % p);
        for (int e = threadIdx.x; e < p * m; e += blockDim.x) Bs[e] = at(B, z, e / m, e % m);
        __syncthreads();
        // Up to 64 x 64 outputs: groups of 4 x 256, each thread up to four chains at a time.
        for (int o0 = 0; o0 < n * m; o0 += 4 * (int)blockDim.x) {
            int r[4], c[4];
            double acc[4];
            const int per = block_dot_any(As, Bs, n, p, m, o0, r, c, acc);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (i < per && o0 + (int)threadIdx.x + i * (int)blockDim.x < n * m) put(C, z, r[i], c[i], acc[i]);
        }
        __syncthreads();
    }
}

// The product walk of one level: child, then up to four (block, sign, first
// touch) targets; the walk order makes every C block's sum the paper's
// left-to-right one (see blocks()).
struct Step {
    int child, nt, quad[4], sign[4], first[4];
};
__host__ __device__ constexpr Step walk_step(int V, int s) {
    return V == 0 ? (s == 0   ? Step{0, 2, {0, 3, 0, 0}, {1, 1, 0, 0}, {1, 1, 0, 0}}     // H1: C11 = , C22 =
                     : s == 1 ? Step{2, 2, {1, 3, 0, 0}, {1, 1, 0, 0}, {1, 0, 0, 0}}     // H3: C12 = , C22 +=
                     : s == 2 ? Step{1, 2, {2, 3, 0, 0}, {1, -1, 0, 0}, {1, 0, 0, 0}}    // H2: C21 = , C22 -=
                     : s == 3 ? Step{3, 2, {0, 2, 0, 0}, {1, 1, 0, 0}, {0, 0, 0, 0}}     // H4: C11 +=, C21 +=
                     : s == 4 ? Step{4, 2, {0, 1, 0, 0}, {-1, 1, 0, 0}, {0, 0, 0, 0}}    // H5: C11 -=, C12 +=
                     : s == 5 ? Step{5, 1, {3, 0, 0, 0}, {1, 0, 0, 0}, {0, 0, 0, 0}}     // H6: C22 +=
                              : Step{6, 1, {0, 0, 0, 0}, {1, 0, 0, 0}, {0, 0, 0, 0}})    // H7: C11 +=
                  : (s == 0   ? Step{0, 4, {0, 1, 2, 3}, {1, 1, 1, 1}, {1, 1, 1, 1}}     // H1: all four =
                     : s == 1 ? Step{1, 1, {0, 0, 0, 0}, {1, 0, 0, 0}, {0, 0, 0, 0}}     // H2: C11 +=
                     : s == 2 ? Step{2, 3, {1, 2, 3, 0}, {1, 1, 1, 0}, {0, 0, 0, 0}}     // H3: C12, C21, C22 +=
                     : s == 3 ? Step{3, 2, {1, 3, 0, 0}, {1, 1, 0, 0}, {0, 0, 0, 0}}     // H4: C12, C22 +=
                     : s == 4 ? Step{4, 2, {2, 3, 0, 0}, {1, 1, 0, 0}, {0, 0, 0, 0}}     // H5: C21, C22 +=
                     : s == 5 ? Step{5, 1, {1, 0, 0, 0}, {1, 0, 0, 0}, {0, 0, 0, 0}}     // H6: C12 +=
                              : Step{6, 1, {2, 0, 0, 0}, {1, 0, 0, 0}, {0, 0, 0, 0}});   // H7: C21 +=
}

// C block `Q` of output i := +-h (first touch) or C + (+-h), in registers.
template <int Q, int kSign, int kFirst>
__device__ __forceinline__ void target(double (&cq)[4][4], int i, double h) {
    const double v = kSign > 0 ? h : -h;
    cq[i][Q] = kFirst ? v : add(cq[i][Q], v);
}

// Step S of the walk: the operand sums of its product into shared memory, the
// naive product of the n x p and p x m blocks, and the product added into its
// C blocks, which each thread keeps in registers for its outputs (a thread
// owns the same positions in every step).
template <int V, int S, int PER>
__device__ __forceinline__ void leaf_level_step(const double *As, const double *Bs, double *Ss, double *Ts,
                                                double (&cq)[4][4], int (&r)[4], int (&c)[4], int n, int p, int m) {
    constexpr int child = walk_step(V, S).child, nt = walk_step(V, S).nt;
    const int P2 = 2 * p, M2 = 2 * m;
    for (int e = threadIdx.x; e < n * p; e += blockDim.x) {
        const int rr = e / p, cc = e - (e / p) * p;
        double o[7];
        children<V, true>(As[rr * P2 + cc], As[rr * P2 + cc + p], As[(rr + n) * P2 + cc],
                          As[(rr + n) * P2 + cc + p], o);
        Ss[e] = o[child];
    }
    for (int e = threadIdx.x; e < p * m; e += blockDim.x) {
        const int rr = e / m, cc = e - (e / m) * m;
        double o[7];
        children<V, false>(Bs[rr * M2 + cc], Bs[rr * M2 + cc + m], Bs[(rr + p) * M2 + cc],
                           Bs[(rr + p) * M2 + cc + m], o);
        Ts[e] = o[child];
    }
    __syncthreads();
    double acc[4];
    block_dot<PER>(Ss, Ts, n, p, m, 0, r, c, acc);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        target<walk_step(V, S).quad[0], walk_step(V, S).sign[0], walk_step(V, S).first[0]>(cq, i, acc[i]);
        if constexpr (nt > 1)
            target<walk_step(V, S).quad[1], walk_step(V, S).sign[1], walk_step(V, S).first[1]>(cq, i, acc[i]);
        if constexpr (nt > 2)
            target<walk_step(V, S).quad[2], walk_step(V, S).sign[2], walk_step(V, S).first[2]>(cq, i, acc[i]);
        if constexpr (nt > 3)
            target<walk_step(V, S).quad[3], walk_step(V, S).sign[3], walk_step(V, S).first[3]>(cq, i, acc[i]);
    }
    __syncthreads();  // Ss and Ts are rewritten by the next step
    if constexpr (S < 6) leaf_level_step<V, S + 1, PER>(As, Bs, Ss, Ts, cq, r, c, n, p, m);
}

// The last recursion level with naive products of blocks <= 32, in shared
// memory: node z's operands are 2n x 2p and 2p x 2m, its result 2n x 2m.
// PER = ceil(n m / 256) outputs per thread (1..4), a template parameter so
// small blocks (the paper's 17 to 22) keep few registers and many CTAs per SM.
template <int V, int PER>
__global__ void __launch_bounds__(256, PER <= 2 ? 4 : 2)
    leaf_level_kernel(const Mat A, const Mat B, const Out C, int64_t nodes, int n, int p, int m) {
    extern __shared__ double sm[];
    double *As = sm, *Bs = As + 4 * n * p, *Ss = Bs + 4 * p * m, *Ts = Ss + n * p;
    const int N2 = 2 * n, P2 = 2 * p, M2 = 2 * m;
    for (int64_t z = blockIdx.x; z < nodes; z += gridDim.x) {
        for (int e = threadIdx.x; e < N2 * P2; e += blockDim.x) As[e] = at(A, z, e / P2, e % P2);
        for (int e = threadIdx.x; e < P2 * M2; e += blockDim.x) Bs[e] = at(B, z, e / M2, e % M2);
        __syncthreads();
        double cq[4][4];
        int r[4], c[4];
        leaf_level_step<V, 0, PER>(As, Bs, Ss, Ts, cq, r, c, n, p, m);
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            if ((int)threadIdx.x + i * (int)blockDim.x >= n * m) break;
#pragma unroll
            for (int q = 0; q < 4; ++q) put(C, z, r[i] + (q >> 1) * n, c[i] + (q & 1) * m, cq[i][q]);
        }
        // the next node's staging waits at the first step's barrier
    }
}

size_t leaf_level_smem(int n, int p, int m) { return (size_t)(5 * n * p + 5 * p * m) * 8; }
size_t leaf_naive_smem(int n, int p, int m) { return (size_t)(n * p + p * m) * 8; }

// ------------------------------------------------------------------ host plan

int64_t pow7(int e) {
    int64_t v = 1;
    while (e-- > 0) v *= 7;
    return v;
}

size_t al(size_t bytes) { return mm::align_up(bytes, 256); }

enum LeafMode { kLeafLevel, kLeafNaive, kFusedLevel, kNaiveProduct };

// The breadth-first part of a plan: a subtree of depth D whose root blocks are
// n0 x p0 and p0 x m0.
struct Sub {
    int D, e;  // depth; level whose nodes the leaf kernel takes
    LeafMode mode;
    int64_t n0, p0, m0;
    std::vector<int> bounds;  // levels whose operands and results are stored: 0 < b1 < ... < e
};

Sub make_sub(int D, int64_t n0, int64_t p0, int64_t m0) {
    Sub s{};
    s.D = D;
    s.n0 = n0, s.p0 = p0, s.m0 = m0;
    const int64_t big = std::max(n0 >> D, std::max(p0 >> D, m0 >> D));
    if (D >= 1 && big <= 32) {
        s.mode = kLeafLevel, s.e = D - 1;
    } else if (big <= 64) {
        s.mode = kLeafNaive, s.e = D;
    } else if (D >= 1) {
        s.mode = kFusedLevel, s.e = D - 1;
    } else {  // a depth-first child with no level left: one plain product of dense blocks
        s.mode = kNaiveProduct, s.e = 0;
    }
    for (int b = 0; b < s.e;) {
        b += (s.e - b >= 2) ? 2 : 1;
        s.bounds.push_back(b);
    }
    return s;
}

size_t sub_bytes(const Sub &s) {
    size_t t = 0;
    for (int b : s.bounds) {
        const int64_t z = pow7(b), n = s.n0 >> b, p = s.p0 >> b, m = s.m0 >> b;
        t += al((size_t)z * n * p * 8) + al((size_t)z * p * m * 8) + al((size_t)z * n * m * 8);
    }
    return t;
}

// Workspace of one depth-first level whose children are n x p by p x m: one
// child's two operands and all seven children's products.
size_t df_level_bytes(int64_t n, int64_t p, int64_t m) {
    return al((size_t)n * p * 8) + al((size_t)p * m * 8) + al((size_t)7 * n * m * 8);
}

struct Plan {
    int depth, top;
    int64_t Np, Pp, Mp;
    Sub sub;
    size_t bytes;
};

Plan make_plan(int depth, int64_t Np, int64_t Pp, int64_t Mp) {
    Plan pl{};
    pl.depth = depth;
    pl.Np = Np, pl.Pp = Pp, pl.Mp = Mp;
    const size_t cap = breadth_cap();
    for (int top = 0; top <= depth; ++top) {
        pl.top = top;
        pl.sub = make_sub(depth - top, Np >> top, Pp >> top, Mp >> top);
        size_t b = sub_bytes(pl.sub);
        for (int j = 1; j <= top; ++j) b += df_level_bytes(Np >> j, Pp >> j, Mp >> j);
        pl.bytes = b;
        if (sub_bytes(pl.sub) <= cap) break;
    }
    return pl;
}

unsigned grid_for(int64_t threads) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(mm::ceil_div(threads, 256), 16 * (int64_t)mm::sm_count()));
}

struct Run {
    int V;
    const Plan *pl;
    cudaStream_t st;
};

int launch_expand(const Run &r, bool sideA, int L, const Mat &src, double *dst, int64_t nodes, int64_t R,
                  int64_t Cc, int only) {
    const unsigned g = grid_for(nodes * (R >> L) * (Cc >> L));
    return mm::launch("strassen_expand", r.st, [&] {
#define MM_EXPAND(V_, A_, L_) expand_kernel<V_, A_, L_><<<g, 256, 0, r.st>>>(src, dst, nodes, R, Cc, only)
        if (r.V == 0) {
            if (sideA) {
                if (L == 1) MM_EXPAND(0, true, 1); else MM_EXPAND(0, true, 2);
            } else {
                if (L == 1) MM_EXPAND(0, false, 1); else MM_EXPAND(0, false, 2);
            }
        } else {
            if (sideA) {
                if (L == 1) MM_EXPAND(1, true, 1); else MM_EXPAND(1, true, 2);
            } else {
                if (L == 1) MM_EXPAND(1, false, 1); else MM_EXPAND(1, false, 2);
            }
        }
#undef MM_EXPAND
    });
}

int launch_combine(const Run &r, int L, const double *H, const Out &dst, int64_t nodes, int64_t R, int64_t Cc) {
    const unsigned g = grid_for(nodes * (R >> L) * (Cc >> L));
    return mm::launch("strassen_combine", r.st, [&] {
        if (r.V == 0) {
            if (L == 1) combine_kernel<0, 1><<<g, 256, 0, r.st>>>(H, dst, nodes, R, Cc);
            else combine_kernel<0, 2><<<g, 256, 0, r.st>>>(H, dst, nodes, R, Cc);
        } else {
            if (L == 1) combine_kernel<1, 1><<<g, 256, 0, r.st>>>(H, dst, nodes, R, Cc);
            else combine_kernel<1, 2><<<g, 256, 0, r.st>>>(H, dst, nodes, R, Cc);
        }
    });
}

cudaError_t leaf_smem_attributes() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        const int most = (int)leaf_level_smem(32, 32, 32);
        const void *fns[8] = {(const void *)leaf_level_kernel<0, 1>, (const void *)leaf_level_kernel<0, 2>,
                              (const void *)leaf_level_kernel<0, 3>, (const void *)leaf_level_kernel<0, 4>,
                              (const void *)leaf_level_kernel<1, 1>, (const void *)leaf_level_kernel<1, 2>,
                              (const void *)leaf_level_kernel<1, 3>, (const void *)leaf_level_kernel<1, 4>};
        for (int i = 0; i < 8 && err == cudaSuccess; ++i)
            err = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute((const void *)leaf_naive_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)leaf_naive_smem(64, 64, 64));
    });
    return err;
}

Mat dense_mat(const double *p, int64_t rows, int64_t cols) { return Mat{p, cols, rows, cols, rows * cols}; }
Out dense_out(double *p, int64_t rows, int64_t cols) { return Out{p, cols, rows, cols, rows * cols}; }

// One subtree breadth-first: A (n0 x p0) and B (p0 x m0) of its root to C.
int run_sub(const Run &r, const Sub &s, const Mat &A, const Mat &B, const Out &C, char *ws) {
    const int nb = (int)s.bounds.size();
    std::vector<double *> arrA(nb), arrB(nb), arrC(nb);
    for (int k = 0; k < nb; ++k) {
        const int b = s.bounds[k];
        const int64_t z = pow7(b), n = s.n0 >> b, p = s.p0 >> b, m = s.m0 >> b;
        arrA[k] = (double *)ws;
        ws += al((size_t)z * n * p * 8);
        arrB[k] = (double *)ws;
        ws += al((size_t)z * p * m * 8);
        arrC[k] = (double *)ws;
        ws += al((size_t)z * n * m * 8);
    }
    // Operand sums down to level e.
    Mat curA = A, curB = B;
    int prev = 0;
    for (int k = 0; k < nb; ++k) {
        const int b = s.bounds[k], L = b - prev;
        const int64_t nodes = pow7(prev);
        int rc = launch_expand(r, true, L, curA, arrA[k], nodes, s.n0 >> prev, s.p0 >> prev, -1);
        if (!rc) rc = launch_expand(r, false, L, curB, arrB[k], nodes, s.p0 >> prev, s.m0 >> prev, -1);
        if (rc) return rc;
        curA = dense_mat(arrA[k], s.n0 >> b, s.p0 >> b);
        curB = dense_mat(arrB[k], s.p0 >> b, s.m0 >> b);
        prev = b;
    }
    // The bottom.
    const int e = s.e;
    const int64_t nodes = pow7(e);
    const Out outE = nb ? dense_out(arrC[nb - 1], s.n0 >> e, s.m0 >> e) : C;
    if (s.mode == kNaiveProduct) {
        int rc = mm::run_naive(s.n0, s.p0, s.m0, curA.p, curA.ld, curB.p, curB.ld, outE.p, outE.ld, r.st);
        if (rc) return rc;
    } else if (s.mode == kFusedLevel) {
        const int64_t n = s.n0 >> (e + 1), p = s.p0 >> (e + 1), m = s.m0 >> (e + 1);
        int rc = mm::run_strassen_level(r.V, nodes, n, p, m, curA.p, curA.ld, curA.rows, curA.cols, curA.zs, curB.p,
                                        curB.ld, curB.rows, curB.cols, curB.zs, outE.p, outE.ld, outE.rows,
                                        outE.cols, outE.zs, r.st);
        if (rc) return rc;
    } else {
        cudaError_t ae = leaf_smem_attributes();
        if (ae != cudaSuccess) return mm::cuda_fail(ae, "Strassen: shared memory attribute");
        const bool level = s.mode == kLeafLevel;
        const int sh = level ? e + 1 : e;
        const int n = (int)(s.n0 >> sh), p = (int)(s.p0 >> sh), m = (int)(s.m0 >> sh);
        const size_t smem = level ? leaf_level_smem(n, p, m) : leaf_naive_smem(n, p, m);
        const int per_sm = std::max(2, std::min(8, (int)(200000 / std::max<size_t>(smem, 1))));
        const unsigned g = (unsigned)std::min<int64_t>(nodes, (int64_t)per_sm * mm::sm_count());
        int rc = mm::launch(level ? "strassen_leaf_level" : "strassen_leaf_naive", r.st, [&] {
            if (!level)
                leaf_naive_kernel<<<g, 256, smem, r.st>>>(curA, curB, outE, nodes, n, p, m);
            else {
                const int per = (n * m + 255) / 256;  // outputs per thread, 1..4 (blocks <= 32 x 32)
#define MM_LEAF(V_, P_) leaf_level_kernel<V_, P_><<<g, 256, smem, r.st>>>(curA, curB, outE, nodes, n, p, m)
                if (r.V == 0) {
                    if (per <= 1) MM_LEAF(0, 1); else if (per == 2) MM_LEAF(0, 2); else if (per == 3) MM_LEAF(0, 3);
                    else MM_LEAF(0, 4);
                } else {
                    if (per <= 1) MM_LEAF(1, 1); else if (per == 2) MM_LEAF(1, 2); else if (per == 3) MM_LEAF(1, 3);
                    else MM_LEAF(1, 4);
                }
#undef MM_LEAF
            }
        });
        if (rc) return rc;
    }
    // C blocks back up to the root.
    for (int k = nb - 1; k >= 0; --k) {
        const int b = s.bounds[k], up = k ? s.bounds[k - 1] : 0;
        const Out dst = k ? dense_out(arrC[k - 1], s.n0 >> up, s.m0 >> up) : C;
        const int rc = launch_combine(r, b - up, arrC[k], dst, pow7(up), s.n0 >> up, s.m0 >> up);
        if (rc) return rc;
    }
    return MM_OK;
}

// Depth-first level j: the node's A (n x p) and B (p x m) to C.
int run_df(const Run &r, int j, const Mat &A, const Mat &B, const Out &C, int64_t n, int64_t p, int64_t m,
           char *ws) {
    const Plan &pl = *r.pl;
    if (j == pl.top) return run_sub(r, pl.sub, A, B, C, ws);
    const int64_t h = n / 2, q = p / 2, w = m / 2;
    double *S = (double *)ws;
    ws += al((size_t)h * q * 8);
    double *T = (double *)ws;
    ws += al((size_t)q * w * 8);
    double *H = (double *)ws;  // the seven children's products, one dense array
    ws += al((size_t)7 * h * w * 8);
    for (int i = 0; i < 7; ++i) {
        int rc = launch_expand(r, true, 1, A, S, 1, n, p, i);
        if (!rc) rc = launch_expand(r, false, 1, B, T, 1, p, m, i);
        if (!rc) rc = run_df(r, j + 1, dense_mat(S, h, q), dense_mat(T, q, w), dense_out(H + i * h * w, h, w), h, q, w, ws);
        if (rc) return rc;
    }
    return launch_combine(r, 1, H, C, 1, n, m);
}

}  // namespace

namespace mm {

// Depth and padded sizes of the recursion (see mm_strassen in mm.h).
int strassen_plan(int variant, int64_t N, int64_t P, int64_t M, int32_t cutoff, int *depth, int64_t *Np,
                  int64_t *Pp, int64_t *Mp) {
    const int64_t X = std::max(N, std::max(P, M));
    int d = 0;
    if (cutoff == 0) {  // the paper's rule, square embedding
        int lg = -1;
        for (int64_t t = X; t > 0; t >>= 1) ++lg;
        d = std::max(0, lg - 4);
        const int64_t Y = ((X >> d) + 1) << d;
        *depth = d;
        *Np = *Pp = *Mp = Y;
    } else {
        if (cutoff > 0) {
            while (ceil_div(X, (int64_t)1 << d) > cutoff) ++d;
        } else if (!tuned_strassen_depth(variant, N, P, M, &d)) {
            // untuned default: the paper's depth floor(log2) - 4, taken on the
            // smallest dimension (blocks of 16 to 31 there), fastest on GB300;
            // at most kWinogradSafeDepth levels of Winograd's variant
            int lg = -1;
            for (int64_t t = std::min(N, std::min(P, M)); t > 0; t >>= 1) ++lg;
            d = std::max(0, lg - 4);
            if (variant == 1) d = std::min(d, kWinogradSafeDepth);
        }
        const int64_t q = (int64_t)1 << d;
        *depth = d;
        *Np = ceil_div(N, q) * q;
        *Pp = ceil_div(P, q) * q;
        *Mp = ceil_div(M, q) * q;
    }
    if (*depth > 16) return fail(MM_ERR_UNSUPPORTED, "Strassen depth %d exceeds 16", *depth);
    return MM_OK;
}

size_t strassen_ws_bytes(int variant, int depth, int64_t Np, int64_t Pp, int64_t Mp) {
    (void)variant;
    if (depth == 0) return 0;
    return make_plan(depth, Np, Pp, Mp).bytes;
}

int run_strassen(int variant, int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                 int64_t ldb, double *C, int64_t ldc, int depth, int64_t Np, int64_t Pp, int64_t Mp, void *ws,
                 cudaStream_t st) {
    if (depth == 0) return run_naive(N, P, M, A, lda, B, ldb, C, ldc, st);
    const Plan pl = make_plan(depth, Np, Pp, Mp);
    const Run r{variant, &pl, st};
    return run_df(r, 0, Mat{A, lda, N, P, 0}, Mat{B, ldb, P, M, 0}, Out{C, ldc, N, M, 0}, Np, Pp, Mp, (char *)ws);
}

}  // namespace mm
