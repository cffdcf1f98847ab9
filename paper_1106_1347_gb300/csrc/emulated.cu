// FP64-accurate product emulated from BF16 slices on the tcgen05 tensor cores.
//
// Not in the paper; its power-of-two row/column scaling generalises the exact
// scaling of section "WinogradScaled" from one global lambda to one exponent
// per row of A (e_i) and per column of B (f_j).  Definition (identical to the
// CPU oracle's):
//   V_ik = RN(A_ik 2^(beta s - 1 - e_i)),  |V| <= 2^(beta s - 1),  beta = 7;
//   V = sum_t v_t 2^(beta t) in balanced digits (low digits in [-64, 64),
//   top digit in [-64, 64]); slice sigma holds the digit of weight
//   2^(beta (s-1-sigma)) as an exact BF16; B is cut per column likewise;
//   T_d = sum_k sum_{sigma+tau=d} a^(sigma)_ik b^(tau)_kj  for d = 0..s-1;
//   C_ij = RN(sum_d T_d 2^(beta (s-1-d))) * 2^(e_i + f_j + 2 - beta (s+1)).
//
// Kernels (all integer work on the FP64 bit patterns; FP64 arithmetic on this
// part runs at ~1/100 of the BF16 tensor rate, so none is spent per slice):
//   split_rows  -- one CTA per row of A: max |A_ik| by integer max on the bit
//                  patterns, then the digits (the row re-read from L2),
//                  written as slices [s][N][P] (K-major, 16-byte stores).
//   col_max / split_cols -- per-column maxima of B, then each thread turns
//                  32 consecutive k of one column into digits and stores them
//                  as K-major slice rows [s][M][P] (the transpose happens in
//                  registers).
//   slice_gemm  -- (slice_gemm.cuh, instantiated per format and slice count)
//                  persistent, one CTA per SM looping over 128x64 output
//                  tiles.  Warp 0 issues TMA loads of all s slices of a
//                  32-wide K-block of A and B (3-D boxes, 64-byte swizzle)
//                  into a ring of shared-memory stages; warp 1 (one elected
//                  lane, warp-uniform operands) issues tcgen05.mma kind::f16
//                  for every pair with sigma + tau = d into TMEM accumulator d
//                  (s x 64 FP32 columns), two adjacent diagonals per N = 128
//                  MMA where it can; eight epilogue warps read each
//                  accumulator out before its partial sums could leave the
//                  integers FP32 holds exactly (|x| <= 2^24), into two int64
//                  registers per output, and at the tile's end round the
//                  exact 128-bit integer once to double and apply
//                  2^(e_i + f_j ...) while the next tile's MMAs run.
// Every mbarrier wait is bounded; on timeout the kernel raises the device
// status word, waits (bounded) for its own copies and MMAs, frees TMEM and exits.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "slice_gemm.cuh"

using namespace emu;

namespace {


__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}
// |x| as its bit pattern (order-preserving for the non-negative doubles).
__device__ __forceinline__ unsigned long long absbits(double x) {
    return (unsigned long long)__double_as_longlong(x) & ~(1ull << 63);
}

// frexp's exponent of a finite double from its magnitude's bit pattern: the e
// with |x| = f 2^e, f in [1/2, 1) (0 for x = 0).  Normal: e = E - 1022 for the
// biased exponent E; subnormal: |x| = frac 2^-1074, so e = bitlength(frac) -
// 1074.
__device__ __forceinline__ int frexp_exp_bits(unsigned long long absbits) {
    if (absbits == 0) return 0;
    const int E = (int)(absbits >> 52);
    return E ? E - 1022 : (64 - __clzll((long long)absbits)) - 1074;
}

// RN(x * 2^sh) as an integer, computed on the bit pattern (ties to even):
// |x| = m 2^(E' - 1075) with E' = max(E, 1), so the result is m shifted left by
// e2 = E' - 1075 + sh when e2 >= 0, else RN(m / 2^r) for r = -e2, which is
// floor((m + 2^(r-1) - 1 + lsb(floor(m / 2^r))) / 2^r): the added amount carries
// into bit r exactly when the remainder is above half, or equal to it with an
// odd quotient (m < 2^53, so nothing overflows; r >= 64 gives 0).
__device__ __forceinline__ int64_t round_scaled(double x, int sh) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    const uint64_t m = (b & ((1ull << 52) - 1)) | (E ? 1ull << 52 : 0ull);
    const int e2 = max(E, 1) - 1075 + sh;
    uint64_t q;
    if (e2 >= 0) {
        q = m << min(e2, 63);
    } else {
        const int r = min(-e2, 63);
        q = (m + ((1ull << (r - 1)) - 1) + ((m >> r) & 1)) >> r;
    }
    return (b >> 63) ? -(int64_t)q : (int64_t)q;
}

// Digit d (|d| < 2^22) as a float, exactly: the bits of 1.5 * 2^23 + d (floats
// in [2^23, 2^24) are spaced by one) minus 1.5 * 2^23.  `biased` = d + bias
// with 0 <= biased < 2^22 may be passed instead, with the bias subtracted too.
constexpr uint32_t kMagicBits = 0x4B400000u;  // 1.5 * 2^23
constexpr float kMagic = 12582912.0f;

// One slice's eight digits (as exact floats) as one vector store: 16 bytes of
// BF16 or 8 bytes of E4M3 at dst (16-byte aligned for BF16, 8 for E4M3).  A
// digit has at most 8 significant bits, so its BF16 is the float's upper half
// (the lower 16 bits are zero) and its E4M3 conversion is exact.
template <int KIND>
__device__ __forceinline__ void store_slice8(const float (&f)[8], unsigned char *dst) {
    if (KIND == MM_SLICE_FP8E4M3) {
        uint32_t w[2] = {0u, 0u};
#pragma unroll
        for (int u = 0; u < 8; ++u)
            w[u >> 2] |= (uint32_t)__nv_cvt_float_to_fp8(f[u], __NV_SATFINITE, __NV_E4M3) << (8 * (u & 3));
        *reinterpret_cast<uint2 *>(dst) = make_uint2(w[0], w[1]);
    } else {
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) w[u] = __byte_perm(__float_as_uint(f[2 * u]), __float_as_uint(f[2 * u + 1]), 0x7632);
        *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Eight consecutive elements of one slice row at a time.  V[u] holds
// RN(x_u 2^sh) on entry.  Its balanced base-2^beta digits d_0 .. d_(s-2) lie in
// [-2^(beta-1), 2^(beta-1)) and the top digit d_(s-1) is the rest, so with
// H = 2^(beta-1) (1 + 2^beta + ... + 2^(beta(s-2))) the low beta(s-1) bits of
// V + H hold the ordinary digits d_t + 2^(beta-1) and the bits above them,
// read as a signed number, are d_(s-1): every digit is one shift and mask of
// V + H, with no carry from one to the next.  Digit t of all eight goes to
// slice s-1-t as one vector store at dst0 + (s-1-t) * stride (dst0: slice 0
// at this row and column).  Every index is a compile-time constant, so nothing
// leaves registers.
template <int KIND>
__device__ __forceinline__ void store_digits8(const int64_t (&V)[8], int s, unsigned char *dst0, int64_t stride) {
    constexpr int beta = fmt_beta(KIND), half = 1 << (beta - 1);
    constexpr uint32_t mask = (1u << beta) - 1;
    uint64_t H = 0;
#pragma unroll
    for (int t = 0; t + 1 < fmt_max_slices(KIND); ++t)
        if (t + 1 < s) H |= (uint64_t)half << (beta * t);
    uint64_t z[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) z[u] = (uint64_t)V[u] + H;
#pragma unroll
    for (int t = 0; t < fmt_max_slices(KIND); ++t) {
        if (t < s) {
            float f[8];
            if (t + 1 < s) {
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    f[u] = __uint_as_float(((uint32_t)(z[u] >> (beta * t)) & mask) | kMagicBits) - (kMagic + half);
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    f[u] = __uint_as_float(kMagicBits + (uint32_t)(int32_t)((int64_t)z[u] >> (beta * t))) - kMagic;
            }
            store_slice8<KIND>(f, dst0 + (int64_t)(s - 1 - t) * stride);
        }
    }
}

// x[c .. c+8) of a row (zeros at and past P), with 16-byte loads when the row
// start is 16-byte aligned and all eight lie before P.
__device__ __forceinline__ void load8(const double *__restrict__ a, int64_t c, int64_t P, bool vec, double (&v)[8]) {
    if (vec && c + 8 <= P) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const double2 x = __ldg(reinterpret_cast<const double2 *>(a + c) + u);
            v[2 * u] = x.x;
            v[2 * u + 1] = x.y;
        }
    } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = (c + u < P) ? __ldg(a + c + u) : 0.0;
    }
}

constexpr int kRowThreads = 256;
// Rows of at most kQuarterRowMax (padded) elements are split by 8 threads each
// (4 rows per warp, 32 per CTA), rows of at most kWarpRowMax by one warp each
// (8 rows per CTA), longer ones by a whole CTA: every thread has 8 elements
// of its row to load at a time, whatever the row length.
constexpr int64_t kQuarterRowMax = 64, kWarpRowMax = 1024;

// One row of A by T threads (a whole CTA of 256, one warp, or 8 lanes of one):
// max |A_ik| by
// integer max on the bit patterns, then the digits, written as slices
// [s][Nr][Pp] (BF16 or FP8-E4M3); columns [P, Pp) get zero digits so every
// K-block read is defined.  The digit pass reads the row again, from L2: with
// one row per CTA only a few rows per SM are in flight (about 40 MB over the
// GPU at 8192 columns), so A crosses HBM once.  `tid` is the thread's index
// among the T; with T = 256 `red` is 8 words of shared memory (unused for a
// warp).  With T = 8 the warp's four groups reduce among themselves, so every
// lane of the warp must call it: a group past the last row passes valid =
// false and only takes part in the reduction.
template <int KIND, int T>
__device__ __forceinline__ void split_row(const SplitA &p, int64_t row, int tid, unsigned long long *red,
                                          bool valid = true) {
    const int64_t off = valid ? row * p.lda : 0;
    const int64_t P = valid ? p.P : 0, Pp = valid ? p.Pp : 0;
    const int s = p.s;
    const bool vec = (((uintptr_t)(p.A + off)) & 15) == 0;
    unsigned long long mx = 0;
    for (int64_t c = 8 * tid; c < P; c += 8 * T) {
        double x[8];
        load8(p.A + off, c, P, vec, x);
#pragma unroll
        for (int u = 0; u < 8; ++u) mx = umax64(mx, absbits(x[u]));
    }
#pragma unroll
    for (int o = (T < 32 ? T : 32) / 2; o > 0; o >>= 1)  // within the T (or 32) lanes of the row
        mx = umax64(mx, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)mx, o));
    if (T > 32) {
        if ((tid & 31) == 0) red[tid >> 5] = mx;
        __syncthreads();
#pragma unroll
        for (int w = 0; w < T / 32; ++w) mx = umax64(mx, red[w]);
        __syncthreads();  // `red` is reused by the next row
    }
    const int e = frexp_exp_bits(mx);
    if (tid == 0 && valid) p.ea[row] = e;
    constexpr int beta = fmt_beta(KIND), es = fmt_esize(KIND);
    const int sh = beta * s - 1 - e;
    const int64_t stride = (int64_t)p.Nr * p.Pp * es;
    unsigned char *row0 = p.slices + (valid ? row : 0) * p.Pp * es;
    // Pp is a multiple of 8 (BF16) or 16 (E4M3) elements: a group of eight
    // starting before Pp ends by Pp.
    for (int64_t c = 8 * tid; c < Pp; c += 8 * T) {
        double x[8];
        load8(p.A + off, c, P, vec, x);
        int64_t V[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) V[u] = round_scaled(x[u], sh);
        store_digits8<KIND>(V, s, row0 + c * es, stride);
    }
}

template <int KIND>
__global__ void __launch_bounds__(kRowThreads, 4) split_rows_kernel(const SplitA p) {
    __shared__ unsigned long long red[kRowThreads / 32];
    split_row<KIND, kRowThreads>(p, blockIdx.x, threadIdx.x, red);
}

// Short rows (Pp <= kWarpRowMax): one warp per row, 8 rows per CTA.
template <int KIND>
__global__ void __launch_bounds__(kRowThreads, 4) split_rows_warp_kernel(const SplitA p) {
    const int64_t row = (int64_t)blockIdx.x * (kRowThreads / 32) + (threadIdx.x >> 5);
    if (row < p.N) split_row<KIND, 32>(p, row, threadIdx.x & 31, nullptr);
}

// Very short rows (Pp <= kQuarterRowMax): 8 threads per row, 32 rows per CTA.
template <int KIND>
__global__ void __launch_bounds__(kRowThreads, 4) split_rows_quarter_kernel(const SplitA p) {
    const int64_t row = (int64_t)blockIdx.x * (kRowThreads / 8) + (threadIdx.x >> 3);
    if (((int64_t)blockIdx.x * (kRowThreads / 8) + ((threadIdx.x & ~31u) >> 3)) >= p.N) return;  // whole warp
    split_row<KIND, 8>(p, row, threadIdx.x & 7, nullptr, row < p.N);
}


// Column maxima of rows [k0, k0 + 256) folded into colmax with atomicMax on the bits.
__device__ __forceinline__ void col_max_part(const SplitB &p, int64_t j, int64_t k0) {
    if (j >= p.M) return;
    const int64_t k1 = min(p.P, k0 + 256);
    unsigned long long mx = 0;
    for (int64_t k = k0; k < k1; ++k) mx = umax64(mx, absbits(p.B[k * p.ldb + j]));
    if (mx) atomicMax(p.colmax + j, mx);
}

__global__ void __launch_bounds__(128) col_max_kernel(const SplitB p) {
    col_max_part(p, (int64_t)blockIdx.x * 128 + threadIdx.x, (int64_t)blockIdx.y * 256);
}

// Column split tiles: 64 columns of B by 128 k.  Lane l of warp w owns column
// j = j0 + 8 w + l / 4 and the k-groups of eight g = l % 4 + 4 r (r < 4): it
// reads them down its column and writes each group's digits straight into
// the K-major slice row j as one vector store per slice -- the transpose
// happens in registers.  Four adjacent lanes cover 32 consecutive k of one
// column, so each load instruction reads 64-byte runs of four rows of B and
// each store fills whole 32-byte sectors (64 bytes of BF16 or 32 of E4M3 per
// slice row).
constexpr int SC_J = 64, SC_K = 128;

template <int KIND>
__device__ __forceinline__ void split_cols_tile(const SplitB &p, int64_t jt, int64_t kt) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, kg = lane & 3;
    const int64_t j = jt * SC_J + 8 * warp + (lane >> 2);
    if (j >= p.M) return;
    const int64_t P = p.P, Pp = p.Pp, ldb = p.ldb;
    const int s = p.s;
    const int f = frexp_exp_bits(p.colmax[j]);
    if (kt == 0 && kg == 0) p.fb[j] = f;
    constexpr int beta = fmt_beta(KIND), es = fmt_esize(KIND);
    const int sh = beta * s - 1 - f;
    const double *__restrict__ bj = p.B + j;
    unsigned char *row0 = p.slices + j * Pp * es;
    const int64_t stride = (int64_t)p.Mr * Pp * es;
    // All 32 loads first, so they are in flight together.
    double x[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t k0 = kt * SC_K + 8 * (kg + 4 * r);
#pragma unroll
        for (int u = 0; u < 8; ++u) x[r][u] = (k0 + u < P) ? __ldg(bj + (k0 + u) * ldb) : 0.0;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t k0 = kt * SC_K + 8 * (kg + 4 * r);
        if (k0 >= Pp) break;  // Pp is a multiple of 8 (BF16) or 16 (E4M3)
        int64_t V[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) V[u] = round_scaled(x[r][u], sh);
        store_digits8<KIND>(V, s, row0 + k0 * es, stride);
    }
}

template <int KIND>
__global__ void __launch_bounds__(256) split_cols_kernel(const SplitB p) {
    split_cols_tile<KIND>(p, blockIdx.x, blockIdx.y);
}


// The grouped split kernels stride over their units (grid-stride loops), so
// one fixed grid serves any batch and a CUDA graph captured once per slice
// format and count is replayed for every batch.
__global__ void __launch_bounds__(256) group_zero_colmax_kernel(const EmuProblem *tab, const int64_t *begin,
                                                                const GroupHeader *hdr) {
    const int64_t units = hdr->units[U_ZERO];
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const int g = find_problem(begin, hdr->count, u);
        const SplitB &p = tab[g].spb;
        const int64_t j = (u - begin[g]) * 256 + threadIdx.x;
        if (j < p.M) p.colmax[j] = 0ull;
    }
}

template <int KIND>
__global__ void __launch_bounds__(kRowThreads, 4) group_split_rows_kernel(const EmuProblem *tab,
                                                                          const int64_t *begin,
                                                                          const GroupHeader *hdr) {
    __shared__ unsigned long long red[kRowThreads / 32];
    const int64_t units = hdr->units[U_ROWS];
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const int g = find_problem(begin, hdr->count, u);
        const SplitA &p = tab[g].spa;
        if (p.Pp <= kQuarterRowMax) {  // 32 rows per unit, 8 threads per row (the whole CTA takes this branch)
            const int64_t row = (u - begin[g]) * (kRowThreads / 8) + (threadIdx.x >> 3);
            const int64_t warp_row0 = (u - begin[g]) * (kRowThreads / 8) + ((threadIdx.x & ~31u) >> 3);
            if (warp_row0 < p.N) split_row<KIND, 8>(p, row, threadIdx.x & 7, nullptr, row < p.N);
        } else if (p.Pp <= kWarpRowMax) {  // 8 rows per unit, one per warp
            const int64_t row = (u - begin[g]) * (kRowThreads / 32) + (threadIdx.x >> 5);
            if (row < p.N) split_row<KIND, 32>(p, row, threadIdx.x & 31, nullptr);
        } else {  // one row per unit
            split_row<KIND, kRowThreads>(p, u - begin[g], threadIdx.x, red);
        }
    }
}

__global__ void __launch_bounds__(128) group_col_max_kernel(const EmuProblem *tab, const int64_t *begin,
                                                            const GroupHeader *hdr) {
    const int64_t units = hdr->units[U_COLMAX];
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const int g = find_problem(begin, hdr->count, u);
        const SplitB &p = tab[g].spb;
        const int64_t local = u - begin[g], nj = (p.M + 127) / 128;
        col_max_part(p, (local % nj) * 128 + threadIdx.x, (local / nj) * 256);
    }
}

template <int KIND>
__global__ void __launch_bounds__(256) group_split_cols_kernel(const EmuProblem *tab, const int64_t *begin,
                                                               const GroupHeader *hdr) {
    const int64_t units = hdr->units[U_SPLITCOLS];
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const int g = find_problem(begin, hdr->count, u);
        const SplitB &p = tab[g].spb;
        const int64_t local = u - begin[g], nj = (p.M + SC_J - 1) / SC_J;
        split_cols_tile<KIND>(p, local % nj, local / nj);
    }
}

cudaError_t slice_smem_attributes();

struct Layout {
    int s;
    int64_t Nr, Mr, Pp;
    size_t off_ea, off_fb, off_colmax, off_a, off_b, total;
};

// Slice rows are Pp elements long: a multiple of 16 bytes (TMA strides) and at
// least one K-block.
Layout layout(int64_t N, int64_t P, int64_t M, int s, int kind) {
    Layout L{};
    L.s = s;
    const int es = fmt_esize(kind), q = 16 / es;
    L.Nr = mm::ceil_div(std::max<int64_t>(N, 1), BM) * BM;
    L.Mr = mm::ceil_div(std::max<int64_t>(M, 1), BN) * BN;
    L.Pp = std::max<int64_t>(mm::ceil_div(std::max<int64_t>(P, 1), q) * q, fmt_bke(kind));
    size_t o = 0;
    L.off_ea = o;
    o += mm::align_up((size_t)L.Nr * 4, 1024);
    L.off_fb = o;
    o += mm::align_up((size_t)L.Mr * 4, 1024);
    L.off_colmax = o;
    o += mm::align_up((size_t)L.Mr * 8, 1024);
    L.off_a = o;
    o += mm::align_up((size_t)s * L.Nr * L.Pp * es, 1024);
    L.off_b = o;
    o += mm::align_up((size_t)s * L.Mr * L.Pp * es, 1024);
    L.total = o;
    return L;
}

// Slices [s][rows][Pp] of the slice format (FP8 as bytes); the K extent is Pp
// (zero-padded by the split kernels), K-blocks past Pp read the TMA zero fill.
// `slice_rows` is the row count from one slice to the next (>= rows; larger for
// a block of rows inside a taller slice).
int encode_slices(CUtensorMap *map, void *base, int64_t rows, int64_t Pp, int s, int box_rows, int kind,
                  int64_t slice_rows = 0) {
    mm::EncodeTiledFn enc = mm::encode_tiled_fn();
    if (!enc) return mm::fail(MM_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    const int es = fmt_esize(kind);
    if (slice_rows < rows) slice_rows = rows;
    cuuint64_t dims[3] = {(cuuint64_t)Pp, (cuuint64_t)rows, (cuuint64_t)s};
    cuuint64_t strides[2] = {(cuuint64_t)Pp * es, (cuuint64_t)(slice_rows * Pp * es)};
    cuuint32_t box[3] = {(cuuint32_t)fmt_bke(kind), (cuuint32_t)box_rows, (cuuint32_t)s};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = kind == MM_SLICE_FP8E4M3 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = enc(map, dt, 3, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return mm::fail(MM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return MM_OK;
}

// Per-launch constants shared by every problem of one slice format and count
// (the rest -- stages, exact chunk, TMEM columns -- follow from s at compile time).
void fill_common(EmuParams &prm, int s) { prm.s = s; }

size_t slice_smem_bytes(int s, int bn) { return (size_t)slice_stages(s, bn) * slice_stage_bytes(s, bn) + 1024; }


}  // namespace

namespace mm {

// Slice count for a tier, or for an explicit count: MM_ERR_ARG for an unknown
// format or an invalid request, MM_ERR_UNSUPPORTED when the tier needs more
// slices than the format's kernel holds (8 BF16 accumulators of 64 TMEM
// columns; 10 FP8-E4M3 ones of 32).
int emulated_slices(int32_t kind, int32_t nslices, double tier) {
    if (kind != MM_SLICE_BF16 && kind != MM_SLICE_FP8E4M3) return MM_ERR_ARG;
    if (nslices > 0) return nslices <= fmt_max_slices(kind) ? nslices : MM_ERR_ARG;
    if (!(tier > 0.0)) return MM_ERR_ARG;
    // beta*s - 1 bits of each row/column; about 8 more bits than -log2(tier) keep the
    // normwise error below the tier on wide-exponent inputs.
    const double need = (-log2(tier) + 9.0) / fmt_beta(kind);
    const int s = std::max(1, (int)ceil(need));
    if (s > fmt_max_slices(kind)) return MM_ERR_UNSUPPORTED;
    return s;
}

size_t emulated_ws_bytes(int64_t N, int64_t P, int64_t M, int s, int kind) {
    return layout(N, P, M, s, kind).total;
}

}  // namespace mm

namespace {

// Pointers of one product's split workspace (layout()).
struct EmuWork {
    Layout L;
    int32_t *ea, *fb;
    unsigned long long *colmax;
    unsigned char *sa, *sb;
};

EmuWork emu_work(int64_t N, int64_t P, int64_t M, int s, int kind, void *ws) {
    EmuWork w;
    w.L = layout(N, P, M, s, kind);
    char *b = (char *)ws;
    w.ea = (int32_t *)(b + w.L.off_ea);
    w.fb = (int32_t *)(b + w.L.off_fb);
    w.colmax = (unsigned long long *)(b + w.L.off_colmax);
    w.sa = (unsigned char *)(b + w.L.off_a);
    w.sb = (unsigned char *)(b + w.L.off_b);
    return w;
}

// Column exponents and slices of columns [c0, c0 + m) of B (B points at
// column c0; c0 = 0 and m = M for all of B).
int split_b(const EmuWork &w, int64_t c0, int64_t P, int64_t m, const double *B, int64_t ldb, int s, int kind,
            cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(w.colmax + c0, 0, (size_t)m * 8, st);
    if (e != cudaSuccess) return mm::cuda_fail(e, "mm_emulated");
    const SplitB spb{P, m, ldb, w.L.Mr, w.L.Pp, B, s, w.colmax + c0, w.fb + c0,
                     w.sb + (size_t)c0 * w.L.Pp * fmt_esize(kind)};
    int rc = mm::launch("emu_col_max", st, [&] {
        dim3 g((unsigned)mm::ceil_div(m, 128), (unsigned)mm::ceil_div(P, 256));
        col_max_kernel<<<g, 128, 0, st>>>(spb);
    });
    if (rc) return rc;
    return mm::launch("emu_split_cols", st, [&] {
        dim3 g((unsigned)mm::ceil_div(m, SC_J), (unsigned)mm::ceil_div(w.L.Pp, SC_K));
        if (kind == MM_SLICE_FP8E4M3)
            split_cols_kernel<MM_SLICE_FP8E4M3><<<g, 256, 0, st>>>(spb);
        else
            split_cols_kernel<MM_SLICE_BF16><<<g, 256, 0, st>>>(spb);
    });
}

// Rows [r0, r0 + n) of A (A points at row r0): exponents and slices.
int split_a_rows(const EmuWork &w, int64_t r0, int64_t n, int64_t P, const double *A, int64_t lda, int s, int kind,
                 cudaStream_t st) {
    const SplitA spa{n, P, lda, w.L.Nr, w.L.Pp, A, s, w.ea + r0,
                     w.sa + (size_t)r0 * w.L.Pp * fmt_esize(kind)};
    return mm::launch("emu_split_rows", st, [&] {
        const bool fp8 = kind == MM_SLICE_FP8E4M3;
        if (w.L.Pp <= kQuarterRowMax) {
            const unsigned g = (unsigned)mm::ceil_div(n, kRowThreads / 8);
            if (fp8)
                split_rows_quarter_kernel<MM_SLICE_FP8E4M3><<<g, kRowThreads, 0, st>>>(spa);
            else
                split_rows_quarter_kernel<MM_SLICE_BF16><<<g, kRowThreads, 0, st>>>(spa);
        } else if (w.L.Pp <= kWarpRowMax) {
            const unsigned g = (unsigned)mm::ceil_div(n, kRowThreads / 32);
            if (fp8)
                split_rows_warp_kernel<MM_SLICE_FP8E4M3><<<g, kRowThreads, 0, st>>>(spa);
            else
                split_rows_warp_kernel<MM_SLICE_BF16><<<g, kRowThreads, 0, st>>>(spa);
        } else if (fp8) {
            split_rows_kernel<MM_SLICE_FP8E4M3><<<(unsigned)n, kRowThreads, 0, st>>>(spa);
        } else {
            split_rows_kernel<MM_SLICE_BF16><<<(unsigned)n, kRowThreads, 0, st>>>(spa);
        }
    });
}

// The slice product for rows [r0, r0 + n) and columns [c0, c0 + m) of C (r0
// a multiple of the tile height, c0 of the tile width; C points at (r0, c0)).
int slice_product(const EmuWork &w, int64_t r0, int64_t n, int64_t c0, int64_t m, int64_t P, double *C, int64_t ldc,
                  int s, int kind, cudaStream_t st, int bn) {
    CUtensorMap tmA, tmB;
    const size_t es = fmt_esize(kind);
    const int64_t nr = mm::ceil_div(n, BM) * BM, mr = mm::ceil_div(m, bn) * bn;
    int rc = encode_slices(&tmA, w.sa + (size_t)r0 * w.L.Pp * es, nr, w.L.Pp, s, BM, kind, w.L.Nr);
    if (!rc) rc = encode_slices(&tmB, w.sb + (size_t)c0 * w.L.Pp * es, mr, w.L.Pp, s, bn, kind, w.L.Mr);
    if (rc) return rc;
    EmuParams prm{};
    fill_common(prm, s);
    prm.N = n;
    prm.P = P;
    prm.M = m;
    prm.tiles_m = (int)mm::ceil_div(n, BM);
    prm.tiles_n = (int)mm::ceil_div(m, bn);
    prm.ea = w.ea + r0;
    prm.fb = w.fb + c0;
    prm.C = C;
    prm.ldc = ldc;
    prm.status = mm::device_status_ptr();
    const size_t smem = slice_smem_bytes(s, bn);
    const cudaError_t attr_err = slice_smem_attributes();
    if (attr_err != cudaSuccess) return mm::cuda_fail(attr_err, "mm_emulated: shared memory attribute");
    const int64_t tiles = (int64_t)prm.tiles_m * prm.tiles_n;
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, mm::sm_count());  // persistent: one CTA per SM
    const bool fp8 = kind == MM_SLICE_FP8E4M3;
    cudaError_t le = cudaSuccess;
    rc = mm::launch(fp8 ? "emu_slice_gemm_tcgen05_fp8" : "emu_slice_gemm_tcgen05", st, [&] {
        le = fp8 ? launch_slice_gemm_fp8(s, bn, grid, smem, st, tmA, tmB, prm)
                 : launch_slice_gemm_bf16(s, bn, grid, smem, st, tmA, tmB, prm);
    });
    if (!rc && le != cudaSuccess) return mm::cuda_fail(le, "mm_emulated: slice count");
    return rc;
}

}  // namespace

namespace mm {

int run_emulated(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                 double *C, int64_t ldc, int s, int kind, void *ws, cudaStream_t st, int bn) {
    if (bn == 0) bn = slice_bn(s);
    if (!slice_bn_ok(s, bn))
        return fail(MM_ERR_ARG, "mm_emulated: tile width %d (64 up to 8 slices, or 32)", bn);
    const EmuWork w = emu_work(N, P, M, s, kind, ws);
    int rc = split_a_rows(w, 0, N, P, A, lda, s, kind, st);
    if (!rc) rc = split_b(w, 0, P, M, B, ldb, s, kind, st);
    if (!rc) rc = slice_product(w, 0, N, 0, M, P, C, ldc, s, kind, st, bn);
    return rc;
}

// Host operands: device copies of A, B and C and the split workspace are carved
// from ws.  One copy stream carries the first row block of A, the column
// blocks of B, then the other row blocks of A; each block of A or B is split
// on the caller's stream as soon as it lands, each block product of C follows
// the splits it needs, and its block of C comes back on a second copy stream
// as soon as it is done, so transfers overlap the products of other blocks.
// The caller's stream waits for the last copy back, and the copy streams wait
// for the caller's earlier work, so consecutive calls on one stream stay
// ordered.  Every block of C is computed exactly as in the one-launch product.
size_t emulated_host_ws_bytes(int64_t N, int64_t P, int64_t M, int s, int kind) {
    return align_up((size_t)N * P * 8, 1024) + align_up((size_t)P * M * 8, 1024) + align_up((size_t)N * M * 8, 1024) +
           layout(N, P, M, s, kind).total;
}

namespace {
struct CopyStreams {
    cudaStream_t up = nullptr, down = nullptr;
};
std::mutex g_copy_mu;
std::vector<CopyStreams> g_copy;

int copy_streams(CopyStreams *out) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(g_copy_mu);
    if ((int)g_copy.size() <= dev) g_copy.resize(dev + 1);
    CopyStreams &c = g_copy[dev];
    if (!c.up) {
        cudaError_t e = cudaStreamCreateWithFlags(&c.up, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.down, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "mm_emulated_host: copy streams");
    }
    *out = c;
    return MM_OK;
}
}  // namespace

int run_emulated_host(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                      double *C, int64_t ldc, int s, int kind, void *ws, cudaStream_t st) {
    CopyStreams cs;
    int rc = copy_streams(&cs);
    if (rc) return rc;
    char *w8 = (char *)ws;
    double *dA = (double *)w8;
    w8 += align_up((size_t)N * P * 8, 1024);
    double *dB = (double *)w8;
    w8 += align_up((size_t)P * M * 8, 1024);
    double *dC = (double *)w8;
    w8 += align_up((size_t)N * M * 8, 1024);
    const EmuWork w = emu_work(N, P, M, s, kind, w8);
    // C in blocks: up to 8 row blocks of whole tiles, and for large products
    // (N >= 4096, M >= 2048) two column blocks, with row blocks sized so each
    // block product fills whole waves (four column blocks throughout measured
    // slower: 16 launches of 4 waves each).  B goes up in pieces -- the first
    // column block in two halves, then the second block -- and the first row
    // block is multiplied by each piece as it lands, so the first product waits
    // for one block of A and a quarter of B; the last block's copy back trails
    // the products.
    const int64_t cb = N >= 4096 && M >= 2048 ? 2 : 1;
    const int64_t nb = std::max<int64_t>(1, std::min<int64_t>(8 / cb, ceil_div(N, 512 * cb)));
    int64_t R = ceil_div(ceil_div(N, nb), BM) * BM;
    const int64_t Mh = ceil_div(ceil_div(M, cb), (int64_t)BN) * BN;  // column block width
    if (cb > 1) {
        // Row blocks of 8 to 24 tile rows, the height whose block products come
        // closest to whole waves of the persistent kernel (ties: the shorter, so
        // the first product starts sooner); e.g. 19 tile rows x 64 tile columns
        // = 8 waves of 152 SMs.
        const int64_t tn = ceil_div(Mh, (int64_t)slice_bn(s)), sms = sm_count();
        double best = 2.0;
        for (int64_t tr = 8; tr <= 24; ++tr) {
            const int64_t t = tr * tn;
            const double waste = (double)(ceil_div(t, sms) * sms - t) / (double)t;
            if (waste < best - 1e-9) best = waste, R = tr * BM;
        }
    }
    // Column blocks (every row block but the first) and pieces of B (the first
    // row block): [c0, c0 + width).
    const int64_t Q = cb > 1 ? ceil_div(ceil_div(Mh, 2), (int64_t)BN) * BN : M;
    const int64_t blk_c0[2] = {0, Mh}, blk_m[2] = {std::min(Mh, M), cb > 1 ? M - Mh : 0};
    const int64_t pc_c0[3] = {0, Q, Mh}, pc_m[3] = {Q, cb > 1 ? Mh - Q : 0, cb > 1 ? M - Mh : 0};
    std::vector<cudaEvent_t> ev;
    auto event = [&](cudaEvent_t *e) {
        cudaError_t r = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
        if (r == cudaSuccess) ev.push_back(*e);
        return r;
    };
    auto done = [&](int r) {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);  // released once their work completes
        return r;
    };
    // All uploads go through one copy stream in the order they are needed: the
    // first block of A, the pieces of B, then the other blocks of A, so the
    // link is not shared with blocks that cannot start yet.
    cudaEvent_t e0, eB[3] = {}, eA, eC, eEnd;
    cudaError_t e = event(&e0);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs.up, e0, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs.down, e0, 0);
    if (e != cudaSuccess) return done(cuda_fail(e, "mm_emulated_host"));
    auto upload_b = [&](int j) {
        if (pc_m[j] <= 0) return cudaSuccess;
        cudaError_t r = cudaMemcpy2DAsync(dB + pc_c0[j], (size_t)M * 8, B + pc_c0[j], (size_t)ldb * 8,
                                          (size_t)pc_m[j] * 8, P, cudaMemcpyHostToDevice, cs.up);
        if (r == cudaSuccess) r = event(&eB[j]);
        if (r == cudaSuccess) r = cudaEventRecord(eB[j], cs.up);
        return r;
    };
    // The block product of rows [r0, r0 + n) and columns [c0, c0 + m), and its copy back.
    auto product = [&](int64_t r0, int64_t n, int64_t c0, int64_t m) {
        int r = slice_product(w, r0, n, c0, m, P, dC + r0 * M + c0, M, s, kind, st, slice_bn(s));
        if (r) return r;
        cudaError_t x = event(&eC);
        if (x == cudaSuccess) x = cudaEventRecord(eC, st);
        if (x == cudaSuccess) x = cudaStreamWaitEvent(cs.down, eC, 0);
        if (x == cudaSuccess)
            x = cudaMemcpy2DAsync(C + r0 * ldc + c0, (size_t)ldc * 8, dC + r0 * M + c0, (size_t)M * 8,
                                  (size_t)m * 8, n, cudaMemcpyDeviceToHost, cs.down);
        return x == cudaSuccess ? MM_OK : cuda_fail(x, "mm_emulated_host");
    };
    for (int64_t r0 = 0; r0 < N; r0 += R) {
        const int64_t n = std::min(R, N - r0);
        e = cudaMemcpy2DAsync(dA + r0 * P, (size_t)P * 8, A + r0 * lda, (size_t)lda * 8, (size_t)P * 8, n,
                              cudaMemcpyHostToDevice, cs.up);
        if (e == cudaSuccess) e = event(&eA);
        if (e == cudaSuccess) e = cudaEventRecord(eA, cs.up);
        if (r0 == 0)
            for (int j = 0; j < 3 && e == cudaSuccess; ++j) e = upload_b(j);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, eA, 0);
        if (e != cudaSuccess) return done(cuda_fail(e, "mm_emulated_host"));
        rc = split_a_rows(w, r0, n, P, dA + r0 * P, P, s, kind, st);
        if (rc) return done(rc);
        if (r0 == 0) {  // each piece of B is split as soon as it lands, then multiplied
            for (int j = 0; j < 3; ++j) {
                if (pc_m[j] <= 0) continue;
                e = cudaStreamWaitEvent(st, eB[j], 0);
                if (e != cudaSuccess) return done(cuda_fail(e, "mm_emulated_host"));
                rc = split_b(w, pc_c0[j], P, pc_m[j], dB + pc_c0[j], M, s, kind, st);
                if (!rc) rc = product(r0, n, pc_c0[j], pc_m[j]);
                if (rc) return done(rc);
            }
            continue;
        }
        for (int j = 0; j < 2; ++j) {
            if (blk_m[j] <= 0) continue;
            rc = product(r0, n, blk_c0[j], blk_m[j]);
            if (rc) return done(rc);
        }
    }
    e = event(&eEnd);
    if (e == cudaSuccess) e = cudaEventRecord(eEnd, cs.down);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, eEnd, 0);
    if (e != cudaSuccess) return done(cuda_fail(e, "mm_emulated_host"));
    return done(MM_OK);
}

}  // namespace mm

// ------------------------------------------------------- grouped host side

namespace {

size_t slices_bytes(int64_t rows_padded, int64_t Pp, int s, int kind) {
    return mm::align_up((size_t)s * rows_padded * Pp * fmt_esize(kind), 1024);
}


cudaError_t slice_smem_attributes() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        err = slice_gemm_smem_attributes_bf16(kSmemLimit - 1024);
        if (err == cudaSuccess) err = slice_gemm_smem_attributes_fp8(kSmemLimit - 1024);
    });
    return err;
}

}  // namespace

namespace mm {

// A grouped launch's memory: a table part (problem table, header, prefix
// arrays), and per problem a data region [column maxima | e | f | A slices |
// B slices].  mm_emulated_group places the data regions right after the
// table; the serving loop keeps each request's region with its operands.
// The table part is laid out for a fixed capacity (>= the problem count) so
// that its header and prefix arrays sit at the same addresses for every
// batch: a CUDA graph captured for one batch is replayed for others.
struct GroupLayout {
    size_t off_table, off_hdr, off_begin[5], table_bytes;
};

static GroupLayout group_layout(int count) {
    GroupLayout g{};
    size_t o = 0;
    g.off_table = o;
    o += align_up((size_t)count * sizeof(EmuProblem), 256);
    g.off_hdr = o;
    o += align_up(sizeof(GroupHeader), 256);
    for (int k = 0; k < 5; ++k) {
        g.off_begin[k] = o;
        o += align_up((size_t)(count + 1) * 8, 256);
    }
    g.table_bytes = align_up(o, 1024);
    return g;
}

size_t group_table_bytes(int count) { return group_layout(count).table_bytes; }

size_t problem_data_bytes(const mm_problem &q, int s, int kind) {
    const Layout L = layout(q.N, q.P, q.M, s, kind);
    return align_up((size_t)L.Mr * 8, 1024) + align_up((size_t)L.Nr * 4, 1024) + align_up((size_t)L.Mr * 4, 1024) +
           slices_bytes(L.Nr, L.Pp, s, kind) + slices_bytes(L.Mr, L.Pp, s, kind);
}

size_t group_data_bytes(const mm_problem *probs, int count, int s, int kind) {
    size_t d = 0;
    for (int i = 0; i < count; ++i) d += problem_data_bytes(probs[i], s, kind);
    return d;
}

size_t emulated_group_ws_bytes(const mm_problem *probs, int count, int s, int kind) {
    if (count <= 0) return 0;
    return group_table_bytes(count) + group_data_bytes(probs, count, s, kind);
}

// The five kernels of a grouped launch (no memset or copy: capturable).
// Fixed grid of each grouped kernel: enough CTAs to fill the GPU, each
// striding over the units (the slice product is persistent, one CTA per SM).
int64_t group_grid_cap(int kernel) {
    const int64_t sms = sm_count();
    switch (kernel) {
    case U_TILES:
        return sms;
    case U_SPLITCOLS:
        return 4 * sms;
    default:
        return 8 * sms;
    }
}

int group_kernels(const GroupLaunch &gl, cudaStream_t st) {
    cudaError_t e = slice_smem_attributes();
    if (e != cudaSuccess) return cuda_fail(e, "grouped emulated product: shared memory attribute");
    int rc = MM_OK;
    if (gl.grid[U_ZERO] > 0)
        rc = launch("emu_group_zero_colmax", st, [&] {
            group_zero_colmax_kernel<<<(unsigned)gl.grid[U_ZERO], 256, 0, st>>>(
                (const EmuProblem *)gl.tab, gl.begin[U_ZERO], (const GroupHeader *)gl.hdr);
        });
    if (rc) return rc;
    if (gl.grid[U_ROWS] > 0)
        rc = launch("emu_group_split_rows", st, [&] {
            const auto k = gl.kind == MM_SLICE_FP8E4M3 ? group_split_rows_kernel<MM_SLICE_FP8E4M3>
                                                       : group_split_rows_kernel<MM_SLICE_BF16>;
            k<<<(unsigned)gl.grid[U_ROWS], kRowThreads, 0, st>>>((const EmuProblem *)gl.tab, gl.begin[U_ROWS],
                                                         (const GroupHeader *)gl.hdr);
        });
    if (rc) return rc;
    if (gl.grid[U_COLMAX] > 0)
        rc = launch("emu_group_col_max", st, [&] {
            group_col_max_kernel<<<(unsigned)gl.grid[U_COLMAX], 128, 0, st>>>((const EmuProblem *)gl.tab,
                                                                                gl.begin[U_COLMAX],
                                                                                (const GroupHeader *)gl.hdr);
        });
    if (rc) return rc;
    if (gl.grid[U_SPLITCOLS] > 0)
        rc = launch("emu_group_split_cols", st, [&] {
            const auto k = gl.kind == MM_SLICE_FP8E4M3 ? group_split_cols_kernel<MM_SLICE_FP8E4M3>
                                                       : group_split_cols_kernel<MM_SLICE_BF16>;
            k<<<(unsigned)gl.grid[U_SPLITCOLS], 256, 0, st>>>(
                (const EmuProblem *)gl.tab, gl.begin[U_SPLITCOLS], (const GroupHeader *)gl.hdr);
        });
    if (rc) return rc;
    const unsigned tiles_grid = (unsigned)std::min<int64_t>(gl.grid[U_TILES], sm_count());  // persistent
    if (gl.grid[U_TILES] > 0) {
        const bool fp8 = gl.kind == MM_SLICE_FP8E4M3;
        cudaError_t le = cudaSuccess;
        rc = launch(fp8 ? "emu_group_slice_gemm_tcgen05_fp8" : "emu_group_slice_gemm_tcgen05", st, [&] {
            const auto *tab = (const EmuProblem *)gl.tab;
            const auto *hdr = (const GroupHeader *)gl.hdr;
            const size_t smem = slice_smem_bytes(gl.s, gl.bn);
            le = fp8 ? launch_group_slice_gemm_fp8(gl.s, gl.bn, tiles_grid, smem, st, tab, gl.begin[U_TILES], hdr)
                     : launch_group_slice_gemm_bf16(gl.s, gl.bn, tiles_grid, smem, st, tab, gl.begin[U_TILES], hdr);
        });
        if (!rc && le != cudaSuccess) return cuda_fail(le, "grouped emulated product: slice count");
    }
    return rc;
}

// Builds the host image of the table part for the problems (all N, P, M >= 1)
// -- to be copied to `table_dev` -- and the launch description.  data[i] is
// problem i's data region of problem_data_bytes(probs[i], s, kind) bytes; the
// table is laid out for `capacity` problems (>= count).
int group_build(const mm_problem *probs, int count, int capacity, int s, void *table_dev, char *const *data,
                std::vector<unsigned char> &image, GroupLaunch &gl, int kind, int bn) {
    if (capacity < count) return fail(MM_ERR_ARG, "grouped launch: %d problems exceed capacity %d", count, capacity);
    if (bn == 0) bn = slice_bn(s);
    if (!slice_bn_ok(s, bn)) return fail(MM_ERR_ARG, "grouped launch: tile width %d", bn);
    const GroupLayout G = group_layout(capacity);
    char *t = (char *)table_dev;
    image.assign(G.table_bytes, 0);
    EmuProblem *tab = (EmuProblem *)(image.data() + G.off_table);
    GroupHeader *hdr = (GroupHeader *)(image.data() + G.off_hdr);
    int64_t *begin[5];
    for (int k = 0; k < 5; ++k) begin[k] = (int64_t *)(image.data() + G.off_begin[k]);
    int64_t units[5] = {0, 0, 0, 0, 0};
    int *status = device_status_ptr();
    // Table order = launch order: the persistent slice kernel deals tiles out
    // round-robin in table order, so the problems with the longest inner
    // dimension (the longest tiles) go first and the short ones fill the end,
    // which evens out the CTAs' finishing times.  Each problem keeps its own
    // data region; any order gives the same results.
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return probs[x].P > probs[y].P; });
    for (int i = 0; i < count; ++i) {
        const mm_problem &q = probs[order[i]];
        const Layout L = layout(q.N, q.P, q.M, s, kind);
        EmuProblem &e = tab[i];
        char *w = data[order[i]];
        unsigned long long *cm = (unsigned long long *)w;
        w += align_up((size_t)L.Mr * 8, 1024);
        int32_t *ea = (int32_t *)w;
        w += align_up((size_t)L.Nr * 4, 1024);
        int32_t *fb = (int32_t *)w;
        w += align_up((size_t)L.Mr * 4, 1024);
        unsigned char *sa = (unsigned char *)w;
        w += slices_bytes(L.Nr, L.Pp, s, kind);
        unsigned char *sb = (unsigned char *)w;
        e.spa = SplitA{q.N, q.P, q.lda, L.Nr, L.Pp, q.A, s, ea, sa};
        e.spb = SplitB{q.P, q.M, q.ldb, L.Mr, L.Pp, q.B, s, cm, fb, sb};
        fill_common(e.prm, s);
        e.prm.N = q.N;
        e.prm.P = q.P;
        e.prm.M = q.M;
        e.prm.tiles_m = (int)ceil_div(q.N, BM);
        e.prm.tiles_n = (int)ceil_div(q.M, bn);
        e.prm.ea = ea;
        e.prm.fb = fb;
        e.prm.C = q.C;
        e.prm.ldc = q.ldc;
        e.prm.status = status;
        int rc = encode_slices(&e.tmA, sa, L.Nr, L.Pp, s, BM, kind);
        if (!rc) rc = encode_slices(&e.tmB, sb, L.Mr, L.Pp, s, bn, kind);
        if (rc) return rc;
        for (int k = 0; k < 5; ++k) begin[k][i] = units[k];
        units[U_ROWS] += L.Pp <= kQuarterRowMax ? ceil_div(q.N, kRowThreads / 8)
                         : L.Pp <= kWarpRowMax  ? ceil_div(q.N, kRowThreads / 32)
                                                : q.N;
        units[U_COLMAX] += ceil_div(q.M, 128) * ceil_div(q.P, 256);
        units[U_SPLITCOLS] += ceil_div(q.M, SC_J) * ceil_div(L.Pp, SC_K);
        units[U_TILES] += (int64_t)e.prm.tiles_m * e.prm.tiles_n;
        units[U_ZERO] += ceil_div(q.M, 256);
    }
    hdr->count = count;
    for (int k = 0; k < 5; ++k) {
        begin[k][count] = units[k];
        hdr->units[k] = units[k];
        gl.grid[k] = std::min(units[k], group_grid_cap(k));
        gl.begin[k] = (const int64_t *)(t + G.off_begin[k]);
    }
    gl.tab = t + G.off_table;
    gl.hdr = t + G.off_hdr;
    gl.s = s;
    gl.kind = kind;
    gl.bn = bn;
    return MM_OK;
}

int run_emulated_group(const mm_problem *probs, int count, int s, int kind, void *ws, cudaStream_t st) {
    std::vector<mm_problem> live;
    live.reserve(count);
    for (int i = 0; i < count; ++i) {
        const mm_problem &q = probs[i];
        if (q.N == 0 || q.M == 0) continue;
        if (q.P == 0) {
            int rc = run_zero(q.N, q.M, q.C, q.ldc, st);
            if (rc) return rc;
            continue;
        }
        live.push_back(q);
    }
    if (live.empty()) return MM_OK;
    std::vector<unsigned char> image;
    GroupLaunch gl{};
    std::vector<char *> data(live.size());
    char *d = (char *)ws + group_table_bytes((int)live.size());
    for (size_t i = 0; i < live.size(); ++i) {
        data[i] = d;
        d += problem_data_bytes(live[i], s, kind);
    }
    int rc = group_build(live.data(), (int)live.size(), (int)live.size(), s, ws, data.data(), image, gl, kind);
    if (rc) return rc;
    // Pageable source: the copy is staged before cudaMemcpyAsync returns, so `image` may go.
    cudaError_t e = cudaMemcpyAsync((void *)gl.tab, image.data(), image.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "grouped emulated product: table upload");
    return group_kernels(gl, st);
}

}  // namespace mm

// ---------------------------------------------------------------------------
// Allocation-free variant of the emulated product.
//
// Some callers cannot allocate device memory for a workspace: for example a
// host application that owns every byte of the device's memory through its
// own pool and forbids other allocations, or a latency-critical loop in which
// an allocation (and the synchronisation it can imply) is not acceptable.
// For them the scratch space -- the row/column exponents, the column maxima
// and the BF16 slices -- lives in this fixed device array instead of a
// caller-supplied workspace.  Every GPU that loads the library holds these
// 64 MiB until the process exits.  All calls share the array, so calls that
// overlap on the GPU (different streams, or different host threads on the same
// device) race on it and must be serialised by the caller.
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on the current device, looked up once per
// device (the first call on each device does this set-up).
static int noalloc_scratch_ptr(void **out) {
    static std::mutex mu;
    static void *ptrs[64] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return mm::cuda_fail(e, "mm_emulated_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) return mm::fail(MM_ERR_UNSUPPORTED, "mm_emulated_noalloc: device index %d", dev);
    std::lock_guard<std::mutex> g(mu);
    if (!ptrs[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return mm::cuda_fail(e, "mm_emulated_noalloc: cudaGetSymbolAddress");
        ptrs[dev] = p;
    }
    *out = ptrs[dev];
    return MM_OK;
}

namespace mm {

size_t emulated_noalloc_capacity() { return kNoAllocScratchBytes; }

int run_emulated_noalloc(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                         int64_t ldb, double *C, int64_t ldc, int s, int kind, cudaStream_t st) {
    const size_t need = emulated_ws_bytes(N, P, M, s, kind);
    if (need > kNoAllocScratchBytes)
        return fail(MM_ERR_NOMEM,
                    "mm_emulated_noalloc: this product needs %zu bytes of scratch, more than the %zu-byte static "
                    "array; call mm_emulated with a workspace instead",
                    need, kNoAllocScratchBytes);
    void *scratch = nullptr;
    int rc = noalloc_scratch_ptr(&scratch);
    if (rc) return rc;
    // The only region that must start at zero (the column maxima) is cleared by
    // run_emulated itself on every call; everything else is fully rewritten.
    return run_emulated(N, P, M, A, lda, B, ldb, C, ldc, s, kind, scratch, st);
}

}  // namespace mm
