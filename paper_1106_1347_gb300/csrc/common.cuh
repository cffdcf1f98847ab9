// Internal helpers shared by the libmm translation units: status reporting,
// kernel-timing hooks, and the inline-PTX wrappers (mbarrier, TMA, tcgen05)
// used by the sm_103a kernels.  Nothing here is part of the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "mm.h"

namespace mm {

// ---------------------------------------------------------------- host status

void set_error(const char *fmt, ...);
int fail(int status, const char *fmt, ...);  // set_error + return status
int cuda_fail(cudaError_t e, const char *what);

// Device status word the kernels raise when a bounded wait gives up.
int *device_status_ptr();
// Streaming multiprocessors of the current device (cached per device).
int sm_count();

constexpr int kStatusTimeoutTma = 1;
constexpr int kStatusTimeoutMma = 2;
constexpr int kStatusTimeoutEpi = 4;
constexpr int kStatusTimeoutSelftest = 8;  // mm_selftest_wait_timeout
int run_selftest_wait(void *stream);

// Kernel timing: begin/end bracket one launch on `stream` when profiling is on.
void prof_begin(const char *name, cudaStream_t stream);
void prof_end(cudaStream_t stream);

template <typename F>
int launch(const char *name, cudaStream_t stream, F &&body) {
    prof_begin(name, stream);
    body();
    cudaError_t e = cudaGetLastError();
    prof_end(stream);
    if (e != cudaSuccess) return cuda_fail(e, name);
    return MM_OK;
}

// Driver entry point for cuTensorMapEncodeTiled (no -lcuda needed).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn();

inline bool ranges_overlap(const void *a, size_t abytes, const void *b, size_t bbytes) {
    uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
    return a0 < b0 + bbytes && b0 < a0 + abytes;
}
inline size_t span_bytes(int64_t rows, int64_t cols, int64_t ld) {
    if (rows <= 0 || cols <= 0) return 0;
    return (size_t)((rows - 1) * ld + cols) * sizeof(double);
}
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Side of the square output tile of a CUDA-core or FP64-MMA kernel, from
// `sides` (largest first): the one whose grid of tiles fills the SMs' waves
// best (ctas / (waves * SMs), waves = ceil(ctas / SMs)), the larger one when
// two are within 2% (fewer operand reloads); `batch` grids of that size run
// together.  Small products then take small tiles and keep every SM busy.
inline int pick_tile(int64_t N, int64_t M, const int *sides, int count, int64_t batch = 1) {
    const int64_t sms = sm_count();
    int best = sides[0];
    double best_eff = -1.0;
    for (int i = 0; i < count; ++i) {
        const int64_t ctas = ceil_div(N, sides[i]) * ceil_div(M, sides[i]) * batch;
        const double eff = (double)ctas / (double)(ceil_div(ctas, sms) * sms);
        if (eff > best_eff + 0.02) {
            best = sides[i];
            best_eff = eff;
        }
    }
    return best;
}

// Checks shared by every C = A B entry point.  Returns MM_OK or MM_ERR_ARG.
int check_gemm_args(const char *fn, int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                    int64_t ldb, const double *C, int64_t ldc);

// Launchers (one per translation unit).
int run_norm_inf(int64_t N, int64_t P, const double *A, int64_t lda, double *out, cudaStream_t st);
int run_zero(int64_t N, int64_t M, double *C, int64_t ldc, cudaStream_t st);
int run_naive(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
              int64_t ldc, cudaStream_t st);
int run_unrolled(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                 double *C, int64_t ldc, int unroll, cudaStream_t st);
int run_kahan(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
              int64_t ldc, cudaStream_t st);
// mode: 0 WinogradOriginal, 1 Brent's global lambda, 2 per-row/column exponents.
size_t winograd_ws_bytes(int64_t N, int64_t P, int64_t M, int mode);
int run_winograd(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                 double *C, int64_t ldc, int mode, int32_t *lambda_out, void *ws, cudaStream_t st);
int strassen_plan(int variant, int64_t N, int64_t P, int64_t M, int32_t cutoff, int *depth, int64_t *Np,
                  int64_t *Pp, int64_t *Mp);
bool tuned_strassen_depth(int variant, int64_t N, int64_t P, int64_t M, int *depth);
// Deepest Strassen-Winograd recursion chosen without being asked for by
// depth (cutoff -1: the default and the tuner): its normwise error about
// doubles per level on uniform inputs (measured 3.0e-15 at 6 levels and
// 3.5e-14 at 9, 8192^3), so 6 levels keep a margin under 1e-14.
constexpr int kWinogradSafeDepth = 6;
// The emulated product's slice format, count and Strassen-Winograd levels for
// a tier (tune.cu): the tuned entry of the shape bucket (returns 1), else the
// model (returns 0); negative for an invalid or unreachable tier.
int emulated_choice(int64_t N, int64_t P, int64_t M, double tier, int *kind, int *slices, int *levels, int *tile);
size_t strassen_ws_bytes(int variant, int depth, int64_t Np, int64_t Pp, int64_t Mp);
int run_strassen(int variant, int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                 int64_t ldb, double *C, int64_t ldc, int depth, int64_t Np, int64_t Pp, int64_t Mp, void *ws,
                 cudaStream_t st);
// One fused recursion level (gemm_f64.cu) for `nodes` equal nodes at fixed
// element strides za, zb, zc: node z's operands are 2n x 2p (reads past
// arows x acols are 0) and 2p x 2m, its result 2n x 2m (writes past
// crows x ccols dropped).
int run_strassen_level(int variant, int64_t nodes, int64_t n, int64_t p, int64_t m, const double *A, int64_t lda,
                       int64_t arows, int64_t acols, int64_t za, const double *B, int64_t ldb, int64_t brows,
                       int64_t bcols, int64_t zb, double *C, int64_t ldc, int64_t crows, int64_t ccols, int64_t zc,
                       cudaStream_t st);
int emulated_slices(int32_t kind, int32_t nslices, double tier);
// kind: MM_SLICE_BF16 or MM_SLICE_FP8E4M3.
size_t emulated_ws_bytes(int64_t N, int64_t P, int64_t M, int s, int kind);
// bn: the slice product's tile width (64 or 32 columns; 0: 64 up to 8 slices, 32 beyond).
int run_emulated(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                 double *C, int64_t ldc, int s, int kind, void *ws, cudaStream_t st,
                 int bn = 0);
size_t emulated_group_ws_bytes(const mm_problem *probs, int count, int s, int kind);
size_t emulated_host_ws_bytes(int64_t N, int64_t P, int64_t M, int s, int kind);
int run_emulated_host(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                      double *C, int64_t ldc, int s, int kind, void *ws, cudaStream_t st);

// Pieces of a grouped emulated launch, for runtimes that place the table part
// (problem table, header, prefix arrays) and the data part (column maxima,
// exponents, slices) themselves and replay the kernels from CUDA graphs.
struct GroupLaunch {
    const void *tab, *hdr;    // device table and header (table part)
    const int64_t *begin[5];  // device prefix arrays
    int64_t grid[5];          // CTAs per kernel (grid-stride kernels: any size works)
    int s, kind;              // slice count and format
    int bn;                   // tile width of the slice product
};
size_t group_table_bytes(int count);
size_t problem_data_bytes(const mm_problem &q, int s, int kind = MM_SLICE_BF16);
size_t group_data_bytes(const mm_problem *probs, int count, int s, int kind = MM_SLICE_BF16);
int group_build(const mm_problem *probs, int count, int capacity, int s, void *table_dev, char *const *data,
                std::vector<unsigned char> &image, GroupLaunch &gl, int kind = MM_SLICE_BF16, int bn = 0);
int group_kernels(const GroupLaunch &gl, cudaStream_t st);
int64_t group_grid_cap(int kernel);  // fixed grid of grouped kernel `kernel` (0..4)
void prof_suspend(bool on);  // skip kernel timing while a stream is being captured
int run_emulated_group(const mm_problem *probs, int count, int s, int kind, void *ws, cudaStream_t st);
// Strassen (variant 0) / Strassen-Winograd (1) levels over the emulated product.
int strassen_emulated_levels(int levels, int64_t N, int64_t P, int64_t M);  // resolves levels == -1
size_t strassen_emulated_ws_bytes(int variant, int levels, int64_t N, int64_t P, int64_t M, int s, int kind);
int run_strassen_emulated(int variant, int levels, int64_t N, int64_t P, int64_t M, const double *A, int64_t lda,
                          const double *B, int64_t ldb, double *C, int64_t ldc, int s, int kind, void *ws,
                          cudaStream_t st);
size_t emulated_noalloc_capacity();
int run_emulated_noalloc(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                         int64_t ldb, double *C, int64_t ldc, int s, int kind, cudaStream_t st);

}  // namespace mm

// ------------------------------------------------------------ device helpers

namespace mmdev {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Largest number of polls of one mbarrier phase before a wait is declared
// stuck (roughly seconds of wall time; normal waits need a few thousand).
constexpr uint32_t kMaxPolls = 1u << 22;

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: true when the phase completed, false after max_polls polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t max_polls = kMaxPolls) {
    for (uint32_t i = 0; i < max_polls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int32_t c0, int32_t c1,
                                            int32_t c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
            "r"(smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int32_t c0,
                                            int32_t c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}
// Makes a tensor map that lives in global memory, and was written through the
// generic proxy (host copy or device store), visible to the TMA unit.
__device__ __forceinline__ void tmap_acquire(const CUtensorMap *map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}
__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}

// tcgen05 (5th-generation tensor core) wrappers, cta_group::1.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem desc] * B[smem desc], kind::f16 (BF16 inputs, FP32
// accumulate).  Called by a whole converged warp: elect.sync picks the one lane
// that issues, so descriptors and addresses stay warp-uniform (a single-lane
// branch around the issue loop costs the MMA warp several times the issue time).
__device__ __forceinline__ void mma_bf16_elect(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred e, p;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// The same for kind::f8f6f4 with E4M3 A and B (K = 32 per instruction).
__device__ __forceinline__ void mma_e4m3_elect(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred e, p;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive once on `bar` when every tcgen05.mma issued so far by the warp's
// elected lane completes.  Called by a whole converged warp.
__device__ __forceinline__ void mma_commit_elect(uint64_t *bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}
// 32 lanes x 32 consecutive 32-bit columns: thread i of the warp gets lane (base lane + i).
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}
// 32 lanes x 16 consecutive 32-bit columns.
__device__ __forceinline__ void tmem_ld_32x32b_x16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor for tcgen05 (K-major operand, swizzled):
// start address >> 4 in bits 0-13, leading byte offset >> 4 in 16-29 (unused
// for swizzled K-major), stride byte offset >> 4 in 32-45 (distance between
// 8-row groups), version 1 in bits 46-47, base offset 0, layout type in bits
// 61-63 (4 = 64-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc_kmajor(uint32_t saddr, uint32_t row_bytes, uint32_t layout) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(16 >> 4) << 16;
    d |= (uint64_t)((8 * row_bytes) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)layout << 61;
    return d;
}
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t saddr) { return smem_desc_kmajor(saddr, 64, 4); }

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in
// bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(uint32_t M, uint32_t N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
// kind::f8f6f4: FP32 accumulator, A and B E4M3 (format code 0 in bits 7-9 and
// 10-12), both K-major.
__host__ __device__ constexpr uint32_t idesc_e4m3_f32(uint32_t M, uint32_t N) {
    return (1u << 4) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

}  // namespace mmdev
