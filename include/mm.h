/*
 * mm.h -- C ABI of libmm, a GB300 (sm_103a) library for the dense product
 * C = A B of an N x P by a P x M double matrix in the methods described in
 * I. Hedtke, "Methods of Matrix Multiplication" (arXiv:1106.1347), plus an
 * FP64-accurate product emulated from BF16 or FP8-E4M3 slices on the tcgen05
 * tensor cores.
 *
 * Common conventions (every entry point below):
 *  - Matrices are row-major double with leading dimensions in elements:
 *    element (i, j) of A is A[i * lda + j].  Required: lda >= max(1, P),
 *    ldb >= max(1, M), ldc >= max(1, M); N, P, M >= 0.
 *  - Matrix, vector and workspace pointers are DEVICE pointers on the current
 *    CUDA device, owned by the caller.  The library never allocates, frees or
 *    retains caller memory; scratch space is passed in as (ws, ws_bytes) and
 *    sized by the matching *_workspace_bytes query.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    enqueue work and return without synchronising.
 *  - C is overwritten (C := A B; there is no alpha/beta).  N == 0 or M == 0 is
 *    a no-op; P == 0 writes C = 0.
 *  - Argument errors are detected before anything is enqueued and return
 *    MM_ERR_ARG (negative sizes, short leading dimensions, NULL pointers with
 *    non-zero extent, C overlapping A or B by address range, short workspace).
 *    A CUDA launch failure returns MM_ERR_CUDA.  mm_last_error() then holds a
 *    thread-local message.
 *  - Inputs must be finite; Inf/NaN propagate in method-dependent ways.
 */
#ifndef MM_H
#define MM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MM_OK = 0,
    MM_ERR_ARG = -1,         /* bad argument; nothing was enqueued */
    MM_ERR_CUDA = -2,        /* a CUDA call or launch failed */
    MM_ERR_NOMEM = -3,       /* a fixed capacity was exceeded */
    MM_ERR_UNSUPPORTED = -4, /* valid request the library does not implement */
    MM_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    MM_ERR_WORKSPACE = -6    /* ws_bytes smaller than the *_workspace_bytes query */
} mm_status;

typedef enum { MM_SLICE_BF16 = 0, MM_SLICE_FP8E4M3 = 1 } mm_slice_kind;

/* Library version as 10000*major + 100*minor + patch. */
int mm_version(void);

/* Thread-local text of the last non-OK status returned on this thread. */
const char *mm_last_error(void);

/* Reads and clears the device status word the kernels set when a bounded wait
 * gives up (current device).  Synchronises `stream`.  Returns MM_OK or
 * MM_ERR_TIMEOUT; *code_out (may be NULL) receives the raw word. */
int mm_device_status(void *stream, int32_t *code_out);

/* Failure-detection self-test: enqueues on `stream` a kernel whose bounded
 * wait on a barrier that nothing completes runs out (2^16 polls), so it sets
 * the device status word (code 8) and returns; the next mm_device_status then
 * reports MM_ERR_TIMEOUT and the context stays usable.  Returns MM_OK once
 * enqueued. */
int mm_selftest_wait_timeout(void *stream);

/*
 * Section "NormInf": *out = ||A||_inf = max_i sum_j |A_ij| for the N x P
 * matrix A.  Each row is summed in index order, so the value is bit-identical
 * to a sequential CPU evaluation.  `out` is one device double; N == 0 or
 * P == 0 gives 0.
 */
int mm_norm_inf(int64_t N, int64_t P, const double *A, int64_t lda, double *out, void *stream);

/*
 * Section "The naive method" (NaivStandard): C_ij = sum_k A_ik B_kj.
 * Runs on the FP64 tensor-core MMA (mma.sync m8n8k4 f64); exact on integer
 * inputs whose partial sums stay below 2^53, otherwise within the usual
 * inner-product rounding error (products are fused, order is blocked).
 */
int mm_naive(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
             double *C, int64_t ldc, void *stream);

/*
 * Section "NaivKahan": the naive product with every dot product summed by the
 * paper's compensated update (err = err + x; t = sum + err;
 * err = (sum - t) + err; sum = t) over x = RN(A_ik B_kj), k in order.
 * Bit-identical to the sequential CPU evaluation.
 */
int mm_kahan(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
             double *C, int64_t ldc, void *stream);

/*
 * Sections "NaivStandard", "NaivOnArray" and "Loop unrolling": the naive sum in
 * the paper's evaluation orders, every product and sum rounded on its own (no
 * FMA), bit-identical to the sequential CPU evaluation.
 *   unroll = 1: aux = aux + A_ik B_kj for k in order (NaivStandard; NaivOnArray
 *               accumulates in C itself and gives the same value);
 *   unroll = 2, 3, 4: NaivLoopUnrollingTwo/Three/Four -- u products summed left
 *               to right, the group added to aux, then the P mod u leftover
 *               products added one by one.
 * Other unroll values return MM_ERR_ARG.  The FP64-pipe kernel runs at about
 * half the rate of mm_naive (no FMA, 2 operations per k); use mm_naive for speed.
 */
int mm_naive_unrolled(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                      double *C, int64_t ldc, int32_t unroll, void *stream);

/*
 * Section "WinogradOriginal": with gamma = floor(P/2),
 *   y_i = sum_j A_i,2j-1 A_i,2j,  z_k = sum_j B_2j-1,k B_2j,k   (1-based),
 *   C_ik = (sum_j (A_i,2j-1 + B_2j,k)(A_i,2j + B_2j-1,k) - y_i) - z_k
 * plus A_i,P B_P,k when P is odd.  y and z are bit-identical to a sequential
 * evaluation; the paired sum uses FMA.  Workspace: mm_winograd_workspace_bytes.
 */
size_t mm_winograd_workspace_bytes(int64_t N, int64_t P, int64_t M);
int mm_winograd(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                double *C, int64_t ldc, void *ws, size_t ws_bytes, void *stream);

/*
 * Section "WinogradScaled": lambda = the smallest integer with
 * 1/2 <= 4^lambda ||A||_inf / ||B||_inf <= 2 (0 if either norm is 0), computed
 * on the device from bit-exact norms (no host synchronisation), then
 * Winograd's form on 2^lambda A and 2^-lambda B; the power-of-two scalings
 * (MultiplyWithScalar) are applied while operand tiles are staged.
 * `lambda_out` is an optional device int32 (NULL to skip).
 */
size_t mm_winograd_scaled_workspace_bytes(int64_t N, int64_t P, int64_t M);
int mm_winograd_scaled(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                       int64_t ldb, double *C, int64_t ldc, int32_t *lambda_out, void *ws, size_t ws_bytes,
                       void *stream);

/*
 * Per-row/column power-of-two scaling of Winograd's form (no counterpart in
 * the paper; it takes the exact scaling of section "WinogradScaled" from one
 * global pair of norms to every row of A and every column of B):
 *   e_i = frexp exponent of max_j |A_ij|, f_k = that of max_j |B_jk| (0 for a
 *   zero row or column), A' = 2^-e_i A_i,:, B' = 2^-f_k B_:,k,
 *   C_ik = 2^(e_i + f_k) WinogradOriginal(A', B')_ik.
 * Every paired sum then adds terms of like magnitude, which keeps the error of
 * each C_ik relative to its own row and column scales (rows and columns of
 * widely different magnitude).  y' and z' are bit-identical to a sequential
 * evaluation over A' and B'; the paired sum uses FMA.  Scalings are exact
 * unless a scaled entry leaves the normal range.
 * Workspace: mm_winograd_rowcol_scaled_workspace_bytes.
 */
size_t mm_winograd_rowcol_scaled_workspace_bytes(int64_t N, int64_t P, int64_t M);
int mm_winograd_rowcol_scaled(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                              int64_t ldb, double *C, int64_t ldc, void *ws, size_t ws_bytes, void *stream);

/*
 * Sections "StrassenNaiv" and "StrassenWinograd": recursive block products
 * with 7 half-size products per level (H1..H7; 18 additions for Strassen's
 * form, 15 for Winograd's variant), down to a base product on the FP64
 * tensor-core MMA.
 *   cutoff == 0: the paper's rule -- X = max{N,P,M}, k = max(0, floor(log2 X) - 4),
 *                embed in Y x Y with Y = (floor(X/2^k) + 1) 2^k, recurse k levels;
 *   cutoff  > 0: the smallest depth at which every padded dimension / 2^depth
 *                is <= cutoff, each dimension padded to a multiple of 2^depth;
 *   cutoff == -1: the depth mm_tune_strassen recorded for this shape bucket,
 *                else the paper's depth taken on the smallest dimension,
 *                max(0, floor(log2 min(N, P, M)) - 4), at most 6 for
 *                mm_strassen_winograd (its normwise error about doubles per
 *                level: 3e-15 at 6 levels, 3.5e-14 at 9 on uniform 8192^3);
 *                each dimension padded to a multiple of 2^depth.
 * Padding is virtual (out-of-range elements read as zero).  Every node of a
 * recursion level is processed by the same launch (breadth-first):
 *   - the operand sums (Plus/Minus) of one or two levels are formed in one
 *     pass over all nodes of a level, each sum rounded as the section's
 *     Aux matrices are, in the printed order;
 *   - blocks of at most 32 at the bottom: the last level runs in shared
 *     memory (operand sums, seven naive FMA block products, C-block sums);
 *     blocks of at most 64: naive block products in shared memory; larger
 *     blocks: the last level forms its operand sums while staging tiles for
 *     the FP64 MMA and adds +-H_i into the C quadrants in its epilogue;
 *   - the C blocks of one or two levels are formed in one pass, left to
 *     right as printed.
 * When a plan's breadth-first arrays would exceed 8 GiB (environment variable
 * MM_STRASSEN_BREADTH_CAP, in bytes, read at each call and each workspace
 * query, overrides this), its top levels run depth-first, one child at a
 * time; the result is the same.  Depth is limited to 16 levels; deeper
 * requests return MM_ERR_UNSUPPORTED.  On integer inputs whose sums stay
 * below 2^53 the result is exact; otherwise it differs from a sequential
 * evaluation only by the FMA rounding of the block products.
 */
size_t mm_strassen_workspace_bytes(int64_t N, int64_t P, int64_t M, int32_t cutoff);
int mm_strassen(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                double *C, int64_t ldc, int32_t cutoff, void *ws, size_t ws_bytes, void *stream);
size_t mm_strassen_winograd_workspace_bytes(int64_t N, int64_t P, int64_t M, int32_t cutoff);
int mm_strassen_winograd(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                         int64_t ldb, double *C, int64_t ldc, int32_t cutoff, void *ws, size_t ws_bytes,
                         void *stream);

/*
 * Autotuner for the Strassen depth used by cutoff == -1 (not in the paper,
 * which fixes the depth by its padding rule).
 * mm_tune_strassen times the recursion at every depth 0, 1, ... whose blocks
 * stay at least 16 in every dimension (at most 6 for StrassenWinograd; each
 * dimension padded to a multiple of 2^depth) on the given operands, writing C
 * each time, and records the fastest depth for (variant,
 * floor(log2 max(N, P, M))); it synchronises
 * `stream`.  variant: 0 = StrassenNaiv, 1 = StrassenWinograd.  ws must hold
 * mm_tune_strassen_workspace_bytes(N, P, M) bytes (depths whose workspace does
 * not fit are skipped).  The table (Strassen depths and the emulated choices
 * below) persists with mm_tune_save / mm_tune_load (text, one entry per line);
 * if MM_TUNE_CACHE is set, that file is loaded at first use.  mm_tune_load
 * returns the number of entries read; mm_tune_clear empties the table.
 */
size_t mm_tune_strassen_workspace_bytes(int64_t N, int64_t P, int64_t M);
int mm_tune_strassen(int32_t variant, int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                     int64_t ldb, double *C, int64_t ldc, void *ws, size_t ws_bytes, void *stream,
                     int32_t *best_depth, double *best_ms);
int mm_tune_save(const char *path);
int mm_tune_load(const char *path);
int mm_tune_clear(void);

/*
 * FP64-accurate product emulated from slices (not in the paper; its
 * per-row/per-column power-of-two scaling generalises section
 * "WinogradScaled").  Each row i of A is scaled by 2^-e_i (e_i the frexp
 * exponent of max_k |A_ik|), rounded to an integer V_ik with beta*s - 1 bits
 * and cut into s balanced base-2^beta digits; B is split per column the same
 * way.  The slice pairs (sigma, tau) with sigma + tau <= s - 1 are multiplied
 * on tcgen05 with FP32 accumulation in TMEM, read out before any partial sum
 * can leave the integers FP32 holds exactly (|x| <= 2^24), accumulated exactly
 * in integers, and rounded once to double with the 2^(e_i + f_j) scaling.
 * The result equals, bit for bit, RN(sum of the kept digit products) scaled --
 * see the oracle's definition.
 *   kind:     MM_SLICE_BF16 (beta = 7, digits |d| <= 64, kind::f16 MMA) or
 *             MM_SLICE_FP8E4M3 (beta = 5, digits |d| <= 16, kind::f8f6f4 MMA at
 *             twice the rate per pair); anything else returns MM_ERR_ARG;
 *   nslices:  1..8 (BF16) or 1..10 (FP8-E4M3), or 0 to choose from `tier`:
 *             s = ceil((log2(1/tier) + 9) / beta);
 *   tier:     target ||C - AB||_inf / (||A||_inf ||B||_inf) when nslices == 0
 *             (<= 1e-14 selects 8 BF16 slices; FP8 reaches tiers down to about
 *             1e-12 with 10 slices -- a tier that needs more slices than the
 *             format holds returns MM_ERR_UNSUPPORTED: the kernel keeps one TMEM
 *             accumulator per diagonal, 64 columns wide up to 8 slices, 32
 *             wide for 9 and 10, and TMEM holds 512 columns).
 * Requires N, M >= 1 and P <= 2^20 (larger P returns MM_ERR_UNSUPPORTED).
 */
size_t mm_emulated_workspace_bytes(int64_t N, int64_t P, int64_t M, int32_t kind, int32_t nslices, double tier);
int mm_emulated(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                double *C, int64_t ldc, int32_t kind, int32_t nslices, double tier, void *ws, size_t ws_bytes,
                void *stream);

/*
 * mm_emulated with the slice product's output tile width chosen by the caller
 * (no counterpart in the paper): tile_n = 64 (up to 8 slices; the default),
 * 32 (any slice count: half the column padding on narrow products, at the
 * N = 64 MMA rate, about 2/3 of the 64-column one), or 0 for the default.
 * Same arguments, workspace (mm_emulated_workspace_bytes) and result bit for
 * bit as mm_emulated; MM_ERR_ARG for any other width.  mm_tune_emulated picks
 * the width per shape bucket and mm_emulated_auto uses the pick.
 */
int mm_emulated_tiled(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                      double *C, int64_t ldc, int32_t kind, int32_t nslices, double tier, int32_t tile_n, void *ws,
                      size_t ws_bytes, void *stream);

/*
 * mm_emulated with HOST operands: A, B and C are host pointers (pinned memory
 * lets the copies overlap the products), `ws` is a device workspace of
 * mm_emulated_host_workspace_bytes bytes holding the device copies of A, B, C
 * and the split.  C is computed in blocks: up to 8 row blocks, and for
 * N >= 4096 and M >= 2048 two column blocks, with row blocks of whole waves of
 * tiles.  One internal copy
 * stream carries the first row block of A, B in pieces (with two column
 * blocks: the first one in two halves, then the second), then the other row
 * blocks of A; each block is split as soon as it lands, the first row block is
 * multiplied by each piece of B as it lands, each later block product follows
 * the splits it needs, and its block of C is copied back on a second internal
 * stream while later blocks run.  Asynchronous on `stream`
 * (which waits for the last copy back); the
 * host buffers must stay valid and C unread until the stream completes.  With
 * P == 0 the call synchronises `stream` and writes C = 0 on the host.  Results are
 * bit-identical to mm_emulated.  Errors as for mm_emulated.
 */
size_t mm_emulated_host_workspace_bytes(int64_t N, int64_t P, int64_t M, int32_t kind, int32_t nslices,
                                        double tier);
int mm_emulated_host(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                     double *C, int64_t ldc, int32_t kind, int32_t nslices, double tier, void *ws, size_t ws_bytes,
                     void *stream);

/* Slice count mm_emulated uses for (kind, nslices, tier). */
int mm_emulated_slices(int32_t kind, int32_t nslices, double tier);

/*
 * Allocation-free variant of mm_emulated (the paper has no counterpart; this
 * is a deployment convenience).  For callers that cannot allocate a device
 * workspace -- a host application that owns the device's whole memory pool,
 * or a loop that must not allocate -- the scratch space lives in a fixed
 * static device array of mm_emulated_noalloc_capacity() bytes (64 MiB) that
 * every GPU loading the library holds until the process exits.  Same
 * arguments and result as mm_emulated minus (ws, ws_bytes).
 *   - Products whose mm_emulated_workspace_bytes exceeds the capacity return
 *     MM_ERR_NOMEM (about N = P = M = 1400 with 8 slices); use mm_emulated.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Calls never allocate or free memory, but they all share the one array:
 *     calls that overlap on the GPU (other streams, other threads on the same
 *     device) race on it, so the caller must serialise them.
 */
int mm_emulated_noalloc(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                        int64_t ldb, double *C, int64_t ldc, int32_t kind, int32_t nslices, double tier,
                        void *stream);
size_t mm_emulated_noalloc_capacity(void);

/*
 * Autotuned FP64-accurate product (not in the paper).  For a requested tier
 * the candidates are the two slice formats, each with the slice count the tier
 * needs (mm_emulated_slices; a format that cannot reach the tier is skipped),
 * times 0, 1 or 2 levels of Strassen-Winograd over the product (each level
 * leaving blocks of at least 512), and for the direct product (0 levels) the
 * two tile widths of mm_emulated_tiled (64 and 32; 32 only past 8 slices).
 *   mm_tune_emulated times every candidate that fits ws (the faster of two
 *     runs after a warm-up, CUDA events on `stream`, which it synchronises) on
 *     the given operands, writing C each time, and records the fastest for the
 *     bucket (floor(log2 N), floor(log2 P), floor(log2 M), round(-log10 tier));
 *     the chosen format, slice count, level count, time and tile width are
 *     written to the optional outputs.  ws: mm_tune_emulated_workspace_bytes
 *     bytes.
 *   mm_tune_emulated_choice (host only, no device work) reports the choice for
 *     a shape and tier: the recorded one (returns 1) or, with none recorded,
 *     the model's (returns 0): the format whose slice pairs cost less at the
 *     nominal rates (an FP8-E4M3 pair at half a BF16 pair), the level count
 *     of mm_strassen_emulated's levels = -1, and the 32-column tile only where
 *     the 64-column one would pad M by more than 3/2 of the 32-column padding
 *     (in practice M <= 32).  `tile` (optional) receives the tile width (the
 *     default width when levels > 0).  Negative status for a tier <= 0 or one
 *     neither format reaches.
 *   mm_emulated_auto computes C = A B with that choice (the direct product for
 *     0 levels, with the chosen tile width, else mm_strassen_emulated's
 *     variant 1); `used` (optional, 4 host int32) receives format, slice
 *     count, levels and tile width.  Its result meets
 *     the tier like mm_emulated's; it is bit-identical to the mm_emulated /
 *     mm_strassen_emulated call with the same choice.  Workspace:
 *     mm_emulated_auto_workspace_bytes.  Errors as for mm_emulated.
 */
size_t mm_tune_emulated_workspace_bytes(int64_t N, int64_t P, int64_t M, double tier);
int mm_tune_emulated(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                     double *C, int64_t ldc, double tier, void *ws, size_t ws_bytes, void *stream, int32_t *best_kind,
                     int32_t *best_slices, int32_t *best_levels, double *best_ms, int32_t *best_tile);
int mm_tune_emulated_choice(int64_t N, int64_t P, int64_t M, double tier, int32_t *kind, int32_t *slices,
                            int32_t *levels, int32_t *tile);
size_t mm_emulated_auto_workspace_bytes(int64_t N, int64_t P, int64_t M, double tier);
int mm_emulated_auto(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                     double *C, int64_t ldc, double tier, void *ws, size_t ws_bytes, void *stream, int32_t *used);

/*
 * Grouped FP64-accurate products (batching; no counterpart in the
 * paper): `count` independent products C_g = A_g B_g of uneven shapes, each
 * with the mm_emulated definition and one common slice count, in one launch
 * of each of the four kernels (split of A, column maxima and split of B, slice
 * products).  Each problem obeys the mm_emulated argument rules; problems
 * with N == 0 or M == 0 are skipped and P == 0 writes zeros.  The outputs must
 * not overlap each other or any input.  Results are bit-identical to calling
 * mm_emulated on each problem.  The host writes a table of the problems into
 * the workspace with one host-to-device copy before the launches.
 */
typedef struct {
    int64_t N, P, M;
    const double *A;
    int64_t lda;
    const double *B;
    int64_t ldb;
    double *C;
    int64_t ldc;
} mm_problem;
size_t mm_emulated_group_workspace_bytes(const mm_problem *probs, int32_t count, int32_t kind, int32_t nslices,
                                         double tier);
int mm_emulated_group(const mm_problem *probs, int32_t count, int32_t kind, int32_t nslices, double tier, void *ws,
                      size_t ws_bytes, void *stream);

/*
 * Strassen levels over the FP64-accurate emulated product (no counterpart in
 * the paper as such: the recursion of sections "StrassenNaiv" (variant 0) and
 * "StrassenWinograd" (variant 1) with mm_emulated's split product as the base
 * case instead of NaivStandard).  C = A B with
 *   - A and B embedded in zero matrices whose sizes Np, Pp, Mp are the
 *     smallest multiples of 2^levels >= N, P, M;
 *   - at each of `levels` levels (0..4) the operands of H1..H7 formed by the
 *     FP64 additions of the section's formulas, in the printed order, and
 *     the C quadrants by its printed sums of the H's, left to right;
 *   - the 7^levels products at the bottom computed as mm_emulated does (slice
 *     format `kind`, slice count from nslices / tier as for mm_emulated), all
 *     in one grouped launch.
 * levels = 0 is mm_emulated itself; levels = -1 picks the count by the
 * smallest of N, P, M (0 below 5120, 1 below 12288, else 2: the measured
 * crossovers on GB300 with 8 BF16 slices).  The result is bit-identical to the CPU
 * oracle's restatement of this definition.  Normwise error: the base
 * product's plus a few units of 2^-53 ||A|| ||B|| per level from the FP64
 * sums.  Workspace (device, caller-owned): the padded copies when padding is
 * needed, every level's operand sums and H blocks, and the grouped product's
 * workspace, as mm_strassen_emulated_workspace_bytes reports (0 for invalid
 * arguments).  Argument rules and errors as mm_emulated; MM_ERR_ARG for a
 * variant other than 0 or 1 or levels outside -1..4.
 */
size_t mm_strassen_emulated_workspace_bytes(int64_t N, int64_t P, int64_t M, int32_t variant, int32_t levels,
                                            int32_t kind, int32_t nslices, double tier);
int mm_strassen_emulated(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                         double *C, int64_t ldc, int32_t variant, int32_t levels, int32_t kind, int32_t nslices,
                         double tier, void *ws, size_t ws_bytes, void *stream);

/*
 * Serving loop (no counterpart in the paper).  A server
 * owns a worker thread and K streams and serves requests C = A B with host
 * operands and a requested accuracy tier:
 *   - `arena` (device, caller-owned, arena_bytes) is the server's entire HBM
 *     budget: per-stream batch tables, every admitted request's device copies
 *     of A, B, C and every running batch's split workspace are carved from it;
 *     the server allocates no device memory itself;
 *   - requests are admitted in arrival order (later ones may pass one that does
 *     not fit yet) once their A, B and C fit; a request that can never fit
 *     completes with MM_ERR_NOMEM;
 *   - continuous batching: whenever a stream is free, all admitted requests of
 *     the oldest request's slice format and count (up to max_batch and, past
 *     the first request, up to 4 ms of estimated work -- copies at 200 GB/s,
 *     slice pairs at 1.2 (BF16) or 2.4 (FP8) PFLOP/s; the environment variable
 *     MM_SERVER_BATCH_MS, read at creation, sets that cap, 0 lifts it, and
 *     MM_SERVER_CLASS_RATIO keeps to requests within that factor of the
 *     oldest one's estimated time, a factor in (0, 1) counting as 1; the
 *     oldest request is always taken) run as one grouped emulated
 *     launch, replayed from a CUDA graph cached per stream, slice format and
 *     count when use_graphs != 0;
 *   - method 0: BF16 slices, the tier's count (mm_emulated_slices);
 *     method 2: per request the format and count of mm_tune_emulated_choice
 *     for its shape and tier (the autotuner's entry when one is recorded,
 *     else the format whose slice pairs cost less, an FP8 pair at half a
 *     BF16 pair (three quarters past 8 FP8 slices) -- e.g. 6 FP8 slices for
 *     1e-6 against 5 BF16 ones); method 1 runs one request at a time with
 *     mm_naive's FP64 kernel (a baseline);
 *   - per request: host-to-device copies of A and B, the product, and the copy
 *     of C back into the caller's host buffer, whose completion ends the
 *     request's latency (measured from mm_server_submit).
 * Host buffers must stay valid until the request completes; pinned host
 * memory lets copies overlap.  Each result is bit-identical to mm_emulated on
 * the same operands with the slice format and count the completion reports
 * (or to mm_naive for method 1).
 */
typedef struct mm_server mm_server;
typedef struct {
    int64_t N, P, M;
    const double *A; /* host, row-major, lda >= P */
    int64_t lda;
    const double *B; /* host, row-major, ldb >= M */
    int64_t ldb;
    double *C; /* host output, ldc >= M */
    int64_t ldc;
    double tier; /* requested ||C - AB||_inf / (||A||_inf ||B||_inf) (methods 0 and 2) */
    int64_t tag; /* caller's identifier, echoed in the completion */
} mm_request;
typedef struct {
    int64_t tag;
    int32_t status; /* MM_OK, MM_ERR_NOMEM (never fits), MM_ERR_TIMEOUT (cancelled), MM_ERR_CUDA */
    int32_t slices; /* slice count used (0 for method 1) */
    int32_t kind;   /* slice format used (mm_slice_kind) */
    int32_t reserved;
    double queue_ms;   /* submit -> launch */
    double latency_ms; /* submit -> C in the host buffer */
} mm_completion;
typedef struct {
    int64_t submitted, completed, rejected, batches, graph_replays;
    double p50_ms, p99_ms, mean_ms, max_ms;
    double busy_s; /* first submit -> last completion */
    double flops;  /* sum of 2NPM over completed requests */
    int64_t peak_arena_bytes;
    /* From CUDA events recorded before each batch's first copy and after its
     * last: device time covered by at least one batch, and by at least two
     * batches at once (batches on different streams overlapping). */
    double device_busy_ms, overlap_ms;
} mm_server_stats_t;
int mm_server_create(void *arena, size_t arena_bytes, int32_t max_batch, int32_t nstreams, int32_t use_graphs,
                     int32_t method, mm_server **out);
int mm_server_submit(mm_server *server, const mm_request *request); /* returns at once */
int mm_server_poll(mm_server *server, mm_completion *out, int32_t cap); /* number of completions written */
int mm_server_wait(mm_server *server, int64_t timeout_ms); /* MM_ERR_TIMEOUT if requests remain */
int mm_server_stats(mm_server *server, mm_server_stats_t *out);
/* Text of the first failure the server hit ("" if none); valid until destroy. */
const char *mm_server_error(mm_server *server);
/* Cancels requests that have not started (status MM_ERR_TIMEOUT), waits for
 * running batches, frees the server.  The arena may be reused afterwards. */
int mm_server_destroy(mm_server *server);

/*
 * FP64 peak probe (measurement support; the paper has no counterpart): the
 * rate of this device's FP64 pipe, the denominator of FP64 roofline
 * fractions.  Runs a kernel of independent DFMA chains and one of independent
 * mma.sync m8n8k4 f64 accumulators on every SM, each timed with CUDA events
 * on `stream` after a warm-up and lengthened until one run lasts at least
 * target_ms (0 < target_ms <= 10000).  Writes the rates in TFLOP/s (2 flop per
 * FMA, 512 per MMA) to *dfma_tflops and *dmma_tflops (either may be NULL).
 * Synchronises `stream`; allocates nothing.
 */
int mm_probe_fp64_peak(double target_ms, double *dfma_tflops, double *dmma_tflops, void *stream);

/*
 * Kernel-level timing (measurement support).  While enabled, every kernel the
 * library launches on any stream is bracketed by CUDA events recorded on that
 * stream.  mm_profile_read synchronises those events and fills up to `cap`
 * entries (kernel name, launch count, total milliseconds), returning the
 * number of distinct kernels; it also resets the record.
 */
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
} mm_kernel_stat;
int mm_profile_enable(int on);
int mm_profile_read(mm_kernel_stat *out, int32_t cap);

#ifdef __cplusplus
}
#endif

#endif /* MM_H */
