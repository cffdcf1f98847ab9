// libmm C ABI: argument checking, status reporting, kernel timing and dispatch
// to the per-method launchers.  See include/mm.h for the contract.
#include <atomic>
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "slice_gemm.cuh"

// Device status word raised by bounded waits (one per device context).
static __device__ int g_device_status;

namespace mm {

int sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n <= 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

static thread_local std::string t_err;

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
}

int fail(int status, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return status;
}

int cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return MM_ERR_CUDA;
}

int *device_status_ptr() {
    static std::mutex mu;
    static std::map<int, int *> per_dev;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    auto it = per_dev.find(dev);
    if (it != per_dev.end()) return it->second;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_status) != cudaSuccess) return nullptr;
    per_dev[dev] = (int *)p;
    return (int *)p;
}

EncodeTiledFn encode_tiled_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// ------------------------------------------------------------ kernel timing

namespace {
struct ProfRec {
    std::string name;
    cudaEvent_t start, stop;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_recs;
std::vector<cudaEvent_t> g_event_pool;
thread_local int t_open = -1;

cudaEvent_t take_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

namespace {
thread_local bool t_prof_suspended = false;
}

void prof_suspend(bool on) { t_prof_suspended = on; }

void prof_begin(const char *name, cudaStream_t stream) {
    if (t_prof_suspended) return;
    std::lock_guard<std::mutex> g(g_prof_mu);
    if (!g_prof_on) return;
    ProfRec r{name, take_event(), take_event()};
    cudaEventRecord(r.start, stream);
    g_prof_recs.push_back(r);
    t_open = (int)g_prof_recs.size() - 1;
}

void prof_end(cudaStream_t stream) {
    if (t_prof_suspended) return;
    std::lock_guard<std::mutex> g(g_prof_mu);
    if (!g_prof_on || t_open < 0) return;
    cudaEventRecord(g_prof_recs[t_open].stop, stream);
    t_open = -1;
}

int check_gemm_args(const char *fn, int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                    int64_t ldb, const double *C, int64_t ldc) {
    if (N < 0 || P < 0 || M < 0) return fail(MM_ERR_ARG, "%s: negative size (N=%lld P=%lld M=%lld)", fn,
                                             (long long)N, (long long)P, (long long)M);
    if (lda < std::max<int64_t>(1, P) || ldb < std::max<int64_t>(1, M) || ldc < std::max<int64_t>(1, M))
        return fail(MM_ERR_ARG, "%s: leading dimension too small (lda=%lld ldb=%lld ldc=%lld)", fn, (long long)lda,
                    (long long)ldb, (long long)ldc);
    if ((N > 0 && P > 0 && !A) || (P > 0 && M > 0 && !B) || (N > 0 && M > 0 && !C))
        return fail(MM_ERR_ARG, "%s: NULL pointer with non-zero extent", fn);
    size_t cb = span_bytes(N, M, ldc);
    if (cb && (ranges_overlap(C, cb, A, span_bytes(N, P, lda)) || ranges_overlap(C, cb, B, span_bytes(P, M, ldb))))
        return fail(MM_ERR_ARG, "%s: C overlaps A or B", fn);
    return MM_OK;
}

}  // namespace mm

using namespace mm;

extern "C" {

int mm_version(void) { return 100; }

const char *mm_last_error(void) { return t_err.c_str(); }

int mm_device_status(void *stream, int32_t *code_out) {
    int *p = device_status_ptr();
    if (!p) return fail(MM_ERR_CUDA, "mm_device_status: no device status symbol");
    int v = 0;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&v, p, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "mm_device_status");
    if (code_out) *code_out = v;
    if (v) return fail(MM_ERR_TIMEOUT, "a device-side wait gave up (code %d)", v);
    return MM_OK;
}

int mm_selftest_wait_timeout(void *stream) { return run_selftest_wait(stream); }

int mm_norm_inf(int64_t N, int64_t P, const double *A, int64_t lda, double *out, void *stream) {
    if (N < 0 || P < 0) return fail(MM_ERR_ARG, "mm_norm_inf: negative size");
    if (lda < std::max<int64_t>(1, P)) return fail(MM_ERR_ARG, "mm_norm_inf: lda too small");
    if (!out || (N > 0 && P > 0 && !A)) return fail(MM_ERR_ARG, "mm_norm_inf: NULL pointer");
    return run_norm_inf(N, P, A, lda, out, (cudaStream_t)stream);
}

int mm_naive(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
             int64_t ldc, void *stream) {
    int rc = check_gemm_args("mm_naive", N, P, M, A, lda, B, ldb, C, ldc);
    if (rc) return rc;
    if (N == 0 || M == 0) return MM_OK;
    if (P == 0) return run_zero(N, M, C, ldc, (cudaStream_t)stream);
    return run_naive(N, P, M, A, lda, B, ldb, C, ldc, (cudaStream_t)stream);
}

int mm_naive_unrolled(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                      double *C, int64_t ldc, int32_t unroll, void *stream) {
    if (unroll < 1 || unroll > 4) return fail(MM_ERR_ARG, "mm_naive_unrolled: unroll must be 1, 2, 3 or 4 (got %d)", unroll);
    int rc = check_gemm_args("mm_naive_unrolled", N, P, M, A, lda, B, ldb, C, ldc);
    if (rc) return rc;
    if (N == 0 || M == 0) return MM_OK;
    if (P == 0) return run_zero(N, M, C, ldc, (cudaStream_t)stream);
    return run_unrolled(N, P, M, A, lda, B, ldb, C, ldc, unroll, (cudaStream_t)stream);
}

int mm_kahan(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
             int64_t ldc, void *stream) {
    int rc = check_gemm_args("mm_kahan", N, P, M, A, lda, B, ldb, C, ldc);
    if (rc) return rc;
    if (N == 0 || M == 0) return MM_OK;
    if (P == 0) return run_zero(N, M, C, ldc, (cudaStream_t)stream);
    return run_kahan(N, P, M, A, lda, B, ldb, C, ldc, (cudaStream_t)stream);
}

size_t mm_winograd_workspace_bytes(int64_t N, int64_t P, int64_t M) { return winograd_ws_bytes(N, P, M, 0); }

size_t mm_winograd_scaled_workspace_bytes(int64_t N, int64_t P, int64_t M) { return winograd_ws_bytes(N, P, M, 1); }

size_t mm_winograd_rowcol_scaled_workspace_bytes(int64_t N, int64_t P, int64_t M) {
    return winograd_ws_bytes(N, P, M, 2);
}

static int winograd_common(const char *fn, int mode, int64_t N, int64_t P, int64_t M, const double *A,
                           int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc, int32_t *lambda_out,
                           void *ws, size_t ws_bytes, void *stream) {
    const bool scaled = mode == 1;
    int rc = check_gemm_args(fn, N, P, M, A, lda, B, ldb, C, ldc);
    if (rc) return rc;
    size_t need = winograd_ws_bytes(N, P, M, mode);
    if (ws_bytes < need || (need && !ws))
        return fail(MM_ERR_WORKSPACE, "%s: workspace %zu bytes < %zu required", fn, ws_bytes, need);
    cudaStream_t st = (cudaStream_t)stream;
    if (N == 0 || M == 0) {
        if (scaled && lambda_out) {
            cudaError_t e = cudaMemsetAsync(lambda_out, 0, sizeof(int32_t), st);
            if (e != cudaSuccess) return cuda_fail(e, fn);
        }
        return MM_OK;
    }
    return run_winograd(N, P, M, A, lda, B, ldb, C, ldc, mode, lambda_out, ws, st);
}

int mm_winograd(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                double *C, int64_t ldc, void *ws, size_t ws_bytes, void *stream) {
    return winograd_common("mm_winograd", 0, N, P, M, A, lda, B, ldb, C, ldc, nullptr, ws, ws_bytes, stream);
}

int mm_winograd_scaled(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                       double *C, int64_t ldc, int32_t *lambda_out, void *ws, size_t ws_bytes, void *stream) {
    return winograd_common("mm_winograd_scaled", 1, N, P, M, A, lda, B, ldb, C, ldc, lambda_out, ws, ws_bytes,
                           stream);
}

int mm_winograd_rowcol_scaled(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                              int64_t ldb, double *C, int64_t ldc, void *ws, size_t ws_bytes, void *stream) {
    return winograd_common("mm_winograd_rowcol_scaled", 2, N, P, M, A, lda, B, ldb, C, ldc, nullptr, ws, ws_bytes,
                           stream);
}

static size_t strassen_ws_query(int variant, int64_t N, int64_t P, int64_t M, int32_t cutoff) {
    int depth;
    int64_t Np, Pp, Mp;
    if (N <= 0 || P <= 0 || M <= 0) return 0;
    if (strassen_plan(variant, N, P, M, cutoff, &depth, &Np, &Pp, &Mp) != MM_OK) return 0;
    return strassen_ws_bytes(variant, depth, Np, Pp, Mp);
}

size_t mm_strassen_workspace_bytes(int64_t N, int64_t P, int64_t M, int32_t cutoff) {
    return strassen_ws_query(0, N, P, M, cutoff);
}
size_t mm_strassen_winograd_workspace_bytes(int64_t N, int64_t P, int64_t M, int32_t cutoff) {
    return strassen_ws_query(1, N, P, M, cutoff);
}

static int strassen_common(const char *fn, int variant, int64_t N, int64_t P, int64_t M, const double *A,
                           int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc, int32_t cutoff,
                           void *ws, size_t ws_bytes, void *stream) {
    int rc = check_gemm_args(fn, N, P, M, A, lda, B, ldb, C, ldc);
    if (rc) return rc;
    if (cutoff < -1) return fail(MM_ERR_ARG, "%s: cutoff must be -1, 0 or positive", fn);
    cudaStream_t st = (cudaStream_t)stream;
    if (N == 0 || M == 0) return MM_OK;
    if (P == 0) return run_zero(N, M, C, ldc, st);
    int depth;
    int64_t Np, Pp, Mp;
    rc = strassen_plan(variant, N, P, M, cutoff, &depth, &Np, &Pp, &Mp);
    if (rc) return rc;
    size_t need = strassen_ws_bytes(variant, depth, Np, Pp, Mp);
    if (ws_bytes < need || (need && !ws))
        return fail(MM_ERR_WORKSPACE, "%s: workspace %zu bytes < %zu required", fn, ws_bytes, need);
    return run_strassen(variant, N, P, M, A, lda, B, ldb, C, ldc, depth, Np, Pp, Mp, ws, st);
}

int mm_strassen(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                double *C, int64_t ldc, int32_t cutoff, void *ws, size_t ws_bytes, void *stream) {
    return strassen_common("mm_strassen", 0, N, P, M, A, lda, B, ldb, C, ldc, cutoff, ws, ws_bytes, stream);
}

int mm_strassen_winograd(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                         int64_t ldb, double *C, int64_t ldc, int32_t cutoff, void *ws, size_t ws_bytes,
                         void *stream) {
    return strassen_common("mm_strassen_winograd", 1, N, P, M, A, lda, B, ldb, C, ldc, cutoff, ws, ws_bytes,
                           stream);
}

int mm_emulated_slices(int32_t kind, int32_t nslices, double tier) { return emulated_slices(kind, nslices, tier); }

size_t mm_emulated_workspace_bytes(int64_t N, int64_t P, int64_t M, int32_t kind, int32_t nslices, double tier) {
    int s = emulated_slices(kind, nslices, tier);
    if (s <= 0 || N < 0 || P < 0 || M < 0) return 0;
    return emulated_ws_bytes(N, P, M, s, kind);
}

// Slice count of a request, or the failure (with its message) when the format,
// the count or the tier is invalid or the tier needs more than 8 slices.
static int slices_or_fail(const char *fn, int32_t kind, int32_t nslices, double tier) {
    if (kind != MM_SLICE_BF16 && kind != MM_SLICE_FP8E4M3) return fail(MM_ERR_ARG, "%s: unknown slice kind %d", fn, kind);
    const int most = kind == MM_SLICE_FP8E4M3 ? 10 : 8;
    if (nslices < 0 || nslices > most) return fail(MM_ERR_ARG, "%s: nslices must be 0..%d for this format", fn, most);
    if (nslices == 0 && !(tier > 0.0)) return fail(MM_ERR_ARG, "%s: tier must be > 0 when nslices == 0", fn);
    const int s = emulated_slices(kind, nslices, tier);
    if (s == MM_ERR_UNSUPPORTED)
        return fail(MM_ERR_UNSUPPORTED, "%s: tier %g needs more than %d %s slices", fn, tier, most,
                    kind == MM_SLICE_FP8E4M3 ? "FP8-E4M3" : "BF16");
    if (s <= 0) return fail(MM_ERR_ARG, "%s: invalid slice request", fn);
    return s;
}

static int emulated_call(const char *fn, int64_t N, int64_t P, int64_t M, const double *A, int64_t lda,
                         const double *B, int64_t ldb, double *C, int64_t ldc, int32_t kind, int32_t nslices,
                         double tier, int32_t tile_n, void *ws, size_t ws_bytes, void *stream) {
    int rc = check_gemm_args(fn, N, P, M, A, lda, B, ldb, C, ldc);
    if (rc) return rc;
    const int s = slices_or_fail(fn, kind, nslices, tier);
    if (s < 0) return s;
    if (tile_n != 0 && !emu::slice_bn_ok(s, tile_n))
        return fail(MM_ERR_ARG, "%s: tile width %d (0, 32, or 64 up to 8 slices)", fn, (int)tile_n);
    if (P > (int64_t(1) << 20)) return fail(MM_ERR_UNSUPPORTED, "%s: P > 2^20", fn);
    cudaStream_t st = (cudaStream_t)stream;
    if (N == 0 || M == 0) return MM_OK;
    if (P == 0) return run_zero(N, M, C, ldc, st);
    size_t need = emulated_ws_bytes(N, P, M, s, kind);
    if (ws_bytes < need || !ws)
        return fail(MM_ERR_WORKSPACE, "%s: workspace %zu bytes < %zu required", fn, ws_bytes, need);
    return run_emulated(N, P, M, A, lda, B, ldb, C, ldc, s, kind, ws, st, tile_n);
}

int mm_emulated(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                double *C, int64_t ldc, int32_t kind, int32_t nslices, double tier, void *ws, size_t ws_bytes,
                void *stream) {
    return emulated_call("mm_emulated", N, P, M, A, lda, B, ldb, C, ldc, kind, nslices, tier, 0, ws, ws_bytes, stream);
}

int mm_emulated_tiled(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                      double *C, int64_t ldc, int32_t kind, int32_t nslices, double tier, int32_t tile_n, void *ws,
                      size_t ws_bytes, void *stream) {
    return emulated_call("mm_emulated_tiled", N, P, M, A, lda, B, ldb, C, ldc, kind, nslices, tier, tile_n, ws,
                         ws_bytes, stream);
}

size_t mm_emulated_host_workspace_bytes(int64_t N, int64_t P, int64_t M, int32_t kind, int32_t nslices,
                                        double tier) {
    const int s = emulated_slices(kind, nslices, tier);
    if (s <= 0 || N < 0 || P < 0 || M < 0) return 0;
    return emulated_host_ws_bytes(N, P, M, s, kind);
}

int mm_emulated_host(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                     double *C, int64_t ldc, int32_t kind, int32_t nslices, double tier, void *ws, size_t ws_bytes,
                     void *stream) {
    int rc = check_gemm_args("mm_emulated_host", N, P, M, A, lda, B, ldb, C, ldc);
    if (rc) return rc;
    const int s = slices_or_fail("mm_emulated_host", kind, nslices, tier);
    if (s < 0) return s;
    if (P > (int64_t(1) << 20)) return fail(MM_ERR_UNSUPPORTED, "mm_emulated_host: P > 2^20");
    cudaStream_t st = (cudaStream_t)stream;
    if (N == 0 || M == 0) return MM_OK;
    if (P == 0) {  // C = 0 in host memory, after the stream's earlier work (which may still write C)
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "mm_emulated_host");
        for (int64_t i = 0; i < N; ++i) memset(C + i * ldc, 0, (size_t)M * 8);
        return MM_OK;
    }
    const size_t need = emulated_host_ws_bytes(N, P, M, s, kind);
    if (ws_bytes < need || !ws)
        return fail(MM_ERR_WORKSPACE, "mm_emulated_host: workspace %zu bytes < %zu required", ws_bytes, need);
    return run_emulated_host(N, P, M, A, lda, B, ldb, C, ldc, s, kind, ws, st);
}

int mm_emulated_noalloc(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                        int64_t ldb, double *C, int64_t ldc, int32_t kind, int32_t nslices, double tier,
                        void *stream) {
    int rc = check_gemm_args("mm_emulated_noalloc", N, P, M, A, lda, B, ldb, C, ldc);
    if (rc) return rc;
    const int s = slices_or_fail("mm_emulated_noalloc", kind, nslices, tier);
    if (s < 0) return s;
    if (P > (int64_t(1) << 20)) return fail(MM_ERR_UNSUPPORTED, "mm_emulated_noalloc: P > 2^20");
    cudaStream_t st = (cudaStream_t)stream;
    if (N == 0 || M == 0) return MM_OK;
    if (P == 0) return run_zero(N, M, C, ldc, st);
    return run_emulated_noalloc(N, P, M, A, lda, B, ldb, C, ldc, s, kind, st);
}

size_t mm_emulated_noalloc_capacity(void) { return emulated_noalloc_capacity(); }

static int check_group(const char *fn, const mm_problem *probs, int32_t count, int32_t kind, int32_t nslices,
                       double tier) {
    if (count < 0 || (count > 0 && !probs)) return fail(MM_ERR_ARG, "%s: bad problem list", fn);
    const int s = slices_or_fail(fn, kind, nslices, tier);
    if (s < 0) return s;
    for (int32_t i = 0; i < count; ++i) {
        const mm_problem &q = probs[i];
        int rc = check_gemm_args(fn, q.N, q.P, q.M, q.A, q.lda, q.B, q.ldb, q.C, q.ldc);
        if (rc) return fail(rc, "%s: problem %d: %s", fn, (int)i, mm_last_error());
        if (q.P > (int64_t(1) << 20)) return fail(MM_ERR_UNSUPPORTED, "%s: problem %d has P > 2^20", fn, (int)i);
    }
    for (int32_t i = 0; i < count; ++i) {  // outputs must not overlap one another
        const size_t bi = span_bytes(probs[i].N, probs[i].M, probs[i].ldc);
        for (int32_t j = i + 1; j < count && bi; ++j)
            if (ranges_overlap(probs[i].C, bi, probs[j].C, span_bytes(probs[j].N, probs[j].M, probs[j].ldc)))
                return fail(MM_ERR_ARG, "%s: outputs of problems %d and %d overlap", fn, (int)i, (int)j);
    }
    return MM_OK;
}

size_t mm_emulated_group_workspace_bytes(const mm_problem *probs, int32_t count, int32_t kind, int32_t nslices,
                                         double tier) {
    const int s = emulated_slices(kind, nslices, tier);
    if (s <= 0 || count <= 0 || !probs) return 0;
    return emulated_group_ws_bytes(probs, count, s, kind);
}

int mm_emulated_group(const mm_problem *probs, int32_t count, int32_t kind, int32_t nslices, double tier, void *ws,
                      size_t ws_bytes, void *stream) {
    int rc = check_group("mm_emulated_group", probs, count, kind, nslices, tier);
    if (rc) return rc;
    if (count == 0) return MM_OK;
    const int s = emulated_slices(kind, nslices, tier);
    const size_t need = emulated_group_ws_bytes(probs, count, s, kind);
    if (ws_bytes < need || !ws)
        return fail(MM_ERR_WORKSPACE, "mm_emulated_group: workspace %zu bytes < %zu required", ws_bytes, need);
    return run_emulated_group(probs, count, s, kind, ws, (cudaStream_t)stream);
}

size_t mm_strassen_emulated_workspace_bytes(int64_t N, int64_t P, int64_t M, int32_t variant, int32_t levels,
                                            int32_t kind, int32_t nslices, double tier) {
    const int s = emulated_slices(kind, nslices, tier);
    if (s <= 0 || N < 0 || P < 0 || M < 0 || variant < 0 || variant > 1 || levels < -1 || levels > 4) return 0;
    if (N == 0 || M == 0 || P == 0) return 0;
    return strassen_emulated_ws_bytes(variant, strassen_emulated_levels(levels, N, P, M), N, P, M, s, kind);
}

int mm_strassen_emulated(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                         double *C, int64_t ldc, int32_t variant, int32_t levels, int32_t kind, int32_t nslices,
                         double tier, void *ws, size_t ws_bytes, void *stream) {
    const char *fn = "mm_strassen_emulated";
    int rc = check_gemm_args(fn, N, P, M, A, lda, B, ldb, C, ldc);
    if (rc) return rc;
    if (variant < 0 || variant > 1) return fail(MM_ERR_ARG, "%s: variant must be 0 or 1", fn);
    if (levels < -1 || levels > 4) return fail(MM_ERR_ARG, "%s: levels must be -1 (automatic) or 0..4", fn);
    const int s = slices_or_fail(fn, kind, nslices, tier);
    if (s < 0) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (N == 0 || M == 0) return MM_OK;
    if (P == 0) return run_zero(N, M, C, ldc, st);
    levels = strassen_emulated_levels(levels, N, P, M);
    const size_t need = strassen_emulated_ws_bytes(variant, levels, N, P, M, s, kind);
    if (ws_bytes < need || !ws)
        return fail(MM_ERR_WORKSPACE, "%s: workspace %zu bytes < %zu required", fn, ws_bytes, need);
    return run_strassen_emulated(variant, levels, N, P, M, A, lda, B, ldb, C, ldc, s, kind, ws, st);
}

size_t mm_emulated_auto_workspace_bytes(int64_t N, int64_t P, int64_t M, double tier) {
    int kind, s, levels, tile;
    if (N <= 0 || P <= 0 || M <= 0 || emulated_choice(N, P, M, tier, &kind, &s, &levels, &tile) < 0) return 0;
    return levels == 0 ? emulated_ws_bytes(N, P, M, s, kind)
                       : strassen_emulated_ws_bytes(1, levels, N, P, M, s, kind);
}

int mm_emulated_auto(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                     double *C, int64_t ldc, double tier, void *ws, size_t ws_bytes, void *stream, int32_t *used) {
    const char *fn = "mm_emulated_auto";
    int rc = check_gemm_args(fn, N, P, M, A, lda, B, ldb, C, ldc);
    if (rc) return rc;
    if (!(tier > 0.0)) return fail(MM_ERR_ARG, "%s: tier must be > 0", fn);
    if (P > (int64_t(1) << 20)) return fail(MM_ERR_UNSUPPORTED, "%s: P > 2^20", fn);
    cudaStream_t st = (cudaStream_t)stream;
    if (N == 0 || M == 0) return MM_OK;
    if (P == 0) return run_zero(N, M, C, ldc, st);
    int kind, s, levels, tile;
    if (emulated_choice(N, P, M, tier, &kind, &s, &levels, &tile) < 0)
        return fail(MM_ERR_UNSUPPORTED, "%s: tier %g needs more slices than either format holds", fn, tier);
    const size_t need = levels == 0 ? emulated_ws_bytes(N, P, M, s, kind)
                                    : strassen_emulated_ws_bytes(1, levels, N, P, M, s, kind);
    if (ws_bytes < need || !ws)
        return fail(MM_ERR_WORKSPACE, "%s: workspace %zu bytes < %zu required", fn, ws_bytes, need);
    if (used) {
        used[0] = kind;
        used[1] = s;
        used[2] = levels;
        used[3] = levels == 0 ? tile : emu::slice_bn(s);
    }
    return levels == 0 ? run_emulated(N, P, M, A, lda, B, ldb, C, ldc, s, kind, ws, st, tile)
                       : run_strassen_emulated(1, levels, N, P, M, A, lda, B, ldb, C, ldc, s, kind, ws, st);
}

int mm_profile_enable(int on) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof_on = on != 0;
    return MM_OK;
}

int mm_profile_read(mm_kernel_stat *out, int32_t cap) {
    std::vector<ProfRec> recs;
    {
        std::lock_guard<std::mutex> g(g_prof_mu);
        recs.swap(g_prof_recs);
    }
    std::vector<mm_kernel_stat> stats;
    int rc = MM_OK;
    for (auto &r : recs) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.stop);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.start, r.stop);
        if (e != cudaSuccess) rc = cuda_fail(e, "mm_profile_read");
        auto it = std::find_if(stats.begin(), stats.end(),
                               [&](const mm_kernel_stat &s) { return r.name == s.name; });
        if (it == stats.end()) {
            mm_kernel_stat s{};
            snprintf(s.name, sizeof s.name, "%s", r.name.c_str());
            stats.push_back(s);
            it = stats.end() - 1;
        }
        it->launches += 1;
        it->total_ms += ms;
    }
    {
        std::lock_guard<std::mutex> g(g_prof_mu);
        for (auto &r : recs) {
            g_event_pool.push_back(r.start);
            g_event_pool.push_back(r.stop);
        }
    }
    if (rc != MM_OK) return rc;
    for (int32_t i = 0; i < cap && i < (int32_t)stats.size(); ++i) out[i] = stats[i];
    return (int)stats.size();
}

}  // extern "C"
