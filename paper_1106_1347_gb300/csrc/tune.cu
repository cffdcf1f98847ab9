// Autotuner: the Strassen recursion depth per (variant, shape bucket), chosen
// by timing depths 0..3 on the device, kept in an in-library table that
// mm_strassen / mm_strassen_winograd consult for cutoff == -1, and persisted
// as a small text file (one "strassen <variant> <bucket> <depth>" line per
// entry; MM_TUNE_CACHE names a file loaded at first use).  The slice count of
// the emulated product needs no search: it follows from the requested tier.
#include <stdio.h>
#include <stdlib.h>

#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"

namespace {

std::mutex g_mu;
std::map<std::pair<int, int>, int> g_depth;  // (variant, bucket) -> depth
bool g_env_loaded = false;

int bucket_of(int64_t N, int64_t P, int64_t M) {
    int64_t X = std::max(N, std::max(P, M));
    int b = 0;
    while (X > 1) {
        X >>= 1;
        ++b;
    }
    return b;  // floor(log2 max dim)
}

int load_file(const char *path) {
    FILE *f = fopen(path, "r");
    if (!f) return mm::fail(MM_ERR_ARG, "mm_tune_load: cannot open %s", path);
    char kind[32];
    int variant, bucket, depth, n = 0;
    while (fscanf(f, "%31s %d %d %d", kind, &variant, &bucket, &depth) == 4) {
        if (std::string(kind) != "strassen" || variant < 0 || variant > 1 || depth < 0 || depth > 10) continue;
        g_depth[{variant, bucket}] = depth;
        ++n;
    }
    fclose(f);
    return n;
}

void load_env_once() {
    if (g_env_loaded) return;
    g_env_loaded = true;
    const char *p = getenv("MM_TUNE_CACHE");
    if (p && *p) (void)load_file(p);
}

}  // namespace

namespace mm {

bool tuned_strassen_depth(int variant, int64_t N, int64_t P, int64_t M, int *depth) {
    std::lock_guard<std::mutex> g(g_mu);
    load_env_once();
    auto it = g_depth.find({variant, bucket_of(N, P, M)});
    if (it == g_depth.end()) return false;
    *depth = it->second;
    return true;
}

}  // namespace mm

extern "C" {

size_t mm_tune_strassen_workspace_bytes(int64_t N, int64_t P, int64_t M) {
    if (N <= 0 || P <= 0 || M <= 0) return 0;
    size_t most = 0;
    for (int d = 1; d <= 3; ++d) {
        const int64_t q = (int64_t)1 << d;
        for (int v = 0; v < 2; ++v)
            most = std::max(most, mm::strassen_ws_bytes(v, d, mm::ceil_div(N, q) * q, mm::ceil_div(P, q) * q,
                                                        mm::ceil_div(M, q) * q));
    }
    return most;
}

int mm_tune_strassen(int32_t variant, int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B,
                     int64_t ldb, double *C, int64_t ldc, void *ws, size_t ws_bytes, void *stream, int32_t *best_depth,
                     double *best_ms) {
    if (variant < 0 || variant > 1) return mm::fail(MM_ERR_ARG, "mm_tune_strassen: variant must be 0 or 1");
    int rc = mm::check_gemm_args("mm_tune_strassen", N, P, M, A, lda, B, ldb, C, ldc);
    if (rc) return rc;
    if (N == 0 || P == 0 || M == 0) return mm::fail(MM_ERR_ARG, "mm_tune_strassen: empty product");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = -1;
    float best_t = 0.f;
    for (int d = 0; d <= 3; ++d) {
        const int64_t q = (int64_t)1 << d;
        const int64_t Np = mm::ceil_div(N, q) * q, Pp = mm::ceil_div(P, q) * q, Mp = mm::ceil_div(M, q) * q;
        if (d > 0 && (N < 2 * q || P < 2 * q || M < 2 * q)) break;  // blocks smaller than 2 rows: stop
        if (mm::strassen_ws_bytes(variant, d, Np, Pp, Mp) > ws_bytes) break;
        float t = 0.f;
        for (int rep = 0; rep < 2 && rc == MM_OK; ++rep) {  // the first run warms up
            cudaEventRecord(e0, st);
            rc = mm::run_strassen(variant, N, P, M, A, lda, B, ldb, C, ldc, d, Np, Pp, Mp, ws, st);
            cudaEventRecord(e1, st);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) rc = mm::cuda_fail(e, "mm_tune_strassen");
            if (rc == MM_OK) cudaEventElapsedTime(&t, e0, e1);
        }
        if (rc) break;
        if (best < 0 || t < best_t) {
            best = d;
            best_t = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> g(g_mu);
        load_env_once();
        g_depth[{variant, bucket_of(N, P, M)}] = best;
    }
    if (best_depth) *best_depth = best;
    if (best_ms) *best_ms = best_t;
    return MM_OK;
}

int mm_tune_save(const char *path) {
    if (!path) return mm::fail(MM_ERR_ARG, "mm_tune_save: NULL path");
    std::lock_guard<std::mutex> g(g_mu);
    FILE *f = fopen(path, "w");
    if (!f) return mm::fail(MM_ERR_ARG, "mm_tune_save: cannot open %s", path);
    for (auto &kv : g_depth) fprintf(f, "strassen %d %d %d\n", kv.first.first, kv.first.second, kv.second);
    fclose(f);
    return MM_OK;
}

int mm_tune_load(const char *path) {
    if (!path) return mm::fail(MM_ERR_ARG, "mm_tune_load: NULL path");
    std::lock_guard<std::mutex> g(g_mu);
    g_env_loaded = true;
    return load_file(path);
}

int mm_tune_clear(void) {
    std::lock_guard<std::mutex> g(g_mu);
    g_depth.clear();
    g_env_loaded = true;
    return MM_OK;
}

}  // extern "C"
