// Autotuner (not in the paper, which fixes its choices by rule):
//   - the Strassen recursion depth per (variant, shape bucket), chosen by
//     timing every depth whose blocks stay at least 16 wide (at most
//     kWinogradSafeDepth levels of Winograd's variant, whose error grows
//     about twice per level), consulted by mm_strassen / mm_strassen_winograd
//     for cutoff == -1;
//   - for the FP64-accurate emulated product, per (shape bucket, tier): the
//     slice format (BF16 or FP8-E4M3, each with the slice count the tier
//     needs), the number of Strassen-Winograd levels over it and, for the
//     direct product, the slice product's tile width (64 or 32 columns),
//     chosen by timing every candidate; consulted by mm_emulated_auto and (for
//     format and count) by the serving loop's method 2.
// Both live in one in-library table, persisted as a small text file, one entry
// per line:
//   strassen <variant> <log2 max dim> <depth>
//   emulated <log2 N> <log2 P> <log2 M> <tier decade> <format> <slices> <levels> <tile width>
// (lines without the tile width, as earlier files wrote them, take the default).
// MM_TUNE_CACHE names a file loaded at first use.  Without an entry the
// choices fall back to models: the paper's depth floor(log2 X) - 4 for
// Strassen; for the emulated product the format whose slice pairs cost less at
// the nominal rates (an FP8 pair costs half a BF16 one, three quarters past 8
// slices), the measured level crossovers of strassen_emulated_levels, and the
// 32-column tile only where a 64-column one would be at most half used.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>

#include "common.cuh"
#include "slice_gemm.cuh"

namespace {

struct EmuChoice {
    int kind, slices, levels, tile;  // tile: the slice product's tile width (0: the default)
    double ms;
};
using EmuKey = std::tuple<int, int, int, int>;  // log2 N, log2 P, log2 M, tier decade

std::mutex g_mu;
std::map<std::pair<int, int>, int> g_depth;  // (variant, bucket) -> depth
std::map<EmuKey, EmuChoice> g_emu;
bool g_env_loaded = false;

int lg2(int64_t x) {
    int b = 0;
    while (x > 1) {
        x >>= 1;
        ++b;
    }
    return b;
}

int bucket_of(int64_t N, int64_t P, int64_t M) { return lg2(std::max(N, std::max(P, M))); }

int tier_decade(double tier) { return (int)lround(-log10(tier)); }

EmuKey emu_key(int64_t N, int64_t P, int64_t M, double tier) {
    return EmuKey{lg2(N), lg2(P), lg2(M), tier_decade(tier)};
}

int load_file(const char *path) {
    FILE *f = fopen(path, "r");
    if (!f) return mm::fail(MM_ERR_ARG, "mm_tune_load: cannot open %s", path);
    char line[256];
    int n = 0;
    while (fgets(line, sizeof line, f)) {
        char kind[32];
        int a[8];
        if (sscanf(line, "%31s", kind) != 1) continue;
        if (std::string(kind) == "strassen" && sscanf(line, "%*s %d %d %d", &a[0], &a[1], &a[2]) == 3) {
            if (a[0] < 0 || a[0] > 1 || a[2] < 0 || a[2] > 16) continue;
            g_depth[{a[0], a[1]}] = a[2];
            ++n;
        } else if (std::string(kind) == "emulated") {
            const int got =
                sscanf(line, "%*s %d %d %d %d %d %d %d %d", &a[0], &a[1], &a[2], &a[3], &a[4], &a[5], &a[6], &a[7]);
            if (got < 7) continue;
            if (got == 7) a[7] = 0;
            if ((a[4] != MM_SLICE_BF16 && a[4] != MM_SLICE_FP8E4M3) || a[5] < 1 || a[5] > (a[4] ? 10 : 8) ||
                a[6] < 0 || a[6] > 4 || (a[7] != 0 && !emu::slice_bn_ok(a[5], a[7])))
                continue;
            g_emu[EmuKey{a[0], a[1], a[2], a[3]}] = EmuChoice{a[4], a[5], a[6], a[7], 0.0};
            ++n;
        }
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

// Deepest Strassen depth the tuner tries: blocks of at least 16 in every dimension.
int max_tuned_depth(int64_t N, int64_t P, int64_t M) {
    const int64_t lo = std::min(N, std::min(P, M));
    int d = 0;
    while (d < 16 && (lo >> (d + 1)) >= 16) ++d;
    return d;
}

// The model's emulated choice for a tier (no table entry): the format whose
// slice pairs cost less, an FP8-E4M3 pair at half a BF16 pair up to 8 slices
// (both issue N = 128 MMAs) and at three quarters past 8 (N = 64 MMAs on
// 32-column accumulators, which issue at about 2/3 of the N = 128 rate).
int model_emulated(int64_t N, int64_t P, int64_t M, double tier, int *kind, int *slices, int *levels, int *tile) {
    const int sb = mm::emulated_slices(MM_SLICE_BF16, 0, tier);
    const int s8 = mm::emulated_slices(MM_SLICE_FP8E4M3, 0, tier);
    if (sb < 0 && s8 < 0) return sb;
    *kind = MM_SLICE_BF16;
    *slices = sb;
    const double cost8 = s8 > 0 ? s8 * (s8 + 1) * (s8 > 8 ? 0.75 : 0.5) : 1e30;
    const double cost16 = sb > 0 ? (double)sb * (sb + 1) : 1e30;
    if (cost8 < cost16) {
        *kind = MM_SLICE_FP8E4M3;
        *slices = s8;
    }
    *levels = mm::strassen_emulated_levels(-1, N, P, M);
    // A 32-column tile issues its MMAs at about 2/3 of the 64-column rate, so
    // it pays only where it saves more than a third of the padded columns.
    const int64_t w64 = mm::ceil_div(M, (int64_t)64) * 64, w32 = mm::ceil_div(M, (int64_t)32) * 32;
    *tile = (*levels == 0 && *slices <= 8 && 3 * w32 < 2 * w64) ? 32 : emu::slice_bn(*slices);
    return MM_OK;
}

// Candidate levels of Strassen-Winograd over the emulated product: each level
// must leave blocks of at least 512 in every dimension.
int max_emulated_levels(int64_t N, int64_t P, int64_t M) {
    const int64_t lo = std::min(N, std::min(P, M));
    int L = 0;
    while (L < 2 && (lo >> (L + 1)) >= 512) ++L;
    return L;
}

size_t emulated_candidate_bytes(int64_t N, int64_t P, int64_t M, int kind, int s, int levels) {
    return levels == 0 ? mm::emulated_ws_bytes(N, P, M, s, kind)
                       : mm::strassen_emulated_ws_bytes(1, levels, N, P, M, s, kind);
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

// The emulated product's format, slice count, Strassen levels and tile width
// for a tier: the tuned entry of the shape bucket, else the model.  Returns 1 (tuned),
// 0 (model) or a negative status for an invalid tier.
int emulated_choice(int64_t N, int64_t P, int64_t M, double tier, int *kind, int *slices, int *levels, int *tile) {
    if (!(tier > 0.0)) return MM_ERR_ARG;
    {
        std::lock_guard<std::mutex> g(g_mu);
        load_env_once();
        auto it = g_emu.find(emu_key(N, P, M, tier));
        if (it != g_emu.end()) {
            *kind = it->second.kind;
            *slices = it->second.slices;
            *levels = it->second.levels;
            *tile = it->second.tile ? it->second.tile : emu::slice_bn(it->second.slices);
            return 1;
        }
    }
    const int rc = model_emulated(N, P, M, tier, kind, slices, levels, tile);
    return rc < 0 ? rc : 0;
}

}  // namespace mm

extern "C" {

size_t mm_tune_strassen_workspace_bytes(int64_t N, int64_t P, int64_t M) {
    if (N <= 0 || P <= 0 || M <= 0) return 0;
    size_t most = 0;
    for (int d = 1; d <= max_tuned_depth(N, P, M); ++d) {
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
    const int dmax = variant == 1 ? std::min(max_tuned_depth(N, P, M), mm::kWinogradSafeDepth)
                                  : max_tuned_depth(N, P, M);
    for (int d = 0; d <= dmax; ++d) {
        const int64_t q = (int64_t)1 << d;
        const int64_t Np = mm::ceil_div(N, q) * q, Pp = mm::ceil_div(P, q) * q, Mp = mm::ceil_div(M, q) * q;
        if (mm::strassen_ws_bytes(variant, d, Np, Pp, Mp) > ws_bytes) continue;
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

size_t mm_tune_emulated_workspace_bytes(int64_t N, int64_t P, int64_t M, double tier) {
    if (N <= 0 || P <= 0 || M <= 0 || !(tier > 0.0)) return 0;
    size_t most = 0;
    for (int kind = MM_SLICE_BF16; kind <= MM_SLICE_FP8E4M3; ++kind) {
        const int s = mm::emulated_slices(kind, 0, tier);
        if (s < 0) continue;
        for (int L = 0; L <= max_emulated_levels(N, P, M); ++L)
            most = std::max(most, emulated_candidate_bytes(N, P, M, kind, s, L));
    }
    return most;
}

int mm_tune_emulated(int64_t N, int64_t P, int64_t M, const double *A, int64_t lda, const double *B, int64_t ldb,
                     double *C, int64_t ldc, double tier, void *ws, size_t ws_bytes, void *stream, int32_t *best_kind,
                     int32_t *best_slices, int32_t *best_levels, double *best_ms, int32_t *best_tile) {
    int rc = mm::check_gemm_args("mm_tune_emulated", N, P, M, A, lda, B, ldb, C, ldc);
    if (rc) return rc;
    if (N == 0 || P == 0 || M == 0) return mm::fail(MM_ERR_ARG, "mm_tune_emulated: empty product");
    if (!(tier > 0.0)) return mm::fail(MM_ERR_ARG, "mm_tune_emulated: tier must be > 0");
    if (P > (int64_t(1) << 20)) return mm::fail(MM_ERR_UNSUPPORTED, "mm_tune_emulated: P > 2^20");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    EmuChoice best{-1, 0, 0, 0, 0.0};
    for (int kind = MM_SLICE_BF16; kind <= MM_SLICE_FP8E4M3 && rc == MM_OK; ++kind) {
        const int s = mm::emulated_slices(kind, 0, tier);
        if (s < 0) continue;  // the tier needs more slices than this format holds
        for (int L = 0; L <= max_emulated_levels(N, P, M) && rc == MM_OK; ++L) {
            if (emulated_candidate_bytes(N, P, M, kind, s, L) > ws_bytes) continue;
            // The direct product tries both tile widths its slice count allows.
            for (int tile : {emu::slice_bn(s), 32}) {
                if (tile == 32 && (L > 0 || emu::slice_bn(s) == 32)) continue;
                float t = 0.f, tmin = 0.f;
                for (int rep = 0; rep < 3 && rc == MM_OK; ++rep) {  // one warm-up, the faster of two timed runs
                    cudaEventRecord(e0, st);
                    rc = L == 0 ? mm::run_emulated(N, P, M, A, lda, B, ldb, C, ldc, s, kind, ws, st, tile)
                                : mm::run_strassen_emulated(1, L, N, P, M, A, lda, B, ldb, C, ldc, s, kind, ws, st);
                    cudaEventRecord(e1, st);
                    cudaError_t e = cudaEventSynchronize(e1);
                    if (e != cudaSuccess) rc = mm::cuda_fail(e, "mm_tune_emulated");
                    if (rc == MM_OK) cudaEventElapsedTime(&t, e0, e1);
                    if (rep == 1 || (rep == 2 && t < tmin)) tmin = t;
                }
                if (rc == MM_OK && (best.kind < 0 || tmin < best.ms)) best = EmuChoice{kind, s, L, tile, (double)tmin};
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (best.kind < 0) return mm::fail(MM_ERR_WORKSPACE, "mm_tune_emulated: no candidate fits %zu bytes", ws_bytes);
    {
        std::lock_guard<std::mutex> g(g_mu);
        load_env_once();
        g_emu[emu_key(N, P, M, tier)] = best;
    }
    if (best_kind) *best_kind = best.kind;
    if (best_slices) *best_slices = best.slices;
    if (best_levels) *best_levels = best.levels;
    if (best_ms) *best_ms = best.ms;
    if (best_tile) *best_tile = best.tile;
    return MM_OK;
}

int mm_tune_emulated_choice(int64_t N, int64_t P, int64_t M, double tier, int32_t *kind, int32_t *slices,
                            int32_t *levels, int32_t *tile) {
    if (N < 0 || P < 0 || M < 0) return mm::fail(MM_ERR_ARG, "mm_tune_emulated_choice: negative size");
    int k = 0, s = 0, l = 0, w = 0;
    const int rc = mm::emulated_choice(N, P, M, tier, &k, &s, &l, &w);
    if (rc < 0) return mm::fail(rc, "mm_tune_emulated_choice: tier must be > 0 and within the formats' reach");
    if (kind) *kind = k;
    if (slices) *slices = s;
    if (levels) *levels = l;
    if (tile) *tile = w;
    return rc;
}

int mm_tune_save(const char *path) {
    if (!path) return mm::fail(MM_ERR_ARG, "mm_tune_save: NULL path");
    std::lock_guard<std::mutex> g(g_mu);
    FILE *f = fopen(path, "w");
    if (!f) return mm::fail(MM_ERR_ARG, "mm_tune_save: cannot open %s", path);
    for (auto &kv : g_depth) fprintf(f, "strassen %d %d %d\n", kv.first.first, kv.first.second, kv.second);
    for (auto &kv : g_emu)
        fprintf(f, "emulated %d %d %d %d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first),
                std::get<2>(kv.first), std::get<3>(kv.first), kv.second.kind, kv.second.slices, kv.second.levels,
                kv.second.tile);
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
    g_emu.clear();
    g_env_loaded = true;
    return MM_OK;
}

}  // extern "C"
