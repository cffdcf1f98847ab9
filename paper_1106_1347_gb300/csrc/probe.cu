// Measurement support (not in the paper): the peak rate of this device's FP64
// pipe, the denominator of every FP64 roofline fraction.  Two kernels keep
// the pipe busy with independent work and nothing else:
//   dfma  -- every thread runs 8 independent FMA chains x <- x * a + b (|a| < 1,
//            so the values stay bounded); 2 flop per FMA;
//   dmma  -- every warp runs 4 independent mma.sync m8n8k4 f64 accumulators;
//            512 flop per MMA (8 x 8 x 4 multiply-adds).
// Each runs on 4 CTAs of 256 threads per SM (32 warps per SM, 8 per
// scheduler), enough independent instructions to cover the pipe's latency.
// The chains end in a comparison with a value they never reach, whose store
// would go to a static device word: the compiler must keep every operation,
// and nothing is allocated.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace {

__device__ double g_probe_sink;

constexpr int kProbeThreads = 256, kProbeCtasPerSm = 4, kChains = 8, kMmaAcc = 4, kInner = 16;

__global__ void __launch_bounds__(kProbeThreads) dfma_probe_kernel(int32_t outer, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (double)(threadIdx.x + c);
    for (int32_t i = 0; i < outer; ++i) {
#pragma unroll
        for (int r = 0; r < kInner; ++r)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.0) g_probe_sink = s;  // never true: the chains stay positive
}

__device__ __forceinline__ void dmma(double (&c)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(c[0]), "+d"(c[1])
                 : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(kProbeThreads) dmma_probe_kernel(int32_t outer, double a, double b) {
    double acc[kMmaAcc][2];
#pragma unroll
    for (int c = 0; c < kMmaAcc; ++c) acc[c][0] = acc[c][1] = 0.0;
    const double av = a * (double)((threadIdx.x & 31) + 1), bv = b;
    for (int32_t i = 0; i < outer; ++i) {
#pragma unroll
        for (int r = 0; r < kInner; ++r)
#pragma unroll
            for (int c = 0; c < kMmaAcc; ++c) dmma(acc[c], av, bv);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kMmaAcc; ++c) s += acc[c][0] + acc[c][1];
    if (s == -1.0) g_probe_sink = s;  // never true: every product is positive
}

// Times `launch(outer)` with events on st: one warm-up run, then repeats the
// timed run with `outer` grown until it lasts at least target_ms.  Returns the
// time of the last run in ms and its `outer` in *outer_used.
template <class F>
int time_probe(F &&launch, double target_ms, cudaStream_t st, float *ms, int32_t *outer_used) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return mm::cuda_fail(e, "mm_probe_fp64_peak: events");
    int32_t outer = 64;
    int rc = launch(outer);
    float t = 0.f;
    for (int tries = 0; rc == MM_OK && tries < 12; ++tries) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) rc = launch(outer);
        if (rc == MM_OK && e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (rc == MM_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (rc == MM_OK && e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e != cudaSuccess) rc = mm::cuda_fail(e, "mm_probe_fp64_peak");
        if (rc != MM_OK || t >= target_ms || outer >= (1 << 24)) break;
        const double grow = t > 0.f ? std::min(16.0, 1.2 * target_ms / t) : 16.0;
        outer = (int32_t)std::min<double>((double)(1 << 24), std::ceil(outer * grow));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = t;
    *outer_used = outer;
    return rc;
}

}  // namespace

extern "C" int mm_probe_fp64_peak(double target_ms, double *dfma_tflops, double *dmma_tflops, void *stream) {
    if (!(target_ms > 0.0) || target_ms > 10000.0)
        return mm::fail(MM_ERR_ARG, "mm_probe_fp64_peak: target_ms must be in (0, 10000]");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t ctas = (int64_t)kProbeCtasPerSm * mm::sm_count();
    const double a = 0.999999, b = 1e-9;
    float ms = 0.f;
    int32_t outer = 0;
    int rc = time_probe(
        [&](int32_t o) {
            return mm::launch("fp64_probe_dfma", st,
                              [&] { dfma_probe_kernel<<<(unsigned)ctas, kProbeThreads, 0, st>>>(o, a, b); });
        },
        target_ms, st, &ms, &outer);
    if (rc) return rc;
    const double fma_count = (double)ctas * kProbeThreads * kChains * kInner * (double)outer;
    if (dfma_tflops) *dfma_tflops = ms > 0.f ? 2.0 * fma_count / (ms * 1e-3) / 1e12 : 0.0;
    rc = time_probe(
        [&](int32_t o) {
            return mm::launch("fp64_probe_dmma", st,
                              [&] { dmma_probe_kernel<<<(unsigned)ctas, kProbeThreads, 0, st>>>(o, 1e-3, 1e-3); });
        },
        target_ms, st, &ms, &outer);
    if (rc) return rc;
    const double mma_count = (double)ctas * (kProbeThreads / 32) * kMmaAcc * kInner * (double)outer;
    if (dmma_tflops) *dmma_tflops = ms > 0.f ? 512.0 * mma_count / (ms * 1e-3) / 1e12 : 0.0;
    return MM_OK;
}
