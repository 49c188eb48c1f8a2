// Pipe-throughput probe: the measured denominators of the FP32 and SFU
// (MUFU) rooflines the objective kernels are reported against.
//
// Each probe kernel keeps many independent dependency chains of one
// operation per thread (so latency is hidden) over a full-occupancy grid
// sized in whole waves of the device's SMs, and is timed with CUDA events
// (best of several launches).  Rates are thread-level operations per second;
// a packed FP32x2 FMA counts as two FMAs.  The results feed no computation of
// the library: they exist so that fractions of peak are fractions of what this
// GPU measurably does, not of nominal unit counts.
#include <cuda_runtime.h>
#include <stdint.h>

#include "musr.h"
#include "musr_internal.h"

namespace musr {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeIters = 2048;
constexpr int kChains = 16;

__global__ void __launch_bounds__(kProbeThreads) probe_ffma(float a, float b, float* sink) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
#pragma unroll 2
    for (int i = 0; i < kProbeIters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1.2345678f) sink[0] = s;  // never true for the probe's inputs; keeps the chains alive
}

__global__ void __launch_bounds__(kProbeThreads) probe_ffma2(float a, float b, float* sink) {
    float2 x[kChains / 2];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) x[c] = make_float2((float)(threadIdx.x + c) * 1e-3f, (float)c * 1e-3f);
#pragma unroll 2
    for (int i = 0; i < kProbeIters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) s += x[c].x + x[c].y;
    if (s == 1.2345678f) sink[0] = s;
}

// SFU operations as single PTX instructions; the FP32 operation that keeps
// each chain bounded runs on the FMA pipe, not the SFU
enum SfuOp { kEx2 = 0, kSin = 1, kCos = 2, kRcp = 3, kLg2 = 4 };

template <int OP>
__device__ __forceinline__ float sfu(float x) {
    float y;
    if (OP == kEx2) asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
    else if (OP == kSin) asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    else if (OP == kCos) asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    else if (OP == kRcp) asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x + 1.f));
    else asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x + 2.f));
    return y;
}

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) probe_sfu(float* sink) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0.25f + (float)(threadIdx.x + c) * 1e-4f;
#pragma unroll 2
    for (int i = 0; i < kProbeIters / 4; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = sfu<OP>(x[c]);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1.2345678f) sink[0] = s;
}

// Best-of-`reps` seconds of one launch of `launch` (after one warm-up launch).
template <class F>
cudaError_t time_best(F launch, cudaStream_t st, int reps, double* seconds) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        launch();
        e = cudaGetLastError();
    }
    double best = 1e30;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms > 0.f && ms * 1e-3 < best) best = ms * 1e-3;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *seconds = best;
    return e;
}

}  // namespace
}  // namespace musr

using namespace musr;

extern "C" int musr_pipe_rates(double* rates, int32_t n_rates) {
    if (!rates || n_rates < MUSR_RATE_COUNT) return MUSR_EINVAL;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(e);
    float* sink = nullptr;
    e = cudaMalloc(&sink, sizeof(float));
    if (e != cudaSuccess) return cuda_status(e);
    cudaStream_t st = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    // 8 resident 256-thread blocks per SM (64 warps), 4 waves
    const int blocks = sms * 8 * 4;
    const double threads = (double)blocks * kProbeThreads;
    double s = 0.0;
    if (e == cudaSuccess) {
        e = time_best([&] { probe_ffma<<<blocks, kProbeThreads, 0, st>>>(0.999f, 1e-3f, sink); }, st, 5, &s);
        rates[MUSR_RATE_FFMA] = threads * kChains * kProbeIters / s;
    }
    if (e == cudaSuccess) {
        e = time_best([&] { probe_ffma2<<<blocks, kProbeThreads, 0, st>>>(0.999f, 1e-3f, sink); }, st, 5, &s);
        rates[MUSR_RATE_FFMA2] = threads * kChains * kProbeIters / s;
    }
    const double sfu_ops = threads * kChains * (kProbeIters / 4);
    if (e == cudaSuccess) {
        e = time_best([&] { probe_sfu<kEx2><<<blocks, kProbeThreads, 0, st>>>(sink); }, st, 5, &s);
        rates[MUSR_RATE_EX2] = sfu_ops / s;
    }
    if (e == cudaSuccess) {
        e = time_best([&] { probe_sfu<kSin><<<blocks, kProbeThreads, 0, st>>>(sink); }, st, 5, &s);
        rates[MUSR_RATE_SIN] = sfu_ops / s;
    }
    if (e == cudaSuccess) {
        e = time_best([&] { probe_sfu<kCos><<<blocks, kProbeThreads, 0, st>>>(sink); }, st, 5, &s);
        rates[MUSR_RATE_COS] = sfu_ops / s;
    }
    if (e == cudaSuccess) {
        e = time_best([&] { probe_sfu<kRcp><<<blocks, kProbeThreads, 0, st>>>(sink); }, st, 5, &s);
        rates[MUSR_RATE_RCP] = sfu_ops / s;
    }
    if (e == cudaSuccess) {
        e = time_best([&] { probe_sfu<kLg2><<<blocks, kProbeThreads, 0, st>>>(sink); }, st, 5, &s);
        rates[MUSR_RATE_LG2] = sfu_ops / s;
    }
    if (st) cudaStreamDestroy(st);
    cudaFree(sink);
    return cuda_status(e);
}
