// Synthetic histograms on the device: Poisson counts of the Eq. 1 theory,
// summed over groups of `rebin` bins, for many parameter vectors at once
// (the training data of the learned start proposer), and a plain Poisson
// sampler for given means.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011), a
// counter-based generator, so every variate is a pure function of (seed,
// sample, histogram, group, attempt) and any subset can be regenerated.
// Poisson variates: inversion by sequential search for mean < 12, and Hormann's
// transformed rejection PTRS (1993) above; the PTRS acceptance test uses the
// log-probability in the cancellation-free Stirling form
//     log p = -mu h(y) + 1/2 log1p(y) - 1/2 log(2 pi mu) - 1/(12 n) + 1/(360 n^3),
//     n = k + 1, y = (n - mu)/mu, h(y) = (1 + y) log1p(y) - y,
// so FP32 keeps it accurate at any mean.  Every floating-point operation of the
// sampler is written with an explicit rounding intrinsic (no contraction), and
// the logarithm and exponential are built from basic IEEE operations, so the
// integers drawn are a fixed function of the mean.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "eval_kernel.cuh"
#include "musr.h"
#include "musr_internal.h"
#include "run_impl.h"

namespace musr {
namespace {

__device__ __forceinline__ void philox_round(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0;
    const uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

__device__ __forceinline__ void philox4x32_10(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        philox_round(c, k0, k1);
    }
}

// uniform in (0, 1): ((r >> 9) + 1/2) 2^-23, exact, never 0 or 1
__device__ __forceinline__ float u01(uint32_t r) {
    return __fmul_rn(__fadd_rn((float)(r >> 9), 0.5f), 1.1920928955078125e-07f);
}

// natural logarithm of a positive normal float by 2 atanh((m-1)/(m+1))
__device__ __forceinline__ float s_log(float x) {
    const uint32_t b = __float_as_uint(x);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float m = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);
    if (m > 1.41421356f) {
        m = __fmul_rn(m, 0.5f);
        e = e + 1;
    }
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float s2 = __fmul_rn(s, s);
    float p = __fmaf_rn(s2, 0.111111111f, 0.142857143f);
    p = __fmaf_rn(s2, p, 0.2f);
    p = __fmaf_rn(s2, p, 0.333333333f);
    p = __fmul_rn(p, s2);
    const float two_s = __fadd_rn(s, s);
    const float lm = __fmaf_rn(two_s, p, two_s);
    const float fe = (float)e;
    return __fmaf_rn(fe, 0.693145752f, __fmaf_rn(fe, 1.42860677e-06f, lm));
}

// exp(x), x in [-88, 0]: 2^n e^(f ln 2) with a 10-term Taylor polynomial
__device__ __forceinline__ float s_exp(float x) {
    const float y = __fmul_rn(x, 1.44269504f);
    const float n = floorf(y);
    const float t = __fmul_rn(__fsub_rn(y, n), 0.693147181f);
    float p = __fmaf_rn(t, 0.1f, 1.0f);
    p = __fmaf_rn(__fmul_rn(t, 0.111111111f), p, 1.0f);
    p = __fmaf_rn(__fmul_rn(t, 0.125f), p, 1.0f);
    p = __fmaf_rn(__fmul_rn(t, 0.142857143f), p, 1.0f);
    p = __fmaf_rn(__fmul_rn(t, 0.166666667f), p, 1.0f);
    p = __fmaf_rn(__fmul_rn(t, 0.2f), p, 1.0f);
    p = __fmaf_rn(__fmul_rn(t, 0.25f), p, 1.0f);
    p = __fmaf_rn(__fmul_rn(t, 0.333333333f), p, 1.0f);
    p = __fmaf_rn(__fmul_rn(t, 0.5f), p, 1.0f);
    p = __fmaf_rn(t, p, 1.0f);
    const int ni = (int)n;
    if (ni < -126) return 0.0f;
    return __uint_as_float(__float_as_uint(p) + (uint32_t)(ni * (1 << 23)));
}

// (1 + y) log1p(y) - y
__device__ __forceinline__ float s_h(float y) {
    if (fabsf(y) < 0.125f) {
        float h = __fmaf_rn(y, -1.0f / 72.0f, 1.0f / 56.0f);
        h = __fmaf_rn(y, h, -1.0f / 42.0f);
        h = __fmaf_rn(y, h, 1.0f / 30.0f);
        h = __fmaf_rn(y, h, -1.0f / 20.0f);
        h = __fmaf_rn(y, h, 1.0f / 12.0f);
        h = __fmaf_rn(y, h, -1.0f / 6.0f);
        h = __fmaf_rn(y, h, 0.5f);
        return __fmul_rn(__fmul_rn(h, y), y);
    }
    const float u = s_log(__fadd_rn(1.0f, y));
    return __fmaf_rn(y, u, __fsub_rn(u, y));
}

// log p(k; mu), mu >= 12
__device__ float s_log_pmf(int k, float mu, float log_mu) {
    if (k < 10) {
        float lf = 0.0f;
        for (int i = 2; i <= k; ++i) lf = __fadd_rn(lf, s_log((float)i));
        return __fsub_rn(__fmaf_rn((float)k, log_mu, -mu), lf);
    }
    const float n = (float)(k + 1);
    const float y = __fdiv_rn(__fsub_rn(n, mu), mu);
    const float l1p = s_log(__fadd_rn(1.0f, y));
    const float rn = __fdiv_rn(1.0f, n);
    float v = -__fmul_rn(mu, s_h(y));
    v = __fmaf_rn(0.5f, l1p, v);
    v = __fsub_rn(v, __fmul_rn(0.5f, s_log(__fmul_rn(6.28318531f, mu))));
    v = __fsub_rn(v, __fmul_rn(rn, 0.0833333333f));
    v = __fmaf_rn(__fmul_rn(__fmul_rn(rn, rn), rn), 0.00277777778f, v);
    return v;
}

// Poisson variate for mean mu; (c1, c2, c3) identify the draw, the first
// counter word counts the Philox blocks it uses.
__device__ int32_t poisson_one(float mu, uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3) {
    if (!(mu > 0.0f)) return 0;
    if (mu < 12.0f) {
        uint32_t c[4] = {0u, c1, c2, c3};
        philox4x32_10(c, k0, k1);
        const float u = u01(c[0]);
        float p = s_exp(-mu);
        float F = p;
        int32_t k = 0;
        while (u > F && k < 1000) {
            k = k + 1;
            p = __fdiv_rn(__fmul_rn(p, mu), (float)k);
            F = __fadd_rn(F, p);
        }
        return k;
    }
    const float slam = __fsqrt_rn(mu);
    const float log_mu = s_log(mu);
    const float b = __fmaf_rn(2.53f, slam, 0.931f);
    const float a = __fmaf_rn(0.02483f, b, -0.059f);
    const float inv_alpha = __fadd_rn(1.1239f, __fdiv_rn(1.1328f, __fsub_rn(b, 3.4f)));
    const float vr = __fsub_rn(0.9277f, __fdiv_rn(3.6224f, __fsub_rn(b, 2.0f)));
    for (uint32_t it = 0; it < 64u; ++it) {
        uint32_t c[4] = {it, c1, c2, c3};
        philox4x32_10(c, k0, k1);
        const float U = __fsub_rn(u01(c[0]), 0.5f);
        const float V = u01(c[1]);
        const float us = __fsub_rn(0.5f, fabsf(U));
        const float kf = floorf(__fmaf_rn(__fadd_rn(__fdiv_rn(__fadd_rn(a, a), us), b), U, __fadd_rn(mu, 0.43f)));
        if (us >= 0.07f && V <= vr) return (int32_t)kf;
        if (kf < 0.0f || (us < 0.013f && V > us)) continue;
        const float lhs = s_log(__fdiv_rn(__fmul_rn(V, inv_alpha), __fadd_rn(__fdiv_rn(a, __fmul_rn(us, us)), b)));
        if (lhs <= s_log_pmf((int)kf, mu, log_mu)) return (int32_t)kf;
    }
    return (int32_t)floorf(__fadd_rn(mu, 0.5f));
}

__global__ void poisson_kernel(const float* __restrict__ mu, int64_t n, uint32_t k0, uint32_t k1,
                               int32_t* __restrict__ counts) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        counts[i] = poisson_one(mu[i], k0, k1, (uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0xffffffffu);
}

struct GenParams {
    const int32_t* hist_nbins;    // [K]
    const int32_t* role_theta;    // [K][kMaxRoles][2]
    const int64_t* group_off;     // [K] offset of histogram k's groups within a sample
    const double* thetas;         // [n_samples][P]
    RunConst rc;
    float dt, t0;
    int K, P, rebin, log1p_out;
    int64_t row_stride;           // floats between consecutive samples in out / mu_out
    uint32_t k0, k1;
    uint64_t sample_offset;
    float* out;                   // [n_samples][row_stride]
    float* mu_out;                // same layout, or null
    const float* etab;            // the run's lifetime factor at every chunk start
};

// One block per (sample, histogram): stage the constants once, then each
// thread sums the theory over its groups of `rebin` bins and draws a count.
template <int NE, int NG, int NS, int KT>
__global__ void __launch_bounds__(kMaxThreads) generate_kernel(const __grid_constant__ GenParams p) {
    constexpr int NPART = stage_parts<NE, NG, NS, KT>();
    __shared__ HistConst hc;
    const int k = blockIdx.x % p.K;
    const int64_t s = blockIdx.x / p.K;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    {
        const double* theta = p.thetas + s * p.P;
        const int32_t* rt = p.role_theta + (size_t)k * kMaxRoles * 2;
        for (int part = warp; part < NPART; part += nwarps)
            stage_part<NE, NG, NS, KT>(part, ThetaByRow{rt, theta}, p.rc, hc, 0, lane);
    }
    __syncthreads();
    const int M = p.hist_nbins[k];
    const int groups = (M + p.rebin - 1) / p.rebin;
    const float zero[kBinsPerThread] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int j = threadIdx.x; j < groups; j += blockDim.x) {
        const int g0 = j * p.rebin, g1 = min(g0 + p.rebin, M);
        float acc[1] = {0.f};
        bool bad = false;
        for (int n0 = g0; n0 < g1; n0 += kBinsPerThread)
            eval_chunk<NE, NG, NS, KT, kSum, 1>(hc, n0, g1, zero, lifetime_from_table(p.etab, n0, hc.qE), MUSR_CHI2,
                                                p.dt, p.t0, acc, bad, nullptr);
        const float mu = acc[0];
        const int32_t cnt = poisson_one(mu, p.k0, p.k1, (uint32_t)j, (uint32_t)k,
                                        (uint32_t)(p.sample_offset + (uint64_t)s));
        const int64_t o = s * p.row_stride + p.group_off[k] + j;
        p.out[o] = p.log1p_out ? log1pf((float)cnt) : (float)cnt;
        if (p.mu_out) p.mu_out[o] = mu;
    }
}

cudaError_t launch_generate(const Signature& s, int blocks, int threads, cudaStream_t st, const GenParams& p) {
#define MUSR_CASE(NE, NG, NS, KT)                                   \
    if (s.ne == NE && s.ng == NG && s.ns == NS && s.kt == KT) {     \
        generate_kernel<NE, NG, NS, KT><<<blocks, threads, 0, st>>>(p); \
        return cudaGetLastError();                                  \
    }
    MUSR_FOR_EACH_SIGNATURE(MUSR_CASE)
#undef MUSR_CASE
    return cudaErrorInvalidValue;
}

// Parameter vectors drawn uniformly from [lo_j, hi_j] for the learned
// entries (learned[q] = j), fixed entries at lo_j; targets[s][q] = 2u - 1.
// u has 53 random bits from two Philox words: counter (sample low, sample
// high, q / 2, 0xfffffffe) under the key (seed low ^ 0x0A5F00D1, seed high).
__global__ void sample_thetas_kernel(const double* __restrict__ lo, const double* __restrict__ hi,
                                     const int32_t* __restrict__ learned, int n_learned, int P, int n,
                                     uint32_t k0, uint32_t k1, uint64_t offset, double* __restrict__ thetas,
                                     float* __restrict__ targets) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    double* th = thetas + (size_t)s * P;
    for (int j = 0; j < P; ++j) th[j] = lo[j];
    const uint64_t id = offset + (uint64_t)s;
    for (int q = 0; q < n_learned; q += 2) {
        uint32_t c[4] = {(uint32_t)id, (uint32_t)(id >> 32), (uint32_t)(q >> 1), 0xfffffffeu};
        philox4x32_10(c, k0 ^ 0x0A5F00D1u, k1);
        for (int h = 0; h < 2 && q + h < n_learned; ++h) {
            const uint32_t wa = c[2 * h], wb = c[2 * h + 1];
            const double u = __dmul_rn(__dadd_rn(__dadd_rn(__dmul_rn((double)(wa >> 5), 67108864.0), (double)(wb >> 6)),
                                                 0.5),
                                       1.1102230246251565e-16);
            const int j = learned[q + h];
            th[j] = __dadd_rn(lo[j], __dmul_rn(__dsub_rn(hi[j], lo[j]), u));
            if (targets) targets[(size_t)s * n_learned + q + h] = (float)__dsub_rn(__dadd_rn(u, u), 1.0);
        }
    }
}

// Rebinned measured histograms: counts summed over groups of `rebin` bins
// (exact in FP32 below 2^24 per group), in the generator's layout.
__global__ void rebin_sum_kernel(const float* __restrict__ data, const int64_t* __restrict__ hist_off,
                                 const int32_t* __restrict__ hist_nbins, const int64_t* __restrict__ group_off,
                                 int rebin, float* __restrict__ out) {
    const int k = blockIdx.y;
    const int M = hist_nbins[k];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int g0 = j * rebin;
    if (g0 >= M) return;
    const int g1 = min(g0 + rebin, M);
    const float* d = data + hist_off[k];
    float sum = 0.f;
    for (int i = g0; i < g1; ++i) sum += d[i];
    out[group_off[k] + j] = sum;
}

}  // namespace

int ensure_groups(musr_run run, int rebin) {
    if (run->d_group_off && run->gen_rebin == rebin) return MUSR_OK;
    std::vector<int64_t> off(run->K);
    int64_t o = 0;
    for (int k = 0; k < run->K; ++k) {
        off[k] = o;
        o += (run->n_bins[k] + rebin - 1) / rebin;
    }
    int st = MUSR_OK;
    if (!run->d_group_off) st = cuda_status(cudaMalloc(&run->d_group_off, sizeof(int64_t) * std::max(run->K, 1)));
    if (st == MUSR_OK)
        st = cuda_status(cudaMemcpy(run->d_group_off, off.data(), sizeof(int64_t) * run->K, cudaMemcpyHostToDevice));
    if (st != MUSR_OK) return st;
    run->gen_rebin = rebin;
    run->gen_per_sample = o;
    return MUSR_OK;
}

int sample_uniform_thetas(const double* lo_dev, const double* hi_dev, const int32_t* learned_dev, int n_learned,
                          int P, int n, uint64_t seed, uint64_t offset, double* thetas_dev, float* targets_dev,
                          cudaStream_t st) {
    if (n <= 0) return MUSR_OK;
    sample_thetas_kernel<<<(n + 127) / 128, 128, 0, st>>>(lo_dev, hi_dev, learned_dev, n_learned, P, n, (uint32_t)seed,
                                                         (uint32_t)(seed >> 32), offset, thetas_dev, targets_dev);
    return cuda_status(cudaGetLastError());
}

int rebin_sum_row(musr_run run, int rebin, float* out_dev, cudaStream_t st) {
    int rc = ensure_groups(run, rebin);
    if (rc != MUSR_OK || run->K == 0) return rc;
    int64_t max_groups = 1;
    for (int k = 0; k < run->K; ++k) max_groups = std::max<int64_t>(max_groups, (run->n_bins[k] + rebin - 1) / rebin);
    dim3 grid((unsigned)((max_groups + 127) / 128), (unsigned)run->K);
    rebin_sum_kernel<<<grid, 128, 0, st>>>(run->d_data, run->d_hist_off, run->d_hist_nbins, run->d_group_off, rebin,
                                          out_dev);
    return cuda_status(cudaGetLastError());
}

}  // namespace musr

using namespace musr;

extern "C" int musr_poisson_sample(const float* mu_dev, int64_t n, uint64_t seed, int32_t* counts_dev,
                                   void* stream) {
    if (n < 0 || (n > 0 && (!mu_dev || !counts_dev))) return MUSR_EINVAL;
    if (n == 0) return MUSR_OK;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256;
    const int blocks = (int)std::min<int64_t>(want, (int64_t)sms * 16);
    poisson_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(mu_dev, n, (uint32_t)seed,
                                                                          (uint32_t)(seed >> 32), counts_dev);
    return cuda_status(cudaGetLastError());
}

int musr::generate_rows(musr_run run, const double* thetas_dev, int n_samples, int rebin, uint64_t seed,
                        uint64_t sample_offset, int log1p_out, float* out_dev, float* mu_dev, int64_t row_stride,
                        cudaStream_t stream) {
    if (!run || n_samples < 0 || rebin < 1) return MUSR_EINVAL;
    if (run->F > 0) return MUSR_ENOTSUP;  // function values are formed per host call
    if (n_samples == 0 || run->K == 0) return MUSR_OK;
    if (!thetas_dev || !out_dev) return MUSR_EINVAL;
    if ((int64_t)n_samples * run->K > (int64_t)0x7fffffff) return MUSR_ENOTSUP;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != run->device) cudaSetDevice(run->device);
    int st = ensure_groups(run, rebin);
    if (st == MUSR_OK) {
        GenParams p;
        memset(&p, 0, sizeof(p));
        p.hist_nbins = run->d_hist_nbins;
        p.role_theta = run->d_role_theta;
        p.group_off = run->d_group_off;
        p.thetas = thetas_dev;
        p.rc = run->rc;
        p.etab = run->d_etab;
        p.dt = (float)run->dt;
        p.t0 = (float)run->t0;
        p.K = run->K;
        p.P = run->P;
        p.rebin = rebin;
        p.row_stride = row_stride > 0 ? row_stride : run->gen_per_sample;
        p.log1p_out = log1p_out;
        p.k0 = (uint32_t)seed;
        p.k1 = (uint32_t)(seed >> 32);
        p.sample_offset = sample_offset;
        p.out = out_dev;
        p.mu_out = mu_dev;
        int64_t max_groups = 1;
        for (int k = 0; k < run->K; ++k) max_groups = std::max<int64_t>(max_groups, (run->n_bins[k] + rebin - 1) / rebin);
        const int threads = (int)std::min<int64_t>(kMaxThreads, std::max<int64_t>(64, (max_groups + 31) / 32 * 32));
        if (row_stride > 0 && row_stride < run->gen_per_sample) st = MUSR_EINVAL;
        cudaStream_t s = stream ? stream : run->stream;
        if (st == MUSR_OK) st = cuda_status(launch_generate(run->sig, n_samples * run->K, threads, s, p));
    }
    if (cur != run->device) cudaSetDevice(cur);
    return st;
}

extern "C" int musr_generate(musr_run run, const double* thetas_dev, int32_t n_samples, int32_t rebin,
                             uint64_t seed, uint64_t sample_offset, int32_t log1p_out, float* out_dev,
                             float* mu_dev, void* stream) {
    return musr::generate_rows(run, thetas_dev, n_samples, rebin, seed, sample_offset, log1p_out, out_dev, mu_dev,
                               0, static_cast<cudaStream_t>(stream));
}
