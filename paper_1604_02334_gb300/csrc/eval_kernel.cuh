// Fused objective / adjoint kernel for the muSR fit (sm_103a).
//
// One launch evaluates, for every bin of every histogram, the Eq. 1 theory
// (Sec. 4.1), the Eq. 3 chi2 or Eq. 4 deviance term, and (by mode) the
// per-bin partial derivatives of N with respect to each parameter ROLE of the
// histogram (N0, bkg, and amplitude / rate / frequency / phase of each line,
// amplitude / width of the Kubo-Toyabe term), accumulated into the gradient
// and the Gauss-Newton matrix.  Everything is reduced to FP64 inside the same
// launch and mapped to theta through the map array (Sec. 4.2.1), in a fixed
// order, so the result is bitwise repeatable.
//
// The paper's kernel (Sec. 4.2.2) uses one thread per bin, FP64, a temporary
// per-bin array and a cuBLAS sum per data set.  Here instead:
//   * each thread owns 8 consecutive bins, loaded as two 128-bit loads;
//   * exponential envelopes and the precession rotations are stepped from bin
//     to bin by exact recurrences (delta form x += x * q), re-seeded every 8
//     bins from exact per-chunk values, so the SFU does one exp2 / sincos per
//     chunk instead of per bin; Gaussian envelopes use one SFU exp2 per bin;
//   * the precession phase at each chunk start is computed in 64-bit fixed
//     point turns, so it is exact at any t (no FP32 phase drift at wt ~ 600);
//   * the deviance uses N h(r), h(r) = (1+r) ln(1+r) - r, r = (d - N)/N, with
//     a short series for small |r| so that FP32 keeps full relative accuracy;
//   * warp shuffles reduce FP32 partials, FP64 sums combine warps, tiles,
//     histograms; the last block of each histogram and then the last block
//     overall finish the sums (no second launch, no atomics on values).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "musr_internal.h"

namespace musr {

// Per-histogram constants staged into shared memory (Sec. 4.2.2 keeps the
// parameter / map values in shared memory for the same reason: every thread
// reads them many times).
struct OscConst {
    float amp, rate, cenv, a_hi, a_lo, b_hi, b_lo, q, cm1, sn;
    unsigned long long ph0, step;
};

struct HistConst {
    float n0, n0_lo, bkg, cE, aE_hi, aE_lo, qE;  // N0 = n0 + n0_lo (FP32 pair)
    float kfreq;  // 2 pi gamma: dN/dB = dN/d(omega) * 2 pi gamma
    OscConst osc[kMaxOsc];
    float kt_amp, kt_rate, kt_cenv, kt_a_hi, kt_a_lo, kt_b_hi, kt_b_lo;
};

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void split_hi_lo(double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// y in [0, 1) to 64-bit fixed-point turns.
__device__ __forceinline__ unsigned long long turns_to_fixed(double x) {
    double y = x - floor(x);
    if (!(y >= 0.0) || y >= 1.0) y = 0.0;
    double s = y * 4294967296.0;  // exact scaling by 2^32
    double hi = floor(s);
    double lo = floor((s - hi) * 4294967296.0);
    return ((unsigned long long)hi << 32) | (unsigned long long)lo;
}

// Sum of the (up to two) theta entries a role reads.
__device__ __forceinline__ double role_value(const int32_t* rt, const double* theta, int r) {
    int i0 = rt[2 * r], i1 = rt[2 * r + 1];
    double v = 0.0;
    if (i0 >= 0) v += theta[i0];
    if (i1 >= 0) v += theta[i1];
    return v;
}

// Stage part `part` of histogram k's constants (part 0: N0, bkg, lifetime;
// 1..NOSC: precession lines; NOSC+1: Kubo-Toyabe).  FP64 for every argument,
// FP32 accurate functions for the small step factors.
struct TimeGrid {
    double t0, dt, inv_tau, gamma;
};

template <int NE, int NG, int KT>
__device__ void stage_hist(int part, const int32_t* rt, const double* theta, const TimeGrid& tg,
                           HistConst& hc) {
    constexpr int NOSC = NE + NG;
    const double LOG2E = 1.4426950408889634074;
    const double dt = tg.dt, t0 = tg.t0, it = tg.inv_tau;
    if (part == 0) {
        split_hi_lo(role_value(rt, theta, 0), hc.n0, hc.n0_lo);
        hc.bkg = (float)role_value(rt, theta, 1);
        split_hi_lo(dt * it * LOG2E, hc.aE_hi, hc.aE_lo);
        hc.qE = expm1f((float)(-dt * it));
        hc.cE = expf((float)(-t0 * it));
        hc.kfreq = (float)(2.0 * 3.14159265358979323846 * tg.gamma);
    } else if (part <= NOSC) {
        const int c = part - 1;
        const int r = 2 + 4 * c;
        const double amp = role_value(rt, theta, r);
        const double rate = role_value(rt, theta, r + 1);
        const double field = role_value(rt, theta, r + 2);
        const double phi = role_value(rt, theta, r + 3);
        OscConst& o = hc.osc[c];
        o.amp = (float)amp;
        o.rate = (float)rate;
        if (c < NE) {  // exp(-(1/tau + lambda) t)
            const double rt_ = it + rate;
            split_hi_lo(rt_ * dt * LOG2E, o.a_hi, o.a_lo);
            o.b_hi = o.b_lo = 0.f;
            o.q = expm1f((float)(-rt_ * dt));
            o.cenv = expf((float)(-rt_ * t0));
        } else {       // exp(-t/tau - sigma^2 t^2 / 2), t = t0 + n dt
            const double s2 = rate * rate;
            split_hi_lo((it + s2 * t0) * dt * LOG2E, o.a_hi, o.a_lo);
            split_hi_lo(0.5 * s2 * dt * dt * LOG2E, o.b_hi, o.b_lo);
            o.q = 0.f;
            o.cenv = expf((float)(-t0 * it - 0.5 * s2 * t0 * t0));
        }
        const double f = tg.gamma * field;  // turns per microsecond
        o.ph0 = turns_to_fixed(f * t0 + phi * 0.15915494309189533577);
        const double stp = f * dt;          // turns per bin
        o.step = turns_to_fixed(stp);
        const float red = (float)(stp - rint(stp));  // in [-0.5, 0.5]
        const float sh = sinpif(red);
        o.cm1 = -2.f * sh * sh;               // cos(step) - 1
        o.sn = sinpif(2.f * red);             // sin(step)
    } else if (KT && part == NOSC + 1) {
        const int r = 2 + 4 * NOSC;
        const double amp = role_value(rt, theta, r);
        const double dl = role_value(rt, theta, r + 1);
        const double s2 = dl * dl;
        hc.kt_amp = (float)amp;
        hc.kt_rate = (float)dl;
        split_hi_lo((it + s2 * t0) * dt * LOG2E, hc.kt_a_hi, hc.kt_a_lo);
        split_hi_lo(0.5 * s2 * dt * dt * LOG2E, hc.kt_b_hi, hc.kt_b_lo);
        hc.kt_cenv = expf((float)(-t0 * it - 0.5 * s2 * t0 * t0));
    }
}

template <int NACC>
__device__ __forceinline__ void warp_sum(float (&v)[NACC]) {
#pragma unroll
    for (int a = 0; a < NACC; ++a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[a] += __shfl_xor_sync(0xffffffffu, v[a], o);
    }
}

// One thread's chunk of kBinsPerThread consecutive bins starting at bin n0 of a
// histogram with M bins: theory (Eq. 1), objective term (Eq. 3 / Eq. 4) and,
// by mode, the role partials accumulated into the gradient and GN matrix.
template <int NE, int NG, int KT, int MODE, int NACC>
__device__ __forceinline__ void eval_chunk(const HistConst& hc, int n0, int M,
                                           const float (&d)[kBinsPerThread], int obj, float dtf,
                                           float t0f, float (&acc)[NACC], bool& bad,
                                           float* model_dst) {
    constexpr int NOSC = NE + NG;
    constexpr int R = 2 + 4 * NOSC + 2 * KT;
    constexpr int G = kBinsPerThread;
    const float nf0 = (float)n0;
    const float n0p = hc.n0, n0lo = hc.n0_lo, bkg = hc.bkg;
    float E = hc.cE * ex2_approx(-fmaf(nf0, hc.aE_hi, nf0 * hc.aE_lo));
    float env[NOSC > 0 ? NOSC : 1], cs[NOSC > 0 ? NOSC : 1], sn[NOSC > 0 ? NOSC : 1];
#pragma unroll
    for (int c = 0; c < NOSC; ++c) {
        const OscConst& o = hc.osc[c];
        if (c < NE) env[c] = o.cenv * ex2_approx(-fmaf(nf0, o.a_hi, nf0 * o.a_lo));
        const unsigned long long ph = o.ph0 + (unsigned long long)n0 * o.step;
        const float x = (float)(int)(ph >> 32) * 2.3283064365386963e-10f;  // turns in [-1/2, 1/2)
        __sincosf(6.28318530717958647692f * x, &sn[c], &cs[c]);
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const float nf = nf0 + (float)g;
        const float t = fmaf(nf, dtf, t0f);
        const float nn = nf * nf;
        float S = E;
#pragma unroll
        for (int c = 0; c < NOSC; ++c) {
            const OscConst& o = hc.osc[c];
            if (c >= NE)
                env[c] = o.cenv * ex2_approx(-fmaf(nn, o.b_hi, fmaf(nf, o.a_hi, fmaf(nn, o.b_lo, nf * o.a_lo))));
            S = fmaf(o.amp * env[c], cs[c], S);
        }
        float envk = 0.f, xk = 0.f, GE = 0.f;
        if (KT) {
            envk = hc.kt_cenv *
                   ex2_approx(-fmaf(nn, hc.kt_b_hi, fmaf(nf, hc.kt_a_hi, fmaf(nn, hc.kt_b_lo, nf * hc.kt_a_lo))));
            const float dtk = hc.kt_rate * t;
            xk = dtk * dtk;
            GE = fmaf(0.666666667f * (1.f - xk), envk, 0.333333333f * E);
            S = fmaf(hc.kt_amp, GE, S);
        }
        // N0 carried as an FP32 pair so its rounding does not bias every bin
        const float N = fmaf(n0p, S, fmaf(n0lo, S, bkg));

        if (MODE == kModel) {
            if (n0 + g < M) model_dst[n0 + g] = N;
        } else if (n0 + g < M) {
            const float dv = d[g];
            float term, wg, wh;
            if (obj == MUSR_CHI2) {
                const float w = rcp_approx(fmaxf(dv, 1.f));
                const float r = dv - N;
                term = r * r * w;
                wg = -2.f * r * w;
                wh = 2.f * w;
            } else {
                if (dv > 0.f) {
                    if (!(N > 0.f)) {
                        bad = true;
                        term = wg = wh = 0.f;
                    } else {
                        const float rN = rcp_approx(N);
                        const float rho = (dv - N) * rN;
                        float h;
                        if (fabsf(rho) < 0.125f) {
                            // sum_{j>=2} (-1)^j rho^j / (j (j-1)), truncated after j = 9
                            h = fmaf(rho, -1.f / 72.f, 1.f / 56.f);
                            h = fmaf(rho, h, -1.f / 42.f);
                            h = fmaf(rho, h, 1.f / 30.f);
                            h = fmaf(rho, h, -1.f / 20.f);
                            h = fmaf(rho, h, 1.f / 12.f);
                            h = fmaf(rho, h, -1.f / 6.f);
                            h = fmaf(rho, h, 0.5f);
                            h = h * rho * rho;
                        } else {
                            const float u = log1pf(rho);
                            h = fmaf(rho, u, u - rho);
                        }
                        term = 2.f * N * h;
                        wg = -2.f * rho;
                        wh = 2.f * rN;
                    }
                } else {
                    if (!(N >= 0.f)) bad = true;
                    term = 2.f * N;
                    wg = 2.f;
                    wh = N > 0.f ? 2.f * rcp_approx(N) : 0.f;
                }
            }
            acc[0] += term;
            if (MODE >= kGrad) {
                float pr[R];
                pr[0] = S;
                pr[1] = 1.f;
#pragma unroll
                for (int c = 0; c < NOSC; ++c) {
                    const OscConst& o = hc.osc[c];
                    const float m = n0p * env[c];
                    const float pa = m * cs[c];
                    const float q = o.amp * pa;
                    pr[2 + 4 * c] = pa;
                    pr[2 + 4 * c + 1] = (c < NE) ? -t * q : -o.rate * t * t * q;
                    const float ps = -o.amp * m * sn[c];
                    pr[2 + 4 * c + 2] = ps * t * hc.kfreq;
                    pr[2 + 4 * c + 3] = ps;
                }
                if (KT) {
                    pr[2 + 4 * NOSC] = n0p * GE;
                    pr[2 + 4 * NOSC + 1] =
                        n0p * hc.kt_amp * 0.666666667f * hc.kt_rate * t * t * (xk - 3.f) * envk;
                }
#pragma unroll
                for (int r = 0; r < R; ++r) acc[1 + r] = fmaf(wg, pr[r], acc[1 + r]);
                if (MODE == kGN) {
                    int a = 1 + R;
#pragma unroll
                    for (int r1 = 0; r1 < R; ++r1) {
                        const float qv = wh * pr[r1];
#pragma unroll
                        for (int r2 = r1; r2 < R; ++r2) {
                            acc[a] = fmaf(qv, pr[r2], acc[a]);
                            ++a;
                        }
                    }
                }
            }
        }
        // step the recurrences to the next bin
        E = fmaf(E, hc.qE, E);
#pragma unroll
        for (int c = 0; c < NOSC; ++c) {
            const OscConst& o = hc.osc[c];
            if (c < NE) env[c] = fmaf(env[c], o.q, env[c]);
            const float c2 = fmaf(cs[c], o.cm1, fmaf(-sn[c], o.sn, cs[c]));
            const float s2 = fmaf(sn[c], o.cm1, fmaf(cs[c], o.sn, sn[c]));
            cs[c] = c2;
            sn[c] = s2;
        }
    }
}

template <int NE, int NG, int KT, int MODE>
__global__ void __launch_bounds__(kMaxThreads) eval_kernel(const EvalParams p) {
    constexpr int NOSC = NE + NG;
    constexpr int R = 2 + 4 * NOSC + 2 * KT;
    constexpr int NACC = MODE == kValue ? 1 : MODE == kGrad ? 1 + R : MODE == kGN ? 1 + R + R * (R + 1) / 2 : 1;
    constexpr int G = kBinsPerThread;

    __shared__ HistConst hc;
    __shared__ float red[kMaxWarps][NACC];
    __shared__ int s_last;

    const int tile = blockIdx.x;
    const int k = p.tile_hist[tile];
    const int M = p.hist_nbins[k];
    const int n0 = p.tile_start[tile] + (int)threadIdx.x * G;
    const bool active = n0 < M;

    // issue the histogram loads first so their latency overlaps the staging
    float d[G];
    if (MODE != kModel && active) {
        const float4* src = reinterpret_cast<const float4*>(p.data + p.hist_off[k] + n0);
        float4 a = __ldg(src), b = __ldg(src + 1);
        d[0] = a.x; d[1] = a.y; d[2] = a.z; d[3] = a.w;
        d[4] = b.x; d[5] = b.y; d[6] = b.z; d[7] = b.w;
    } else {
#pragma unroll
        for (int g = 0; g < G; ++g) d[g] = 0.f;
    }

    if (threadIdx.x < 2 + NOSC) {
        const TimeGrid tg{p.t0, p.dt, p.inv_tau, p.gamma};
        stage_hist<NE, NG, KT>(threadIdx.x, p.role_theta + (size_t)k * kMaxRoles * 2, p.theta, tg, hc);
    }
    __syncthreads();

    float acc[NACC];
#pragma unroll
    for (int a = 0; a < NACC; ++a) acc[a] = 0.f;
    bool bad = false;

    if (active)
        eval_chunk<NE, NG, KT, MODE, NACC>(hc, n0, M, d, p.obj, (float)p.dt, (float)p.t0, acc, bad,
                                           MODE == kModel ? p.model_out + p.model_off[k] : nullptr);
    if (MODE == kModel) return;

    // ---- block reduction: FP32 within the warp, FP64 across warps ----
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    warp_sum<NACC>(acc);
    if (lane == 0) {
#pragma unroll
        for (int a = 0; a < NACC; ++a) red[warp][a] = acc[a];
    }
    const int any_bad = __syncthreads_or(bad);
    for (int a = threadIdx.x; a < NACC; a += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += (double)red[w][a];
        p.partial[(size_t)tile * NACC + a] = s;
    }
    if (threadIdx.x == 0 && any_bad) atomicOr(p.flags, 1u);
    __threadfence();  // every writer publishes its partials before the ticket
    __syncthreads();

    // ---- last tile of this histogram sums the histogram ----
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(&p.hist_count[k], 1u);
        s_last = (prev == (unsigned)p.hist_ntiles[k] - 1u);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    {
        const int ft = p.hist_first_tile[k], nt = p.hist_ntiles[k];
        for (int a = threadIdx.x; a < NACC; a += blockDim.x) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int j = 0;
            for (; j + 4 <= nt; j += 4) {
                const double* q = p.partial + (size_t)(ft + j) * NACC + a;
                s0 += __ldcg(q);
                s1 += __ldcg(q + NACC);
                s2 += __ldcg(q + 2 * NACC);
                s3 += __ldcg(q + 3 * NACC);
            }
            for (; j < nt; ++j) s0 += __ldcg(p.partial + (size_t)(ft + j) * NACC + a);
            p.hist_sum[(size_t)k * NACC + a] = (s0 + s1) + (s2 + s3);
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        p.hist_count[k] = 0u;
        const unsigned prev = atomicAdd(p.global_count, 1u);
        s_last = (prev == (unsigned)p.K - 1u);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // ---- last histogram maps roles to theta (fixed-order CSR sums) ----
    for (int o = threadIdx.x; o < p.n_out; o += blockDim.x) {
        double s = 0.0;
        const int e = p.csr_ptr[o + 1];
        for (int j = p.csr_ptr[o]; j < e; ++j) s += __ldcg(p.hist_sum + p.csr_src[j]);
        p.out[o] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *p.global_count = 0u;
        unsigned f = atomicExch(p.flags, 0u);
        if (!isfinite(p.out[0])) f |= 2u;
        if (p.status_out) *p.status_out = (int32_t)f;
    }
}

template <int NE, int NG, int KT, int MODE>
cudaError_t launch_one(int threads, int n_tiles, cudaStream_t stream, const EvalParams& p) {
    eval_kernel<NE, NG, KT, MODE><<<n_tiles, threads, 0, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace musr
