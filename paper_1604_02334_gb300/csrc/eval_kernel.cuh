// Fused objective / adjoint kernel for the muSR fit (sm_103a).
//
// One launch evaluates, for every bin of every histogram, the Eq. 1 theory
// (Sec. 4.1), the Eq. 3 chi2 or Eq. 4 deviance term, and (by mode) the
// per-bin partial derivatives of N with respect to each parameter ROLE of the
// histogram (N0, bkg, and amplitude / rate / frequency / phase of each line,
// amplitude / width of the Kubo-Toyabe term), accumulated into the gradient
// and the Gauss-Newton matrix.  The sums are finished inside the same launch
// and mapped to theta through the map array (Sec. 4.2.1) in a fixed order, so
// the result is bitwise repeatable.
//
// The paper's kernel (Sec. 4.2.2) uses one thread per bin, FP64, a temporary
// per-bin array and a cuBLAS sum per data set.  GB300 has a strong FP32 / SFU
// datapath and a very narrow FP64 one (an FP64 warp instruction occupies the
// pipe for tens of cycles), so here instead:
//   * each thread owns 8 consecutive bins, loaded as two 128-bit loads;
//   * exponential envelopes and the precession rotations are stepped from bin
//     to bin by exact recurrences (delta form x += x * q), re-seeded every 8
//     bins from exact per-chunk values, so the SFU does one exp2 / sincos per
//     chunk instead of per bin; Gaussian envelopes use one SFU exp2 per bin;
//   * the precession phase at each chunk start is computed in 64-bit fixed
//     point turns, so it is exact at any t (no FP32 phase drift at wt ~ 600);
//   * the deviance uses N h(r), h(r) = (1+r) ln(1+r) - r, r = (d - N)/N, with
//     a short series for small |r| so that FP32 keeps full relative accuracy;
//   * per-histogram constants (the only FP64-heavy arithmetic) are staged once
//     per call -- on the host for host calls, by a small stage kernel chained
//     with programmatic dependent launch for device calls -- not per block;
//   * sums beyond the warp use FP32 double-float pairs (TwoSum, ~44-bit
//     significand) instead of FP64: warps -> block -> 8-block cluster (read
//     through distributed shared memory) -> last cluster leader, which forms
//     the per-histogram sums and the theta-space outputs, converting each
//     output to FP64 once.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "musr_internal.h"

namespace musr {

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

__host__ __device__ __forceinline__ void split_hi_lo(double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// x mod 1 as 64-bit fixed-point turns.
__host__ __device__ __forceinline__ unsigned long long turns_to_fixed(double x) {
    double y = x - floor(x);
    if (!(y >= 0.0) || y >= 1.0) y = 0.0;
    double s = y * 4294967296.0;  // exact scaling by 2^32
    double hi = floor(s);
    double lo = floor((s - hi) * 4294967296.0);
    return ((unsigned long long)hi << 32) | (unsigned long long)lo;
}

// Sum of the (up to two) theta entries a role reads.
__host__ __device__ __forceinline__ double role_value(const int32_t* rt, const double* theta, int r) {
    int i0 = rt[2 * r], i1 = rt[2 * r + 1];
    double v = 0.0;
    if (i0 >= 0) v += theta[i0];
    if (i1 >= 0) v += theta[i1];
    return v;
}

// Per-histogram constants in NPART independent parts (so that different
// threads can compute them concurrently):
//   part 0        N0 (hi/lo), bkg, lifetime recurrence, 2 pi gamma
//   part 1 + 2c   envelope of precession line c
//   part 2 + 2c   phase of precession line c (64-bit fixed-point turns)
//   part 1 + 2 NOSC  static Gaussian Kubo-Toyabe term
// Every argument is formed in FP64.  PRECISE (host) evaluates the few
// transcendental step factors in FP64 too; the device variant uses FP32
// accurate functions of the FP64 arguments (FP64 functions are slow there).
struct TimeGrid {
    double t0, dt, inv_tau, gamma;
};

template <int NE, int NG, int KT>
__host__ __device__ constexpr int stage_parts() {
    return 2 + 2 * (NE + NG);
}

template <bool PRECISE>
__host__ __device__ __forceinline__ float st_expm1(double x) {
#ifdef __CUDA_ARCH__
    if (!PRECISE) return expm1f((float)x);
#endif
    return (float)expm1(x);
}
template <bool PRECISE>
__host__ __device__ __forceinline__ float st_exp(double x) {
#ifdef __CUDA_ARCH__
    if (!PRECISE) return expf((float)x);
#endif
    return (float)exp(x);
}
// sin(pi x) for x in [-1, 1]
template <bool PRECISE>
__host__ __device__ __forceinline__ float st_sinpi(double x) {
#ifdef __CUDA_ARCH__
    if (!PRECISE) return sinpif((float)x);
#endif
    return (float)sin(3.14159265358979323846 * x);
}

template <int NE, int NG, int KT, bool PRECISE>
__host__ __device__ void stage_hist(int part, const int32_t* rt, const double* theta, const TimeGrid& tg,
                                    HistConst& hc) {
    constexpr int NOSC = NE + NG;
    const double LOG2E = 1.4426950408889634074;
    const double dt = tg.dt, t0 = tg.t0, it = tg.inv_tau;
    if (part == 0) {
        split_hi_lo(role_value(rt, theta, 0), hc.n0, hc.n0_lo);
        hc.bkg = (float)role_value(rt, theta, 1);
        split_hi_lo(dt * it * LOG2E, hc.aE_hi, hc.aE_lo);
        hc.qE = st_expm1<PRECISE>(-dt * it);
        hc.cE = st_exp<PRECISE>(-t0 * it);
        hc.kfreq = (float)(2.0 * 3.14159265358979323846 * tg.gamma);
    } else if (part <= 2 * NOSC) {
        const int c = (part - 1) >> 1;
        const int r = 2 + 4 * c;
        OscConst& o = hc.osc[c];
        if (part & 1) {  // envelope
            const double amp = role_value(rt, theta, r);
            const double rate = role_value(rt, theta, r + 1);
            o.amp = (float)amp;
            o.rate = (float)rate;
            if (c < NE) {  // exp(-(1/tau + lambda) t)
                const double rt_ = it + rate;
                split_hi_lo(rt_ * dt * LOG2E, o.a_hi, o.a_lo);
                o.b_hi = o.b_lo = 0.f;
                o.q = st_expm1<PRECISE>(-rt_ * dt);
                o.cenv = st_exp<PRECISE>(-rt_ * t0);
            } else {  // exp(-t/tau - sigma^2 t^2 / 2), t = t0 + n dt
                const double s2 = rate * rate;
                split_hi_lo((it + s2 * t0) * dt * LOG2E, o.a_hi, o.a_lo);
                split_hi_lo(0.5 * s2 * dt * dt * LOG2E, o.b_hi, o.b_lo);
                o.q = 0.f;
                o.cenv = st_exp<PRECISE>(-t0 * it - 0.5 * s2 * t0 * t0);
            }
        } else {  // phase
            const double field = role_value(rt, theta, r + 2);
            const double phi = role_value(rt, theta, r + 3);
            const double f = tg.gamma * field;  // turns per microsecond
            o.ph0 = turns_to_fixed(f * t0 + phi * 0.15915494309189533577);
            const double stp = f * dt;  // turns per bin
            o.step = turns_to_fixed(stp);
            const double red = stp - rint(stp);  // in [-0.5, 0.5]
            const float sh = st_sinpi<PRECISE>(red);
            o.cm1 = -2.f * sh * sh;                  // cos(step) - 1
            o.sn = st_sinpi<PRECISE>(2.0 * red);     // sin(step)
        }
    } else if (KT && part == 2 * NOSC + 1) {
        const int r = 2 + 4 * NOSC;
        const double amp = role_value(rt, theta, r);
        const double dl = role_value(rt, theta, r + 1);
        const double s2 = dl * dl;
        hc.kt_amp = (float)amp;
        hc.kt_rate = (float)dl;
        split_hi_lo((it + s2 * t0) * dt * LOG2E, hc.kt_a_hi, hc.kt_a_lo);
        split_hi_lo(0.5 * s2 * dt * dt * LOG2E, hc.kt_b_hi, hc.kt_b_lo);
        hc.kt_cenv = st_exp<PRECISE>(-t0 * it - 0.5 * s2 * t0 * t0);
    }
}

// Double-float (hi + lo) accumulation on the FP32 pipe: TwoSum of the high
// parts, low parts added into the error, renormalised (Knuth / Dekker).
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float v = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, e);
    return DF{h, __fsub_rn(e, __fsub_rn(h, s))};
}

// Block-wide copy of n elements from global (L2) to shared memory with eight
// loads in flight per thread: a plain loop would wait one L2 round trip per
// element before issuing the next load.
template <class T>
__device__ __forceinline__ void copy_to_smem(T* dst, const T* src, int n) {
    for (int base = threadIdx.x; base < n; base += 8 * blockDim.x) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = base + u * blockDim.x;
            if (i < n) v[u] = __ldcg(src + i);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = base + u * blockDim.x;
            if (i < n) dst[i] = v[u];
        }
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


// Device-path staging: one block per histogram; part q of its constants is
// computed by lane 0 of warp q.  It lets the dependent objective kernel
// launch at once (programmatic dependent launch); that kernel waits for the
// staged constants before it reads them.
template <int NE, int NG, int KT>
__global__ void stage_kernel(const double* theta, const int32_t* role_theta, TimeGrid tg, HistConst* out) {
    asm volatile("griddepcontrol.launch_dependents;");
    constexpr int NPART = stage_parts<NE, NG, KT>();
    const int k = blockIdx.x;
    const int part = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0 && part < NPART)
        stage_hist<NE, NG, KT, false>(part, role_theta + (size_t)k * kMaxRoles * 2, theta, tg, out[k]);
}

template <int NE, int NG, int KT, int MODE>
__global__ void __launch_bounds__(kMaxThreads) eval_kernel(const __grid_constant__ EvalParams p) {
    namespace cg = cooperative_groups;
    constexpr int NOSC = NE + NG;
    constexpr int R = 2 + 4 * NOSC + 2 * KT;
    constexpr int NACC = MODE == kValue ? 1 : MODE == kGrad ? 1 + R : MODE == kGN ? 1 + R + R * (R + 1) / 2 : 1;
    constexpr int G = kBinsPerThread;

    __shared__ HistConst hc;
    __shared__ float red[kMaxWarps][NACC];
    __shared__ DF bpart[NACC];  // this block's sums; the cluster leader reads them
    __shared__ int s_last;
    extern __shared__ __align__(16) unsigned char dyn_smem[];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
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

    // histogram k's constants: inline in the launch parameters (host calls) or
    // written by the preceding stage kernel (device calls)
    {
        const unsigned* src;
        if (p.hconst_inline_n > 0) {
            src = reinterpret_cast<const unsigned*>(&p.hconst_inline[k]);
        } else {
            asm volatile("griddepcontrol.wait;" ::: "memory");
            src = reinterpret_cast<const unsigned*>(p.hconst + k);
        }
        unsigned* dst = reinterpret_cast<unsigned*>(&hc);
        for (int i = threadIdx.x; i < (int)(sizeof(HistConst) / 4); i += blockDim.x)
            dst[i] = p.hconst_inline_n > 0 ? src[i] : __ldcg(src + i);
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

    // ---- block: FP32 warp sums, double-float across warps ----
    warp_sum<NACC>(acc);
    if (lane == 0) {
#pragma unroll
        for (int a = 0; a < NACC; ++a) red[warp][a] = acc[a];
    }
    const int any_bad = __syncthreads_or(bad);
    for (int a = threadIdx.x; a < NACC; a += blockDim.x) {
        DF v{red[0][a], 0.f};
        for (int w = 1; w < nwarps; ++w) v = df_add(v, DF{red[w][a], 0.f});
        bpart[a] = v;
    }
    if (threadIdx.x == 0 && any_bad) atomicOr(p.flags, 1u);

    // ---- cluster: the leader sums its blocks through distributed shared memory ----
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    const unsigned rank = cl.block_rank(), csize = cl.num_blocks();
    DF* partial = reinterpret_cast<DF*>(p.partial);
    if (rank == 0) {
        const int cidx = blockIdx.x / (int)csize;
        for (int a = threadIdx.x; a < NACC; a += blockDim.x) {
            DF rv[8];  // all remote reads in flight before the (ordered) adds
#pragma unroll
            for (unsigned r = 0; r < 8; ++r) rv[r] = r < csize ? cl.map_shared_rank(bpart, r)[a] : DF{0.f, 0.f};
            DF v = rv[0];
#pragma unroll
            for (unsigned r = 1; r < 8; ++r)
                if (r < csize) v = df_add(v, rv[r]);
            partial[(size_t)cidx * NACC + a] = v;
        }
    }
    cl.sync();  // keep every block's shared memory alive until the leader has read it
    if (rank != 0) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(p.global_count, 1u);
        s_last = (prev == (unsigned)p.n_clusters - 1u);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // ---- last cluster leader: histogram sums (fixed order), then theta via the map ----
    const int W = p.win_doubles;  // window of cluster partials, a multiple of NACC
    DF* win = reinterpret_cast<DF*>(dyn_smem);
    DF* hsum = p.hsum_in_smem ? win + W : reinterpret_cast<DF*>(p.hist_sum);
    for (int i = threadIdx.x; i < p.K * NACC; i += blockDim.x) hsum[i] = DF{0.f, 0.f};
    const int total = p.n_clusters * NACC;
    for (int i0 = 0; i0 < total; i0 += W) {
        const int n = min(W, total - i0);
        __syncthreads();
        copy_to_smem(reinterpret_cast<float2*>(win), reinterpret_cast<const float2*>(partial + i0), n);
        __syncthreads();
        const int c0 = i0 / NACC, c1 = c0 + n / NACC;
        const int k0 = p.cluster_hist[c0], k1 = p.cluster_hist[c1 - 1];
        for (int q = threadIdx.x; q < (k1 - k0 + 1) * NACC; q += blockDim.x) {
            const int kk = k0 + q / NACC, a = q % NACC;
            const int first = p.hist_first_cluster[kk];
            const int lo = max(first, c0), hi = min(first + p.hist_nclusters[kk], c1);
            DF s = hsum[kk * NACC + a];
            for (int c = lo; c < hi; ++c) s = df_add(s, win[(c - c0) * NACC + a]);
            hsum[kk * NACC + a] = s;
        }
    }
    __syncthreads();
    const int32_t* cptr = p.csr_ptr;
    const int32_t* csrc = p.csr_src;
    if (p.csr_in_smem) {
        int32_t* sp = reinterpret_cast<int32_t*>(win + W + (p.hsum_in_smem ? p.K * NACC : 0));
        copy_to_smem(sp, p.csr_ptr, p.n_out + 1);
        copy_to_smem(sp + p.n_out + 1, p.csr_src, p.n_src);
        __syncthreads();
        cptr = sp;
        csrc = sp + p.n_out + 1;
    }
    for (int o = threadIdx.x; o < p.n_out; o += blockDim.x) {
        DF s{0.f, 0.f};
        const int e = cptr[o + 1];
        for (int j = cptr[o]; j < e; ++j) s = df_add(s, hsum[csrc[j]]);
        p.out[o] = (double)s.hi + (double)s.lo;  // exact: |lo| <= ulp(hi) / 2
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *p.global_count = 0u;
        unsigned f = atomicExch(p.flags, 0u);
        if (!isfinite(p.out[0])) f |= 2u;
        if (p.status_out) *p.status_out = (int32_t)f;
    }
}

// Launch the objective kernel in clusters of p.cluster blocks.  With the
// constants not inline (device calls) the stage kernel runs first and the
// objective kernel follows as its programmatic dependent.  n_tiles == 0 only
// sets the kernel's shared-memory attribute (call it outside stream capture).
template <int NE, int NG, int KT, int MODE>
cudaError_t launch_one(int threads, int n_tiles, cudaStream_t stream, const EvalParams& p) {
    const size_t smem = (size_t)p.smem_bytes;
    if (n_tiles == 0) {
        // the attribute is per kernel, shared by every run: only ever raise it
        // (to the device's opt-in maximum), never lower it below another run's need
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, eval_kernel<NE, NG, KT, MODE>);
        if (e != cudaSuccess) return e;
        const int avail = optin - (int)fa.sharedSizeBytes;
        if ((int)smem > avail) return cudaErrorInvalidValue;
        if (fa.maxDynamicSharedSizeBytes >= avail) return cudaSuccess;
        return cudaFuncSetAttribute(eval_kernel<NE, NG, KT, MODE>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, avail);
    }
    const bool staged = p.hconst_inline_n == 0 && !p.hconst_ready;
    if (staged) {
        const TimeGrid tg{p.t0, p.dt, p.inv_tau, p.gamma};
        stage_kernel<NE, NG, KT><<<p.K, 32 * stage_parts<NE, NG, KT>(), 0, stream>>>(
            p.theta, p.role_theta, tg, p.hconst);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_tiles);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = p.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = staged ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, eval_kernel<NE, NG, KT, MODE>, p);
}

}  // namespace musr
