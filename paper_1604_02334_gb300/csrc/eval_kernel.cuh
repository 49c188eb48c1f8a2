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
//   * envelopes and precession rotations are stepped from bin to bin by
//     recurrences re-seeded every 8 bins from exact per-chunk values: each
//     line is carried as the scaled rotation (env cos, env sin), advanced by a
//     constant 2 x 2 step (exponential envelope) or by the rotation and the
//     envelope ratio 1 + gq with gq' = gq Q + (Q - 1) (Gaussian envelope), so
//     the SFU does one exp2 / sincos per line per chunk, not per bin;
//   * the adjoint accumulates w x_role with x_role cheap per bin and applies
//     the per-histogram factor of each role once, after the reduction;
//   * the precession phase at each chunk start is computed in 64-bit fixed
//     point turns, so it is exact at any t (no FP32 phase drift at wt ~ 600);
//   * the deviance uses N h(r), h(r) = (1+r) ln(1+r) - r, r = (d - N)/N, with
//     a short series for small |r| so that FP32 keeps full relative accuracy;
//   * every block stages its histogram's constants itself, with few FP64
//     instructions: double-float FP32 pairs where precision matters and
//     integer fixed point for phases, spread over several warps so the
//     dependency chains overlap (with the first data loads in flight);
//   * the lifetime factor exp(-t/tau), which multiplies every bin, is seeded
//     per chunk from a per-run table rounded once from FP64, so no coherent
//     bias enters N (the gradient sums cancel ~100-fold and would amplify it);
//   * the value and gradient modes evaluate the even and odd bins of a chunk
//     as the two lanes of packed FP32 instructions (FFMA2 and kin);
//   * reduction: FP32 warp shuffles, FP64 across the block's warps (with the
//     histogram's role factors applied), then each block adds its FP64
//     partials as 126-bit fixed-point integers into per-histogram
//     accumulators; integer sums do not depend on the order in which blocks
//     finish, so the last block's FP64 conversion and the map to theta give
//     bitwise repeatable results without cluster barriers or partial arrays.
#pragma once

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

__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The theta entries of a histogram's roles, slot 2 r + j (j = 0, 1) of role
// r, 0 where the map row has no entry: read through the row from theta ...
struct ThetaByRow {
    const int32_t* rt;
    const double* theta;
    __device__ __forceinline__ double operator()(int slot) const {
        const int i = rt[slot];
        return i >= 0 ? theta[i] : 0.0;
    }
};
// ... or gathered beforehand (into shared memory).
struct ThetaGathered {
    const double* v;
    __device__ __forceinline__ double operator()(int slot) const { return v[slot]; }
};

// Sum of the (up to two) theta entries a role reads (at most one FP64 add).
template <class TH>
__device__ __forceinline__ double role_value(const TH& th, int r) {
    return th(2 * r) + th(2 * r + 1);
}

// ---- double-float (hi + lo) arithmetic on the FP32 pipe (Knuth TwoSum,
// Dekker TwoProd with FMA); about 44 significant bits ----
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

__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float h = __fadd_rn(p, e);
    return DF{h, __fsub_rn(e, __fsub_rn(h, p))};
}

__device__ __forceinline__ DF df_from(double x) {
    const float hi = __double2float_rn(x);
    return DF{hi, __double2float_rn(x - (double)hi)};
}

__device__ __forceinline__ DF df_of(const float2 v) { return DF{v.x, v.y}; }

// frac(x * c) in 64-bit fixed-point turns, c = c.x + c.y * 2^-64 (unsigned
// 64.64), by exact integer arithmetic on x's significand (truncated at
// 2^-64 turns).  The phase of every precession line is formed this way, so it
// is exact at any t without FP64 arithmetic.
__device__ __forceinline__ unsigned long long fixmul(double x, ulonglong2 c) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7ff);
    if (e == 0 || e == 0x7ff) return 0ull;  // zero / subnormal / non-finite
    const unsigned long long m = (bits & 0xfffffffffffffull) | (1ull << 52);
    // P = m * (c.x * 2^64 + c.y), 192 bits, in units of 2^-64 turns per 2^sh
    const unsigned long long l1 = m * c.y, h1 = __umul64hi(m, c.y);
    const unsigned long long l2 = m * c.x, h2 = __umul64hi(m, c.x);
    const unsigned long long p0 = l1;
    const unsigned long long p1 = h1 + l2;
    const unsigned long long p2 = h2 + (p1 < h1 ? 1ull : 0ull);
    const int sh = e - 1075;  // x = m * 2^sh
    unsigned long long r;
    if (sh >= 0) {
        r = sh < 64 ? (p0 << sh) : 0ull;
    } else {
        const int s = -sh;
        if (s < 64) r = (p0 >> s) | (p1 << (64 - s));
        else if (s == 64) r = p1;
        else if (s < 128) r = (p1 >> (s - 64)) | (p2 << (128 - s));
        else if (s == 128) r = p2;
        else if (s < 192) r = p2 >> (s - 128);
        else r = 0ull;
    }
    return (bits >> 63) ? (0ull - r) : r;
}

// expm1(x) and sin(pi x): Taylor series for the small per-bin step
// arguments (expm1: |x| < 1/4, terms to x^9, truncation below 3e-13
// relative; sin: |x| < 1/32, below 3e-15), the FP32 library functions
// otherwise.
__device__ __forceinline__ float step_expm1(float x) {
    if (fabsf(x) >= 0.25f) return expm1f(x);
    float r = fmaf(x, 1.f / 9.f, 1.f);
    r = fmaf(x * 0.125f, r, 1.f);
    r = fmaf(x * (1.f / 7.f), r, 1.f);
    r = fmaf(x * (1.f / 6.f), r, 1.f);
    r = fmaf(x * 0.2f, r, 1.f);
    r = fmaf(x * 0.25f, r, 1.f);
    r = fmaf(x * (1.f / 3.f), r, 1.f);
    r = fmaf(x * 0.5f, r, 1.f);
    return x * r;
}

__device__ __forceinline__ float step_sinpi(float x) {
    if (fabsf(x) >= 0.03125f) return sinpif(x);
    const float y = 3.14159265358979323846f * x, y2 = y * y;
    float r = fmaf(-y2, 1.f / 42.f, 1.f);
    r = fmaf(-y2 * 0.05f, r, 1.f);
    r = fmaf(-y2 * (1.f / 6.f), r, 1.f);
    return y * r;
}

// Per-histogram constants in NPART independent parts, each computed by lane 0
// of its own warp so the parts overlap:
//   part 0        N0 (hi/lo), bkg, lifetime recurrence
//   part 1 + 2c   envelope of precession line c
//   part 2 + 2c   phase of precession line c (64-bit fixed-point turns)
//   part 1 + 2 NOSC  static Gaussian Kubo-Toyabe term
// Only FP32 (double-float where precision matters), integer arithmetic and
// FP32 accurate functions: no chains of FP64 operations.
template <int NE, int NG, int NS, int KT>
__host__ __device__ constexpr int stage_parts() {
    return 2 + 2 * (NE + NG + NS);
}

// Out-of-line copies of the staging's functions: the staging runs once per
// block, and an inlined copy at every call site multiplies the prologue's
// code, which a block fetches cold while the other block on its SM runs the
// bin loop.
static __device__ __noinline__ float stage_expm1(float x) { return step_expm1(x); }
static __device__ __noinline__ float stage_sinpi(float x) { return step_sinpi(x); }
static __device__ __noinline__ unsigned long long stage_fixmul(double x, ulonglong2 c) { return fixmul(x, c); }
static __device__ __noinline__ float stage_exp(float x) { return expf(x); }

// N independent evaluations of a staging function: by one thread in turn
// (lane < 0), or by the lanes of a warp at once, lane j evaluating the j-th
// (every lane of the warp takes part, and every lane receives all N results).
// Both ways evaluate the same function on the same arguments.
template <int N>
__device__ __forceinline__ void stage_expm1_n(const float (&x)[N], float (&y)[N], int lane) {
    if (lane < 0) {
#pragma unroll
        for (int j = 0; j < N; ++j) y[j] = stage_expm1(x[j]);
        return;
    }
    float xi = x[0];
#pragma unroll
    for (int j = 1; j < N; ++j)
        if (lane == j) xi = x[j];
    const float yi = stage_expm1(xi);
#pragma unroll
    for (int j = 0; j < N; ++j) y[j] = __shfl_sync(0xffffffffu, yi, j);
}
template <int N>
__device__ __forceinline__ void stage_sinpi_n(const float (&x)[N], float (&y)[N], int lane) {
    if (lane < 0) {
#pragma unroll
        for (int j = 0; j < N; ++j) y[j] = stage_sinpi(x[j]);
        return;
    }
    float xi = x[0];
#pragma unroll
    for (int j = 1; j < N; ++j)
        if (lane == j) xi = x[j];
    const float yi = stage_sinpi(xi);
#pragma unroll
    for (int j = 0; j < N; ++j) y[j] = __shfl_sync(0xffffffffu, yi, j);
}
// the first n of N products (all N by a warp: the lanes beyond n cost nothing)
template <int N>
__device__ __forceinline__ void stage_fixmul_n(const double (&x)[N], const ulonglong2 (&c)[N],
                                               unsigned long long (&y)[N], int n, int lane) {
    if (lane < 0) {
#pragma unroll
        for (int j = 0; j < N; ++j) y[j] = j < n ? stage_fixmul(x[j], c[j]) : 0ull;
        return;
    }
    double xi = x[0];
    ulonglong2 ci = c[0];
#pragma unroll
    for (int j = 1; j < N; ++j)
        if (lane == j) {
            xi = x[j];
            ci = c[j];
        }
    const unsigned long long yi = stage_fixmul(xi, ci);
#pragma unroll
    for (int j = 0; j < N; ++j) y[j] = j < n ? __shfl_sync(0xffffffffu, yi, j) : 0ull;
}

// stripe > 0: bins between a thread's consecutive chunks (for the Gaussian
// ratio carried from chunk to chunk, see GqCarry); 0 when nothing is carried.
// lane < 0: one thread stages the part; lane >= 0: all 32 lanes of a warp
// call with the same part and their lane index, and share its independent
// function evaluations (every lane stores the same values).
template <int NE, int NG, int NS, int KT, class TH>
__device__ void stage_part(int part, const TH& th, const RunConst& rc, HistConst& hc, int stripe = 0,
                           int lane = -1) {
    constexpr int NOSC = NE + NG + NS;
    const DF it = df_of(rc.inv_tau), dtL = df_of(rc.dt_log2e), dt = df_of(rc.dt);
    if (part == 0) {
        const DF n0 = df_from(role_value(th, 0));
        hc.n0 = n0.hi;
        hc.n0_lo = n0.lo;
        hc.bkg = __double2float_rn(role_value(th, 1));
        hc.qE = rc.qE;
        hc.qE2 = rc.qE * (2.f + rc.qE);
        hc.kfreq = rc.kfreq;
    } else if (part <= 2 * NOSC) {
        const int c = (part - 1) >> 1;
        const int r = 2 + 4 * c;
        OscConst& o = hc.osc[c];
        if (part & 1) {  // envelope
            const DF rate = df_from(role_value(th, r + 1));
            o.amp = __double2float_rn(role_value(th, r));
            o.rate = rate.hi;
            if (c >= NE + NG) {  // exp(-(lambda t)^beta), evaluated per bin; the rotation alone is stepped
                o.beta = __double2float_rn(role_value(th, 2 + 4 * NOSC));
                o.a_hi = o.a_lo = o.b_hi = o.b_lo = o.q = o.qs = o.q2 = o.qs2 = 0.f;
                o.cenv = 1.f;
            } else if (c < NE) {  // exp(-(1/tau + lambda) t)
                const DF rtot = df_add(it, rate);
                const DF a = df_mul(rtot, dtL);
                o.a_hi = a.hi;
                o.a_lo = a.lo;
                o.b_hi = o.b_lo = 0.f;
                o.q = stage_expm1(-df_mul(rtot, dt).hi);
                o.q2 = o.q * (2.f + o.q);
                o.qs = o.qs2 = 0.f;
                o.cenv = rc.t0_zero ? 1.f : stage_exp(-df_mul(rtot, df_of(rc.t0)).hi);
            } else {  // exp(-t/tau - sigma^2 t^2 / 2), t = t0 + n dt
                const DF s2 = df_mul(rate, rate);
                const DF a = df_add(df_mul(it, dtL), df_mul(s2, df_of(rc.t0_dt_log2e)));
                const DF b = df_mul(s2, df_of(rc.half_dt2_log2e));
                o.a_hi = a.hi;
                o.a_lo = a.lo;
                o.b_hi = b.hi;
                o.b_lo = b.lo;
                // 2^(-2 b) - 1, its change over a stripe, 2^(-8 b) - 1, the 2-bin change over a stripe
                const float xq[4] = {-1.38629436111989061883f * (b.hi + b.lo),
                                     -1.38629436111989061883f * (float)stripe * (b.hi + b.lo),
                                     -5.54517744447956247532f * (b.hi + b.lo),
                                     -2.77258872223978123767f * (float)stripe * (b.hi + b.lo)};
                float yq[4];
                stage_expm1_n<4>(xq, yq, lane);
                o.q = yq[0];
                o.qs = yq[1];
                o.q2 = yq[2];
                o.qs2 = yq[3];
                if (rc.t0_zero) {
                    o.cenv = 1.f;
                } else {
                    const DF t0 = df_of(rc.t0);
                    const DF x = df_add(df_mul(t0, it), df_mul(df_mul(s2, t0), DF{0.5f * t0.hi, 0.5f * t0.lo}));
                    o.cenv = stage_exp(-x.hi);
                }
            }
        } else {  // phase: sums of fixed-point products are exact mod 1 turn
            // an absent entry reads 0, whose fixed-point product is 0
            const double f0 = th(2 * (r + 2)), f1 = th(2 * (r + 2) + 1), phi = th(2 * (r + 3));
            const double xf[5] = {f0, f1, phi, f0, f1};
            const ulonglong2 cf[5] = {rc.turns_per_bin, rc.turns_per_bin, rc.inv_two_pi, rc.turns_at_t0,
                                      rc.turns_at_t0};
            unsigned long long yf[5];
            stage_fixmul_n<5>(xf, cf, yf, rc.t0_zero ? 3 : 5, lane);
            const unsigned long long step = yf[0] + yf[1];
            const unsigned long long ph0 = yf[2] + (yf[3] + yf[4]);
            o.ph0 = ph0;
            o.step = step;
            o.step_s = step * (unsigned long long)stripe;  // mod 2^64: whole turns drop out
            const float red = (float)(long long)step * 5.42101086242752217e-20f;  // turns in [-1/2, 1/2)
            const float xs[3] = {red, 2.f * red, 4.f * red};
            float ys[3];
            stage_sinpi_n<3>(xs, ys, lane);
            o.cm1 = -2.f * ys[0] * ys[0];    // cos(step) - 1
            o.sn = ys[1];                    // sin(step)
            o.cm1_2 = -2.f * ys[1] * ys[1];  // cos(2 step) - 1
            o.sn_2 = ys[2];
        }
    } else if (KT && part == 2 * NOSC + 1) {
        const int r = 2 + 4 * NOSC + NS;
        const DF dl = df_from(role_value(th, r + 1));
        const DF s2 = df_mul(dl, dl);
        hc.kt_amp = __double2float_rn(role_value(th, r));
        hc.kt_rate = dl.hi;
        const DF a = df_add(df_mul(it, dtL), df_mul(s2, df_of(rc.t0_dt_log2e)));
        const DF b = df_mul(s2, df_of(rc.half_dt2_log2e));
        hc.kt_a_hi = a.hi;
        hc.kt_a_lo = a.lo;
        hc.kt_b_hi = b.hi;
        hc.kt_b_lo = b.lo;
        const float xq[4] = {-1.38629436111989061883f * (b.hi + b.lo),
                             -1.38629436111989061883f * (float)stripe * (b.hi + b.lo),
                             -5.54517744447956247532f * (b.hi + b.lo),
                             -2.77258872223978123767f * (float)stripe * (b.hi + b.lo)};
        float yq[4];
        stage_expm1_n<4>(xq, yq, lane);
        hc.kt_q = yq[0];
        hc.kt_qs = yq[1];
        hc.kt_q2 = yq[2];
        hc.kt_qs2 = yq[3];
        if (rc.t0_zero) {
            hc.kt_cenv = 1.f;
        } else {
            const DF t0 = df_of(rc.t0);
            const DF x = df_add(df_mul(t0, it), df_mul(df_mul(s2, t0), DF{0.5f * t0.hi, 0.5f * t0.lo}));
            hc.kt_cenv = stage_exp(-x.hi);
        }
    }
}

// Asynchronous global -> shared copies (completed by cp_async_wait_all in the
// issuing thread; other threads see the data after a barrier that follows).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int NACC>
__device__ __forceinline__ void warp_sum(float (&v)[NACC]) {
#pragma unroll
    for (int a = 0; a < NACC; ++a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[a] += __shfl_xor_sync(0xffffffffu, v[a], o);
    }
}

// Reduce-scatter of N accumulators over the warp by recursive halving: at
// step s every lane keeps half of its values (the upper half where bit s of
// its lane index is set) and adds the partner's (lane ^ 2^s) copy of that
// half, so the warp does ~N shuffles instead of the butterfly's 5 N.  On
// return lane L holds the warp sums of accumulators j + (NP / 32) bitrev5(L),
// j < NP / 32, in v[0 .. NP / 32) (NP = N rounded up to a multiple of 32;
// the padding is zero).
template <int N>
struct WarpSplit {
    static constexpr int NP = (N + 31) / 32 * 32;
    static constexpr int PER = NP / 32;
    float v[NP];
};
template <int N>
__device__ __forceinline__ void warp_reduce_scatter(WarpSplit<N>& w, int lane) {
    constexpr int NP = WarpSplit<N>::NP;
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int M = NP >> s, H = M >> 1;
        const bool up = (lane >> s) & 1;
#pragma unroll
        for (int i = 0; i < H; ++i) {
            const float keep = up ? w.v[i + H] : w.v[i];
            const float send = up ? w.v[i] : w.v[i + H];
            w.v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 1 << s);
        }
    }
}
__device__ __forceinline__ int bitrev5(int x) {
    return ((x & 1) << 4) | ((x & 2) << 2) | (x & 4) | ((x & 8) >> 2) | ((x & 16) >> 4);
}

// One thread's chunk of kBinsPerThread consecutive bins starting at bin n0 of a
// histogram with M bins: theory (Eq. 1), objective term (Eq. 3 / Eq. 4) and,
// by mode, the role partials accumulated into the gradient and GN matrix.
//
// Each precession line is carried as the scaled rotation (env cos, env sin):
// an exponential line advances by one constant 2 x 2 step per bin (rotation
// times the envelope's step), a Gaussian line by the rotation and the
// envelope ratio (1 + gq), itself stepped by gq' = gq Q + (Q - 1).  Role
// partials dN/d(role) = f_role x_role with f_role constant per histogram
// (acc_factor, which also carries the objective's weight factor -2 / 2) and
// x_role cheap per bin: the accumulators collect sum w' x_role, w' = wg / -2.
// The Gaussian step ratios at a thread's next chunk (one stripe further):
// gq(n0 + stripe) = gq(n0) Qs + (Qs - 1), Qs = 2^(-2 b stripe), so only a
// thread's first chunk evaluates them from scratch.
template <int NOSC>
struct GqCarry {
    float gq[NOSC > 0 ? NOSC : 1];
    float gqk;
    unsigned long long ph[NOSC > 0 ? NOSC : 1];  // fixed-point phase at the next chunk (exact 64-bit sums)
    bool valid;
};

// ---- packed FP32 pairs (sm_100 FFMA2 / FMUL2 / FADD2): two values per instruction ----
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Gauss-Newton accumulators of one thread, packed: the gradient sums
// g[r] += w' x[r] as pairs g2[i] = (g[2i], g[2i+1]), and the upper triangle
// h[r1][r2] += (wh x[r1]) x[r2], r2 >= r1, row by row: entries from an even
// column in adjacent pairs (one FFMA2 against the aligned pair
// (x[c], x[c+1])), the diagonal of an odd row and the last entry of a row
// of odd length singly.  gn_scatter writes them in the standard layout.
constexpr int gn_pairs(int R) {
    int n = 0;
    for (int r1 = 0; r1 < R; ++r1) n += (R - (r1 + (r1 & 1))) / 2;
    return n;
}
constexpr int gn_singles(int R) {
    int n = 0;
    for (int r1 = 0; r1 < R; ++r1) n += (r1 & 1) + ((R - (r1 + (r1 & 1))) & 1);
    return n;
}
template <int R>
struct GnAcc {
    static constexpr int RX = (R + 1) / 2;
    static constexpr int NP = gn_pairs(R);
    static constexpr int NSG = gn_singles(R);
    float2 g2[RX];
    float2 p[NP > 0 ? NP : 1];
    float s[NSG > 0 ? NSG : 1];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < RX; ++i) g2[i] = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < NP; ++i) p[i] = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < NSG; ++i) s[i] = 0.f;
    }
};

// acc[1 + r] = g[r]; acc[1 + R + ...] = the triangle row by row.
template <int R, int NACC>
__device__ __forceinline__ void gn_scatter(const GnAcc<R>& G, float (&acc)[NACC]) {
#pragma unroll
    for (int r = 0; r < R; ++r) acc[1 + r] = (r & 1) ? G.g2[r >> 1].y : G.g2[r >> 1].x;
    int a = 1 + R, pi = 0, si = 0;
#pragma unroll
    for (int r1 = 0; r1 < R; ++r1) {
        int c = r1;
        if (c & 1) {
            acc[a++] = G.s[si++];
            ++c;
        }
#pragma unroll
        for (; c + 1 < R; c += 2) {
            acc[a++] = G.p[pi].x;
            acc[a++] = G.p[pi].y;
            ++pi;
        }
        if (c < R) acc[a++] = G.s[si++];
    }
}

// The lifetime factor at any bin n0 from the run's table of chunk starts,
// stepped by the per-bin recurrence over the n0 mod 8 bins past the start.
__device__ __forceinline__ float lifetime_from_table(const float* etab, int n0, float qE) {
    float E = __ldg(etab + (n0 >> 3));
    for (int r = n0 & 7; r > 0; --r) E = fmaf(E, qE, E);
    return E;
}

// 2-bin ratio minus 1 of a Gaussian envelope exp2(-(a n + b n^2)) at bin n:
// 2^(-(2 a + 4 b (n + 1))) - 1.
__device__ __forceinline__ float gauss_ratio2(float a_hi, float a_lo, float b_hi, float b_lo, int n) {
    const float k4 = 4.f * (float)(n + 1);
    return step_expm1(-0.693147180559945309f * fmaf(k4, b_hi, fmaf(k4, b_lo, 2.f * (a_hi + a_lo))));
}

// First-chunk seeds of a Gaussian ratio recurrence (a Gaussian envelope or
// the Kubo-Toyabe term), exp2(-(a n + b n^2)) at bin n0: the 1-bin ratio
// minus 1, 2^(-(a + b (2 n0 + 1))) - 1, and the 2-bin ratios at n0 and n0 + 1.
// Out of line: a thread that carries the ratios from chunk to chunk computes
// them once, and inlined copies would enlarge the bin loop's code.
struct GaussSeed {
    float q1, r0, r1;
};
static __device__ __noinline__ float gauss_seed1(float a_hi, float a_lo, float b_hi, float b_lo, int n0) {
    const float k1 = fmaf(2.f, (float)n0, 1.f);
    return step_expm1(-0.693147180559945309f * fmaf(k1, b_hi, fmaf(k1, b_lo, a_hi + a_lo)));
}
static __device__ __noinline__ GaussSeed gauss_seed(float a_hi, float a_lo, float b_hi, float b_lo, int n0) {
    const float k1 = fmaf(2.f, (float)n0, 1.f);
    GaussSeed g;
    g.q1 = step_expm1(-0.693147180559945309f * fmaf(k1, b_hi, fmaf(k1, b_lo, a_hi + a_lo)));
    g.r0 = gauss_ratio2(a_hi, a_lo, b_hi, b_lo, n0);
    g.r1 = gauss_ratio2(a_hi, a_lo, b_hi, b_lo, n0 + 1);
    return g;
}

// E0: the lifetime factor exp(-t/tau) at bin n0 (from the run's lifetime table)
template <int NE, int NG, int NS, int KT, int MODE, int NACC, bool FULL>
__device__ __forceinline__ void eval_chunk_body(const HistConst& hc, int n0, int M,
                                                const float (&d)[kBinsPerThread], float E0, int obj, float dtf,
                                                float t0f, float (&acc)[NACC], bool& bad,
                                                float* model_dst, GqCarry<NE + NG + NS>* carry,
                                                GnAcc<2 + 4 * (NE + NG + NS) + NS + 2 * KT>* gn) {
    constexpr int NOSC = NE + NG + NS;
    constexpr int R = 2 + 4 * NOSC + NS + 2 * KT;
    constexpr int CS = NE + NG;    // index of the stretched line (when NS)
    constexpr int RB = 2 + 4 * NOSC;  // role of its exponent beta
    constexpr int RK = RB + NS;       // first Kubo-Toyabe role
    constexpr int G = kBinsPerThread;
    constexpr bool NEED_TT = KT || (NG > 0 && MODE >= kGrad);
    const float nf0 = (float)n0;
    const float n0p = hc.n0, n0lo = hc.n0_lo, bkg = hc.bkg;
    float E = E0;
    float C[NOSC > 0 ? NOSC : 1], Sn[NOSC > 0 ? NOSC : 1], gq[NOSC > 0 ? NOSC : 1];
    float stA[NOSC > 0 ? NOSC : 1], stB[NOSC > 0 ? NOSC : 1];
    const float k1 = fmaf(2.f, nf0, 1.f);  // 2 n0 + 1
    const float nn0 = nf0 * nf0;
#pragma unroll
    for (int c = 0; c < NOSC; ++c) {
        const OscConst& o = hc.osc[c];
        float env;
        if (NS && c >= CS) {
            // stretched line: the rotation alone is carried, its envelope is evaluated per bin
            env = 1.f;
            stA[c] = o.cm1;
            stB[c] = o.sn;
        } else if (c < NE) {
            env = o.cenv * ex2_approx(-fmaf(nf0, o.a_hi, nf0 * o.a_lo));
            // one bin's step: (1 + q) (cos d, sin d) = (1 + A, B)
            stA[c] = fmaf(o.q, o.cm1, o.q + o.cm1);
            stB[c] = fmaf(o.q, o.sn, o.sn);
        } else {
            env = o.cenv * ex2_approx(-fmaf(nn0, o.b_hi, fmaf(nf0, o.a_hi, fmaf(nn0, o.b_lo, nf0 * o.a_lo))));
            if (carry && carry->valid) {
                gq[c] = carry->gq[c];
            } else if (carry) {  // once per thread: out of line
                gq[c] = gauss_seed1(o.a_hi, o.a_lo, o.b_hi, o.b_lo, n0);
            } else {
                gq[c] = step_expm1(-0.693147180559945309f * fmaf(k1, o.b_hi, fmaf(k1, o.b_lo, o.a_hi + o.a_lo)));
            }
            if (carry) carry->gq[c] = fmaf(gq[c], o.qs, gq[c] + o.qs);
            stA[c] = o.cm1;
            stB[c] = o.sn;
        }
        const unsigned long long ph =
            (carry && carry->valid) ? carry->ph[c] : o.ph0 + (unsigned long long)n0 * o.step;
        if (carry) carry->ph[c] = ph + o.step_s;
        const float x = (float)(int)(ph >> 32) * 2.3283064365386963e-10f;  // turns in [-1/2, 1/2)
        float sc, cc;
        __sincosf(6.28318530717958647692f * x, &sc, &cc);
        C[c] = env * cc;
        Sn[c] = env * sc;
    }
    // Kubo-Toyabe: G(t) e^{-t/tau} = E / 3 + (1 - x) e23,  x = (Delta t)^2,
    // e23 = 2/3 exp(-t/tau - x/2), stepped like a Gaussian envelope
    float e23 = 0.f, gqk = 0.f, kr2 = 0.f;
    if (KT) {
        e23 = 0.666666667f * hc.kt_cenv *
              ex2_approx(-fmaf(nn0, hc.kt_b_hi, fmaf(nf0, hc.kt_a_hi, fmaf(nn0, hc.kt_b_lo, nf0 * hc.kt_a_lo))));
        if (carry && carry->valid) {
            gqk = carry->gqk;
        } else if (carry) {  // once per thread: out of line
            gqk = gauss_seed1(hc.kt_a_hi, hc.kt_a_lo, hc.kt_b_hi, hc.kt_b_lo, n0);
        } else {
            gqk = step_expm1(-0.693147180559945309f *
                             fmaf(k1, hc.kt_b_hi, fmaf(k1, hc.kt_b_lo, hc.kt_a_hi + hc.kt_a_lo)));
        }
        if (carry) carry->gqk = fmaf(gqk, hc.kt_qs, gqk + hc.kt_qs);
        kr2 = hc.kt_rate * hc.kt_rate;
    }
    if (carry) carry->valid = true;
    const float ts = fmaf(nf0, dtf, t0f);
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const float t = fmaf((float)g, dtf, ts);
        const float tt = NEED_TT ? t * t : 0.f;
        // this bin's scaled rotation of every line: the carried one, or for the
        // stretched line the rotation times e^{-t/tau} exp(-(lambda t)^beta)
        float Cb[NOSC > 0 ? NOSC : 1], Sb[NOSC > 0 ? NOSC : 1];
        float sp = 0.f, slg = 0.f;  // stretched line: (lambda t)^beta and log2(lambda t), 0 where lambda t <= 0
#pragma unroll
        for (int c = 0; c < NOSC; ++c) {
            if (NS && c >= CS) {
                const float u = hc.osc[c].rate * t;
                const bool pos = u > 0.f;
                const float lg = lg2_approx(u);
                sp = pos ? ex2_approx(hc.osc[c].beta * lg) : 0.f;
                slg = pos ? lg : 0.f;
                const float ev = E * ex2_approx(-1.44269504088896341f * sp);
                Cb[c] = ev * C[c];
                Sb[c] = ev * Sn[c];
            } else {
                Cb[c] = C[c];
                Sb[c] = Sn[c];
            }
        }
        float S = E;
#pragma unroll
        for (int c = 0; c < NOSC; ++c) S = fmaf(hc.osc[c].amp, Cb[c], S);
        float xk = 0.f, GE = 0.f;
        if (KT) {
            xk = kr2 * tt;
            GE = fmaf(E, 0.333333333f, fmaf(-e23, xk, e23));
            S = fmaf(hc.kt_amp, GE, S);
        }
        // N0 carried as an FP32 pair so its rounding does not bias every bin
        const float N = fmaf(n0p, S, fmaf(n0lo, S, bkg));

        if (MODE == kModel) {
            if (FULL || n0 + g < M) model_dst[n0 + g] = N;
        } else if (MODE == kSum) {
            if (FULL || n0 + g < M) acc[0] += N;
        } else if (FULL || n0 + g < M) {
            const float dv = d[g];
            float wq, wh;  // wq = wg / -2 (gradient weight), wh = GN weight / 2
            if (obj == MUSR_CHI2) {
                const float w = rcp_approx(fmaxf(dv, 1.f));
                const float r = dv - N;
                wq = r * w;
                acc[0] = fmaf(r, wq, acc[0]);
                wh = w;
            } else {
                float term;
                if (dv > 0.f) {
                    if (!(N > 0.f)) {
                        bad = true;
                        term = wq = wh = 0.f;
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
                        wq = rho;
                        wh = rN;
                    }
                } else {
                    if (!(N >= 0.f)) bad = true;
                    term = 2.f * N;
                    wq = -1.f;
                    wh = N > 0.f ? rcp_approx(N) : 0.f;
                }
                acc[0] += term;
            }
            if (MODE == kGrad) {
                const float wt = wq * t;
                const float wtt = NEED_TT ? wq * tt : 0.f;
                acc[1] = fmaf(wq, S, acc[1]);
                acc[2] += wq;
#pragma unroll
                for (int c = 0; c < NOSC; ++c) {
                    acc[3 + 4 * c] = fmaf(wq, Cb[c], acc[3 + 4 * c]);
                    if (NS && c >= CS) {
                        const float pc = sp * Cb[c];
                        acc[4 + 4 * c] = fmaf(wq, pc, acc[4 + 4 * c]);
                        acc[1 + RB] = fmaf(wq, pc * slg, acc[1 + RB]);
                    } else {
                        acc[4 + 4 * c] = fmaf(c < NE ? wt : wtt, Cb[c], acc[4 + 4 * c]);
                    }
                    acc[5 + 4 * c] = fmaf(wt, Sb[c], acc[5 + 4 * c]);
                    acc[6 + 4 * c] = fmaf(wq, Sb[c], acc[6 + 4 * c]);
                }
                if (KT) {
                    acc[1 + RK] = fmaf(wq, GE, acc[1 + RK]);
                    acc[2 + RK] = fmaf(wtt, (xk - 3.f) * e23, acc[2 + RK]);
                }
            } else if (MODE == kGN) {
                float x[R];
                x[0] = S;
                x[1] = 1.f;
#pragma unroll
                for (int c = 0; c < NOSC; ++c) {
                    x[2 + 4 * c] = Cb[c];
                    if (NS && c >= CS) {
                        x[3 + 4 * c] = sp * Cb[c];
                        x[RB] = sp * slg * Cb[c];
                    } else {
                        x[3 + 4 * c] = (c < NE ? t : tt) * Cb[c];
                    }
                    x[4 + 4 * c] = t * Sb[c];
                    x[5 + 4 * c] = Sb[c];
                }
                if (KT) {
                    x[RK] = GE;
                    x[RK + 1] = tt * (xk - 3.f) * e23;
                }
                // x as aligned pairs (x[R] = 0 when R is odd)
                constexpr int RX = (R + 1) / 2;
                float2 xp[RX];
#pragma unroll
                for (int i = 0; i < RX; ++i) xp[i] = make_float2(x[2 * i], 2 * i + 1 < R ? x[2 * i + 1] : 0.f);
                const float2 wq2 = bc2(wq);
#pragma unroll
                for (int i = 0; i < RX; ++i) gn->g2[i] = fma2(wq2, xp[i], gn->g2[i]);
                int pi = 0, si = 0;
#pragma unroll
                for (int r1 = 0; r1 < R; ++r1) {
                    const float qv = wh * x[r1];
                    const float2 q2 = bc2(qv);
                    int c = r1;
                    if (c & 1) {
                        gn->s[si] = fmaf(qv, x[c], gn->s[si]);
                        ++si;
                        ++c;
                    }
#pragma unroll
                    for (; c + 1 < R; c += 2) {
                        gn->p[pi] = fma2(q2, xp[c >> 1], gn->p[pi]);
                        ++pi;
                    }
                    if (c < R) {
                        gn->s[si] = fmaf(qv, x[c], gn->s[si]);
                        ++si;
                    }
                }
            }
        }
        // step the recurrences to the next bin
        E = fmaf(E, hc.qE, E);
#pragma unroll
        for (int c = 0; c < NOSC; ++c) {
            const float c2 = fmaf(C[c], stA[c], fmaf(-Sn[c], stB[c], C[c]));
            const float s2 = fmaf(Sn[c], stA[c], fmaf(C[c], stB[c], Sn[c]));
            if (c < NE || c >= CS) {
                C[c] = c2;
                Sn[c] = s2;
            } else {
                C[c] = fmaf(c2, gq[c], c2);
                Sn[c] = fmaf(s2, gq[c], s2);
                gq[c] = fmaf(gq[c], hc.osc[c].q, gq[c] + hc.osc[c].q);
            }
        }
        if (KT) {
            e23 = fmaf(e23, gqk, e23);
            gqk = fmaf(gqk, hc.kt_q, gqk + hc.kt_q);
        }
    }
}

// carry: NULL, or the thread's GqCarry when its successive calls are one
// stripe apart (the staged qs constants must be for that stripe)
template <int NE, int NG, int NS, int KT, int MODE, int NACC>
__device__ __forceinline__ void eval_chunk(const HistConst& hc, int n0, int M, const float (&d)[kBinsPerThread],
                                           float E0, int obj, float dtf, float t0f, float (&acc)[NACC], bool& bad,
                                           float* model_dst, GqCarry<NE + NG + NS>* carry = nullptr,
                                           GnAcc<2 + 4 * (NE + NG + NS) + NS + 2 * KT>* gn = nullptr) {
    if (n0 + kBinsPerThread <= M)
        eval_chunk_body<NE, NG, NS, KT, MODE, NACC, true>(hc, n0, M, d, E0, obj, dtf, t0f, acc, bad, model_dst,
                                                          carry, gn);
    else
        eval_chunk_body<NE, NG, NS, KT, MODE, NACC, false>(hc, n0, M, d, E0, obj, dtf, t0f, acc, bad, model_dst,
                                                           carry, gn);
}

// ---- packed FP32 pairs: two bins per instruction (FFMA2 / FMUL2 / FADD2) ----
//
// The value and adjoint modes step the even and odd bins of a thread's 8-bin
// chunk as the two lanes of float2 operands: lane x holds bins n0, n0+2, n0+4,
// n0+6 and lane y bins n0+1, n0+3, n0+5, n0+7, so the counts come out of the
// two 128-bit loads already paired.  Every recurrence advances a lane by two
// bins (the 2-bin constants staged with the 1-bin ones); lane y is seeded
// from lane x by one 1-bin step.  The arithmetic per bin is that of
// eval_chunk_body, in half the instructions.

// What a thread carries from one chunk to its next, one stripe further, so
// the next chunk's seeds need no multiplication or series: the fixed-point
// phase of every line (advanced by an exact 64-bit addition), the Gaussian
// envelopes' 1-bin ratio at the chunk start (gq(n + stripe) = gq(n) Qs +
// (Qs - 1)) and both lanes' 2-bin ratios (G2(n + stripe) = G2(n) Qs2 +
// (Qs2 - 1)), likewise for the Kubo-Toyabe envelope.
template <int NOSC>
struct G2Carry {
    float2 g2[NOSC > 0 ? NOSC : 1];
    float2 g2k;
    float gq1[NOSC > 0 ? NOSC : 1];
    float gqk1;
    unsigned long long ph[NOSC > 0 ? NOSC : 1];
    bool valid;
};


// One chunk of 8 bins starting at n0 (a multiple of 8) in packed lanes:
// MODE kValue or kGrad.  d holds the chunk's counts, E0 the lifetime factor at
// n0; acc are the per-lane accumulators (lane sums are added after the
// chunks).  FULL: all 8 bins lie below M.
template <int NE, int NG, int NS, int KT, int MODE, int NACC, bool FULL>
__device__ __forceinline__ void eval_pair_body(const HistConst& hc, int n0, int M,
                                               const float (&d)[kBinsPerThread], float E0, int obj, float dtf,
                                               float t0f, float2 (&acc)[NACC], bool& bad,
                                               G2Carry<NE + NG + NS>* carry) {
    static_assert(MODE == kValue || MODE == kGrad, "packed lanes serve the value and gradient modes");
    constexpr int NOSC = NE + NG + NS;
    constexpr int CS = NE + NG;       // index of the stretched line (when NS)
    constexpr int RB = 2 + 4 * NOSC;  // role of its exponent beta
    constexpr int RK = RB + NS;       // first Kubo-Toyabe role
    constexpr bool NEED_TT = KT || (NG > 0 && MODE >= kGrad);
    const float nf0 = (float)n0;
    const float2 n0p = bc2(hc.n0), n0lo = bc2(hc.n0_lo), bkg = bc2(hc.bkg);
    // lifetime factor: lane y one bin further
    float2 E = make_float2(E0, fmaf(E0, hc.qE, E0));
    const float2 qE2 = bc2(hc.qE2);
    float2 C[NOSC > 0 ? NOSC : 1], Sn[NOSC > 0 ? NOSC : 1], g2[NOSC > 0 ? NOSC : 1];
    float2 stA[NOSC > 0 ? NOSC : 1], stB[NOSC > 0 ? NOSC : 1], nstB[NOSC > 0 ? NOSC : 1];
    const float nn0 = nf0 * nf0;
    const bool carried = carry && carry->valid;
#pragma unroll
    for (int c = 0; c < NOSC; ++c) {
        const OscConst& o = hc.osc[c];
        // lane x: exact seed at n0 (fixed-point phase, SFU sincos and exp2)
        const unsigned long long ph = carried ? carry->ph[c] : o.ph0 + (unsigned long long)n0 * o.step;
        if (carry) carry->ph[c] = ph + o.step_s;
        const float x = (float)(int)(ph >> 32) * 2.3283064365386963e-10f;  // turns in [-1/2, 1/2)
        float sc, cc;
        __sincosf(6.28318530717958647692f * x, &sc, &cc);
        // lane y: one 1-bin rotation further
        const float cy = fmaf(cc, o.cm1, fmaf(-sc, o.sn, cc));
        const float sy = fmaf(sc, o.cm1, fmaf(cc, o.sn, sc));
        float env, envy;
        if (NS && c >= CS) {
            env = envy = 1.f;  // the stretched envelope is evaluated per bin
            stA[c] = bc2(o.cm1_2);
            stB[c] = bc2(o.sn_2);
        } else if (c < NE) {
            env = o.cenv * ex2_approx(-fmaf(nf0, o.a_hi, nf0 * o.a_lo));
            envy = fmaf(env, o.q, env);
            // two bins' step: (1 + q2) (cos 2d, sin 2d) = (1 + A, B)
            stA[c] = bc2(fmaf(o.q2, o.cm1_2, o.q2 + o.cm1_2));
            stB[c] = bc2(fmaf(o.q2, o.sn_2, o.sn_2));
        } else {
            env = o.cenv * ex2_approx(-fmaf(nn0, o.b_hi, fmaf(nf0, o.a_hi, fmaf(nn0, o.b_lo, nf0 * o.a_lo))));
            // 1-bin ratio at n0 (lane y's seed), then both lanes' 2-bin ratios
            float gq1;
            if (carried) {
                gq1 = carry->gq1[c];
                g2[c] = carry->g2[c];
            } else {
                const GaussSeed sd = gauss_seed(o.a_hi, o.a_lo, o.b_hi, o.b_lo, n0);
                gq1 = sd.q1;
                g2[c] = make_float2(sd.r0, sd.r1);
            }
            if (carry) carry->gq1[c] = fmaf(gq1, o.qs, gq1 + o.qs);
            envy = fmaf(env, gq1, env);
            if (carry) carry->g2[c] = fma2(g2[c], bc2(o.qs2), add2(g2[c], bc2(o.qs2)));
            stA[c] = bc2(o.cm1_2);
            stB[c] = bc2(o.sn_2);
        }
        nstB[c] = make_float2(-stB[c].x, -stB[c].y);
        C[c] = make_float2(env * cc, envy * cy);
        Sn[c] = make_float2(env * sc, envy * sy);
    }
    // Kubo-Toyabe: G(t) e^{-t/tau} = E / 3 + (1 - x) e23,  x = (Delta t)^2,
    // e23 = 2/3 exp(-t/tau - x/2), stepped like a Gaussian envelope
    float2 e23 = bc2(0.f), g2k = bc2(0.f), nkr2 = bc2(0.f), kr2 = bc2(0.f);
    if (KT) {
        const float ex = 0.666666667f * hc.kt_cenv *
                         ex2_approx(-fmaf(nn0, hc.kt_b_hi, fmaf(nf0, hc.kt_a_hi, fmaf(nn0, hc.kt_b_lo, nf0 * hc.kt_a_lo))));
        float gq1;
        if (carried) {
            gq1 = carry->gqk1;
            g2k = carry->g2k;
        } else {
            const GaussSeed sd = gauss_seed(hc.kt_a_hi, hc.kt_a_lo, hc.kt_b_hi, hc.kt_b_lo, n0);
            gq1 = sd.q1;
            g2k = make_float2(sd.r0, sd.r1);
        }
        if (carry) carry->gqk1 = fmaf(gq1, hc.kt_qs, gq1 + hc.kt_qs);
        e23 = make_float2(ex, fmaf(ex, gq1, ex));
        if (carry) carry->g2k = fma2(g2k, bc2(hc.kt_qs2), add2(g2k, bc2(hc.kt_qs2)));
        const float r2 = hc.kt_rate * hc.kt_rate;
        kr2 = bc2(r2);
        nkr2 = bc2(-r2);
    }
    if (carry) carry->valid = true;
    const float tsx = fmaf(nf0, dtf, t0f);
    const float2 ts = make_float2(tsx, tsx + dtf);
    const float2 dt2 = bc2(2.f * dtf);
    const float2 m1 = bc2(-1.f), one = bc2(1.f), third = bc2(0.333333333f), m3 = bc2(-3.f);
#pragma unroll
    for (int j = 0; j < kBinsPerThread / 2; ++j) {
        const float2 t = fma2(bc2((float)j), dt2, ts);
        const float2 tt = NEED_TT ? mul2(t, t) : bc2(0.f);
        float2 Cb[NOSC > 0 ? NOSC : 1], Sb[NOSC > 0 ? NOSC : 1];
        float2 sp = bc2(0.f), slg = bc2(0.f);  // stretched line: (lambda t)^beta and log2(lambda t) per lane
#pragma unroll
        for (int c = 0; c < NOSC; ++c) {
            if (NS && c >= CS) {
                const float2 u = mul2(bc2(hc.osc[c].rate), t);
                const float lx = lg2_approx(u.x), ly = lg2_approx(u.y);
                sp = make_float2(u.x > 0.f ? ex2_approx(hc.osc[c].beta * lx) : 0.f,
                                 u.y > 0.f ? ex2_approx(hc.osc[c].beta * ly) : 0.f);
                slg = make_float2(u.x > 0.f ? lx : 0.f, u.y > 0.f ? ly : 0.f);
                const float2 ev = mul2(E, make_float2(ex2_approx(-1.44269504088896341f * sp.x),
                                                      ex2_approx(-1.44269504088896341f * sp.y)));
                Cb[c] = mul2(ev, C[c]);
                Sb[c] = mul2(ev, Sn[c]);
            } else {
                Cb[c] = C[c];
                Sb[c] = Sn[c];
            }
        }
        float2 S = E;
#pragma unroll
        for (int c = 0; c < NOSC; ++c) S = fma2(bc2(hc.osc[c].amp), Cb[c], S);
        float2 GE = bc2(0.f), xm3 = bc2(0.f);
        if (KT) {
            const float2 omx = fma2(nkr2, tt, one);  // 1 - (Delta t)^2
            GE = fma2(e23, omx, mul2(E, third));
            if (MODE == kGrad) xm3 = fma2(kr2, tt, m3);  // (Delta t)^2 - 3
            S = fma2(bc2(hc.kt_amp), GE, S);
        }
        // N0 carried as an FP32 pair so its rounding does not bias every bin
        const float2 N = fma2(n0p, S, fma2(n0lo, S, bkg));
        const float2 dv = make_float2(d[2 * j], d[2 * j + 1]);
        const bool vx = FULL || n0 + 2 * j < M, vy = FULL || n0 + 2 * j + 1 < M;
        float2 wq;
        if (obj == MUSR_CHI2) {
            float2 w = make_float2(rcp_approx(fmaxf(dv.x, 1.f)), rcp_approx(fmaxf(dv.y, 1.f)));
            if (!FULL) w = make_float2(vx ? w.x : 0.f, vy ? w.y : 0.f);
            const float2 r = fma2(N, m1, dv);
            wq = mul2(r, w);
            acc[0] = fma2(r, wq, acc[0]);
        } else {
            float term[2], wl[2];
            const float dl[2] = {dv.x, dv.y}, Nl[2] = {N.x, N.y};
            const bool vl[2] = {vx, vy};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                term[h] = wl[h] = 0.f;
                if (!vl[h]) continue;
                if (dl[h] > 0.f) {
                    if (!(Nl[h] > 0.f)) {
                        bad = true;
                    } else {
                        const float rN = rcp_approx(Nl[h]);
                        const float rho = (dl[h] - Nl[h]) * rN;
                        float hh;
                        if (fabsf(rho) < 0.125f) {
                            // sum_{j>=2} (-1)^j rho^j / (j (j-1)), truncated after j = 9
                            hh = fmaf(rho, -1.f / 72.f, 1.f / 56.f);
                            hh = fmaf(rho, hh, -1.f / 42.f);
                            hh = fmaf(rho, hh, 1.f / 30.f);
                            hh = fmaf(rho, hh, -1.f / 20.f);
                            hh = fmaf(rho, hh, 1.f / 12.f);
                            hh = fmaf(rho, hh, -1.f / 6.f);
                            hh = fmaf(rho, hh, 0.5f);
                            hh = hh * rho * rho;
                        } else {
                            const float u = log1pf(rho);
                            hh = fmaf(rho, u, u - rho);
                        }
                        term[h] = 2.f * Nl[h] * hh;
                        wl[h] = rho;
                    }
                } else {
                    if (!(Nl[h] >= 0.f)) bad = true;
                    term[h] = 2.f * Nl[h];
                    wl[h] = -1.f;
                }
            }
            acc[0] = add2(acc[0], make_float2(term[0], term[1]));
            wq = make_float2(wl[0], wl[1]);
        }
        if (MODE == kGrad) {
            const float2 wt = mul2(wq, t);
            const float2 wtt = NEED_TT ? mul2(wq, tt) : bc2(0.f);
            acc[1] = fma2(wq, S, acc[1]);
            acc[2] = add2(acc[2], wq);
#pragma unroll
            for (int c = 0; c < NOSC; ++c) {
                acc[3 + 4 * c] = fma2(wq, Cb[c], acc[3 + 4 * c]);
                if (NS && c >= CS) {
                    const float2 pc = mul2(sp, Cb[c]);
                    acc[4 + 4 * c] = fma2(wq, pc, acc[4 + 4 * c]);
                    acc[1 + RB] = fma2(wq, mul2(pc, slg), acc[1 + RB]);
                } else {
                    acc[4 + 4 * c] = fma2(c < NE ? wt : wtt, Cb[c], acc[4 + 4 * c]);
                }
                acc[5 + 4 * c] = fma2(wt, Sb[c], acc[5 + 4 * c]);
                acc[6 + 4 * c] = fma2(wq, Sb[c], acc[6 + 4 * c]);
            }
            if (KT) {
                acc[1 + RK] = fma2(wq, GE, acc[1 + RK]);
                acc[2 + RK] = fma2(mul2(wtt, xm3), e23, acc[2 + RK]);
            }
        }
        // step every lane by two bins
        E = fma2(E, qE2, E);
#pragma unroll
        for (int c = 0; c < NOSC; ++c) {
            const float2 c2 = fma2(C[c], stA[c], fma2(Sn[c], nstB[c], C[c]));
            const float2 s2 = fma2(Sn[c], stA[c], fma2(C[c], stB[c], Sn[c]));
            if (c < NE || c >= CS) {
                C[c] = c2;
                Sn[c] = s2;
            } else {
                C[c] = fma2(c2, g2[c], c2);
                Sn[c] = fma2(s2, g2[c], s2);
                const float2 q2 = bc2(hc.osc[c].q2);
                g2[c] = fma2(g2[c], q2, add2(g2[c], q2));
            }
        }
        if (KT) {
            e23 = fma2(e23, g2k, e23);
            const float2 q2 = bc2(hc.kt_q2);
            g2k = fma2(g2k, q2, add2(g2k, q2));
        }
    }
}

template <int NE, int NG, int NS, int KT, int MODE, int NACC>
__device__ __forceinline__ void eval_pair(const HistConst& hc, int n0, int M, const float (&d)[kBinsPerThread],
                                          float E0, int obj, float dtf, float t0f, float2 (&acc)[NACC], bool& bad,
                                          G2Carry<NE + NG + NS>* carry) {
    if (n0 + kBinsPerThread <= M)
        eval_pair_body<NE, NG, NS, KT, MODE, NACC, true>(hc, n0, M, d, E0, obj, dtf, t0f, acc, bad, carry);
    else
        eval_pair_body<NE, NG, NS, KT, MODE, NACC, false>(hc, n0, M, d, E0, obj, dtf, t0f, acc, bad, carry);
}

// The per-histogram constant of accumulator a (see eval_chunk): 1 for the
// objective; -2 f_r for the gradient of role r (dN/d role = f_r x_r, the
// accumulators hold sum (wg / -2) x_r); 2 f_r1 f_r2 for the Gauss-Newton
// entry of roles (r1, r2) (they hold sum (wh / 2) x_r1 x_r2).
template <int NE, int NG, int NS, int KT>
__device__ __forceinline__ float role_factor_r(const HistConst& hc, int r) {
    constexpr int NOSC = NE + NG + NS;
    if (r < 2) return 1.f;
    const float n0p = hc.n0;
    if (r < 2 + 4 * NOSC) {
        const int c = (r - 2) >> 2, j = (r - 2) & 3;
        const OscConst& o = hc.osc[c];
        const float an = -o.amp * n0p;
        if (j == 0) return n0p;
        if (j == 1) {
            if (c < NE) return an;
            if (c < NE + NG) return o.rate * an;
            // stretched: d(lambda t)^beta / d lambda = beta (lambda t)^beta / lambda (x = (lambda t)^beta x
            // the line); 0 at lambda = 0, where the envelope is 1 on both sides
            return o.rate != 0.f ? an * o.beta / o.rate : 0.f;
        }
        if (j == 2) return an * hc.kfreq;
        return an;
    }
    if (NS && r == 2 + 4 * NOSC) {
        // stretched exponent: d(lambda t)^beta / d beta = ln 2 log2(lambda t) (lambda t)^beta
        return -hc.osc[NE + NG].amp * n0p * 0.693147180559945309f;
    }
    if (r == 2 + 4 * NOSC + NS) return n0p;
    // x = t^2 (x_KT - 3) e23 with e23 = 2/3 of the envelope
    return n0p * hc.kt_amp * hc.kt_rate;
}

template <int NE, int NG, int NS, int KT, int MODE>
__device__ __forceinline__ float acc_factor(const HistConst& hc, int a) {
    constexpr int R = 2 + 4 * (NE + NG + NS) + NS + 2 * KT;
    if (a == 0 || MODE < kGrad) return 1.f;
    if (a <= R) return -2.f * role_factor_r<NE, NG, NS, KT>(hc, a - 1);
    // Gauss-Newton entry: upper triangle of (r1, r2), row by row
    int q = a - 1 - R, r1 = 0;
    while (q >= R - r1) {
        q -= R - r1;
        ++r1;
    }
    return 2.f * role_factor_r<NE, NG, NS, KT>(hc, r1) * role_factor_r<NE, NG, NS, KT>(hc, r1 + q);
}


// ---- deterministic fixed-point accumulation ----
// Each warp's role-factored FP32 totals become the integers X = v 2^48 (exact
// for |v| >= 2^-24, truncated below; |v| < 2^72); a block sums its warps' X
// in shared memory and adds the block total, split into three 42-bit limbs,
// with 64-bit atomic adds whose results are unused (no round trip).  Integer
// addition is associative, so the per-histogram totals are bitwise the same
// whatever order the blocks finish in; with at most 2^22 additions per
// accumulator no limb overflows.  Sums of totals (the map to theta) are formed on the
// integers too, and each output is converted to FP64 once: no FP64 addition
// chains (FP64 has a long latency on this GPU).
constexpr int kFixFracBits = 48;
constexpr int kFixLimbBits = 42;

// X = v 2^48 as an integer (truncated below 2^-48); false when v is not
// finite or |v| >= 2^72 (X = 0 then).  A block sums at most 8 such values, so
// its total stays below 2^123.
__device__ __forceinline__ bool fix_of(float v, __int128& X) {
    const unsigned bits = __float_as_uint(v);
    const int e = (int)((bits >> 23) & 0xffu);
    X = 0;
    if (e == 0xff || e >= 127 + 72) return false;
    if (e == 0) return true;  // zero or below 2^-126: nothing at the 2^-48 resolution
    const long long m = (long long)((bits & 0x7fffffu) | 0x800000u);
    const int sh = e - 150 + kFixFracBits;  // |v| 2^48 = m 2^sh
    X = sh >= 0 ? ((__int128)m << sh) : (__int128)(m >> min(-sh, 63));
    if (bits >> 31) X = -X;
    return true;
}

// Add X to three 42-bit limbs (atomics whose results are unused).
__device__ __forceinline__ void fix_add(unsigned long long* limbs, __int128 X) {
    const unsigned long long mask = (1ull << kFixLimbBits) - 1ull;
    atomicAdd(limbs + 0, (unsigned long long)X & mask);
    atomicAdd(limbs + 1, (unsigned long long)(X >> kFixLimbBits) & mask);
    atomicAdd(limbs + 2, (unsigned long long)(long long)(X >> (2 * kFixLimbBits)));
}

// The integer total of three accumulated limbs.
__device__ __forceinline__ __int128 fix_total(unsigned long long l0, unsigned long long l1, unsigned long long l2) {
    return (__int128)l0 + ((__int128)l1 << kFixLimbBits) + ((__int128)(long long)l2 << (2 * kFixLimbBits));
}

// X / 2^48 in FP64, rounded once to nearest (ties to even), assembled with
// integer operations only: the FP64 pipe (conversions included) is narrow
// on this GPU, and the tail converts thousands of sums at once.
// |X| < 2^127, so the result is a normal double.
__device__ __forceinline__ double fix_to_double(__int128 X) {
    if (X == 0) return 0.0;
    const unsigned long long sign = X < 0 ? (1ull << 63) : 0ull;
    const unsigned __int128 u = X < 0 ? (unsigned __int128)(-X) : (unsigned __int128)X;
    const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
    const int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);  // leading one
    int e = msb - kFixFracBits;                                                     // result exponent
    unsigned long long m;                                                           // 53-bit significand
    if (msb <= 52) {
        m = (unsigned long long)(u << (52 - msb));
    } else {
        const int sh = msb - 52;  // 1 .. 74 bits dropped
        m = (unsigned long long)(u >> sh);
        const unsigned __int128 rem = u & (((unsigned __int128)1 << sh) - 1);
        const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
        if (rem > half || (rem == half && (m & 1ull))) {
            ++m;
            if (m >> 53) {  // carried into a new leading bit
                m >>= 1;
                ++e;
            }
        }
    }
    return __longlong_as_double(
        (long long)(sign | ((unsigned long long)(e + 1023) << 52) | (m & ((1ull << 52) - 1ull))));
}

template <int NE, int NG, int NS, int KT, int MODE>
__global__ void __launch_bounds__(MODE == kGN ? kMaxThreadsGn : kMaxThreads) eval_kernel(const __grid_constant__ EvalParams p) {
    constexpr int NOSC = NE + NG + NS;
    constexpr int R = 2 + 4 * NOSC + NS + 2 * KT;
    constexpr int NACC = MODE == kValue ? 1 : MODE == kGrad ? 1 + R : MODE == kGN ? 1 + R + R * (R + 1) / 2 : 1;
    constexpr int G = kBinsPerThread;

    __shared__ HistConst hc;
    constexpr int KW = MODE == kGN ? kMaxWarpsGn : kMaxWarps;
    __shared__ float red[KW][NACC];
    __shared__ __align__(16) __int128 xred[KW][NACC];
    __shared__ int s_last;
    extern __shared__ __align__(16) unsigned char dyn_smem[];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    // programmatic dependent launch: this grid may be scheduled while the
    // previous one in the stream finishes.  Nothing that grid may write is
    // read before it has completed (griddepcontrol.wait); what is read earlier
    // is immutable (pre_wait, see EvalParams).  Every thread waits before the
    // block's first global write.
    // the tile's launch parameters are read together, ahead of the wait (a
    // launch's parameters never change): their first reads miss the constant
    // cache, and one miss after another would add up
    const int pre_wait = MODE == kModel ? 0 : p.pre_wait;
    const unsigned uni_tph = (unsigned)p.uni_tph, uni_chunks = (unsigned)p.uni_chunks;
    const int uni_nbins = p.uni_nbins;
    const int64_t uni_stride = p.uni_stride;
    const float* const data = p.data;
    if (pre_wait == 0) asm volatile("griddepcontrol.wait;" ::: "memory");
    // the next grid in the stream may be launched at once: its blocks take SM
    // slots as this grid's blocks leave them (every kernel of this library
    // waits before it touches what this grid writes)
    asm volatile("griddepcontrol.launch_dependents;");
    const int tile = blockIdx.x;
    int k, M, tstart, tend;
    const float* hdata;
    if (uni_tph > 0) {
        // chunk range [j C / T, (j + 1) C / T) in 32-bit arithmetic: the host
        // sets this form only when C T < 2^32
        const unsigned kk = (unsigned)tile / uni_tph, j = (unsigned)tile - kk * uni_tph;
        k = (int)kk;
        M = uni_nbins;
        tstart = (int)(j * uni_chunks / uni_tph) * G;
        tend = (int)((j + 1) * uni_chunks / uni_tph) * G;
        hdata = data + (int64_t)k * uni_stride;
    } else {
        k = p.tile_hist[tile];
        M = p.hist_nbins[k];
        tstart = p.tile_start[tile];
        tend = p.tile_end[tile];
        hdata = p.data + p.hist_off[k];
    }
    // a tile is a range of 8-bin chunks; thread t takes chunks t, t + blockDim, ...
    // (every chunk that starts below tend starts below M)
    const int stripe = (int)blockDim.x * G;
    int n0 = tstart + (int)threadIdx.x * G;

    // the histogram's theta entries (one per role slot, warp 0) come first,
    // alone: queued behind the block's data loads their round trip doubled.
    // theta is inline in the launch parameters for host calls; the role rows
    // are immutable, theta in device memory is read after the wait
    __shared__ double s_th[2 * kMaxRoles];
    if (threadIdx.x < 2 * kMaxRoles) {
        const double* theta = p.theta_inline_n ? p.theta_inline : p.theta;
        const int32_t* rt = (p.rt_inline ? p.rt_rows : p.role_theta) + (size_t)k * kMaxRoles * 2;
        const int i = rt[threadIdx.x];
        if (pre_wait == 1) asm volatile("griddepcontrol.wait;" ::: "memory");
        s_th[threadIdx.x] = i >= 0 ? theta[i] : 0.0;
    }
    __syncthreads();

    // then the first chunk's loads (counts and the lifetime factor at its
    // start), whose latency overlaps the staging arithmetic
    float d[G];
    float E0 = 0.f;
    if (n0 < tend) E0 = __ldg(p.etab + (n0 >> 3));
    if (MODE != kModel && n0 < tend) {
        const float4* src = reinterpret_cast<const float4*>(hdata + n0);
        float4 a = __ldg(src), b = __ldg(src + 1);
        d[0] = a.x; d[1] = a.y; d[2] = a.z; d[3] = a.w;
        d[4] = b.x; d[5] = b.y; d[6] = b.z; d[7] = b.w;
    } else {
#pragma unroll
        for (int g = 0; g < G; ++g) d[g] = 0.f;
    }

    // stage histogram k's constants: one part per warp, so the parts' latency
    // chains overlap, and a part's independent function evaluations spread
    // over the warp's lanes
    {
        constexpr int NPART = stage_parts<NE, NG, NS, KT>();
        for (int part = warp; part < NPART; part += nwarps)
            stage_part<NE, NG, NS, KT>(part, ThetaGathered{s_th}, p.rc, hc, (int)blockDim.x * G, lane);
    }
    __syncthreads();

    // the tail's map into shared memory (when it fits), copied while the bins
    // are evaluated: only the last block reads it, but no block knows yet
    // whether it is last, and the copies cost no registers
    const int n_rows = p.csr_row ? p.n_rows : p.n_out;
    const int cw1 = (n_rows + 1 + 3) >> 2, cw2 = (p.n_src + 3) >> 2;  // 16-byte pieces of pointers, sources
    int32_t* tbl = reinterpret_cast<int32_t*>(dyn_smem + (p.hsum_in_smem ? sizeof(__int128) * p.K * NACC : 0));
    if (MODE != kModel && p.csr_in_smem) {
        const int cw3 = p.csr_row ? (n_rows + 3) >> 2 : 0;
        for (int c = threadIdx.x; c < cw1 + cw2 + cw3; c += blockDim.x) {
            if (c < cw1) cp_async16(tbl + 4 * c, p.csr_ptr + 4 * c);
            else if (c < cw1 + cw2) cp_async16(tbl + 4 * c, p.csr_src + 4 * (c - cw1));
            else cp_async16(tbl + 4 * c, p.csr_row + 4 * (c - cw1 - cw2));
        }
    }

    float acc[NACC];
#pragma unroll
    for (int a = 0; a < NACC; ++a) acc[a] = 0.f;
    bool bad = false;

    if constexpr (MODE == kValue || MODE == kGrad) {
        // packed lanes (even / odd bins), lane sums added after the chunks
        float2 acc2[NACC];
#pragma unroll
        for (int a = 0; a < NACC; ++a) acc2[a] = make_float2(0.f, 0.f);
        G2Carry<NOSC> carry;
        carry.valid = false;
        for (; n0 < tend; n0 += stripe) {
            // the next chunk's loads are in flight while this one is evaluated
            const int n1 = n0 + stripe;
            float dn[G];
            float En = 0.f;
            if (n1 < tend) {
                const float4* src = reinterpret_cast<const float4*>(hdata + n1);
                float4 a = __ldg(src), b = __ldg(src + 1);
                dn[0] = a.x; dn[1] = a.y; dn[2] = a.z; dn[3] = a.w;
                dn[4] = b.x; dn[5] = b.y; dn[6] = b.z; dn[7] = b.w;
                En = __ldg(p.etab + (n1 >> 3));
            } else {
#pragma unroll
                for (int g = 0; g < G; ++g) dn[g] = 0.f;
            }
            eval_pair<NE, NG, NS, KT, MODE, NACC>(hc, n0, M, d, E0, p.obj, (float)p.dt, (float)p.t0, acc2, bad, &carry);
#pragma unroll
            for (int g = 0; g < G; ++g) d[g] = dn[g];
            E0 = En;
        }
#pragma unroll
        for (int a = 0; a < NACC; ++a) acc[a] = acc2[a].x + acc2[a].y;
    } else {
        GqCarry<NOSC> carry;
        carry.valid = false;
        GnAcc<R> gnacc;
        gnacc.zero();
        for (; n0 < tend; n0 += stripe) {
            // the next chunk's loads are in flight while this one is evaluated
            const int n1 = n0 + stripe;
            float dn[G];
            float En = 0.f;
            if (n1 < tend) {
                En = __ldg(p.etab + (n1 >> 3));
                if (MODE != kModel) {
                    const float4* src = reinterpret_cast<const float4*>(hdata + n1);
                    float4 a = __ldg(src), b = __ldg(src + 1);
                    dn[0] = a.x; dn[1] = a.y; dn[2] = a.z; dn[3] = a.w;
                    dn[4] = b.x; dn[5] = b.y; dn[6] = b.z; dn[7] = b.w;
                }
            }
            if (MODE == kModel || !(n1 < tend)) {
#pragma unroll
                for (int g = 0; g < G; ++g) dn[g] = 0.f;
            }
            eval_chunk<NE, NG, NS, KT, MODE, NACC>(hc, n0, M, d, E0, p.obj, (float)p.dt, (float)p.t0, acc, bad,
                                                   MODE == kModel ? p.model_out + p.model_off[k] : nullptr, &carry,
                                                   &gnacc);
#pragma unroll
            for (int g = 0; g < G; ++g) d[g] = dn[g];
            E0 = En;
        }
        if constexpr (MODE == kGN) gn_scatter(gnacc, acc);
    }
    if (MODE == kModel) return;

    // ---- block: FP32 warp sums scaled by the histogram's role factors, as
    // fixed-point integers (one thread per warp and accumulator) summed over
    // the warps, one fixed-point add per accumulator into the histogram's
    // totals ----
    if constexpr (NACC >= 32) {
        // many accumulators (Gauss-Newton): reduce-scatter, each lane stores its share
        WarpSplit<NACC> ws;
#pragma unroll
        for (int a = 0; a < WarpSplit<NACC>::NP; ++a) ws.v[a] = a < NACC ? acc[a] : 0.f;
        warp_reduce_scatter<NACC>(ws, lane);
        const int a0 = WarpSplit<NACC>::PER * bitrev5(lane);
#pragma unroll
        for (int j = 0; j < WarpSplit<NACC>::PER; ++j)
            if (a0 + j < NACC) red[warp][a0 + j] = ws.v[j];
    } else {
        warp_sum<NACC>(acc);
        if (lane == 0) {
#pragma unroll
            for (int a = 0; a < NACC; ++a) red[warp][a] = acc[a];
        }
    }
    const int any_bad = __syncthreads_or(bad);
    // the previous grid has completed (its limbs and counters reset, its
    // output written) before this block adds anything
    if (pre_wait != 0) asm volatile("griddepcontrol.wait;" ::: "memory");
    {
        unsigned flag = (threadIdx.x == 0 && any_bad) ? 1u : 0u;
        for (int q = threadIdx.x; q < nwarps * NACC; q += blockDim.x) {
            const int w = q / NACC, a = q - w * NACC;
            const float f = (MODE >= kGrad && a > 0) ? acc_factor<NE, NG, NS, KT, MODE>(hc, a) : 1.f;
            if (!fix_of(red[w][a] * f, xred[w][a])) flag |= 2u;
        }
        __syncthreads();
        for (int a = threadIdx.x; a < NACC; a += blockDim.x) {
            __int128 X = 0;
            for (int w = 0; w < nwarps; ++w) X += xred[w][a];
            fix_add(p.facc + ((size_t)k * NACC + a) * 3, X);
        }
        if (flag) atomicOr(p.flags, flag);
    }
    // the barrier orders every thread's adds before thread 0's ticket, a
    // release (cumulative: it publishes what the barrier made thread 0
    // observe) and, for the last block, an acquire of every other block's
    // adds, which the second barrier passes on to the whole block
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(p.global_count) : "memory");
        s_last = (prev == gridDim.x - 1u);
    }
    __syncthreads();
    cp_async_wait_all();  // this thread's map copies (long complete)
    if (!s_last) return;

    // ---- last block: per-histogram integer totals (their limbs zeroed for the
    // next launch), then theta via the map (CSR rows of sources; value and
    // gradient: a row per output; Gauss-Newton: a row per output that has
    // sources, whose output index the row table gives), summed as integers.
    // The map is in shared memory already when it fits (copied during the
    // bins); the limbs come in batches of up to eight totals a thread with the
    // whole batch in flight ----
    const unsigned fl = *reinterpret_cast<volatile unsigned*>(p.flags);
    __int128* hsum = p.hsum_in_smem ? reinterpret_cast<__int128*>(dyn_smem) : p.hist_sum;
    const int32_t* cptr = p.csr_in_smem ? tbl : p.csr_ptr;
    const int32_t* csrc = p.csr_in_smem ? tbl + 4 * cw1 : p.csr_src;
    const int32_t* crow = p.csr_row ? (p.csr_in_smem ? tbl + 4 * (cw1 + cw2) : p.csr_row) : nullptr;
    {
        const int n_tot = p.K * NACC;
        for (int base = threadIdx.x; base < n_tot; base += 8 * blockDim.x) {
            unsigned long long lv[8][3];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = base + u * blockDim.x;
                if (i < n_tot) {
                    const unsigned long long* l = p.facc + (size_t)i * 3;
                    lv[u][0] = __ldcg(l);
                    lv[u][1] = __ldcg(l + 1);
                    lv[u][2] = __ldcg(l + 2);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = base + u * blockDim.x;
                if (i < n_tot) {
                    hsum[i] = fix_total(lv[u][0], lv[u][1], lv[u][2]);
                    // the limbs start from zero for the next launch
                    unsigned long long* l = p.facc + (size_t)i * 3;
                    l[0] = 0ull;
                    l[1] = 0ull;
                    l[2] = 0ull;
                }
            }
        }
        // outputs without a row are 0 (the run's own buffers already hold 0
        // there); ordered before the rows' stores by the barrier below
        if (p.csr_row && !p.out_zeroed)
            for (int o = threadIdx.x; o < p.n_out; o += blockDim.x) p.out[o] = 0.0;
    }
    __syncthreads();
    // every block has taken its ticket and set its flags, and every thread
    // here has read the flags (the barrier performs its load): reset both for
    // the next launch
    if (threadIdx.x == 0) {
        *p.global_count = 0u;
        *p.flags = 0u;
    }
    const bool overflow = (fl & 2u) != 0u;
    double out0 = 0.0;  // thread 0 keeps the objective: out may be host memory, slow to read back
    // L = 1, 2 or 4 lanes a row (as many as one pass over the rows allows),
    // each summing every L-th of its sources (integer sums are exact in any
    // order), their partial sums added across the L lanes
    const int nl = (int)blockDim.x >= 4 * n_rows ? 4 : (int)blockDim.x >= 2 * n_rows ? 2 : 1;
    const int lsh = nl >> 1;  // log2(nl)
    for (int rb = 0; rb < n_rows; rb += (int)blockDim.x >> lsh) {
        const int r = rb + ((int)threadIdx.x >> lsh), q = (int)threadIdx.x & (nl - 1);
        const bool live = r < n_rows;
        __int128 X = 0;
        if (live) {
            const int e = cptr[r + 1];
#pragma unroll 4
            for (int j = cptr[r] + q; j < e; j += nl) X += hsum[csrc[j]];
        }
        unsigned long long lo = (unsigned long long)X;
        long long hi = (long long)(X >> 64);
        for (int m = 1; m < nl; m <<= 1) {
            const unsigned long long lo2 = __shfl_xor_sync(0xffffffffu, lo, m);
            const long long hi2 = __shfl_xor_sync(0xffffffffu, hi, m);
            const unsigned long long sum = lo + lo2;
            hi = hi + hi2 + (sum < lo ? 1ll : 0ll);
            lo = sum;
        }
        if (live && q == 0) {
            const int o = crow ? crow[r] : r;
            // Gauss-Newton entries: the rows carry H[i][j], i <= j; the sum is
            // stored at [i][j] and [j][i]
            int om = -1;
            if (MODE == kGN && o > p.P) {
                const int oh = o - 1 - p.P, i = oh / p.P, j = oh - i * p.P;
                if (i < j) om = 1 + p.P + j * p.P + i;
            }
            // NaN when a warp total was not representable (not finite, or >= 2^72)
            const double v = overflow ? __longlong_as_double(0x7ff8000000000000ll)
                                      : fix_to_double(((__int128)hi << 64) | (__int128)lo);
            p.out[o] = v;
            if (om >= 0) p.out[om] = v;
            if (o == 0) out0 = v;
        }
    }
    // results in mapped host memory: visible to the host before the status that announces them
    if (p.status_sys_fence) __threadfence_system();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned f = fl & 1u;
        if (!isfinite(out0)) f |= 2u;
        if (p.status_out) {
            if (p.status_sys_fence) __threadfence_system();
            *reinterpret_cast<volatile int32_t*>(p.status_out) = (int32_t)f;
        }
    }
}

// Launch the objective kernel.  n_tiles == 0 only sets the kernel's
// shared-memory attribute (call it outside capture); n_tiles < 0 only reports
// the kernel's resident blocks per SM.
template <int NE, int NG, int NS, int KT, int MODE>
cudaError_t launch_one(int threads, int n_tiles, cudaStream_t stream, const EvalParams& p) {
    const size_t smem = (size_t)p.smem_bytes;
    if (n_tiles < 0) {
        // occupancy query: resident blocks per SM written to p.status_out (host int)
        int nb = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, eval_kernel<NE, NG, NS, KT, MODE>,
                                                                      threads, smem);
        *reinterpret_cast<int*>(p.status_out) = nb;
        return e;
    }
    if (n_tiles == 0) {
        // the attribute is per kernel, shared by every run: only ever raise it
        // (to the device's opt-in maximum), never lower it below another run's need
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, eval_kernel<NE, NG, NS, KT, MODE>);
        if (e != cudaSuccess) return e;
        const int avail = optin - (int)fa.sharedSizeBytes;
        if ((int)smem > avail) return cudaErrorInvalidValue;
        if (fa.maxDynamicSharedSizeBytes >= avail) return cudaSuccess;
        return cudaFuncSetAttribute(eval_kernel<NE, NG, NS, KT, MODE>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, avail);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_tiles);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, eval_kernel<NE, NG, NS, KT, MODE>, p);
}

}  // namespace musr
