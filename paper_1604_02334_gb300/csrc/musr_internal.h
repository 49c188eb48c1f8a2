// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "musr.h"

namespace musr {

constexpr int kMaxOsc = 2;                         // precession lines per run
constexpr int kMaxRoles = 2 + 4 * kMaxOsc + 1 + 2; // N0, bkg, 4 per line, stretching exponent, 2 for KT
constexpr int kBinsPerThread = 8;                  // consecutive bins per thread (2 x float4)
constexpr int kMaxThreads = 256;                   // block size upper bound
constexpr int kMaxWarps = kMaxThreads / 32;
// the objective kernel's Gauss-Newton mode may also run 384-thread blocks:
// at ~170 registers a thread only 256 fit otherwise, 8 warps an SM
constexpr int kMaxThreadsGn = 384;
constexpr int kMaxWarpsGn = kMaxThreadsGn / 32;
constexpr int kInlineParams = 256;                 // theta passed inside the launch parameters
constexpr int kInlineRoleHist = 32;                // role-map rows passed inside the launch parameters

// Per-histogram constants of the theory, staged into shared memory by every
// block for its histogram at the start of an evaluation (the paper's kernel
// keeps the parameter / map values in shared memory for the same reason,
// Sec. 4.2.2: every thread reads them many times).
struct OscConst {
    // q: per-bin expm1 step of an exponential envelope; for a Gaussian
    // envelope expm1 of the per-bin change of its step ratio, 2^(-2 b) - 1
    float amp, rate, cenv, a_hi, a_lo, b_hi, b_lo, q, cm1, sn;
    float qs;    // Gaussian envelope: 2^(-2 b stripe) - 1, the change of its step ratio over one stripe
    float beta;  // stretched envelope: exponent beta (rate holds lambda)
    // two-bin steps (the packed kernels step even and odd bins as two lanes):
    // q2 = expm1 of the exponential envelope over 2 bins, or for a Gaussian
    // envelope the change of its 2-bin ratio, 2^(-8 b) - 1; cm1_2 / sn_2 the
    // rotation over 2 bins; qs2 = 2^(-4 b stripe) - 1
    float q2, cm1_2, sn_2, qs2;
    unsigned long long ph0, step;  // phase at bin 0 and per bin, 64-bit fixed-point turns
    unsigned long long step_s;     // phase advance over one stripe (a thread's next chunk)
};

struct HistConst {
    float n0, n0_lo, bkg, qE;  // N0 = n0 + n0_lo (FP32 pair); qE = expm1(-dt / tau), the lifetime step
    float qE2;    // expm1(-2 dt / tau)
    float kfreq;  // 2 pi gamma: dN/dB = dN/d(omega) * 2 pi gamma
    OscConst osc[kMaxOsc];
    float kt_amp, kt_rate, kt_cenv, kt_a_hi, kt_a_lo, kt_b_hi, kt_b_lo, kt_q, kt_qs;
    float kt_q2, kt_qs2;  // the Kubo-Toyabe envelope's 2-bin ratio constants (as OscConst q2, qs2)
};

// Theta-independent constants of a run's time grid, prepared on the host in
// FP64 / exact integer arithmetic (float2 = double-float hi, lo).
struct RunConst {
    float2 inv_tau, dt, dt_log2e, t0, t0_dt_log2e, half_dt2_log2e;
    float qE, kfreq;  // lifetime step expm1(-dt / tau), 2 pi gamma
    int t0_zero;
    ulonglong2 turns_per_bin;  // gamma * dt as unsigned 64.64 fixed point (turns per gauss)
    ulonglong2 turns_at_t0;    // gamma * t0
    ulonglong2 inv_two_pi;     // 1 / (2 pi)
};

// Kernel "signature": how many precession lines of each relaxation kind and
// whether a static Gaussian Kubo-Toyabe term is present.  Exponential lines
// come first in the kernel's role order, Gaussian lines second, the stretched
// line (at most one) third; roles: N0, bkg, 4 per line (amplitude, rate,
// field, phase), the stretched line's exponent, then the Kubo-Toyabe pair.
struct Signature {
    int ne = 0, ng = 0, ns = 0, kt = 0;
    int n_osc() const { return ne + ng + ns; }
    int roles() const { return 2 + 4 * n_osc() + ns + 2 * kt; }
    bool operator==(const Signature& o) const { return ne == o.ne && ng == o.ng && ns == o.ns && kt == o.kt; }
    bool operator!=(const Signature& o) const { return !(*this == o); }
};

// A run's components in the kernels' role order: the signature, the component
// index of every line (exponential, Gaussian, stretched) and of the
// Kubo-Toyabe term (-1 if none).
struct RoleLayout {
    Signature sig;
    int osc[kMaxOsc] = {};
    int kt = -1;
};

// Validate the component list against the map width and order it; MUSR_OK,
// MUSR_EINVAL (bad kind or column) or MUSR_ENOTSUP (too many lines).
inline int role_layout(const musr_component* comp, int n_comp, int map_width, RoleLayout& L) {
    int e[kMaxOsc], g[kMaxOsc], st = -1;
    L = RoleLayout{};
    for (int c = 0; c < n_comp; ++c) {
        const musr_component& m = comp[c];
        const int cols[6] = {m.amp, m.rate, m.field, m.field2, m.phase, m.kind == MUSR_TF_STRETCHED ? m.beta : -1};
        for (int j = 0; j < 6; ++j)
            if (cols[j] < -1 || cols[j] >= map_width) return MUSR_EINVAL;
        if (m.kind == MUSR_TF_EXP || m.kind == MUSR_TF_GAUSS || m.kind == MUSR_TF_STRETCHED) {
            if (L.sig.n_osc() >= kMaxOsc) return MUSR_ENOTSUP;
            if (m.kind == MUSR_TF_EXP) e[L.sig.ne++] = c;
            else if (m.kind == MUSR_TF_GAUSS) g[L.sig.ng++] = c;
            else if (st >= 0) return MUSR_ENOTSUP;
            else st = c, L.sig.ns = 1;
        } else if (m.kind == MUSR_KT_STATIC_GAUSS) {
            if (L.kt >= 0) return MUSR_ENOTSUP;
            L.kt = c;
        } else {
            return MUSR_EINVAL;
        }
    }
    L.sig.kt = L.kt >= 0;
    int n = 0;
    for (int i = 0; i < L.sig.ne; ++i) L.osc[n++] = e[i];
    for (int i = 0; i < L.sig.ng; ++i) L.osc[n++] = g[i];
    if (st >= 0) L.osc[n++] = st;
    return MUSR_OK;
}

// Role row of one histogram: rt[2 r] and rt[2 r + 1] are the theta indices
// (or -1) whose sum is role r; map_row is the histogram's map row.
inline void role_row(const RoleLayout& L, const musr_component* comp, const int32_t* map_row, int32_t* rt) {
    auto col = [&](int c) { return c < 0 ? -1 : map_row[c]; };
    for (int i = 0; i < kMaxRoles * 2; ++i) rt[i] = -1;
    rt[0] = col(0);
    rt[2] = col(1);
    const int no = L.sig.n_osc();
    for (int s = 0; s < no; ++s) {
        const musr_component& m = comp[L.osc[s]];
        int32_t* q = rt + 2 * (2 + 4 * s);
        q[0] = col(m.amp);
        q[2] = col(m.rate);
        q[4] = col(m.field);
        q[5] = col(m.field2);
        q[6] = col(m.phase);
        if (m.kind == MUSR_TF_STRETCHED) rt[2 * (2 + 4 * no)] = col(m.beta);
    }
    if (L.kt >= 0) {
        const musr_component& m = comp[L.kt];
        int32_t* q = rt + 2 * (2 + 4 * no + L.sig.ns);
        q[0] = col(m.amp);
        q[2] = col(m.rate);
    }
}

// Every signature a kernel is compiled for: X(NE, NG, NS, KT) with at most
// kMaxOsc lines of which at most one stretched, with and without the
// Kubo-Toyabe term.
#define MUSR_FOR_EACH_SIGNATURE(X)                                                    \
    X(0, 0, 0, 0) X(0, 0, 0, 1) X(1, 0, 0, 0) X(1, 0, 0, 1) X(0, 1, 0, 0) X(0, 1, 0, 1) \
    X(2, 0, 0, 0) X(2, 0, 0, 1) X(1, 1, 0, 0) X(1, 1, 0, 1) X(0, 2, 0, 0) X(0, 2, 0, 1) \
    X(0, 0, 1, 0) X(0, 0, 1, 1) X(1, 0, 1, 0) X(1, 0, 1, 1) X(0, 1, 1, 0) X(0, 1, 1, 1)

// Evaluation modes (kernel template parameter).
enum Mode { kValue = 0, kGrad = 1, kGN = 2, kModel = 3, kSum = 4 };

inline int n_acc(int mode, int R) {
    return mode == kValue ? 1 : mode == kGrad ? 1 + R : mode == kGN ? 1 + R + R * (R + 1) / 2 : 0;
}

// Everything one launch of the objective kernel reads or writes.
struct EvalParams {
    // run layout (device)
    const float* data;            // padded, histogram-major
    const int64_t* hist_off;      // [K] float offset of histogram k in data
    const int32_t* hist_nbins;    // [K]
    const int32_t* tile_hist;     // [n_tiles]
    const int32_t* tile_start;    // [n_tiles] first bin of the tile
    const int32_t* tile_end;      // [n_tiles] bin past the tile (a multiple of 8, or the padded length)
    const int32_t* role_theta;    // [K][kMaxRoles][2] theta indices (or -1) per role
    const double* theta;          // [P] on the device (device calls)
    RunConst rc;
    double t0, dt, inv_tau, gamma;
    int K, P, obj;
    // reduction scratch
    unsigned long long* facc;     // [K][nacc][3] fixed-point limbs of the per-histogram sums (self-resetting)
    __int128* hist_sum;           // [K][nacc] integer totals (when they do not fit in shared memory)
    unsigned* global_count;       // [1]   (self-resetting)
    unsigned* flags;              // [1]   (self-resetting)
    const int32_t* csr_ptr;       // [n_out + 1]
    const int32_t* csr_src;       // sources: k * nacc + acc
    int n_out;
    int n_src;                    // csr_src length
    const int32_t* csr_row;       // [n_rows] output index of each map row, or null: row r is output r
    int n_rows;                   // map rows (when csr_row is set)
    int out_zeroed;               // 1: out holds 0 wherever the map has no row (else the kernel zeroes it)
    int hsum_in_smem, csr_in_smem;
    int smem_bytes;               // dynamic shared memory of the objective kernel
    double* out;                  // [n_out]
    int32_t* status_out;          // [1] or null
    int status_sys_fence;         // 1: out / status_out are mapped host memory the host polls
    int theta_inline_n;           // > 0: theta_inline holds theta (host calls)
    double theta_inline[kInlineParams];
    // What a block may read before the grid-dependency wait of programmatic
    // dependent launch (the previous kernel in the stream may still run):
    //   0  nothing (the wait comes first)
    //   1  the run's tables, counts and lifetime factors (written only by
    //      calls that synchronise before returning); theta after the wait
    //   2  those and theta (inline): staging and the whole bin loop run before
    //      the wait, which then precedes the block's first global write
    // Never 2 in kModel, whose bin loop writes the model.
    int pre_wait;
    // Equal-length histograms (the common layout): tile b belongs to histogram
    // k = b / uni_tph and covers chunks [j C / uni_tph, (j + 1) C / uni_tph)
    // of it, j = b mod uni_tph, C = uni_chunks (8-bin chunks per histogram);
    // histogram k starts at float k * uni_stride.  The tile and histogram
    // tables are then not read, which takes two dependent memory round trips
    // off the start of every block.  0: use the tables.  Set only when
    // C * uni_tph < 2^32 (the kernel divides in 32-bit arithmetic).
    int uni_tph, uni_chunks, uni_nbins;
    int64_t uni_stride;
    // role -> theta rows of the first kInlineRoleHist histograms (when K fits),
    // so staging waits for theta alone
    int rt_inline;
    int32_t rt_rows[kInlineRoleHist * kMaxRoles * 2];
    // model output (kModel)
    float* model_out;
    const int64_t* model_off;     // [K] offsets into model_out
    // lifetime factor exp(-t/tau) at every 8-bin chunk start (see lifetime_table_len)
    const float* etab;
};
// kernel parameters are limited to 32764 bytes
static_assert(sizeof(EvalParams) <= 32000, "EvalParams exceeds the kernel parameter space");


// 32-bit words of the objective kernel's map in shared memory: row pointers
// (n_rows + 1), sources, and the row -> output table when there is one, each
// array starting on a 16-byte boundary (the kernel copies them with cp.async).
inline size_t csr_smem_words(int64_t n_rows, int64_t n_src, bool row_table) {
    auto r4 = [](int64_t n) { return (size_t)((n + 3) / 4 * 4); };
    return r4(n_rows + 1) + r4(n_src) + (row_table ? r4(n_rows) : 0);
}

// Launch the objective kernel for a signature / mode (eval_*.cu).
cudaError_t launch_eval(const Signature& sig, int mode, int threads, int n_tiles,
                        cudaStream_t stream, const EvalParams& p);

// Map a CUDA error to a status code, remembering its name for
// musr_last_cuda_error() (per host thread).
int cuda_status(cudaError_t e);

// Theta-independent constants of a time grid (host, FP64 / integer).
RunConst make_run_const(double t0, double dt, double tau, double gamma);

// The lifetime factor exp(-(t0 + 8 j dt) / tau) at every chunk start j of a
// time grid, evaluated in FP64 and rounded once to FP32.  The kernels seed
// their per-bin lifetime recurrence from it: the factor multiplies every bin
// of the model, so a seed computed in FP32 (an SFU exp2 of a rounded
// argument) would bias N coherently over many bins, and the objective's
// gradient sums, which cancel ~100-fold, would inherit that bias amplified.
inline int64_t lifetime_table_len(int64_t max_bins) { return max_bins / kBinsPerThread + 2; }
cudaError_t fill_lifetime_table(float* tab, int64_t n, double t0, double dt, double tau, cudaStream_t st);

}  // namespace musr
