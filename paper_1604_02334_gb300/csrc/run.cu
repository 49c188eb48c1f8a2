// Run handles and the single-run entry points of the C ABI (include/musr.h).
//
// A run owns the device copy of its histograms (uploaded once, Sec. 4.2), its
// tiling plan, the role -> theta table derived from the map array (Sec. 4.2.1)
// and the scratch of the fused reduction.  Host-pointer calls replay a CUDA
// graph (theta upload -> objective kernel -> result download) so one call
// costs one graph launch and one synchronisation.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <utility>
#include <vector>

#include "eval_kernel.cuh"
#include "musr_internal.h"
#include "run_impl.h"

namespace musr {

cudaError_t launch_eval_mode0(const Signature&, int, int, cudaStream_t, const EvalParams&);
cudaError_t launch_eval_mode1(const Signature&, int, int, cudaStream_t, const EvalParams&);
cudaError_t launch_eval_mode2(const Signature&, int, int, cudaStream_t, const EvalParams&);
cudaError_t launch_eval_mode3(const Signature&, int, int, cudaStream_t, const EvalParams&);

cudaError_t launch_eval(const Signature& s, int mode, int threads, int n_tiles, cudaStream_t st,
                        const EvalParams& p) {
    switch (mode) {
        case kValue: return launch_eval_mode0(s, threads, n_tiles, st, p);
        case kGrad: return launch_eval_mode1(s, threads, n_tiles, st, p);
        case kGN: return launch_eval_mode2(s, threads, n_tiles, st, p);
        case kModel: return launch_eval_mode3(s, threads, n_tiles, st, p);
    }
    return cudaErrorInvalidValue;
}

namespace {
// |a * b| as unsigned 64.64 fixed point, exactly (truncated at 2^-64), from the
// two doubles' significands; *neg receives the product's sign.
ulonglong2 product_fixed(double a, double b, int* neg) {
    *neg = 0;
    if (a == 0.0 || b == 0.0 || !isfinite(a) || !isfinite(b)) return ulonglong2{0ull, 0ull};
    *neg = (a < 0.0) != (b < 0.0);
    int ea, eb;
    const double fa = frexp(fabs(a), &ea), fb = frexp(fabs(b), &eb);  // [0.5, 1)
    const unsigned long long ma = (unsigned long long)ldexp(fa, 53);
    const unsigned long long mb = (unsigned long long)ldexp(fb, 53);
    const unsigned __int128 P = (unsigned __int128)ma * mb;  // |ab| = P * 2^(ea + eb - 106)
    const int sh = ea + eb - 106 + 64;                       // |ab| * 2^64 = P * 2^sh
    unsigned __int128 V;
    if (sh >= 0) V = sh < 22 ? P << sh : ~(unsigned __int128)0;  // |ab| < 2^64 in practice
    else V = -sh < 128 ? P >> -sh : 0;
    return ulonglong2{(unsigned long long)(V >> 64), (unsigned long long)V};
}

float2 df_split(double v) {
    const float hi = (float)v;
    return float2{hi, (float)(v - (double)hi)};
}
}  // namespace

RunConst make_run_const(double t0, double dt, double tau, double gamma) {
    const double LOG2E = 1.4426950408889634074;
    RunConst rc;
    memset(&rc, 0, sizeof(rc));
    rc.inv_tau = df_split(1.0 / tau);
    rc.dt = df_split(dt);
    rc.dt_log2e = df_split(dt * LOG2E);
    rc.t0 = df_split(t0);
    rc.t0_dt_log2e = df_split(t0 * dt * LOG2E);
    rc.half_dt2_log2e = df_split(0.5 * dt * dt * LOG2E);
    rc.qE = (float)expm1(-dt / tau);
    rc.kfreq = (float)(2.0 * 3.14159265358979323846 * gamma);
    rc.t0_zero = t0 == 0.0;
    int neg = 0;
    rc.turns_per_bin = product_fixed(gamma, dt, &neg);  // dt > 0; gamma >= 0 is checked at plan
    rc.turns_at_t0 = product_fixed(gamma, t0, &neg);    // t0 >= 0 is checked at plan
    // 1 / (2 pi) = 0.1591549430918953357688837633725143620344596457404564487476673440588967976342265350901138027662530859560728427267...
    rc.inv_two_pi = ulonglong2{0ull, 2935890503282001226ull};
    return rc;
}

thread_local const char* g_last_cuda_error = "none";

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return MUSR_OK;
    g_last_cuda_error = cudaGetErrorName(e);
    if (e == cudaErrorMemoryAllocation) return MUSR_ENOMEM;
    return MUSR_ECUDA;
}

__global__ void lifetime_table_kernel(float* tab, int64_t n, double t0, double dt8, double inv_tau) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        tab[j] = (float)exp(-(t0 + (double)j * dt8) * inv_tau);
}

cudaError_t fill_lifetime_table(float* tab, int64_t n, double t0, double dt, double tau, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, 1024);
    lifetime_table_kernel<<<blocks, threads, 0, st>>>(tab, n, t0, dt * kBinsPerThread, 1.0 / tau);
    return cudaGetLastError();
}

// Copy concatenated counts (FP32 or FP64, device) into the padded FP32 layout.
__global__ void pack_data_kernel(const void* src, int is_f64, const int64_t* src_off,
                                 const int64_t* dst_off, const int32_t* nbins, int K, float* dst) {
    const int k = blockIdx.y;
    if (k >= K) return;
    const int M = nbins[k];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
        const int64_t s = src_off[k] + i;
        dst[dst_off[k] + i] = is_f64 ? (float)static_cast<const double*>(src)[s]
                                     : static_cast<const float*>(src)[s];
    }
}

}  // namespace musr

using namespace musr;

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// host calls: the status word's value while the kernel runs, and how long the
// host polls it before it blocks in a stream synchronisation instead
constexpr int32_t kStatusPending = INT32_MIN;
constexpr int kStatusSpinUs = 2000;
constexpr int kMinThreadsGn = 128;
// the tiling planner's cost of one wave of blocks, in bins of one SM's work:
// a block's staging and reduction take ~2 us, which an SM spends on ~7000
// bins of the gradient mode
constexpr int64_t kWaveCostBins = 7000;

}  // namespace

// ---------------------------------------------------------------------------
// plan construction
// ---------------------------------------------------------------------------
int musr_run_s::plan(const musr_run_desc* d) {
    K = d->n_hist;
    P = d->n_params;
    W = d->map_width;
    t0 = d->t0_us;
    dt = d->dt_us;
    tau = d->tau_us;
    gamma = d->gamma_mhz_per_g;
    if (K < 0 || P < 0 || P > kMaxParams || W < 2 || W > 32 || d->n_comp < 0) return MUSR_EINVAL;
    if (!(dt > 0.0) || !(tau > 0.0) || !(t0 >= 0.0) || !isfinite(t0) || !(gamma >= 0.0) ||
        !isfinite(gamma))
        return MUSR_EINVAL;
    rc = make_run_const(t0, dt, tau, gamma);
    if (K > 0 && (!d->n_bins || !d->map)) return MUSR_EINVAL;
    if (d->n_comp > 0 && !d->comp) return MUSR_EINVAL;
    n_bins.assign(d->n_bins, d->n_bins + K);
    map.assign(d->map, d->map + (size_t)K * W);
    comp.assign(d->comp, d->comp + d->n_comp);
    // function array: compiled once, evaluated per call on the host
    F = d->n_funcs;
    if (F < 0 || (F > 0 && !d->funcs)) return MUSR_EINVAL;
    if (F > kMaxFuncs || P + F > kMaxParams) return MUSR_ENOTSUP;
    funcs.resize(F);
    for (int j = 0; j < F; ++j)
        if (compile_host_expr(d->funcs[j], P, funcs[j]) != MUSR_OK) return MUSR_EINVAL;
    Pk = P + F;
    // the kernels' map: entry -2 - j (function j) becomes slot P + j
    std::vector<int32_t> kmap(map);
    total_bins = 0;
    for (int k = 0; k < K; ++k) {
        if (n_bins[k] < 0) return MUSR_EINVAL;
        if (n_bins[k] > (int64_t(1) << 24)) return MUSR_ENOTSUP;
        total_bins += n_bins[k];
        for (int c = 0; c < W; ++c) {
            const int i = map[(size_t)k * W + c];
            if (i < -1 - F || i >= P) return MUSR_EINVAL;
            if (i <= -2) kmap[(size_t)k * W + c] = P + (-2 - i);
        }
    }
    // signature (exponential, Gaussian, stretched lines, Kubo-Toyabe) and the role -> theta table
    RoleLayout rl;
    const int st = role_layout(comp.data(), (int)comp.size(), W, rl);
    if (st != MUSR_OK) return st;
    sig = rl.sig;
    R = sig.roles();
    role_theta.assign((size_t)K * kMaxRoles * 2, -1);
    for (int k = 0; k < K; ++k)
        role_row(rl, comp.data(), kmap.data() + (size_t)k * W, role_theta.data() + (size_t)k * kMaxRoles * 2);
    // data layout: every histogram at a multiple of 8 floats
    hist_off.assign(K, 0);
    model_off.assign(K, 0);
    int64_t off = 0, moff = 0;
    for (int k = 0; k < K; ++k) {
        hist_off[k] = off;
        model_off[k] = moff;
        off += round_up(n_bins[k], 8);
        moff += n_bins[k];
    }
    data_floats = (size_t)off + 8;
    return MUSR_OK;
}

std::vector<int64_t> musr_run_s::tiles_per_hist(int t, int64_t target) const {
    int64_t total = 0;
    for (int k = 0; k < K; ++k) total += (n_bins[k] + kBinsPerThread - 1) / kBinsPerThread;
    std::vector<int64_t> tph(K, 1);
    if (total == 0) return tph;
    for (int k = 0; k < K; ++k) {
        const int64_t ck = (n_bins[k] + kBinsPerThread - 1) / kBinsPerThread;
        const int64_t share = ck * target / total;              // proportional, rounded down
        tph[k] = std::max<int64_t>(1, std::min(share, ck / t));  // >= one chunk per thread
    }
    return tph;
}

// Tiles of near-equal chunk ranges, tph[k] of them over histogram k.
void musr_run_s::build_tiles(Tiling& T, int t, const std::vector<int64_t>& tph) const {
    T.threads = t;
    T.tile_hist.clear();
    T.tile_start.clear();
    T.tile_end.clear();
    bool uniform = K > 0;
    for (int k = 0; k < K; ++k) {
        const int64_t ck = (n_bins[k] + kBinsPerThread - 1) / kBinsPerThread;
        for (int64_t j = 0; j < tph[k]; ++j) {
            T.tile_hist.push_back(k);
            T.tile_start.push_back((int32_t)(j * ck / tph[k] * kBinsPerThread));
            T.tile_end.push_back((int32_t)((j + 1) * ck / tph[k] * kBinsPerThread));
        }
        if (n_bins[k] != n_bins[0] || tph[k] != tph[0]) uniform = false;
    }
    T.n_tiles = (int)T.tile_hist.size();
    T.uni_tph = uniform ? (int)tph[0] : 0;
}

// Dynamic shared memory of the objective kernel's tail for a mode: the
// per-histogram totals and the CSR, each when it fits.
int musr_run_s::tail_smem(int mode, int* hsum_smem, int* csr_smem) const {
    const int nacc = n_acc(mode, R);
    const size_t csr_words = csr_smem_words(n_rows[mode], n_src[mode], mode == kGN);
    const int hs = (size_t)K * nacc * 16 <= 64 * 1024;
    const int cs = csr_words * 4 <= 64 * 1024;
    if (hsum_smem) *hsum_smem = hs;
    if (csr_smem) *csr_smem = cs;
    return (int)(16 * (hs ? (size_t)K * nacc : 0) + 4 * (cs ? csr_words : 0));
}

// CSR of output entry -> (histogram, accumulator) sources for one mode.
void musr_run_s::build_csr(int mode, std::vector<int32_t>& ptr, std::vector<int32_t>& src,
                            std::vector<int32_t>& rows) const {
    const int nacc = n_acc(mode, R);
    const int64_t n_out = 1 + (mode >= kGrad ? Pk : 0) + (mode == kGN ? (int64_t)Pk * Pk : 0);
    std::vector<std::pair<int64_t, int32_t>> e;
    for (int k = 0; k < K; ++k) {
        const int32_t* rt = role_theta.data() + (size_t)k * kMaxRoles * 2;
        const int32_t base = k * nacc;
        e.push_back({0, base});
        if (mode >= kGrad) {
            for (int r = 0; r < R; ++r)
                for (int j = 0; j < 2; ++j)
                    if (rt[2 * r + j] >= 0) e.push_back({1 + rt[2 * r + j], base + 1 + r});
        }
        if (mode == kGN) {
            // H[i][j] and H[j][i] have the same sources: only entries with
            // i <= j get them (the kernels store each sum at both places)
            int a = 1 + R;
            for (int r1 = 0; r1 < R; ++r1)
                for (int r2 = r1; r2 < R; ++r2, ++a)
                    for (int j1 = 0; j1 < 2; ++j1)
                        for (int j2 = 0; j2 < 2; ++j2) {
                            const int i = rt[2 * r1 + j1], jj = rt[2 * r2 + j2];
                            if (i < 0 || jj < 0) continue;
                            if (i <= jj) e.push_back({1 + Pk + (int64_t)i * Pk + jj, base + a});
                            if (r1 != r2 && jj <= i) e.push_back({1 + Pk + (int64_t)jj * Pk + i, base + a});
                        }
        }
    }
    std::stable_sort(e.begin(), e.end(),
                     [](const std::pair<int64_t, int32_t>& x, const std::pair<int64_t, int32_t>& y) {
                         return x.first < y.first;
                     });
    src.resize(e.size());
    for (size_t i = 0; i < e.size(); ++i) src[i] = e[i].second;
    rows.clear();
    if (mode != kGN) {
        // one row per output
        ptr.assign(n_out + 1, 0);
        for (size_t i = 0; i < e.size(); ++i) ptr[e[i].first + 1]++;
        for (int64_t o = 0; o < n_out; ++o) ptr[o + 1] += ptr[o];
        return;
    }
    // Gauss-Newton: one row per output that has sources (most of the P^2
    // entries have none); rows[r] is its output index
    ptr.assign(1, 0);
    for (size_t i = 0; i < e.size(); ++i) {
        if (i == 0 || e[i].first != e[i - 1].first) {
            rows.push_back((int32_t)e[i].first);
            ptr.push_back(ptr.back());
        }
        ptr.back()++;
    }
}

// One device allocation holds every per-run array; pieces are 256-byte aligned.
struct Arena {
    size_t size = 0;
    template <class T>
    size_t take(size_t n) {
        size_t o = size;
        size = round_up((int64_t)(size + n * sizeof(T)), 256);
        return o;
    }
};

int musr_run_s::allocate() {
    const int nacc_max = n_acc(Pk <= kMaxGnParams ? kGN : kGrad, R);
    std::vector<int32_t> ptr[3], src[3], rows[3];
    for (int m = 0; m < 3; ++m) {
        if (m == kGN && Pk > kMaxGnParams) continue;
        build_csr(m, ptr[m], src[m], rows[m]);
        n_out[m] = (int)(1 + (m >= kGrad ? Pk : 0) + (m == kGN ? (int64_t)Pk * Pk : 0));
        n_rows[m] = (int)ptr[m].size() - 1;
        n_src[m] = (int)src[m].size();
    }
    // per-mode tiling: for each block size, one wave of resident blocks
    // (resident count from the kernel's occupancy; more waves only for runs
    // beyond 8 chunks a thread) as tiles of near-equal chunk ranges spread over
    // the histograms in proportion to their bins; the block size whose busiest
    // SM holds the fewest bins wins, with a cost per wave for the blocks' fixed
    // work (staging, reduction)
    int dev_sms = 152;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, device);
    for (int m = 0; m < 4; ++m) {
        if (m == kGN && Pk > kMaxGnParams) continue;
        // the Gauss-Newton mode reduces 1 + R + R(R+1)/2 accumulators per block and
        // maps ~P^2 outputs in its tail: blocks of fewer than kMinThreadsGn threads
        // spend more on that than they save in parallelism
        int t_min = m == kGN ? kMinThreadsGn : 32;
        // runs that fill the GPU keep a warp per staging part, so the parts'
        // latency chains run side by side
        if (total_bins >= (int64_t)2 * dev_sms * kMaxThreads * kBinsPerThread)
            while (t_min < kMaxThreads && t_min < 32 * (2 + 2 * sig.n_osc())) t_min <<= 1;
        int best_t = kMaxThreads;
        int64_t best_slots = 1;
        std::vector<int64_t> best_tph;
        int64_t best_cost = INT64_MAX;
        // block sizes 256, 128, ..., t_min; the Gauss-Newton mode tries 384 first
        std::vector<int> sizes;
        if (m == kGN) sizes.push_back(kMaxThreadsGn);
        for (int t = kMaxThreads; t >= t_min; t >>= 1) sizes.push_back(t);
        for (const int t : sizes) {
            int per_sm = 0;
            EvalParams q;
            memset(&q, 0, sizeof(q));
            q.smem_bytes = m == kModel ? 0 : tail_smem(m, nullptr, nullptr);
            q.status_out = reinterpret_cast<int32_t*>(&per_sm);
            if (launch_eval(sig, m, t, -1, stream, q) != cudaSuccess || per_sm < 1) per_sm = 1;
            const int64_t slots = (int64_t)per_sm * dev_sms;
            // one wave of tiles, or several when a run is too large for a wave
            // of tiles of at most 8 chunks a thread
            int64_t total = 0;
            for (int k = 0; k < K; ++k) total += (n_bins[k] + kBinsPerThread - 1) / kBinsPerThread;
            const int64_t waves = std::max<int64_t>(1, (total + slots * t * 8 - 1) / (slots * t * 8));
            const std::vector<int64_t> tph = tiles_per_hist(t, slots * waves);
            int64_t n = 0, max_chunks = 0;
            for (int k = 0; k < K; ++k) {
                const int64_t ck = (n_bins[k] + kBinsPerThread - 1) / kBinsPerThread;
                n += tph[k];
                max_chunks = std::max(max_chunks, (ck + tph[k] - 1) / tph[k]);
            }
            // the busiest SM's bins (its blocks' chunks, spread over its warps)
            const int64_t per_sm_tiles = (n + dev_sms - 1) / dev_sms;
            const int64_t cost = per_sm_tiles * max_chunks * kBinsPerThread + kWaveCostBins * ((n + slots - 1) / slots);
            if (cost < best_cost) {
                best_cost = cost;
                best_t = t;
                best_tph = tph;
                best_slots = slots;
            }
        }
        build_tiles(tl[m], best_t, best_tph);
        // Queued evaluations overlap one another, so their rate is set by the
        // SM time their blocks hold, not by one launch's busiest SM: every
        // tile fewer is one staging and one reduction fewer, and the next
        // evaluations' blocks fill the slots a launch leaves free.  When the
        // planner's tiles fit in one wave they take tiles of twice the chunks
        // a thread (up to 16), else as many chunks a thread (measured: longer
        // blocks lengthen the chain of dependent reductions once a launch
        // spans waves), in the fewest tiles that give no thread more.  One
        // launch alone is better served by the planner's tiles, which spread
        // the bins over more SMs.
        if (tl[m].uni_tph > 0) {
            const int64_t ck = (n_bins[0] + kBinsPerThread - 1) / kBinsPerThread, t = tl[m].threads;
            const int64_t per_thread = ((ck + tl[m].uni_tph - 1) / tl[m].uni_tph + t - 1) / t;
            const bool one_wave = tl[m].n_tiles <= best_slots;
            const int64_t pq = one_wave && per_thread <= 8 ? 2 * per_thread : per_thread;
            tl[m].uni_tph_queued = (int)std::max<int64_t>(1, (ck + pq * t - 1) / (pq * t));
        }

        if (m < 3) smem_bytes[m] = tail_smem(m, &hsum_in_smem[m], &csr_in_smem[m]);
    }
    const int n_out_max = n_out[Pk <= kMaxGnParams ? kGN : kGrad];
    Arena A;
    const size_t o_data = A.take<float>(data_floats);
    const size_t o_hoff = A.take<int64_t>(K + 1);
    const size_t o_moff = A.take<int64_t>(K + 1);
    const size_t o_nb = A.take<int32_t>(K + 1);
    size_t o_th[4], o_ts[4], o_te[4];
    for (int m = 0; m < 4; ++m) {
        o_th[m] = A.take<int32_t>(tl[m].n_tiles + 1);
        o_ts[m] = A.take<int32_t>(tl[m].n_tiles + 1);
        o_te[m] = A.take<int32_t>(tl[m].n_tiles + 1);
    }
    const size_t o_rt = A.take<int32_t>(role_theta.size() + 1);
    const size_t o_map = A.take<int32_t>(map.size() + 1);  // raw map rows (user theories)
    int64_t max_m = 0;
    for (int k = 0; k < K; ++k) max_m = std::max(max_m, n_bins[k]);
    etab_len = lifetime_table_len(max_m);
    const size_t o_etab = A.take<float>((size_t)etab_len);
    size_t o_ptr[3], o_src[3], o_row[3];
    for (int m = 0; m < 3; ++m) {
        o_ptr[m] = A.take<int32_t>(ptr[m].size() + 1);
        o_src[m] = A.take<int32_t>(src[m].size() + 1);
        o_row[m] = A.take<int32_t>(rows[m].size() + 1);
    }
    const size_t o_facc = A.take<unsigned long long>((size_t)(K + 1) * nacc_max * 3);
    const size_t o_hsum = A.take<__int128>((size_t)(K + 1) * nacc_max);
    const size_t o_cnt = A.take<unsigned>(4);
    const size_t o_theta = A.take<double>(Pk + 1);
    const size_t o_out = A.take<double>(n_out_max + 1);
    const size_t o_status = A.take<int32_t>(2);
    const size_t o_tmp = A.take<double>(Pk + 1);
    if (cudaMalloc(&arena, A.size) != cudaSuccess) {
        arena = nullptr;
        return MUSR_ENOMEM;
    }
    char* b = static_cast<char*>(arena);
    d_data = reinterpret_cast<float*>(b + o_data);
    d_hist_off = reinterpret_cast<int64_t*>(b + o_hoff);
    d_model_off = reinterpret_cast<int64_t*>(b + o_moff);
    d_hist_nbins = reinterpret_cast<int32_t*>(b + o_nb);
    for (int m = 0; m < 4; ++m) {
        tl[m].d_tile_hist = reinterpret_cast<int32_t*>(b + o_th[m]);
        tl[m].d_tile_start = reinterpret_cast<int32_t*>(b + o_ts[m]);
        tl[m].d_tile_end = reinterpret_cast<int32_t*>(b + o_te[m]);
    }
    d_role_theta = reinterpret_cast<int32_t*>(b + o_rt);
    d_map = reinterpret_cast<int32_t*>(b + o_map);
    d_etab = reinterpret_cast<float*>(b + o_etab);
    for (int m = 0; m < 3; ++m) {
        d_csr_ptr[m] = reinterpret_cast<int32_t*>(b + o_ptr[m]);
        d_csr_src[m] = reinterpret_cast<int32_t*>(b + o_src[m]);
        d_csr_row[m] = rows[m].empty() ? nullptr : reinterpret_cast<int32_t*>(b + o_row[m]);
    }
    d_facc = reinterpret_cast<unsigned long long*>(b + o_facc);
    d_hist_sum = reinterpret_cast<__int128*>(b + o_hsum);
    d_counters = reinterpret_cast<unsigned*>(b + o_cnt);
    d_theta = reinterpret_cast<double*>(b + o_theta);
    d_out = reinterpret_cast<double*>(b + o_out);
    d_status = reinterpret_cast<int32_t*>(b + o_status);
    d_theta_tmp = reinterpret_cast<double*>(b + o_tmp);

    // host staging, mapped so the kernel writes host-call results straight
    // into it (no copy node after the kernel)
    if (cudaHostAlloc(&h_pinned, sizeof(double) * (size_t)(Pk + 1 + n_out_max + 1) + 64,
                      cudaHostAllocMapped) != cudaSuccess) {
        h_pinned = nullptr;
        return MUSR_ENOMEM;
    }
    h_theta = static_cast<double*>(h_pinned);
    h_out = h_theta + Pk + 1;
    // outputs the Gauss-Newton map never writes (entries without sources) stay 0
    memset(h_out, 0, sizeof(double) * (n_out_max + 1));
    h_status = reinterpret_cast<int32_t*>(h_out + n_out_max + 1);
    if (cudaHostGetDevicePointer((void**)&hd_out, h_out, 0) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&hd_status, h_status, 0) != cudaSuccess)
        return MUSR_ECUDA;

    // static tables
    std::vector<int32_t> nb32(K);
    for (int k = 0; k < K; ++k) nb32[k] = (int32_t)n_bins[k];
    cudaError_t e = cudaSuccess;
    auto up = [&](void* dst, const void* src_, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src_, bytes, cudaMemcpyHostToDevice, stream);
    };
    up(d_hist_off, hist_off.data(), sizeof(int64_t) * K);
    up(d_model_off, model_off.data(), sizeof(int64_t) * K);
    up(d_hist_nbins, nb32.data(), sizeof(int32_t) * K);
    for (int m = 0; m < 4; ++m) {
        const Tiling& T = tl[m];
        if (T.n_tiles == 0) continue;  // a mode without a tiling (Gauss-Newton beyond kMaxGnParams)
        up(T.d_tile_hist, T.tile_hist.data(), sizeof(int32_t) * T.n_tiles);
        up(T.d_tile_start, T.tile_start.data(), sizeof(int32_t) * T.n_tiles);
        up(T.d_tile_end, T.tile_end.data(), sizeof(int32_t) * T.n_tiles);
    }
    up(d_role_theta, role_theta.data(), sizeof(int32_t) * role_theta.size());
    up(d_map, map.data(), sizeof(int32_t) * map.size());
    if (e == cudaSuccess) e = fill_lifetime_table(d_etab, etab_len, t0, dt, tau, stream);
    for (int m = 0; m < 3; ++m) {
        up(d_csr_ptr[m], ptr[m].data(), sizeof(int32_t) * ptr[m].size());
        up(d_csr_src[m], src[m].data(), sizeof(int32_t) * src[m].size());
        if (d_csr_row[m]) up(d_csr_row[m], rows[m].data(), sizeof(int32_t) * rows[m].size());
    }
    // opt the kernels whose reduction tail needs > 48 KB of shared memory in
    for (int m = 0; m < 3 && e == cudaSuccess; ++m) {
        if (m == kGN && Pk > kMaxGnParams) continue;
        EvalParams q = params(MUSR_CHI2, m, d_theta, d_out, d_status);
        e = launch_eval(sig, m, tl[m].threads, 0, stream, q);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(d_counters, 0, sizeof(unsigned) * 4, stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(d_facc, 0, sizeof(unsigned long long) * (size_t)(K + 1) * nacc_max * 3, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_data, 0, sizeof(float) * data_floats, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_out, 0, sizeof(double) * (n_out_max + 1), stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    return cuda_status(e);
}

int musr_run_s::upload(int dtype, const void* data, int on_device) {
    if (!data) return MUSR_OK;
    if (dtype != MUSR_F32 && dtype != MUSR_F64) return MUSR_EINVAL;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        // straight copies into the padded layout (padding stays 0): consecutive
        // histograms whose device and host offsets differ by the same amount
        // (every one before them a multiple of 8 bins long) go in one copy
        const float* src = static_cast<const float*>(data);
        std::vector<float> conv;
        if (dtype == MUSR_F64) {
            conv.resize((size_t)total_bins);
            const double* d64 = static_cast<const double*>(data);
            for (int64_t i = 0; i < total_bins; ++i) conv[i] = (float)d64[i];
            src = conv.data();
        }
        int64_t s = 0, run_src = 0, run_dst = 0, run_len = 0;
        auto flush = [&]() {
            if (run_len > 0 && e == cudaSuccess)
                e = cudaMemcpyAsync(d_data + run_dst, src + run_src, sizeof(float) * run_len,
                                    cudaMemcpyHostToDevice, stream);
            run_len = 0;
        };
        for (int k = 0; k < K; ++k) {
            if (n_bins[k]) {
                if (run_len > 0 && hist_off[k] == run_dst + run_len && s == run_src + run_len) {
                    run_len += n_bins[k];
                } else {
                    flush();
                    run_src = s;
                    run_dst = hist_off[k];
                    run_len = n_bins[k];
                }
            }
            s += n_bins[k];
        }
        flush();
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        return cuda_status(e);
    }
    // device source: pack with a kernel (source offsets in a small temporary buffer)
    std::vector<int64_t> src_off(K);
    int64_t s = 0;
    for (int k = 0; k < K; ++k) {
        src_off[k] = s;
        s += n_bins[k];
    }
    int64_t* d_src_off = nullptr;
    e = cudaMalloc(&d_src_off, sizeof(int64_t) * (K + 1));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_src_off, src_off.data(), sizeof(int64_t) * K, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && K > 0) {
        dim3 grid(64, K);
        pack_data_kernel<<<grid, 256, 0, stream>>>(data, dtype == MUSR_F64, d_src_off, d_hist_off,
                                                   d_hist_nbins, K, d_data);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (d_src_off) cudaFree(d_src_off);
    return cuda_status(e);
}

EvalParams musr_run_s::params(int obj, int mode, const double* theta_dev, double* out_dev,
                              int32_t* status_dev) const {
    EvalParams p;
    memset(&p, 0, sizeof(p));
    p.data = d_data;
    p.hist_off = d_hist_off;
    p.hist_nbins = d_hist_nbins;
    const Tiling& T = tl[mode];
    p.tile_hist = T.d_tile_hist;
    p.tile_start = T.d_tile_start;
    p.tile_end = T.d_tile_end;
    p.role_theta = d_role_theta;
    p.theta = theta_dev;
    p.t0 = t0;
    p.dt = dt;
    p.inv_tau = 1.0 / tau;
    p.gamma = gamma;
    p.rc = rc;
    p.K = K;
    p.P = Pk;
    p.obj = obj;
    p.facc = d_facc;
    p.hist_sum = d_hist_sum;
    p.global_count = d_counters;
    p.flags = d_counters + 1;
    const int m = mode == kModel ? kValue : mode;
    p.csr_ptr = d_csr_ptr[m];
    p.csr_src = d_csr_src[m];
    p.n_out = n_out[m];
    p.n_src = n_src[m];
    p.csr_row = d_csr_row[m];
    p.n_rows = n_rows[m];
    // the run's own output buffers hold 0 wherever the map writes nothing
    p.out_zeroed = out_dev == d_out || out_dev == hd_out;
    p.hsum_in_smem = hsum_in_smem[m];
    p.csr_in_smem = csr_in_smem[m];
    p.smem_bytes = mode == kModel ? 0 : smem_bytes[m];
    // equal-length histograms: tiles and offsets by arithmetic (see EvalParams)
    if (T.uni_tph > 0 && n_bins[0] + kBinsPerThread * (int64_t)T.threads < (int64_t)1 << 30 &&
        (n_bins[0] + kBinsPerThread - 1) / kBinsPerThread * (int64_t)T.uni_tph < (int64_t)1 << 32) {
        p.uni_tph = T.uni_tph;
        p.uni_chunks = (int)((n_bins[0] + kBinsPerThread - 1) / kBinsPerThread);
        p.uni_nbins = (int)n_bins[0];
        p.uni_stride = round_up(n_bins[0], 8);
    }
    if (K <= kInlineRoleHist) {
        p.rt_inline = 1;
        memcpy(p.rt_rows, role_theta.data(), sizeof(int32_t) * (size_t)K * kMaxRoles * 2);
    }
    p.out = out_dev;
    p.status_out = status_dev;
    p.model_off = d_model_off;
    p.etab = d_etab;
    // the run's counts, tables and lifetime factors change only in calls
    // that synchronise before returning: a block may read them before its
    // grid-dependency wait (theta in device memory only after it)
    p.pre_wait = 1;
    return p;
}

int musr_run_s::launch(int obj, int mode, const double* theta_dev, double* out_dev,
                       int32_t* status_dev, cudaStream_t st, float* model_out) {
    if (mode == kGN && Pk > kMaxGnParams) return MUSR_ENOTSUP;
    if (K == 0) return MUSR_OK;
    EvalParams p = params(obj, mode, theta_dev, out_dev, status_dev);
    p.model_out = model_out;
    return cuda_status(launch_eval(sig, mode, tl[mode].threads, tl[mode].n_tiles, st, p));
}

int musr_run_s::extend_theta(const double* theta, double* ext, std::vector<std::vector<double>>* jac) const {
    memcpy(ext, theta, sizeof(double) * P);
    if (jac) jac->assign(F, {});
    for (int j = 0; j < F; ++j) {
        const HostExpr& f = funcs[j];
        ext[P + j] = eval_host_expr(f, theta, -1, nullptr);
        if (!isfinite(ext[P + j])) return MUSR_ENONFINITE;
        if (!jac) continue;
        (*jac)[j].resize(f.refs.size());
        for (size_t r = 0; r < f.refs.size(); ++r) eval_host_expr(f, theta, f.refs[r], &(*jac)[j][r]);
    }
    return MUSR_OK;
}

// Host-pointer evaluation: one launch, theta inline in the launch parameters
// (through device memory beyond kInlineParams), results written by the kernel
// into mapped host memory.  With a function array the kernel works on the
// Pk = P + F slots and the results are folded back onto theta by the chain
// rule: g = g_p + J^T g_f, H = A^T H' A with A = [I; J].
int musr_run_s::eval_host(int obj, int mode, const double* theta, double* out_host, int32_t* flags,
                          const double** view) {
    if (obj != MUSR_CHI2 && obj != MUSR_POISSON) return MUSR_EINVAL;
    if (mode < kValue || mode > kGN) return MUSR_EINVAL;
    if (mode == kGN && Pk > kMaxGnParams) return MUSR_ENOTSUP;
    for (int j = 0; j < P; ++j)
        if (!isfinite(theta[j])) return MUSR_ENONFINITE;
    const int nuser = 1 + (mode >= kGrad ? P : 0) + (mode == kGN ? P * P : 0);
    if (K == 0) {
        memset(out_host, 0, sizeof(double) * nuser);
        *flags = 0;
        return MUSR_OK;
    }
    std::vector<double> ext;
    std::vector<std::vector<double>> jac;
    const double* th = theta;
    if (F > 0) {
        ext.resize(Pk);
        const int st = extend_theta(theta, ext.data(), mode >= kGrad ? &jac : nullptr);
        if (st != MUSR_OK) return st;
        th = ext.data();
    }
    EvalParams p = params(obj, mode, nullptr, hd_out, hd_status);
    cudaError_t e = cudaSuccess;
    if (Pk <= kInlineParams) {
        p.theta_inline_n = Pk;
        memcpy(p.theta_inline, th, sizeof(double) * Pk);
        p.pre_wait = 2;
    } else {
        memcpy(h_theta, th, sizeof(double) * Pk);
        e = cudaMemcpyAsync(d_theta, h_theta, sizeof(double) * Pk, cudaMemcpyHostToDevice, stream);
        p.theta = d_theta;
    }
    // the kernel's last block writes the status word after the results: poll it
    // (a short bounded spin, then a blocking stream synchronisation)
    p.status_sys_fence = 1;
    __atomic_store_n(h_status, kStatusPending, __ATOMIC_RELAXED);
    if (e == cudaSuccess) e = launch_eval(sig, mode, tl[mode].threads, tl[mode].n_tiles, stream, p);
    bool seen = false;
    if (e == cudaSuccess) {
        const auto t0 = std::chrono::steady_clock::now();
        for (int spin = 0; !seen; ++spin) {
            seen = __atomic_load_n(h_status, __ATOMIC_ACQUIRE) != kStatusPending;
            if (!seen && (spin & 255) == 255 &&
                std::chrono::steady_clock::now() - t0 > std::chrono::microseconds(kStatusSpinUs))
                break;
        }
        if (!seen) e = cudaStreamSynchronize(stream);
    }
    if (e != cudaSuccess) return cuda_status(e);
    *flags = __atomic_load_n(h_status, __ATOMIC_ACQUIRE);
    if (F == 0) {
        if (view) *view = h_out;
        else memcpy(out_host, h_out, sizeof(double) * nuser);
        return MUSR_OK;
    }
    out_host[0] = h_out[0];
    if (mode == kValue) return MUSR_OK;
    const double* g = h_out + 1;
    double* go = out_host + 1;
    memcpy(go, g, sizeof(double) * P);
    for (int j = 0; j < F; ++j)
        for (size_t r = 0; r < funcs[j].refs.size(); ++r) go[funcs[j].refs[r]] += jac[j][r] * g[P + j];
    if (mode != kGN) return MUSR_OK;
    const double* H = h_out + 1 + Pk;  // Pk x Pk
    double* Ho = out_host + 1 + P;       // P x P
    for (int a = 0; a < P; ++a) memcpy(Ho + (size_t)a * P, H + (size_t)a * Pk, sizeof(double) * P);
    for (int j = 0; j < F; ++j) {
        const std::vector<int>& rj = funcs[j].refs;
        for (size_t x = 0; x < rj.size(); ++x) {
            const int b = rj[x];
            const double jb = jac[j][x];
            for (int a = 0; a < P; ++a) {
                Ho[(size_t)a * P + b] += H[(size_t)a * Pk + P + j] * jb;
                Ho[(size_t)b * P + a] += jb * H[(size_t)(P + j) * Pk + a];
            }
        }
        for (int l = 0; l < F; ++l) {
            const double hjl = H[(size_t)(P + j) * Pk + P + l];
            const std::vector<int>& rl = funcs[l].refs;
            for (size_t x = 0; x < rj.size(); ++x)
                for (size_t y = 0; y < rl.size(); ++y)
                    Ho[(size_t)rj[x] * P + rl[y]] += jac[j][x] * jac[l][y] * hjl;
        }
    }
    return MUSR_OK;
}

musr_run_s::~musr_run_s() {
    if (fd_batch) musr_batch_destroy(fd_batch);
    if (d_group_off) cudaFree(d_group_off);
    if (arena) cudaFree(arena);
    if (h_pinned) cudaFreeHost(h_pinned);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (own_stream && stream) cudaStreamDestroy(stream);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int musr_create_run(const musr_run_desc* desc, musr_run* out) {
    if (!desc || !out) return MUSR_EINVAL;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MUSR_ECUDA;
    musr_run_s* r = new (std::nothrow) musr_run_s();
    if (!r) return MUSR_ENOMEM;
    r->device = dev;
    int st = r->plan(desc);
    if (st == MUSR_OK) {
        if (desc->stream) {
            r->stream = static_cast<cudaStream_t>(desc->stream);
            r->own_stream = false;
        } else {
            st = cuda_status(cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking));
            r->own_stream = true;
        }
    }
    if (st == MUSR_OK) st = cuda_status(cudaStreamCreateWithFlags(&r->cap_stream, cudaStreamNonBlocking));
    if (st == MUSR_OK) st = r->allocate();
    if (st == MUSR_OK) st = r->upload(desc->data_dtype, desc->data, desc->data_on_device);
    if (st != MUSR_OK) {
        delete r;
        return st;
    }
    *out = r;
    return MUSR_OK;
}

int musr_destroy_run(musr_run run) {
    if (!run) return MUSR_OK;
    DeviceGuard g(run->device);
    cudaStreamSynchronize(run->stream);
    delete run;
    return MUSR_OK;
}

int musr_run_info(musr_run run, int32_t* n_params, int64_t* total_bins, int32_t* n_hist) {
    if (!run) return MUSR_EINVAL;
    if (n_params) *n_params = run->P;
    if (total_bins) *total_bins = run->total_bins;
    if (n_hist) *n_hist = run->K;
    return MUSR_OK;
}

int musr_set_data(musr_run run, int32_t dtype, const void* data, int32_t on_device) {
    if (!run || !data) return MUSR_EINVAL;
    DeviceGuard g(run->device);
    return run->upload(dtype, data, on_device);
}

int musr_chi2(musr_run run, int obj, const double* theta, double* value) {
    if (!run || !theta || !value) return MUSR_EINVAL;
    DeviceGuard g(run->device);
    int32_t flags = 0;
    int st = run->eval_host(obj, kValue, theta, value, &flags);
    if (st != MUSR_OK) return st;
    if (flags & 1) {
        *value = INFINITY;
        return MUSR_EDOMAIN;
    }
    return isfinite(*value) ? MUSR_OK : MUSR_ENONFINITE;
}

int musr_chi2_grad(musr_run run, int obj, const double* theta, double* value, double* grad,
                   double* gn) {
    if (!run || !theta) return MUSR_EINVAL;
    DeviceGuard g(run->device);
    const int mode = gn ? kGN : kGrad;
    std::vector<double> out;
    out.resize(run->n_out[mode == kGN && run->Pk > kMaxGnParams ? kGrad : mode] + 1);
    int32_t flags = 0;
    int st = run->eval_host(obj, mode, theta, out.data(), &flags);
    if (st != MUSR_OK) return st;
    if (value) *value = out[0];
    if (grad) memcpy(grad, out.data() + 1, sizeof(double) * run->P);
    if (gn) memcpy(gn, out.data() + 1 + run->P, sizeof(double) * run->P * run->P);
    if (flags & 1) {
        if (value) *value = INFINITY;
        return MUSR_EDOMAIN;
    }
    return isfinite(out[0]) ? MUSR_OK : MUSR_ENONFINITE;
}

int musr_chi2_grad_device(musr_run run, int obj, int mode, const double* theta_dev, double* out_dev,
                          int32_t* status_dev, void* stream) {
    if (!run || !theta_dev || !out_dev) return MUSR_EINVAL;
    if (obj != MUSR_CHI2 && obj != MUSR_POISSON) return MUSR_EINVAL;
    if (mode < MUSR_VALUE || mode > MUSR_VALUE_GRAD_GN) return MUSR_EINVAL;
    if (run->F > 0) return MUSR_ENOTSUP;  // function values are formed on the host
    DeviceGuard g(run->device);
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : run->stream;
    if (run->K == 0) {
        cudaError_t e = cudaMemsetAsync(out_dev, 0, sizeof(double) * run->n_out[mode], st);
        if (e == cudaSuccess && status_dev) e = cudaMemsetAsync(status_dev, 0, sizeof(int32_t), st);
        return cuda_status(e);
    }
    return run->launch(obj, mode, theta_dev, out_dev, status_dev, st, nullptr);
}

int musr_chi2_grad_async(musr_run run, int obj, int mode, const double* theta, double* out_dev,
                         int32_t* status_dev, void* stream) {
    if (!run || !theta || !out_dev) return MUSR_EINVAL;
    if (obj != MUSR_CHI2 && obj != MUSR_POISSON) return MUSR_EINVAL;
    if (mode < MUSR_VALUE || mode > MUSR_VALUE_GRAD_GN) return MUSR_EINVAL;
    if (run->F > 0 || run->Pk > kInlineParams) return MUSR_ENOTSUP;
    if (mode == kGN && run->Pk > kMaxGnParams) return MUSR_ENOTSUP;
    for (int j = 0; j < run->P; ++j)
        if (!isfinite(theta[j])) return MUSR_ENONFINITE;
    DeviceGuard g(run->device);
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : run->stream;
    if (run->K == 0) {
        cudaError_t e = cudaMemsetAsync(out_dev, 0, sizeof(double) * run->n_out[mode], st);
        if (e == cudaSuccess && status_dev) e = cudaMemsetAsync(status_dev, 0, sizeof(int32_t), st);
        return cuda_status(e);
    }
    // theta by value in the launch parameters: immutable, so the whole bin
    // loop may precede the grid-dependency wait
    EvalParams p = run->params(obj, mode, nullptr, out_dev, status_dev);
    p.theta_inline_n = run->Pk;
    memcpy(p.theta_inline, theta, sizeof(double) * run->Pk);
    p.pre_wait = 2;
    int n_tiles = run->tl[mode].n_tiles;
    if (p.uni_tph > 0 && run->tl[mode].uni_tph_queued > 0) {  // equal histograms: the queued tiling
        p.uni_tph = run->tl[mode].uni_tph_queued;
        n_tiles = run->K * p.uni_tph;
    }
    return cuda_status(launch_eval(run->sig, mode, run->tl[mode].threads, n_tiles, st, p));
}

int musr_model(musr_run run, const double* theta, float* out, int32_t out_on_device) {
    if (!run || !theta || !out) return MUSR_EINVAL;
    DeviceGuard g(run->device);
    for (int j = 0; j < run->P; ++j)
        if (!isfinite(theta[j])) return MUSR_ENONFINITE;
    if (run->K == 0 || run->total_bins == 0) return MUSR_OK;
    std::vector<double> ext(run->Pk);
    const int fst = run->extend_theta(theta, ext.data(), nullptr);
    if (fst != MUSR_OK) return fst;
    cudaError_t e = cudaMemcpyAsync(run->d_theta_tmp, ext.data(), sizeof(double) * run->Pk,
                                    cudaMemcpyHostToDevice, run->stream);
    float* dst = out;
    float* tmp = nullptr;
    if (e == cudaSuccess && !out_on_device) {
        e = cudaMalloc(&tmp, sizeof(float) * run->total_bins);
        dst = tmp;
    }
    int st = cuda_status(e);
    if (st == MUSR_OK) st = run->launch(MUSR_CHI2, kModel, run->d_theta_tmp, nullptr, nullptr, run->stream, dst);
    if (st == MUSR_OK && !out_on_device)
        st = cuda_status(cudaMemcpyAsync(out, tmp, sizeof(float) * run->total_bins,
                                         cudaMemcpyDeviceToHost, run->stream));
    if (st == MUSR_OK) st = cuda_status(cudaStreamSynchronize(run->stream));
    if (tmp) cudaFree(tmp);
    return st;
}

const char* musr_strerror(int code) {
    switch (code) {
        case MUSR_OK: return "ok";
        case MUSR_EINVAL: return "invalid argument or layout";
        case MUSR_ENOMEM: return "out of memory";
        case MUSR_ECUDA: return "CUDA error";
        case MUSR_ENONFINITE: return "non-finite parameter or result";
        case MUSR_EDOMAIN: return "Poisson mean outside its domain (N < 0, or N = 0 with d > 0)";
        case MUSR_ETIMEOUT: return "bounded device wait timed out";
        case MUSR_ENOCONV: return "minimiser did not converge";
        case MUSR_ENOTSUP: return "layout outside the supported limits";
    }
    return "unknown status";
}

const char* musr_version(void) { return "musr-gb300 0.1 (sm_103a)"; }

const char* musr_last_cuda_error(void) { return g_last_cuda_error; }

}  // extern "C"
