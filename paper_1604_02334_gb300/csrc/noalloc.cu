// musr_chi2_grad_noalloc: the objective / adjoint evaluation for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while another framework
// owns the device's memory pool, real-time acquisition processes that forbid
// allocation after start-up, or plug-ins whose host application hands them
// only pre-allocated device buffers.  For them this entry point keeps every
// piece of scratch the evaluation needs (tiling tables, the parameter map,
// the lifetime-factor table, the reduction accumulators and a padded copy of
// the histograms) in one file-scope device array of a fixed size,
// MUSR_NOALLOC_SCRATCH_BYTES.  The array belongs to this library's module:
// every GPU that loads it holds the array until the process exits.  The
// entry point itself calls no cudaMalloc, cudaFree or other allocating
// routine, on the device or on the host.
//
// Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress (that
// device current) and keeps it; later calls reuse it.  With CUDA's lazy
// module loading (the default) that first call is also when the driver loads
// this file's module on the device and reserves the array's memory, so
// callers make it at start-up, before another framework takes the memory.
//
// Each call uploads its tables from a static host plan with cudaMemcpyAsync
// (pageable source), which the next call rewrites: calls made while the
// stream is being captured into a graph are refused (MUSR_ENOTSUP), since a
// captured copy would read that buffer again at every replay.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <atomic>
#include <mutex>

#include "eval_kernel.cuh"
#include "musr.h"
#include "musr_internal.h"

namespace musr {
namespace {

constexpr size_t kScratchBytes = MUSR_NOALLOC_SCRATCH_BYTES;
constexpr int kNaMaxHist = MUSR_NOALLOC_MAX_HIST;
constexpr int kNaMaxParams = MUSR_NOALLOC_MAX_PARAMS;
constexpr int kNaMaxTiles = 1 << 13;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::atomic<unsigned char*> g_scratch_addr[kMaxDevices];

// Host-side plan of one call, built in a static buffer under a mutex (no
// heap use); the device work itself is asynchronous.
struct NaPlan {
    int K, P, R, threads, tile_bins, n_tiles, n_out, n_src;
    Signature sig;
    int64_t hist_off[kNaMaxHist];
    int32_t hist_nbins[kNaMaxHist];
    int32_t role_theta[kNaMaxHist * kMaxRoles * 2];
    int32_t tile_hist[kNaMaxTiles], tile_start[kNaMaxTiles], tile_end[kNaMaxTiles];
    int32_t csr_ptr[kNaMaxParams + 2];
    int32_t csr_src[kNaMaxHist * (1 + 2 * kMaxRoles)];
    int32_t csr_cnt[kNaMaxParams + 2];
    int64_t data_floats;
};
NaPlan g_plan;
std::mutex g_plan_mutex;

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

int plan_call(const musr_run_desc* d, int mode, int sms, NaPlan& pl) {
    pl.K = d->n_hist;
    pl.P = d->n_params;
    if (pl.K < 1 || pl.K > kNaMaxHist || pl.P < 1 || pl.P > kNaMaxParams) return MUSR_ENOTSUP;
    if (d->n_funcs != 0) return MUSR_ENOTSUP;  // function arrays are evaluated by the host entry points
    if (d->map_width < 2 || d->map_width > 32 || d->n_comp < 0 || !d->n_bins || !d->map) return MUSR_EINVAL;
    if (d->n_comp > 0 && !d->comp) return MUSR_EINVAL;
    if (!(d->dt_us > 0.0) || !(d->tau_us > 0.0) || !(d->t0_us >= 0.0) || !(d->gamma_mhz_per_g >= 0.0))
        return MUSR_EINVAL;
    RoleLayout rl;
    const int st = role_layout(d->comp, d->n_comp, d->map_width, rl);
    if (st != MUSR_OK) return st;
    pl.sig = rl.sig;
    pl.R = pl.sig.roles();
    for (int k = 0; k < pl.K; ++k) {
        if (d->n_bins[k] < 0) return MUSR_EINVAL;
        if (d->n_bins[k] > (int64_t(1) << 24)) return MUSR_ENOTSUP;
        for (int c = 0; c < d->map_width; ++c) {
            const int i = d->map[(int64_t)k * d->map_width + c];
            if (i < -1 || i >= pl.P) return MUSR_EINVAL;
        }
        role_row(rl, d->comp, d->map + (int64_t)k * d->map_width, pl.role_theta + (size_t)k * kMaxRoles * 2);
    }
    // tiling: the largest block that still gives >= 2 blocks per SM
    pl.threads = 32;
    for (int t = kMaxThreads; t >= 32; t >>= 1) {
        int64_t tiles = 0;
        for (int k = 0; k < pl.K; ++k)
            tiles += std::max<int64_t>(1, (d->n_bins[k] + t * kBinsPerThread - 1) / (t * kBinsPerThread));
        if (tiles >= 2 * sms) {
            pl.threads = t;
            break;
        }
    }
    pl.tile_bins = pl.threads * kBinsPerThread;
    int64_t off = 0;
    pl.n_tiles = 0;
    for (int k = 0; k < pl.K; ++k) {
        const int64_t M = d->n_bins[k];
        pl.hist_off[k] = off;
        pl.hist_nbins[k] = (int32_t)M;
        off += round_up(M, 8);
        const int64_t nt = std::max<int64_t>(1, (M + pl.tile_bins - 1) / pl.tile_bins);
        if (pl.n_tiles + nt > kNaMaxTiles) return MUSR_ENOTSUP;
        for (int64_t j = 0; j < nt; ++j) {
            pl.tile_hist[pl.n_tiles] = k;
            pl.tile_start[pl.n_tiles] = (int32_t)std::min<int64_t>(j * pl.tile_bins, round_up(M, 8));
            pl.tile_end[pl.n_tiles] = (int32_t)std::min<int64_t>((j + 1) * pl.tile_bins, round_up(M, 8));
            ++pl.n_tiles;
        }
    }
    pl.data_floats = off + 8;
    // CSR of output -> (histogram, accumulator) in (k, role, entry) order, by
    // counting sort (no heap)
    const int nacc = n_acc(mode, pl.R);
    pl.n_out = 1 + (mode >= kGrad ? pl.P : 0);
    for (int o = 0; o <= pl.n_out; ++o) pl.csr_cnt[o] = 0;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            pl.csr_ptr[0] = 0;
            for (int o = 0; o < pl.n_out; ++o) pl.csr_ptr[o + 1] = pl.csr_ptr[o] + pl.csr_cnt[o];
            for (int o = 0; o < pl.n_out; ++o) pl.csr_cnt[o] = pl.csr_ptr[o];
        }
        for (int k = 0; k < pl.K; ++k) {
            const int32_t* rt = pl.role_theta + (size_t)k * kMaxRoles * 2;
            const int32_t base = k * nacc;
            if (pass == 0) pl.csr_cnt[0]++;
            else pl.csr_src[pl.csr_cnt[0]++] = base;
            if (mode < kGrad) continue;
            for (int r = 0; r < pl.R; ++r)
                for (int j = 0; j < 2; ++j) {
                    const int i = rt[2 * r + j];
                    if (i < 0) continue;
                    if (pass == 0) pl.csr_cnt[1 + i]++;
                    else pl.csr_src[pl.csr_cnt[1 + i]++] = base + 1 + r;
                }
        }
    }
    pl.n_src = pl.csr_ptr[pl.n_out];
    return MUSR_OK;
}

cudaError_t launch_na(const Signature& s, int mode, int threads, int n_tiles, cudaStream_t st,
                      const EvalParams& p) {
#define MUSR_CASE(NE, NG, NS, KT)                                                          \
    if (s.ne == NE && s.ng == NG && s.ns == NS && s.kt == KT)                                  \
        return mode == kValue ? launch_one<NE, NG, NS, KT, kValue>(threads, n_tiles, st, p) \
                              : launch_one<NE, NG, NS, KT, kGrad>(threads, n_tiles, st, p);
    MUSR_FOR_EACH_SIGNATURE(MUSR_CASE)
#undef MUSR_CASE
    return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace musr

using namespace musr;

extern "C" int musr_chi2_grad_noalloc(const musr_run_desc* desc, int obj, int mode,
                                      const double* theta_dev, double* out_dev, int32_t* status_dev,
                                      void* stream) {
    if (!desc || !theta_dev || !out_dev) return MUSR_EINVAL;
    if (obj != MUSR_CHI2 && obj != MUSR_POISSON) return MUSR_EINVAL;
    if (mode != MUSR_VALUE && mode != MUSR_VALUE_GRAD) return MUSR_ENOTSUP;
    if (!desc->data || !desc->data_on_device || desc->data_dtype != MUSR_F32) return MUSR_ENOTSUP;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MUSR_ECUDA;
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        const cudaError_t e = cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cs);
        if (e != cudaSuccess) return cuda_status(e);
        if (cs != cudaStreamCaptureStatusNone) return MUSR_ENOTSUP;
    }
    // one-time set-up on this device: the device address of the scratch array
    unsigned char* base = g_scratch_addr[dev].load();
    if (!base) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess || !ptr) return cuda_status(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
        base = static_cast<unsigned char*>(ptr);
        g_scratch_addr[dev].store(base);
    }
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    std::lock_guard<std::mutex> lock(g_plan_mutex);
    NaPlan& pl = g_plan;
    int st = plan_call(desc, mode, sms, pl);
    if (st != MUSR_OK) return st;
    const int nacc = n_acc(mode, pl.R);

    // carve the scratch array; reject calls whose working set does not fit
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = (off + bytes + 255) / 256 * 256;
        return o;
    };
    const size_t o_cnt = take(4 * sizeof(unsigned));
    const size_t o_hoff = take(sizeof(int64_t) * pl.K);
    const size_t o_nb = take(sizeof(int32_t) * pl.K);
    const size_t o_th = take(sizeof(int32_t) * pl.n_tiles);
    const size_t o_ts = take(sizeof(int32_t) * pl.n_tiles);
    const size_t o_te = take(sizeof(int32_t) * pl.n_tiles);
    const size_t o_rt = take(sizeof(int32_t) * pl.K * kMaxRoles * 2);
    const size_t o_cp = take(sizeof(int32_t) * (pl.n_out + 1));
    const size_t o_cs = take(sizeof(int32_t) * (pl.n_src + 1));
    const size_t o_facc = take(sizeof(unsigned long long) * (size_t)pl.K * nacc * 3);
    const size_t o_hsum = take(sizeof(__int128) * (size_t)pl.K * nacc);
    const size_t o_data = take(sizeof(float) * (size_t)pl.data_floats);
    int64_t max_m = 0;
    for (int k = 0; k < pl.K; ++k) max_m = std::max<int64_t>(max_m, pl.hist_nbins[k]);
    const int64_t etab_len = lifetime_table_len(max_m);
    const size_t o_etab = take(sizeof(float) * (size_t)etab_len);
    if (off > kScratchBytes) return MUSR_ENOTSUP;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(base + o_cnt, 0, 4 * sizeof(unsigned), s);  // tickets start at 0
    // the fixed-point accumulators start at 0 (the kernel's last block also leaves them at 0)
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_facc, 0, sizeof(unsigned long long) * (size_t)pl.K * nacc * 3, s);
    auto up = [&](size_t o, const void* src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(base + o, src, bytes, cudaMemcpyHostToDevice, s);
    };
    up(o_hoff, pl.hist_off, sizeof(int64_t) * pl.K);
    up(o_nb, pl.hist_nbins, sizeof(int32_t) * pl.K);
    up(o_th, pl.tile_hist, sizeof(int32_t) * pl.n_tiles);
    up(o_ts, pl.tile_start, sizeof(int32_t) * pl.n_tiles);
    up(o_te, pl.tile_end, sizeof(int32_t) * pl.n_tiles);
    up(o_rt, pl.role_theta, sizeof(int32_t) * pl.K * kMaxRoles * 2);
    up(o_cp, pl.csr_ptr, sizeof(int32_t) * (pl.n_out + 1));
    up(o_cs, pl.csr_src, sizeof(int32_t) * pl.n_src);
    // the histograms, copied into the padded layout the kernel reads
    float* data = reinterpret_cast<float*>(base + o_data);
    const float* src = static_cast<const float*>(desc->data);
    int64_t so = 0;
    for (int k = 0; k < pl.K && e == cudaSuccess; ++k) {
        const int64_t M = desc->n_bins[k];
        if (M) e = cudaMemcpyAsync(data + pl.hist_off[k], src + so, sizeof(float) * M, cudaMemcpyDeviceToDevice, s);
        so += M;
    }
    // the lifetime factor at every chunk start of the time grid
    float* etab = reinterpret_cast<float*>(base + o_etab);
    if (e == cudaSuccess) e = fill_lifetime_table(etab, etab_len, desc->t0_us, desc->dt_us, desc->tau_us, s);
    if (e != cudaSuccess) return cuda_status(e);

    EvalParams p;
    memset(&p, 0, sizeof(p));
    p.data = data;
    p.hist_off = reinterpret_cast<const int64_t*>(base + o_hoff);
    p.hist_nbins = reinterpret_cast<const int32_t*>(base + o_nb);
    p.tile_hist = reinterpret_cast<const int32_t*>(base + o_th);
    p.tile_start = reinterpret_cast<const int32_t*>(base + o_ts);
    p.tile_end = reinterpret_cast<const int32_t*>(base + o_te);
    p.role_theta = reinterpret_cast<const int32_t*>(base + o_rt);
    p.theta = theta_dev;
    p.t0 = desc->t0_us;
    p.dt = desc->dt_us;
    p.inv_tau = 1.0 / desc->tau_us;
    p.gamma = desc->gamma_mhz_per_g;
    p.rc = make_run_const(desc->t0_us, desc->dt_us, desc->tau_us, desc->gamma_mhz_per_g);
    p.K = pl.K;
    p.P = pl.P;
    p.obj = obj;
    p.facc = reinterpret_cast<unsigned long long*>(base + o_facc);
    p.hist_sum = reinterpret_cast<__int128*>(base + o_hsum);
    p.global_count = reinterpret_cast<unsigned*>(base + o_cnt);
    p.flags = reinterpret_cast<unsigned*>(base + o_cnt) + 1;
    p.csr_ptr = reinterpret_cast<const int32_t*>(base + o_cp);
    p.csr_src = reinterpret_cast<const int32_t*>(base + o_cs);
    p.n_out = pl.n_out;
    p.n_src = pl.n_src;
    p.hsum_in_smem = 1;  // K <= 64 and nacc <= 13: at most 13 KB
    p.csr_in_smem = 1;   // at most ~7 KB
    p.smem_bytes = (int)(16 * (size_t)pl.K * nacc + 4 * csr_smem_words(pl.n_out, pl.n_src, false));
    p.out = out_dev;
    p.status_out = status_dev;
    p.etab = etab;
    // allow the tail's shared memory, then stage the constants and evaluate
    e = launch_na(pl.sig, mode, pl.threads, 0, s, p);
    if (e == cudaSuccess) e = launch_na(pl.sig, mode, pl.threads, pl.n_tiles, s, p);
    return cuda_status(e);
}
