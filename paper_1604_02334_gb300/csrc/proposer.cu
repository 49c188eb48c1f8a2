// Learned start proposer: an MLP on the BF16 tensor cores maps rebinned,
// log-scaled histograms of a run to starting parameters for the minimiser.
// Network input of a run with histograms k and groups g of `rebin` bins
// (counts c_kg, histogram totals C_k):
//     u_kg = log(1 + c_kg) - log(1 + C_k),   v_k = log(1 + C_k),
// each standardised by a per-feature mean and standard deviation estimated
// once from generated samples, so that the relative modulation of the
// counts (the precession signal, ~10 %) spans many BF16 ulps instead of two.
// Training data come from the device generator (Eq. 1 theory summed over
// groups of bins, Poisson counts), drawn fresh for every step with parameter
// vectors uniform in a box, so the network never sees a sample twice.  The
// fit from the proposal is judged by its chi2 / ndf; above a threshold the
// plain multi-start fit runs as the fallback.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "musr.h"
#include "musr_internal.h"
#include "run_impl.h"

struct musr_proposer_s {
    musr_run layout = nullptr;
    int P = 0, K = 0, n_learned = 0, rebin = 64, batch = 512, n_groups = 0, n_feat = 0, n_in = 0;
    bool have_norm = false;
    std::vector<double> lo, hi;
    std::vector<int32_t> learned;
    musr_mlp mlp = nullptr;
    uint64_t seed = 1, drawn = 0;
    double box_margin = 0.25;  // learned fits ending outside the widened box fall back
    void* arena = nullptr;
    double *d_lo = nullptr, *d_hi = nullptr, *d_thetas = nullptr;
    int32_t* d_learned = nullptr;
    float *d_x = nullptr, *d_t = nullptr, *d_y = nullptr, *d_g = nullptr, *d_mu = nullptr, *d_isig = nullptr;
    double* d_stats = nullptr;  // [2][n_feat] sums of x and x^2 while estimating the standardisation
    int64_t* d_goff = nullptr;  // group offsets of each histogram within a row
    cudaStream_t stream = nullptr;
};

namespace musr {
int gbatch_n_runs(musr_gbatch b);
musr_run gbatch_run(musr_gbatch b, int r);
int gbatch_has_gn(musr_gbatch b);
}  // namespace musr

namespace {

constexpr uint64_t kNormOffset = 1ull << 62;  // sample indices of the standardisation set
constexpr int kNormBatches = 16;

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

bool same_layout(musr_run a, musr_run b) {
    if (a->K != b->K) return false;
    for (int k = 0; k < a->K; ++k)
        if (a->n_bins[k] != b->n_bins[k]) return false;
    return true;
}

// One block per (row, histogram): total counts (FP64, exact for integers),
// then the standardised features of the histogram's groups and its total.
__global__ void features_kernel(const float* __restrict__ counts, int64_t row_stride_in, const int64_t* __restrict__ group_off,
                                const int32_t* __restrict__ hist_nbins, int rebin, int n_groups,
                                const float* __restrict__ mu, const float* __restrict__ isig, float* __restrict__ x,
                                int64_t row_stride_out) {
    __shared__ double red[32];
    const int k = blockIdx.x, row = blockIdx.y, K = gridDim.x;
    const int G = (hist_nbins[k] + rebin - 1) / rebin;
    const float* c = counts + (size_t)row * row_stride_in + group_off[k];
    double s = 0.0;
    for (int g = threadIdx.x; g < G; g += blockDim.x) s += (double)c[g];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) red[0] = t;
    }
    __syncthreads();
    const float L = (float)log1p(red[0]);
    float* xr = x + (size_t)row * row_stride_out;
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
        const int64_t f = group_off[k] + g;
        xr[f] = (log1pf(c[g]) - L - mu[f]) * isig[f];
    }
    if (threadIdx.x == 0) {
        const int f = n_groups + k;
        xr[f] = (L - mu[f]) * isig[f];
    }
    (void)K;
}

// Column sums of x and x^2 over the rows of a batch (FP64)
__global__ void feature_stats_kernel(const float* __restrict__ x, int rows, int64_t row_stride, int n_feat,
                                     double* __restrict__ stats) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_feat) return;
    double s1 = 0.0, s2 = 0.0;
    for (int r = 0; r < rows; ++r) {
        const double v = (double)x[(size_t)r * row_stride + f];
        s1 += v;
        s2 += v * v;
    }
    stats[f] += s1;
    stats[n_feat + f] += s2;
}

__global__ void finish_stats_kernel(const double* __restrict__ stats, int n_feat, double n, float* __restrict__ mu,
                                    float* __restrict__ isig) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_feat) return;
    const double m = stats[f] / n;
    const double var = fmax(stats[n_feat + f] / n - m * m, 0.0);
    mu[f] = (float)m;
    isig[f] = (float)(1.0 / fmax(sqrt(var), 1e-3));
}

int launch_features(musr_proposer p, const float* counts, int64_t in_stride, int rows, const float* mu,
                    const float* isig, float* x, int64_t out_stride, cudaStream_t st) {
    if (rows <= 0) return MUSR_OK;
    const int threads = 256;
    dim3 grid((unsigned)p->K, (unsigned)rows);
    features_kernel<<<grid, threads, 0, st>>>(counts, in_stride, p->d_goff, p->layout->d_hist_nbins,
                                              p->rebin, p->n_groups, mu, isig, x, out_stride);
    return musr::cuda_status(cudaGetLastError());
}

// Generated histograms of `n` training samples from index `offset` -> d_x rows
// (and the targets into d_t), with the given standardisation.
int make_batch(musr_proposer p, int n, uint64_t offset, const float* mu, const float* isig) {
    int st = musr::sample_uniform_thetas(p->d_lo, p->d_hi, p->d_learned, p->n_learned, p->P, n, p->seed, offset,
                                         p->d_thetas, p->d_t, p->stream);
    if (st == MUSR_OK)
        st = musr::generate_rows(p->layout, p->d_thetas, n, p->rebin, p->seed, offset, 0, p->d_g, nullptr,
                                 p->n_groups, p->stream);
    if (st == MUSR_OK) st = launch_features(p, p->d_g, p->n_groups, n, mu, isig, p->d_x, p->n_in, p->stream);
    return st;
}

// The standardisation: mean and standard deviation of every feature over
// kNormBatches generated batches of sample indices from kNormOffset.
int ensure_norm(musr_proposer p) {
    if (p->have_norm) return MUSR_OK;
    // identity standardisation while measuring: mu = 0 (d_mu zeroed), isig = 1
    std::vector<float> ones(p->n_feat, 1.f);
    int st = musr::cuda_status(cudaMemsetAsync(p->d_mu, 0, sizeof(float) * p->n_feat, p->stream));
    if (st == MUSR_OK)
        st = musr::cuda_status(cudaMemcpyAsync(p->d_isig, ones.data(), sizeof(float) * p->n_feat,
                                               cudaMemcpyHostToDevice, p->stream));
    if (st == MUSR_OK)
        st = musr::cuda_status(cudaMemsetAsync(p->d_stats, 0, sizeof(double) * 2 * p->n_feat, p->stream));
    for (int b = 0; b < kNormBatches && st == MUSR_OK; ++b) {
        st = make_batch(p, p->batch, kNormOffset + (uint64_t)b * p->batch, p->d_mu, p->d_isig);
        if (st == MUSR_OK) {
            feature_stats_kernel<<<(p->n_feat + 255) / 256, 256, 0, p->stream>>>(p->d_x, p->batch, p->n_in, p->n_feat,
                                                                                p->d_stats);
            st = musr::cuda_status(cudaGetLastError());
        }
    }
    if (st == MUSR_OK) {
        finish_stats_kernel<<<(p->n_feat + 255) / 256, 256, 0, p->stream>>>(
            p->d_stats, p->n_feat, (double)kNormBatches * p->batch, p->d_mu, p->d_isig);
        st = musr::cuda_status(cudaGetLastError());
    }
    if (st == MUSR_OK) st = musr::cuda_status(cudaStreamSynchronize(p->stream));
    if (st == MUSR_OK) p->have_norm = true;
    return st;
}

}  // namespace

extern "C" {

int musr_proposer_destroy(musr_proposer p) {
    if (!p) return MUSR_OK;
    if (p->stream) cudaStreamSynchronize(p->stream);
    if (p->mlp) musr_mlp_destroy(p->mlp);
    if (p->arena) cudaFree(p->arena);
    if (p->stream) cudaStreamDestroy(p->stream);
    delete p;
    return MUSR_OK;
}

int musr_proposer_create(musr_run layout, const double* lo, const double* hi, const musr_proposer_opts* opts,
                         musr_proposer* out) {
    if (!layout || !lo || !hi || !out) return MUSR_EINVAL;
    *out = nullptr;
    if (layout->F > 0) return MUSR_ENOTSUP;  // the generator reads parameters only
    musr_proposer_opts o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.rebin <= 0) o.rebin = 64;
    if (o.n_hidden <= 0) o.n_hidden = 512;
    if (o.n_hidden_layers <= 0) o.n_hidden_layers = 3;
    if (o.batch <= 0) o.batch = 512;
    if (!(o.in_scale > 0.f)) o.in_scale = 1.f;
    if (o.seed == 0) o.seed = 1;
    if (!(o.box_margin > 0.f)) o.box_margin = 0.25f;
    if (o.batch % 128 || layout->K <= 0) return MUSR_EINVAL;
    musr_proposer p = new (std::nothrow) musr_proposer_s();
    if (!p) return MUSR_ENOMEM;
    p->layout = layout;
    p->P = layout->P;
    p->K = layout->K;
    p->rebin = o.rebin;
    p->batch = o.batch;
    p->seed = o.seed;
    p->box_margin = o.box_margin;
    p->lo.assign(lo, lo + p->P);
    p->hi.assign(hi, hi + p->P);
    for (int j = 0; j < p->P; ++j) {
        if (!(std::isfinite(lo[j]) && std::isfinite(hi[j])) || hi[j] < lo[j]) {
            delete p;
            return MUSR_EINVAL;
        }
        if (hi[j] > lo[j]) p->learned.push_back(j);
    }
    p->n_learned = (int)p->learned.size();
    std::vector<int64_t> goff(p->K);
    int64_t groups = 0;
    for (int k = 0; k < p->K; ++k) {
        goff[k] = groups;
        groups += (layout->n_bins[k] + o.rebin - 1) / o.rebin;
    }
    p->n_groups = (int)std::min<int64_t>(groups, 1 << 30);
    p->n_feat = p->n_groups + p->K;
    p->n_in = (p->n_feat + 127) / 128 * 128;
    if (p->n_learned == 0 || p->n_learned > 128 || groups == 0 || groups + p->K > (1 << 20)) {
        delete p;
        return MUSR_EINVAL;
    }
    int st = musr_mlp_create(p->n_in, o.n_hidden, o.n_hidden_layers, p->n_learned, p->batch, o.in_scale,
                             o.seed ^ 0x6d6c7000ull, &p->mlp);
    size_t sz = 0;
    auto take = [&](size_t bytes) {
        const size_t at = sz;
        sz += al256(bytes);
        return at;
    };
    const size_t B = p->batch;
    const size_t o_lo = take(sizeof(double) * p->P), o_hi = take(sizeof(double) * p->P);
    const size_t o_th = take(sizeof(double) * p->P * B), o_ln = take(sizeof(int32_t) * p->n_learned);
    const size_t o_x = take(sizeof(float) * (size_t)p->n_in * B), o_t = take(sizeof(float) * p->n_learned * B);
    const size_t o_y = take(sizeof(float) * p->n_learned * B), o_g = take(sizeof(float) * (size_t)p->n_groups * B);
    const size_t o_mu = take(sizeof(float) * p->n_feat), o_is = take(sizeof(float) * p->n_feat);
    const size_t o_st = take(sizeof(double) * 2 * p->n_feat), o_go = take(sizeof(int64_t) * p->K);
    if (st == MUSR_OK && cudaMalloc(&p->arena, sz) != cudaSuccess) {
        p->arena = nullptr;
        st = MUSR_ENOMEM;
    }
    if (st == MUSR_OK) st = musr::cuda_status(cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking));
    if (st == MUSR_OK) {
        char* a = static_cast<char*>(p->arena);
        p->d_lo = reinterpret_cast<double*>(a + o_lo);
        p->d_hi = reinterpret_cast<double*>(a + o_hi);
        p->d_thetas = reinterpret_cast<double*>(a + o_th);
        p->d_learned = reinterpret_cast<int32_t*>(a + o_ln);
        p->d_x = reinterpret_cast<float*>(a + o_x);
        p->d_t = reinterpret_cast<float*>(a + o_t);
        p->d_y = reinterpret_cast<float*>(a + o_y);
        p->d_g = reinterpret_cast<float*>(a + o_g);
        p->d_mu = reinterpret_cast<float*>(a + o_mu);
        p->d_isig = reinterpret_cast<float*>(a + o_is);
        p->d_stats = reinterpret_cast<double*>(a + o_st);
        p->d_goff = reinterpret_cast<int64_t*>(a + o_go);
        cudaError_t e = cudaMemsetAsync(p->arena, 0, sz, p->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->d_lo, lo, sizeof(double) * p->P, cudaMemcpyHostToDevice, p->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->d_hi, hi, sizeof(double) * p->P, cudaMemcpyHostToDevice, p->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->d_learned, p->learned.data(), sizeof(int32_t) * p->n_learned,
                                cudaMemcpyHostToDevice, p->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->d_goff, goff.data(), sizeof(int64_t) * p->K, cudaMemcpyHostToDevice, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
        st = musr::cuda_status(e);
    }
    if (st != MUSR_OK) {
        musr_proposer_destroy(p);
        return st;
    }
    *out = p;
    return MUSR_OK;
}

int musr_proposer_mlp(musr_proposer p, musr_mlp* out) {
    if (!p || !out) return MUSR_EINVAL;
    *out = p->mlp;
    return MUSR_OK;
}

int musr_proposer_info(musr_proposer p, int32_t* n_features, int32_t* n_learned, int32_t* n_inputs) {
    if (!p) return MUSR_EINVAL;
    if (n_features) *n_features = p->n_feat;
    if (n_learned) *n_learned = p->n_learned;
    if (n_inputs) *n_inputs = p->n_in;
    return MUSR_OK;
}

int musr_proposer_get_norm(musr_proposer p, float* mu, float* inv_sigma) {
    if (!p || !mu || !inv_sigma) return MUSR_EINVAL;
    int st = ensure_norm(p);
    if (st == MUSR_OK)
        st = musr::cuda_status(cudaMemcpy(mu, p->d_mu, sizeof(float) * p->n_feat, cudaMemcpyDeviceToHost));
    if (st == MUSR_OK)
        st = musr::cuda_status(cudaMemcpy(inv_sigma, p->d_isig, sizeof(float) * p->n_feat, cudaMemcpyDeviceToHost));
    return st;
}

int musr_proposer_set_norm(musr_proposer p, const float* mu, const float* inv_sigma) {
    if (!p || !mu || !inv_sigma) return MUSR_EINVAL;
    for (int f = 0; f < p->n_feat; ++f)
        if (!std::isfinite(mu[f]) || !std::isfinite(inv_sigma[f])) return MUSR_EINVAL;
    int st = musr::cuda_status(cudaStreamSynchronize(p->stream));
    if (st == MUSR_OK)
        st = musr::cuda_status(cudaMemcpy(p->d_mu, mu, sizeof(float) * p->n_feat, cudaMemcpyHostToDevice));
    if (st == MUSR_OK)
        st = musr::cuda_status(cudaMemcpy(p->d_isig, inv_sigma, sizeof(float) * p->n_feat, cudaMemcpyHostToDevice));
    if (st == MUSR_OK) p->have_norm = true;
    return st;
}

int musr_proposer_sample(musr_proposer p, int32_t n, uint64_t offset, double* thetas_dev, float* targets_dev,
                         void* stream) {
    if (!p || n < 0 || (n > 0 && !thetas_dev)) return MUSR_EINVAL;
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : p->stream;
    return musr::sample_uniform_thetas(p->d_lo, p->d_hi, p->d_learned, p->n_learned, p->P, n, p->seed, offset,
                                       thetas_dev, targets_dev, s);
}

int musr_proposer_features(musr_proposer p, const musr_run* runs, int32_t n_runs, float* out_dev, void* stream) {
    if (!p || n_runs < 0 || (n_runs > 0 && (!runs || !out_dev))) return MUSR_EINVAL;
    for (int r = 0; r < n_runs; ++r)
        if (!runs[r] || !same_layout(p->layout, runs[r])) return MUSR_EINVAL;
    (void)stream;
    int st = ensure_norm(p);
    for (int r0 = 0; r0 < n_runs && st == MUSR_OK; r0 += p->batch) {
        const int n = std::min(p->batch, n_runs - r0);
        for (int r = 0; r < n && st == MUSR_OK; ++r) {
            st = musr::cuda_status(cudaStreamSynchronize(runs[r0 + r]->stream));
            if (st == MUSR_OK)
                st = musr::rebin_sum_row(runs[r0 + r], p->rebin, p->d_g + (size_t)r * p->n_groups, p->stream);
        }
        if (st == MUSR_OK)
            st = launch_features(p, p->d_g, p->n_groups, n, p->d_mu, p->d_isig, out_dev + (size_t)r0 * p->n_feat,
                                 p->n_feat, p->stream);
        if (st == MUSR_OK) st = musr::cuda_status(cudaStreamSynchronize(p->stream));
    }
    return st;
}

int musr_proposer_train(musr_proposer p, int32_t n_steps, float lr_start, float lr_end, float* losses) {
    if (!p || n_steps < 0 || !(lr_start > 0.f) || !(lr_end > 0.f)) return MUSR_EINVAL;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->layout->device) cudaSetDevice(p->layout->device);
    int st = ensure_norm(p);
    const double ratio = (double)lr_end / (double)lr_start;
    for (int s = 0; s < n_steps && st == MUSR_OK; ++s) {
        const double f = n_steps > 1 ? (double)s / (double)(n_steps - 1) : 0.0;
        const float lr = (float)((double)lr_start * pow(ratio, f));
        st = make_batch(p, p->batch, p->drawn, p->d_mu, p->d_isig);
        p->drawn += (uint64_t)p->batch;
        if (st == MUSR_OK)
            st = musr_mlp_train_step(p->mlp, p->d_x, p->d_t, p->batch, lr, losses ? losses + s : nullptr, p->stream);
    }
    if (cur != p->layout->device) cudaSetDevice(cur);
    return st;
}

int musr_proposer_propose(musr_proposer p, const musr_run* runs, int32_t n_runs, double* thetas_out) {
    if (!p || n_runs < 0 || (n_runs > 0 && (!runs || !thetas_out))) return MUSR_EINVAL;
    for (int r = 0; r < n_runs; ++r)
        if (!runs[r] || !same_layout(p->layout, runs[r]) || runs[r]->P != p->P) return MUSR_EINVAL;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->layout->device) cudaSetDevice(p->layout->device);
    int st = ensure_norm(p);
    std::vector<float> y;
    for (int r0 = 0; r0 < n_runs && st == MUSR_OK; r0 += p->batch) {
        const int n = std::min(p->batch, n_runs - r0);
        for (int r = 0; r < n && st == MUSR_OK; ++r) {
            st = musr::cuda_status(cudaStreamSynchronize(runs[r0 + r]->stream));
            if (st == MUSR_OK)
                st = musr::rebin_sum_row(runs[r0 + r], p->rebin, p->d_g + (size_t)r * p->n_groups, p->stream);
        }
        if (st == MUSR_OK)
            st = launch_features(p, p->d_g, p->n_groups, n, p->d_mu, p->d_isig, p->d_x, p->n_in, p->stream);
        const int nb = (n + 127) / 128 * 128;
        if (st == MUSR_OK) st = musr_mlp_forward(p->mlp, p->d_x, nb, p->d_y, p->stream);
        y.resize((size_t)n * p->n_learned);
        if (st == MUSR_OK)
            st = musr::cuda_status(cudaMemcpy(y.data(), p->d_y, sizeof(float) * y.size(), cudaMemcpyDeviceToHost));
        if (st != MUSR_OK) break;
        for (int r = 0; r < n; ++r) {
            double* th = thetas_out + (size_t)(r0 + r) * p->P;
            for (int j = 0; j < p->P; ++j) th[j] = p->lo[j];
            for (int q = 0; q < p->n_learned; ++q) {
                const int j = p->learned[q];
                double u = 0.5 * ((double)y[(size_t)r * p->n_learned + q] + 1.0);
                u = std::isfinite(u) ? std::min(1.0, std::max(0.0, u)) : 0.5;
                th[j] = p->lo[j] + (p->hi[j] - p->lo[j]) * u;
            }
        }
    }
    if (cur != p->layout->device) cudaSetDevice(cur);
    return st;
}

namespace {
// every learned entry of theta inside [lo - m w, hi + m w], w = hi - lo
bool in_widened_box(const musr_proposer_s* p, const double* theta) {
    for (int j : p->learned) {
        const double w = p->hi[j] - p->lo[j], m = p->box_margin * w;
        if (!(theta[j] >= p->lo[j] - m && theta[j] <= p->hi[j] + m)) return false;
    }
    return true;
}

// The fallback grid (n_starts rows of P) shrunk kInformedShrink times about
// its centre and moved onto the proposal: row i, entry j = proposal_j +
// (grid_ij - mean_j) / kInformedShrink.  Entries the grid does not scan
// (equal in every row) take the proposal's value; scanned ones are searched
// finely around it.
constexpr double kInformedShrink = 8.0;
// iteration cap of those fits: from a start near the minimum LM converges in
// tens of iterations; starts that wander are cut off
constexpr int kInformedMaxIter = 100;

musr_fit_opts stage_opts(const musr_fit_opts* opts, int stage) {
    musr_fit_opts o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (stage == 1) o.max_iter = o.max_iter > 0 ? std::min(o.max_iter, kInformedMaxIter) : kInformedMaxIter;
    return o;
}
std::vector<double> informed_starts(const double* grid, int n_starts, int P, const double* proposal) {
    std::vector<double> s((size_t)n_starts * P);
    for (int j = 0; j < P; ++j) {
        double mean = 0.0;
        for (int i = 0; i < n_starts; ++i) mean += grid[(size_t)i * P + j];
        mean /= n_starts;
        for (int i = 0; i < n_starts; ++i) {
            const double g = grid[(size_t)i * P + j];
            s[(size_t)i * P + j] = g == mean ? proposal[j] : proposal[j] + (g - mean) / kInformedShrink;
        }
    }
    return s;
}
}  // namespace

int musr_fit_learned(musr_proposer p, musr_run run, int obj, const uint8_t* free_mask, const musr_fit_opts* opts,
                     double chi2ndf_max, const double* fallback_starts, int32_t n_fallback, double* theta_out,
                     musr_fit_result* out, int32_t* used_fallback) {
    if (!p || !run || !theta_out || !out || n_fallback < 0 || (n_fallback > 0 && !fallback_starts))
        return MUSR_EINVAL;
    if (used_fallback) *used_fallback = 0;
    int st = musr_proposer_propose(p, &run, 1, theta_out);
    if (st != MUSR_OK) return st;
    const std::vector<double> prop0(theta_out, theta_out + p->P);
    st = musr_fit(run, obj, theta_out, free_mask, opts, out);
    // after the first fallback stage only a converged fit counts (its starts are cut off early)
    auto good = [&](int s, bool converged_only = false) {
        return (s == MUSR_OK || (!converged_only && s == MUSR_ENOCONV)) && std::isfinite(out->value) &&
               out->ndf > 0 && out->value / out->ndf <= chi2ndf_max && in_widened_box(p, theta_out);
    };
    if (good(st) || n_fallback == 0) return st;
    if (st == MUSR_ECUDA || st == MUSR_ETIMEOUT) return st;
    // stage 1: the fallback grid shrunk onto the proposal (informed_starts);
    // stage 2 (if still not good): the fallback grid as given
    for (int stage = 1; stage <= 2; ++stage) {
        if (used_fallback) *used_fallback = stage;
        const std::vector<double> starts = stage == 1 ? informed_starts(fallback_starts, n_fallback, p->P, prop0.data())
                                                      : std::vector<double>(fallback_starts,
                                                                            fallback_starts + (size_t)n_fallback * p->P);
        const int nf = out->n_free;
        std::vector<double> th(p->P), cov(out->cov ? (size_t)nf * nf : 0);
        musr_fit_result r;
        memset(&r, 0, sizeof(r));
        r.cov = cov.empty() ? nullptr : cov.data();
        const musr_fit_opts so = stage_opts(opts, stage);
        int st2;
        if (stage == 1) {
            // one start after the other; the first converged fit within the threshold and the box ends the stage
            st2 = MUSR_ENOCONV;
            r.value = INFINITY;
            std::vector<double> t(p->P), c(cov.size());
            for (int i = 0; i < n_fallback; ++i) {
                std::copy(starts.begin() + (size_t)i * p->P, starts.begin() + (size_t)(i + 1) * p->P, t.begin());
                musr_fit_result ri;
                memset(&ri, 0, sizeof(ri));
                ri.cov = c.empty() ? nullptr : c.data();
                const int si = musr_fit(run, obj, t.data(), free_mask, &so, &ri);
                if (si == MUSR_ECUDA || si == MUSR_ETIMEOUT) return si;
                const int32_t it_sum = r.iters + ri.iters, ev_sum = r.n_evals + ri.n_evals;
                const bool ok = (si == MUSR_OK || si == MUSR_ENOCONV) && std::isfinite(ri.value);
                const bool accepted = si == MUSR_OK && ri.ndf > 0 && ri.value / ri.ndf <= chi2ndf_max &&
                                      in_widened_box(p, t.data());
                if (ok && (accepted || ri.value < r.value)) {
                    r = ri;
                    r.cov = cov.empty() ? nullptr : cov.data();
                    std::copy(c.begin(), c.end(), cov.begin());
                    std::copy(t.begin(), t.end(), th.begin());
                    st2 = si;
                }
                r.iters = it_sum;
                r.n_evals = ev_sum;
                if (accepted) break;
            }
        } else {
            st2 = musr_fit_multistart(run, obj, starts.data(), n_fallback, free_mask, &so, th.data(), &r);
        }
        if (st2 == MUSR_ECUDA || st2 == MUSR_ETIMEOUT) return st2;
        const int32_t iters = out->iters + r.iters, evals = out->n_evals + r.n_evals;
        const bool first_ok = (st == MUSR_OK || st == MUSR_ENOCONV) && std::isfinite(out->value);
        const bool second_ok = (st2 == MUSR_OK || st2 == MUSR_ENOCONV) && std::isfinite(r.value);
        if (second_ok && (!first_ok || r.value < out->value)) {
            double* user_cov = out->cov;
            *out = r;
            out->cov = user_cov;
            if (user_cov) std::copy(cov.begin(), cov.end(), user_cov);
            std::copy(th.begin(), th.end(), theta_out);
            st = st2;
        }
        out->iters = iters;
        out->n_evals = evals;
        if (good(st, stage == 1)) break;
    }
    return st;
}

int musr_fit_learned_batch(musr_proposer p, musr_gbatch batch, int obj, const uint8_t* free_masks,
                           const musr_fit_opts* opts, double chi2ndf_max, const double* fallback_starts,
                           int32_t n_fallback, double* thetas_out, musr_fit_result* results, int32_t* used_fallback) {
    if (!p || !batch || !thetas_out || !results || n_fallback < 0 || (n_fallback > 0 && !fallback_starts))
        return MUSR_EINVAL;
    if (!musr::gbatch_has_gn(batch)) return MUSR_EINVAL;
    const int n = musr::gbatch_n_runs(batch);
    std::vector<musr_run> runs(n);
    std::vector<int64_t> toff(n + 1, 0);
    for (int r = 0; r < n; ++r) {
        runs[r] = musr::gbatch_run(batch, r);
        toff[r + 1] = toff[r] + runs[r]->P;
        if (used_fallback) used_fallback[r] = 0;
    }
    int st = musr_proposer_propose(p, runs.data(), n, thetas_out);
    if (st != MUSR_OK) return st;
    const std::vector<double> prop0(thetas_out, thetas_out + toff[n]);
    st = musr_fit_batch(batch, obj, thetas_out, free_masks, opts, results);
    if (st != MUSR_OK && st != MUSR_ENOCONV && st != MUSR_EDOMAIN && st != MUSR_ENONFINITE) return st;
    // after the first fallback stage only a converged fit counts (its starts are cut off early)
    auto good = [&](int r, bool converged_only) {
        const musr_fit_result& x = results[r];
        return (x.status == MUSR_OK || (!converged_only && x.status == MUSR_ENOCONV)) && std::isfinite(x.value) &&
               x.ndf > 0 && x.value / x.ndf <= chi2ndf_max && in_widened_box(p, thetas_out + toff[r]);
    };
    // stage 1: the fallback grid shrunk onto the run's proposal (informed_starts);
    // stage 2, for the runs still not good: the grid as given
    for (int stage = 1; stage <= 2 && n_fallback > 0; ++stage) {
        std::vector<int> bad;
        for (int r = 0; r < n; ++r)
            if (!good(r, stage == 2)) bad.push_back(r);
        if (bad.empty()) break;
        std::vector<musr_run> fr;
        std::vector<double> fs, fth;
        std::vector<uint8_t> fm;
        for (int r : bad) {
            fr.push_back(runs[r]);
            const double* src = fallback_starts + toff[r] * n_fallback;
            const int P = runs[r]->P;
            if (stage == 1) {
                const std::vector<double> s = informed_starts(src, n_fallback, P, prop0.data() + toff[r]);
                fs.insert(fs.end(), s.begin(), s.end());
            } else {
                fs.insert(fs.end(), src, src + (size_t)P * n_fallback);
            }
            if (free_masks) fm.insert(fm.end(), free_masks + toff[r], free_masks + toff[r + 1]);
            fth.resize(fth.size() + P);
        }
        std::vector<musr_fit_result> fres(bad.size());
        for (auto& x : fres) memset(&x, 0, sizeof(x));
        const musr_fit_opts so = stage_opts(opts, stage);
        // stage 1: a run's first converged start within the threshold and the box ends its search
        std::vector<double> ndf(bad.size());
        for (size_t i = 0; i < bad.size(); ++i) {
            const int r = bad[i];
            int nfree = runs[r]->P;
            if (free_masks) {
                nfree = 0;
                for (int j = 0; j < runs[r]->P; ++j) nfree += free_masks[toff[r] + j] ? 1 : 0;
            }
            ndf[i] = (double)(runs[r]->total_bins - nfree);
        }
        const std::function<bool(int, const double*, double)> accept = [&](int i, const double* th, double f) {
            return std::isfinite(f) && ndf[i] > 0 && f / ndf[i] <= chi2ndf_max && in_widened_box(p, th);
        };
        const int st2 = musr::fit_multistart_batch_accept(fr.data(), (int)fr.size(), obj, fs.data(), n_fallback,
                                                          free_masks ? fm.data() : nullptr, &so,
                                                          stage == 1 ? &accept : nullptr, fth.data(), fres.data());
        if (st2 != MUSR_OK && st2 != MUSR_ENOCONV && st2 != MUSR_EDOMAIN && st2 != MUSR_ENONFINITE) return st2;
        int64_t o = 0;
        for (size_t i = 0; i < bad.size(); ++i) {
            const int r = bad[i];
            if (used_fallback) used_fallback[r] = stage;
            const musr_fit_result& x = fres[i];
            const int32_t iters = results[r].iters + x.iters, evals = results[r].n_evals + x.n_evals;
            const bool first_ok = (results[r].status == MUSR_OK || results[r].status == MUSR_ENOCONV) &&
                                  std::isfinite(results[r].value);
            const bool second_ok = (x.status == MUSR_OK || x.status == MUSR_ENOCONV) && std::isfinite(x.value);
            if (second_ok && (!first_ok || x.value < results[r].value)) {
                double* cov = results[r].cov;
                results[r] = x;
                results[r].cov = cov;
                if (cov)
                    for (int e = 0; e < x.n_free * x.n_free; ++e) cov[e] = NAN;
                memcpy(thetas_out + toff[r], fth.data() + o, sizeof(double) * runs[r]->P);
            }
            results[r].iters = iters;
            results[r].n_evals = evals;
            o += runs[r]->P;
        }
    }
    int worst = MUSR_OK;
    for (int r = 0; r < n; ++r)
        if (results[r].status != MUSR_OK && worst == MUSR_OK) worst = results[r].status;
    return worst;
}

}  // extern "C"
