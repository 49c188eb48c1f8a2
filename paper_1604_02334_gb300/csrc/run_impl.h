// The run object behind the opaque musr_run handle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <vector>

#include "musr.h"
#include "musr_internal.h"

namespace musr {
constexpr int kMaxParams = 4096;   // theta length
constexpr int kMaxGnParams = 1024; // Gauss-Newton output is P x P
constexpr int kMaxFuncs = 64;      // function array entries per run

// A function-array expression compiled to a postfix program (funcs.cpp).
struct HostExpr {
    struct Ins {
        int op, i;
        double c;
    };
    std::vector<Ins> code;
    std::vector<int> refs;  // theta indices it reads, ascending
    int depth = 0;          // evaluation stack depth
};
// MUSR_OK or MUSR_EINVAL (syntax, or an index outside theta[0, P)).
int compile_host_expr(const char* text, int P, HostExpr& out);
// Value at theta; with dvar >= 0 also the derivative along theta[dvar].
double eval_host_expr(const HostExpr& e, const double* theta, int dvar, double* deriv);

// Generator body: rebinned Poisson samples of n_samples parameter vectors,
// sample s written at out_dev + s * row_stride (row_stride 0: packed).
int generate_rows(musr_run run, const double* thetas_dev, int n_samples, int rebin, uint64_t seed,
                  uint64_t sample_offset, int log1p_out, float* out_dev, float* mu_dev, int64_t row_stride,
                  cudaStream_t stream);
// Group offsets of a rebin factor, cached in the run (run->d_group_off).
int ensure_groups(musr_run run, int rebin);
// Uniform draws of the learned parameters (see generate.cu) and the matching
// targets 2u - 1; fixed parameters take lo.
int sample_uniform_thetas(const double* lo_dev, const double* hi_dev, const int32_t* learned_dev, int n_learned,
                          int P, int n, uint64_t seed, uint64_t offset, double* thetas_dev, float* targets_dev,
                          cudaStream_t st);
// The run's data summed over groups of `rebin` bins, one row.
int rebin_sum_row(musr_run run, int rebin, float* out_dev, cudaStream_t st);
// musr_fit_multistart_batch; with accept non-null, the first start of run
// r that converges with accept(r, theta, value) true stops r's other starts
// and is r's result (fit.cpp).
int fit_multistart_batch_accept(const musr_run* runs, int n_runs, int obj, const double* starts, int n_starts,
                                const uint8_t* free_masks, const musr_fit_opts* opts,
                                const std::function<bool(int, const double*, double)>* accept, double* thetas_out,
                                musr_fit_result* results);
}  // namespace musr

struct musr_run_s {
    int device = 0;
    // layout (host copy)
    int K = 0, P = 0, W = 0;
    // function array (Sec. 4.2.1): F host expressions whose values the kernels
    // read as parameter slots P .. P + F - 1 (Pk = P + F slots in all)
    int F = 0, Pk = 0;
    std::vector<musr::HostExpr> funcs;
    std::vector<int64_t> n_bins;
    std::vector<int32_t> map;
    std::vector<musr_component> comp;
    double t0 = 0, dt = 0, tau = 0, gamma = 0;
    musr::RunConst rc;  // theta-independent constants of the time grid
    int64_t total_bins = 0;
    musr::Signature sig;
    int R = 0;
    std::vector<int32_t> role_theta;  // [K][kMaxRoles][2]
    // tiling, per mode (value, grad, GN, model): tiles are ranges of 8-bin
    // chunks of one histogram (histogram k split into tph[k] near-equal
    // ranges), sized so a launch is about one wave of resident blocks with an
    // even share of bins per SM
    struct Tiling {
        int threads = 256, n_tiles = 0, uni_tph = 0;  // uni_tph: tiles per histogram when all are equal
        // tiles per histogram for queued evaluations (equal histograms only,
        // else 0): fewer, longer tiles than uni_tph (see the planner)
        int uni_tph_queued = 0;
        std::vector<int32_t> tile_hist, tile_start, tile_end;
        int32_t *d_tile_hist = nullptr, *d_tile_start = nullptr, *d_tile_end = nullptr;
    };
    Tiling tl[4];
    std::vector<int64_t> hist_off, model_off;
    size_t data_floats = 0;
    // device memory (one arena)
    void* arena = nullptr;
    float* d_data = nullptr;
    int64_t *d_hist_off = nullptr, *d_model_off = nullptr;
    int32_t* d_hist_nbins = nullptr;
    int32_t* d_role_theta = nullptr;
    int32_t* d_map = nullptr;  // [K][W] the descriptor's map rows
    float* d_etab = nullptr;   // lifetime factor at every chunk start (lifetime_table_len)
    int64_t etab_len = 0;
    int32_t* d_csr_ptr[3] = {nullptr, nullptr, nullptr};
    int32_t* d_csr_src[3] = {nullptr, nullptr, nullptr};
    // Gauss-Newton: the map's rows are the outputs that have sources (their
    // output index in d_csr_row); value and gradient: row = output, no table
    int32_t* d_csr_row[3] = {nullptr, nullptr, nullptr};
    int n_out[3] = {0, 0, 0};
    int n_src[3] = {0, 0, 0};
    int n_rows[3] = {0, 0, 0};
    // dynamic shared memory of the reduction tail per mode
    int hsum_in_smem[3] = {0, 0, 0}, csr_in_smem[3] = {0, 0, 0};
    int smem_bytes[3] = {0, 0, 0};
    unsigned long long* d_facc = nullptr;  // fixed-point limbs, K x nacc x 3
    __int128* d_hist_sum = nullptr;
    unsigned* d_counters = nullptr;  // [0] global ticket, [1] flags
    double *d_theta = nullptr, *d_out = nullptr, *d_theta_tmp = nullptr;
    int32_t* d_status = nullptr;
    // pinned staging for host-pointer calls
    void* h_pinned = nullptr;
    double *h_theta = nullptr, *h_out = nullptr;
    int32_t* h_status = nullptr;
    double* hd_out = nullptr;     // device view of h_out
    int32_t* hd_status = nullptr; // device view of h_status
    // streams
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    bool own_stream = false;
    // generator: group offsets for the cached rebin factor
    int64_t* d_group_off = nullptr;
    int gen_rebin = 0;
    int64_t gen_per_sample = 0;
    // batched plan over this run alone, used by the central-difference fit
    musr_batch fd_batch = nullptr;
    int fd_batch_vec = 0;

    int plan(const musr_run_desc* d);
    // tiles per histogram for a target tile count (>= 1 each, about
    // proportional to its chunks, each tile at least one chunk per thread)
    std::vector<int64_t> tiles_per_hist(int threads, int64_t target) const;
    void build_tiles(Tiling& t, int threads, const std::vector<int64_t>& tph) const;
    int tail_smem(int mode, int* hsum_smem, int* csr_smem) const;
    void build_csr(int mode, std::vector<int32_t>& ptr, std::vector<int32_t>& src, std::vector<int32_t>& rows) const;
    int allocate();
    int upload(int dtype, const void* data, int on_device);
    musr::EvalParams params(int obj, int mode, const double* theta_dev, double* out_dev,
                            int32_t* status_dev) const;
    int launch(int obj, int mode, const double* theta_dev, double* out_dev, int32_t* status_dev,
               cudaStream_t st, float* model_out);
    // theta (P entries) -> the kernels' Pk slots, and the derivatives of the
    // function slots (jac[j][r] = d f_j / d theta[funcs[j].refs[r]])
    int extend_theta(const double* theta, double* ext, std::vector<std::vector<double>>* jac) const;
    // out_host: value (+ gradient, + Gauss-Newton matrix) over the P parameters
    // view != null and no function array: the results are left in the run's
    // pinned buffer, *view pointing at them (valid until the next call), and
    // out_host is not written
    int eval_host(int obj, int mode, const double* theta, double* out_host, int32_t* flags,
                  const double** view = nullptr);
    ~musr_run_s();
};
