// The run object behind the opaque musr_run handle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "musr.h"
#include "musr_internal.h"

namespace musr {
constexpr int kMaxParams = 4096;   // theta length
constexpr int kMaxGnParams = 1024; // Gauss-Newton output is P x P
}  // namespace musr

struct musr_run_s {
    int device = 0;
    // layout (host copy)
    int K = 0, P = 0, W = 0;
    std::vector<int64_t> n_bins;
    std::vector<int32_t> map;
    std::vector<musr_component> comp;
    double t0 = 0, dt = 0, tau = 0, gamma = 0;
    int64_t total_bins = 0;
    musr::Signature sig;
    int R = 0;
    std::vector<int32_t> role_theta;  // [K][kMaxRoles][2]
    // tiling
    int threads = 256, tile_bins = 2048, n_tiles = 0;
    std::vector<int32_t> tile_hist, tile_start, hist_first_tile, hist_ntiles;
    std::vector<int64_t> hist_off, model_off;
    size_t data_floats = 0;
    // device memory (one arena)
    void* arena = nullptr;
    float* d_data = nullptr;
    int64_t *d_hist_off = nullptr, *d_model_off = nullptr;
    int32_t *d_hist_nbins = nullptr, *d_tile_hist = nullptr, *d_tile_start = nullptr;
    int32_t *d_hist_first_tile = nullptr, *d_hist_ntiles = nullptr, *d_role_theta = nullptr;
    int32_t* d_csr_ptr[3] = {nullptr, nullptr, nullptr};
    int32_t* d_csr_src[3] = {nullptr, nullptr, nullptr};
    int n_out[3] = {0, 0, 0};
    double *d_partial = nullptr, *d_hist_sum = nullptr;
    unsigned* d_counters = nullptr;  // [K] per-histogram tickets, [1] global ticket, [1] flags
    double *d_theta = nullptr, *d_out = nullptr, *d_theta_tmp = nullptr;
    int32_t* d_status = nullptr;
    // pinned staging for host-pointer calls
    void* h_pinned = nullptr;
    double *h_theta = nullptr, *h_out = nullptr;
    int32_t* h_status = nullptr;
    // streams and cached graphs [objective][mode]
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t graphs[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    // batched plan over this run alone, used by the central-difference fit
    musr_batch fd_batch = nullptr;
    int fd_batch_vec = 0;

    int plan(const musr_run_desc* d);
    int build_tiles(int threads);
    void build_csr(int mode, std::vector<int32_t>& ptr, std::vector<int32_t>& src) const;
    int allocate();
    int upload(int dtype, const void* data, int on_device);
    musr::EvalParams params(int obj, int mode, const double* theta_dev, double* out_dev,
                            int32_t* status_dev) const;
    int launch(int obj, int mode, const double* theta_dev, double* out_dev, int32_t* status_dev,
               cudaStream_t st, float* model_out);
    int eval_host(int obj, int mode, const double* theta, double* out_host, int32_t* flags);
    ~musr_run_s();
};
