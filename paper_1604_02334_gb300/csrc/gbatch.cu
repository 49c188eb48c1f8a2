// Host side of the batched adjoint evaluation (see gbatch_kernel.cuh): the
// item plan and LPT schedule per mode, a small autotuner over launch shapes,
// host and device entry points.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <functional>
#include <new>
#include <queue>
#include <vector>

#include "gbatch_kernel.cuh"
#include "musr.h"
#include "musr_internal.h"
#include "run_impl.h"

namespace musr {
template <int MODE>
cudaError_t launch_gbatch_mode(const Signature& s, int blocks, int threads, size_t smem, cudaStream_t st,
                               const GParams& p);
extern template cudaError_t launch_gbatch_mode<kGrad>(const Signature&, int, int, size_t, cudaStream_t,
                                                      const GParams&);
extern template cudaError_t launch_gbatch_mode<kGN>(const Signature&, int, int, size_t, cudaStream_t,
                                                    const GParams&);
}  // namespace musr

using namespace musr;

namespace {

struct GShape {
    int threads = 256, blocks_per_sm = 2, rows = 8;
};

struct GPlan {
    GShape shape;
    int blocks = 0, n_items = 0;
    void* arena = nullptr;
    GRunRef* d_runs = nullptr;
    GWork* d_works = nullptr;
    int32_t *d_block_ptr = nullptr, *d_run_items = nullptr;
    int32_t *d_hist_item_ptr = nullptr, *d_run_nitems = nullptr;
    double* d_partial = nullptr;
    unsigned *d_run_count = nullptr, *d_flags = nullptr;
    bool tuned = false;
    void release() {
        if (arena) cudaFree(arena);
        arena = nullptr;
    }
};

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

int nacc_of(int mode, int R) { return mode == kGrad ? 1 + R : 1 + R + R * (R + 1) / 2; }

}  // namespace

struct musr_gbatch_s {
    int device = 0, sms = 152, with_gn = 0;
    std::vector<musr_run> runs;
    Signature sig;
    int R = 0, K_max = 0;
    std::vector<int64_t> theta_off;
    std::vector<int64_t> out_off[3];
    int64_t total_theta = 0, total_out[3] = {0, 0, 0};
    GPlan plan[3];  // by mode (kGrad, kGN)
    void* io = nullptr;
    double *d_thetas = nullptr, *d_out = nullptr;
    uint8_t* d_active = nullptr;
    int32_t* d_status = nullptr;
    void* h_pinned = nullptr;
    double *h_thetas = nullptr, *h_out = nullptr;
    uint8_t* h_active = nullptr;
    int32_t* h_status = nullptr;
    cudaStream_t stream = nullptr;

    int make_plan(int mode, const GShape& sh);
    GParams params(int mode, int obj, const double* thetas, const uint8_t* active, double* out, int32_t* status) const;
    int launch(int mode, int obj, const double* thetas, const uint8_t* active, double* out, int32_t* status,
               cudaStream_t st) const;
    int tune(int mode, int obj, const double* thetas);
    ~musr_gbatch_s() {
        if (stream) cudaStreamSynchronize(stream);
        for (auto& pl : plan) pl.release();
        if (io) cudaFree(io);
        if (h_pinned) cudaFreeHost(h_pinned);
        if (stream) cudaStreamDestroy(stream);
    }
};

int musr_gbatch_s::make_plan(int mode, const GShape& sh) {
    GPlan& pl = plan[mode];
    pl.release();
    pl.shape = sh;
    const int stripe = sh.threads * kBinsPerThread;
    std::vector<GItem> items;
    std::vector<int32_t> run_items, hist_item_ptr, run_nitems(runs.size());
    std::vector<GRunRef> refs(runs.size());
    for (size_t r = 0; r < runs.size(); ++r) {
        const musr_run_s* run = runs[r];
        GRunRef& Rr = refs[r];
        Rr.hist_ptr_off = (int32_t)hist_item_ptr.size();
        const int first = (int)run_items.size();
        for (int k = 0; k < run->K; ++k) {
            hist_item_ptr.push_back((int32_t)run_items.size());
            const int64_t M = run->n_bins[k];
            const int64_t rows_total = std::max<int64_t>(1, (M + stripe - 1) / stripe);
            for (int64_t r0 = 0; r0 < rows_total; r0 += sh.rows) {
                GItem it;
                it.run = (int32_t)r;
                it.hist = k;
                it.start = (int32_t)(r0 * stripe);
                it.rows = (int32_t)std::min<int64_t>(sh.rows, rows_total - r0);
                run_items.push_back((int32_t)items.size());
                items.push_back(it);
            }
        }
        hist_item_ptr.push_back((int32_t)run_items.size());
        run_nitems[r] = (int32_t)run_items.size() - first;
        Rr.data = run->d_data;
        Rr.hist_off = run->d_hist_off;
        Rr.hist_nbins = run->d_hist_nbins;
        Rr.role_theta = run->d_role_theta;
        Rr.csr_ptr = run->d_csr_ptr[mode];
        Rr.csr_src = run->d_csr_src[mode];
        Rr.csr_row = run->d_csr_row[mode];
        Rr.n_rows = run->n_rows[mode];
        Rr.rc = run->rc;
        Rr.etab = run->d_etab;
        Rr.t0 = run->t0;
        Rr.dt = run->dt;
        Rr.P = run->P;
        Rr.K = run->K;
        Rr.n_out = run->n_out[mode];
        Rr.theta_off = theta_off[r];
        Rr.out_off = out_off[mode][r];
    }
    pl.n_items = (int)items.size();
    pl.blocks = std::max(1, std::min(pl.n_items, sms * sh.blocks_per_sm));
    // LPT: longest item first onto the least-loaded block
    std::vector<int32_t> order(pl.n_items);
    for (int i = 0; i < pl.n_items; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return items[a].rows > items[b].rows; });
    using Load = std::pair<double, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int b = 0; b < pl.blocks; ++b) heap.push({0.0, b});
    std::vector<std::vector<int32_t>> assign(pl.blocks);
    for (int i : order) {
        Load l = heap.top();
        heap.pop();
        assign[l.second].push_back(i);
        heap.push({l.first + 1.0 + (double)items[i].rows, l.second});  // + staging cost of one row
    }
    // the items as the blocks take them: one self-contained descriptor each
    std::vector<int32_t> block_ptr(pl.blocks + 1, 0);
    std::vector<GWork> works;
    works.reserve(items.size());
    for (int b = 0; b < pl.blocks; ++b) {
        for (int32_t i : assign[b]) {
            const GItem& it = items[i];
            const musr_run_s* run = runs[it.run];
            GWork w;
            memset(&w, 0, sizeof(w));
            w.rc = run->rc;
            w.hdata = run->d_data + run->hist_off[it.hist];
            w.etab = run->d_etab;
            w.theta_off = theta_off[it.run];
            w.item = i;
            w.run = it.run;
            w.start = it.start;
            w.rows = it.rows;
            w.M = (int32_t)run->n_bins[it.hist];
            w.dtf = (float)run->dt;
            w.t0f = (float)run->t0;
            memcpy(w.rt, run->role_theta.data() + (size_t)it.hist * kMaxRoles * 2, sizeof(w.rt));
            works.push_back(w);
        }
        block_ptr[b + 1] = (int32_t)works.size();
    }
    const int nacc = nacc_of(mode, R);
    size_t sz = 0;
    auto take = [&](size_t bytes) {
        const size_t at = sz;
        sz += al256(bytes);
        return at;
    };
    const size_t o_runs = take(sizeof(GRunRef) * refs.size()), o_works = take(sizeof(GWork) * works.size());
    const size_t o_bp = take(sizeof(int32_t) * block_ptr.size());
    const size_t o_ri = take(sizeof(int32_t) * run_items.size()), o_hp = take(sizeof(int32_t) * hist_item_ptr.size());
    const size_t o_rn = take(sizeof(int32_t) * run_nitems.size());
    const size_t o_part = take(sizeof(double) * (size_t)pl.n_items * nacc);
    const size_t o_cnt = take(sizeof(unsigned) * runs.size()), o_fl = take(sizeof(unsigned) * runs.size());
    if (cudaMalloc(&pl.arena, sz) != cudaSuccess) {
        pl.arena = nullptr;
        return MUSR_ENOMEM;
    }
    char* a = static_cast<char*>(pl.arena);
    pl.d_runs = reinterpret_cast<GRunRef*>(a + o_runs);
    pl.d_works = reinterpret_cast<GWork*>(a + o_works);
    pl.d_block_ptr = reinterpret_cast<int32_t*>(a + o_bp);
    pl.d_run_items = reinterpret_cast<int32_t*>(a + o_ri);
    pl.d_hist_item_ptr = reinterpret_cast<int32_t*>(a + o_hp);
    pl.d_run_nitems = reinterpret_cast<int32_t*>(a + o_rn);
    pl.d_partial = reinterpret_cast<double*>(a + o_part);
    pl.d_run_count = reinterpret_cast<unsigned*>(a + o_cnt);
    pl.d_flags = reinterpret_cast<unsigned*>(a + o_fl);
    cudaError_t e = cudaMemsetAsync(pl.arena, 0, sz, stream);
    auto up = [&](void* dst, const void* src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream);
    };
    up(pl.d_runs, refs.data(), sizeof(GRunRef) * refs.size());
    up(pl.d_works, works.data(), sizeof(GWork) * works.size());
    up(pl.d_block_ptr, block_ptr.data(), sizeof(int32_t) * block_ptr.size());
    up(pl.d_run_items, run_items.data(), sizeof(int32_t) * run_items.size());
    up(pl.d_hist_item_ptr, hist_item_ptr.data(), sizeof(int32_t) * hist_item_ptr.size());
    up(pl.d_run_nitems, run_nitems.data(), sizeof(int32_t) * run_nitems.size());
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    return cuda_status(e);
}

GParams musr_gbatch_s::params(int mode, int obj, const double* thetas, const uint8_t* active, double* out,
                              int32_t* status) const {
    const GPlan& pl = plan[mode];
    GParams p;
    memset(&p, 0, sizeof(p));
    p.runs = pl.d_runs;
    p.works = pl.d_works;
    p.block_ptr = pl.d_block_ptr;
    p.run_items = pl.d_run_items;
    p.hist_item_ptr = pl.d_hist_item_ptr;
    p.run_nitems = pl.d_run_nitems;
    p.thetas = thetas;
    p.active = active;
    p.obj = obj;
    p.partial = pl.d_partial;
    p.run_count = pl.d_run_count;
    p.flags = pl.d_flags;
    p.out = out;
    p.status = status;
    return p;
}

int musr_gbatch_s::launch(int mode, int obj, const double* thetas, const uint8_t* active, double* out,
                          int32_t* status, cudaStream_t st) const {
    const GPlan& pl = plan[mode];
    const size_t smem = sizeof(double) * (size_t)K_max * nacc_of(mode, R);
    const GParams p = params(mode, obj, thetas, active, out, status);
    cudaError_t e = mode == kGrad ? launch_gbatch_mode<kGrad>(sig, pl.blocks, pl.shape.threads, smem, st, p)
                                  : launch_gbatch_mode<kGN>(sig, pl.blocks, pl.shape.threads, smem, st, p);
    return cuda_status(e);
}

// Time a few launch shapes with the caller's first parameter vectors and keep
// the fastest plan for this mode.
int musr_gbatch_s::tune(int mode, int obj, const double* thetas) {
    const GShape cands[] = {{256, 1, 8}, {256, 1, 16}, {256, 2, 8}, {256, 2, 16},
                            {256, 3, 4}, {256, 3, 8}, {256, 3, 16}, {128, 2, 16}};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return MUSR_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return MUSR_ECUDA;
    }
    float best = INFINITY;
    GShape best_shape = cands[0];
    int st = MUSR_OK;
    for (const GShape& c : cands) {
        st = make_plan(mode, c);
        if (st != MUSR_OK) break;
        st = launch(mode, obj, thetas, nullptr, d_out, d_status, stream);  // warm-up
        float ms = INFINITY;
        for (int rep = 0; rep < 3 && st == MUSR_OK; ++rep) {
            cudaEventRecord(e0, stream);
            st = launch(mode, obj, thetas, nullptr, d_out, d_status, stream);
            cudaEventRecord(e1, stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = MUSR_ECUDA;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = std::min(ms, t);
        }
        if (st != MUSR_OK) break;
        if (ms < best) {
            best = ms;
            best_shape = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == MUSR_OK) st = make_plan(mode, best_shape);
    if (st == MUSR_OK) plan[mode].tuned = true;
    return st;
}

namespace musr {

// Evaluate mode (kGrad / kGN) for every run with active[r] != 0 (active NULL:
// all) from host parameter vectors; host outputs by run (1 + P (+ P*P)) and
// per-run flags (bit 0: deviance domain, bit 1: non-finite).
int gbatch_eval_host(musr_gbatch b, int obj, int mode, const double* thetas, const uint8_t* active, double* out,
                     int32_t* flags) {
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != b->device) cudaSetDevice(b->device);
    const size_t nr = b->runs.size();
    memcpy(b->h_thetas, thetas, sizeof(double) * b->total_theta);
    if (active) memcpy(b->h_active, active, nr);
    cudaError_t e = cudaMemcpyAsync(b->d_thetas, b->h_thetas, sizeof(double) * b->total_theta,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && active)
        e = cudaMemcpyAsync(b->d_active, b->h_active, nr, cudaMemcpyHostToDevice, b->stream);
    int st = cuda_status(e);
    if (st == MUSR_OK && !b->plan[mode].tuned) st = b->tune(mode, obj, b->d_thetas);
    if (st == MUSR_OK) st = b->launch(mode, obj, b->d_thetas, active ? b->d_active : nullptr, b->d_out, b->d_status,
                                      b->stream);
    if (st == MUSR_OK)
        st = cuda_status(cudaMemcpyAsync(b->h_out, b->d_out, sizeof(double) * b->total_out[mode],
                                         cudaMemcpyDeviceToHost, b->stream));
    if (st == MUSR_OK)
        st = cuda_status(cudaMemcpyAsync(b->h_status, b->d_status, sizeof(int32_t) * nr, cudaMemcpyDeviceToHost,
                                         b->stream));
    if (st == MUSR_OK) st = cuda_status(cudaStreamSynchronize(b->stream));
    if (st == MUSR_OK) {
        for (size_t r = 0; r < nr; ++r) {
            if (active && !active[r]) continue;
            const int64_t o = b->out_off[mode][r];
            if (out) memcpy(out + o, b->h_out + o, sizeof(double) * b->runs[r]->n_out[mode]);
            if (flags) flags[r] = b->h_status[r];
        }
    }
    if (cur != b->device) cudaSetDevice(cur);
    return st;
}

// the pinned host copy of the last gbatch_eval_host outputs (valid until the next call)
const double* gbatch_host_out(musr_gbatch b) { return b->h_out; }
int64_t gbatch_out_offset(musr_gbatch b, int mode, int r) { return b->out_off[mode][r]; }
int64_t gbatch_theta_offset(musr_gbatch b, int r) { return b->theta_off[r]; }
int64_t gbatch_total_out(musr_gbatch b, int mode) { return b->total_out[mode]; }
int gbatch_has_gn(musr_gbatch b) { return b->with_gn; }
int gbatch_n_runs(musr_gbatch b) { return (int)b->runs.size(); }
musr_run gbatch_run(musr_gbatch b, int r) { return b->runs[r]; }

}  // namespace musr

extern "C" {

int musr_gbatch_destroy(musr_gbatch b) {
    delete b;
    return MUSR_OK;
}

int musr_gbatch_create(const musr_run* runs, int32_t n_runs, int32_t with_gn, musr_gbatch* out) {
    if (!runs || n_runs <= 0 || !out) return MUSR_EINVAL;
    *out = nullptr;
    for (int r = 0; r < n_runs; ++r) {
        if (!runs[r] || runs[r]->K <= 0) return MUSR_EINVAL;  // a run without histograms has no items
        if (runs[r]->F > 0) return MUSR_ENOTSUP;               // function values are formed per host call
        const Signature& s = runs[r]->sig;
        if (s != runs[0]->sig || runs[r]->device != runs[0]->device)
            return MUSR_EINVAL;
        if (with_gn && runs[r]->P > kMaxGnParams) return MUSR_ENOTSUP;
    }
    musr_gbatch b = new (std::nothrow) musr_gbatch_s();
    if (!b) return MUSR_ENOMEM;
    b->device = runs[0]->device;
    b->with_gn = with_gn ? 1 : 0;
    b->runs.assign(runs, runs + n_runs);
    b->sig = runs[0]->sig;
    b->R = b->sig.roles();
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != b->device) cudaSetDevice(b->device);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    for (int m = 0; m < 3; ++m) b->out_off[m].assign(n_runs, 0);
    for (int r = 0; r < n_runs; ++r) {
        musr_run run = runs[r];
        b->K_max = std::max(b->K_max, run->K);
        b->theta_off.push_back(b->total_theta);
        b->total_theta += run->P;
        for (int m = kGrad; m <= kGN; ++m) {
            b->out_off[m][r] = b->total_out[m];
            b->total_out[m] += run->n_out[m];
        }
    }
    const int top = b->with_gn ? kGN : kGrad;
    int st = MUSR_OK;
    const size_t smem = sizeof(double) * (size_t)b->K_max * nacc_of(top, b->R);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
    if (smem + 16384 > (size_t)optin) st = MUSR_ENOTSUP;
    const size_t n_out = (size_t)b->total_out[top];
    size_t o_th = 0, o_out = al256(sizeof(double) * b->total_theta);
    size_t o_act = o_out + al256(sizeof(double) * n_out), o_st = o_act + al256((size_t)n_runs);
    size_t sz = o_st + al256(sizeof(int32_t) * n_runs);
    if (st == MUSR_OK && cudaMalloc(&b->io, sz) != cudaSuccess) {
        b->io = nullptr;
        st = MUSR_ENOMEM;
    }
    if (st == MUSR_OK && cudaMallocHost(&b->h_pinned, sz) != cudaSuccess) {
        b->h_pinned = nullptr;
        st = MUSR_ENOMEM;
    }
    if (st == MUSR_OK) st = cuda_status(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    if (st == MUSR_OK) {
        char* d = static_cast<char*>(b->io);
        char* h = static_cast<char*>(b->h_pinned);
        b->d_thetas = reinterpret_cast<double*>(d + o_th);
        b->d_out = reinterpret_cast<double*>(d + o_out);
        b->d_active = reinterpret_cast<uint8_t*>(d + o_act);
        b->d_status = reinterpret_cast<int32_t*>(d + o_st);
        b->h_thetas = reinterpret_cast<double*>(h + o_th);
        b->h_out = reinterpret_cast<double*>(h + o_out);
        b->h_active = reinterpret_cast<uint8_t*>(h + o_act);
        b->h_status = reinterpret_cast<int32_t*>(h + o_st);
        st = cuda_status(cudaMemsetAsync(b->io, 0, sz, b->stream));
        if (st == MUSR_OK) st = cuda_status(cudaStreamSynchronize(b->stream));
    }
    for (int m = kGrad; m <= top && st == MUSR_OK; ++m) st = b->make_plan(m, GShape{});
    if (cur != b->device) cudaSetDevice(cur);
    if (st != MUSR_OK) {
        delete b;
        return st;
    }
    *out = b;
    return MUSR_OK;
}

int musr_gbatch_eval(musr_gbatch b, int obj, int mode, const double* thetas, const uint8_t* active, double* out,
                     int32_t* flags) {
    if (!b || !thetas || !out) return MUSR_EINVAL;
    if (obj != MUSR_CHI2 && obj != MUSR_POISSON) return MUSR_EINVAL;
    if (mode != MUSR_VALUE_GRAD && !(mode == MUSR_VALUE_GRAD_GN && b->with_gn)) return MUSR_EINVAL;
    for (int64_t i = 0; i < b->total_theta; ++i)
        if (!std::isfinite(thetas[i])) return MUSR_ENONFINITE;
    return musr::gbatch_eval_host(b, obj, mode, thetas, active, out, flags);
}

int musr_gbatch_eval_device(musr_gbatch b, int obj, int mode, const double* thetas_dev, double* out_dev,
                            int32_t* flags_dev, void* stream) {
    if (!b || !thetas_dev || !out_dev) return MUSR_EINVAL;
    if (obj != MUSR_CHI2 && obj != MUSR_POISSON) return MUSR_EINVAL;
    if (mode != MUSR_VALUE_GRAD && !(mode == MUSR_VALUE_GRAD_GN && b->with_gn)) return MUSR_EINVAL;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != b->device) cudaSetDevice(b->device);
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : b->stream;
    int st = MUSR_OK;
    if (!b->plan[mode].tuned) {
        // tuning synchronises; it runs on the batch's own stream after the caller's work
        cudaEvent_t ev;
        st = cuda_status(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        if (st == MUSR_OK) {
            cudaEventRecord(ev, s);
            cudaStreamWaitEvent(b->stream, ev, 0);
            cudaEventDestroy(ev);
            st = b->tune(mode, obj, thetas_dev);
        }
    }
    if (st == MUSR_OK) st = b->launch(mode, obj, thetas_dev, nullptr, out_dev, flags_dev, s);
    if (cur != b->device) cudaSetDevice(cur);
    return st;
}

}  // extern "C"
