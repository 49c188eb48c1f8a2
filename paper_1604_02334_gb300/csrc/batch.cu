// Batched evaluation: many runs of uneven size, each with many parameter
// vectors (the P + 1 vectors of a Jacobian / line search), in ONE persistent
// launch replayed from a CUDA graph.
//
// Work is cut into items (run, histogram, first bin, rows): a row is one
// block-wide stripe of threads x 8 bins.  A host-side LPT schedule (longest
// item first onto the least-loaded block) gives each persistent block a fixed
// list of items.  For each item the block stages the per-histogram constants
// of ALL the run's vectors into shared memory once, then every thread loads
// its 8 bins once per row and evaluates them for every vector, so the data is
// read from HBM once per launch however many vectors there are.  Per-vector
// FP32 warp sums become FP64 item partials; the last item of each run sums
// its items in a fixed order (bitwise repeatable).  Block size, persistent
// grid and rows per item are chosen by a small autotuner on first use.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <functional>
#include <queue>
#include <vector>

#include "eval_kernel.cuh"
#include "musr.h"
#include "musr_internal.h"
#include "run_impl.h"

namespace musr {

constexpr int kBatchMaxVec = 128;

struct BatchRunRef {
    const float* data;
    const int64_t* hist_off;
    const int32_t* hist_nbins;
    const int32_t* role_theta;
    const float* etab;      // lifetime factor at every chunk start
    RunConst rc;
    double t0, dt;
    int32_t P, V;           // parameters, vectors evaluated this launch
    int64_t theta_off;      // offset of the run's first vector in thetas
    int64_t val_off;        // offset of the run's first value
    int32_t item_first;     // into run_items
    int32_t n_items;
};

struct BatchItem {
    int32_t run, hist, start, rows;
    int64_t slot;  // partial offset (V doubles)
};

struct BatchParams {
    const BatchRunRef* runs;
    const BatchItem* items;
    const int32_t* block_ptr;
    const int32_t* block_items;
    const int32_t* run_items;
    const int64_t* item_slot;  // [n_items] partial offset of each item
    const double* thetas;
    int obj;
    double* partial;
    unsigned* run_count;
    unsigned* flags;  // per value
    double* values;
};

template <int NE, int NG, int NS, int KT>
__global__ void __launch_bounds__(kMaxThreads) batch_kernel(const BatchParams p) {
    constexpr int NPART = stage_parts<NE, NG, NS, KT>();
    constexpr int G = kBinsPerThread;
    extern __shared__ unsigned char smem_raw[];
    HistConst* hcs = reinterpret_cast<HistConst*>(smem_raw);
    __shared__ float red[kMaxWarps][kBatchMaxVec];
    __shared__ int s_last;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int stripe = blockDim.x * G;

    for (int it = p.block_ptr[blockIdx.x]; it < p.block_ptr[blockIdx.x + 1]; ++it) {
        const int item_idx = p.block_items[it];
        const BatchItem item = p.items[item_idx];
        const BatchRunRef& R = p.runs[item.run];
        const int V = R.V;
        const int k = item.hist;
        const int M = R.hist_nbins[k];
        const float* hdata = R.data + R.hist_off[k];

        __syncthreads();  // the previous item is done with hcs / red
        {
            const int32_t* rt = R.role_theta + (size_t)k * kMaxRoles * 2;
            for (int q = threadIdx.x; q < V * NPART; q += blockDim.x) {
                const int v = q / NPART, part = q % NPART;
                stage_part<NE, NG, NS, KT>(part, ThetaByRow{rt, p.thetas + R.theta_off + (int64_t)v * R.P}, R.rc, hcs[v]);
            }
        }
        for (int v = threadIdx.x; v < V; v += blockDim.x)
            for (int w = 0; w < nwarps; ++w) red[w][v] = 0.f;
        __syncthreads();

        const float dtf = (float)R.dt, t0f = (float)R.t0;
        for (int row = 0; row < item.rows; ++row) {
            const int n0 = item.start + row * stripe + (int)threadIdx.x * G;
            const bool active = n0 < M;
            float d[G];
            float E0 = 0.f;
            if (active) {
                E0 = __ldg(R.etab + (n0 >> 3));
                const float4* src = reinterpret_cast<const float4*>(hdata + n0);
                const float4 a = __ldg(src), b = __ldg(src + 1);
                d[0] = a.x; d[1] = a.y; d[2] = a.z; d[3] = a.w;
                d[4] = b.x; d[5] = b.y; d[6] = b.z; d[7] = b.w;
            } else {
#pragma unroll
                for (int g = 0; g < G; ++g) d[g] = 0.f;
            }
            for (int v = 0; v < V; ++v) {
                float acc[1] = {0.f};
                bool bad = false;
                if (active)
                    eval_chunk<NE, NG, NS, KT, kValue, 1>(hcs[v], n0, M, d, E0, p.obj, dtf, t0f, acc, bad, nullptr);
                if (bad) atomicOr(&p.flags[R.val_off + v], 1u);
                float s = acc[0];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) red[warp][v] += s;
            }
        }
        __syncthreads();
        for (int v = threadIdx.x; v < V; v += blockDim.x) {
            double s = 0.0;
            for (int w = 0; w < nwarps; ++w) s += (double)red[w][v];
            p.partial[item.slot + v] = s;
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned prev = atomicAdd(&p.run_count[item.run], 1u);
            s_last = prev == (unsigned)R.n_items - 1u;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            for (int v = threadIdx.x; v < V; v += blockDim.x) {
                double s = 0.0;
                for (int j0 = 0; j0 < R.n_items; j0 += 8) {
                    // eight item partials in flight, then added in order
                    int64_t slot[8];
                    double x[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        slot[u] = j0 + u < R.n_items ? p.item_slot[p.run_items[R.item_first + j0 + u]] : -1;
#pragma unroll
                    for (int u = 0; u < 8; ++u) x[u] = slot[u] >= 0 ? __ldcg(p.partial + slot[u] + v) : 0.0;
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (slot[u] >= 0) s += x[u];
                }
                const unsigned f = atomicExch(&p.flags[R.val_off + v], 0u);
                p.values[R.val_off + v] = f ? (double)INFINITY : s;
            }
            __syncthreads();
            if (threadIdx.x == 0) p.run_count[item.run] = 0u;
        }
    }
}

template <int NE, int NG, int NS, int KT>
cudaError_t launch_batch_sig(int blocks, int threads, size_t smem, cudaStream_t st, const BatchParams& p) {
    auto kern = batch_kernel<NE, NG, NS, KT>;
    // per-kernel attribute shared by every plan: raise it once to the opt-in maximum
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes < smem) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
    }
    kern<<<blocks, threads, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_batch(const Signature& s, int blocks, int threads, size_t smem, cudaStream_t st,
                         const BatchParams& p) {
#define MUSR_CASE(NE, NG, NS, KT)                             \
    if (s.ne == NE && s.ng == NG && s.ns == NS && s.kt == KT) \
        return launch_batch_sig<NE, NG, NS, KT>(blocks, threads, smem, st, p);
    MUSR_FOR_EACH_SIGNATURE(MUSR_CASE)
#undef MUSR_CASE
    return cudaErrorInvalidValue;
}

}  // namespace musr

using namespace musr;

namespace {
}  // namespace

// Launch shape chosen by the autotuner.
struct BatchShape {
    int threads = 256, blocks_per_sm = 2, rows = 4;
};

struct musr_batch_s {
    int device = 0;
    int sms = 152;
    std::vector<musr_run> runs;
    std::vector<int32_t> max_vec;
    Signature sig;
    int vmax = 0;
    std::vector<int64_t> theta_off, val_off;
    int64_t total_theta = 0, total_vals = 0;
    bool tuned = false;
    BatchShape shape;
    int blocks = 0;
    int n_items = 0;
    int64_t partial_len = 0;
    // device
    void* arena = nullptr;   // tables + scratch of the current plan
    void* io = nullptr;      // thetas and values (outlive re-planning)
    BatchRunRef* d_runs = nullptr;
    BatchItem* d_items = nullptr;
    int32_t *d_block_ptr = nullptr, *d_block_items = nullptr, *d_run_items = nullptr;
    int64_t* d_item_slot = nullptr;
    double *d_partial = nullptr, *d_thetas = nullptr, *d_values = nullptr;
    unsigned *d_run_count = nullptr, *d_flags = nullptr;
    void* h_pinned = nullptr;
    double *h_thetas = nullptr, *h_values = nullptr;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    std::vector<BatchRunRef> refs;

    int plan(const BatchShape& sh);
    BatchParams params(int obj, const double* thetas, double* values) const;
    int launch(int obj, const double* thetas, double* values, cudaStream_t st) const;
    int tune(int obj, const double* thetas);
    void free_plan();
    ~musr_batch_s() {
        free_plan();
        if (io) cudaFree(io);
        for (int o = 0; o < 2; ++o)
            if (graph[o]) cudaGraphExecDestroy(graph[o]);
        if (h_pinned) cudaFreeHost(h_pinned);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (stream) cudaStreamDestroy(stream);
    }
};

void musr_batch_s::free_plan() {
    if (arena) cudaFree(arena);
    arena = nullptr;
}

// Build items, the LPT schedule and the device tables for one launch shape.
int musr_batch_s::plan(const BatchShape& sh) {
    free_plan();
    shape = sh;
    const int stripe = sh.threads * kBinsPerThread;
    std::vector<BatchItem> items;
    std::vector<std::vector<int32_t>> per_run(runs.size());
    int64_t slot = 0;
    for (size_t r = 0; r < runs.size(); ++r) {
        const musr_run_s* run = runs[r];
        for (int k = 0; k < run->K; ++k) {
            const int64_t M = run->n_bins[k];
            const int64_t rows_total = std::max<int64_t>(1, (M + stripe - 1) / stripe);
            for (int64_t r0 = 0; r0 < rows_total; r0 += sh.rows) {
                BatchItem it;
                it.run = (int32_t)r;
                it.hist = k;
                it.start = (int32_t)(r0 * stripe);
                it.rows = (int32_t)std::min<int64_t>(sh.rows, rows_total - r0);
                it.slot = slot;
                slot += max_vec[r];
                per_run[r].push_back((int32_t)items.size());
                items.push_back(it);
            }
        }
    }
    n_items = (int)items.size();
    partial_len = slot;
    blocks = std::max(1, std::min(n_items, sms * sh.blocks_per_sm));
    // LPT: longest item first onto the least-loaded block
    std::vector<int32_t> order(n_items);
    for (int i = 0; i < n_items; ++i) order[i] = i;
    auto cost = [&](int i) { return (double)items[i].rows * (double)max_vec[items[i].run]; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    using Load = std::pair<double, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int b = 0; b < blocks; ++b) heap.push({0.0, b});
    std::vector<std::vector<int32_t>> assign(blocks);
    for (int i : order) {
        Load l = heap.top();
        heap.pop();
        assign[l.second].push_back(i);
        heap.push({l.first + cost(i), l.second});
    }
    std::vector<int32_t> block_ptr(blocks + 1, 0), block_items;
    for (int b = 0; b < blocks; ++b) {
        block_items.insert(block_items.end(), assign[b].begin(), assign[b].end());
        block_ptr[b + 1] = (int32_t)block_items.size();
    }
    std::vector<int32_t> run_items;
    refs.assign(runs.size(), BatchRunRef{});
    for (size_t r = 0; r < runs.size(); ++r) {
        const musr_run_s* run = runs[r];
        BatchRunRef& R = refs[r];
        R.data = run->d_data;
        R.hist_off = run->d_hist_off;
        R.hist_nbins = run->d_hist_nbins;
        R.role_theta = run->d_role_theta;
        R.rc = run->rc;
        R.etab = run->d_etab;
        R.t0 = run->t0;
        R.dt = run->dt;
        R.P = run->P;
        R.V = max_vec[r];
        R.theta_off = theta_off[r];
        R.val_off = val_off[r];
        R.item_first = (int32_t)run_items.size();
        R.n_items = (int32_t)per_run[r].size();
        run_items.insert(run_items.end(), per_run[r].begin(), per_run[r].end());
    }
    // one arena for every table and scratch buffer
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    size_t off = 0;
    const size_t o_runs = off; off += al(sizeof(BatchRunRef) * runs.size() + 1);
    const size_t o_items = off; off += al(sizeof(BatchItem) * items.size() + 1);
    const size_t o_bp = off; off += al(sizeof(int32_t) * block_ptr.size());
    const size_t o_bi = off; off += al(sizeof(int32_t) * block_items.size() + 4);
    const size_t o_ri = off; off += al(sizeof(int32_t) * run_items.size() + 4);
    const size_t o_is = off; off += al(sizeof(int64_t) * items.size() + 8);
    const size_t o_part = off; off += al(sizeof(double) * (size_t)(partial_len + 1));
    const size_t o_rc = off; off += al(sizeof(unsigned) * (runs.size() + 1));
    const size_t o_fl = off; off += al(sizeof(unsigned) * (size_t)(total_vals + 1));
    if (cudaMalloc(&arena, off) != cudaSuccess) {
        arena = nullptr;
        return MUSR_ENOMEM;
    }
    char* b = static_cast<char*>(arena);
    d_runs = reinterpret_cast<BatchRunRef*>(b + o_runs);
    d_items = reinterpret_cast<BatchItem*>(b + o_items);
    d_block_ptr = reinterpret_cast<int32_t*>(b + o_bp);
    d_block_items = reinterpret_cast<int32_t*>(b + o_bi);
    d_run_items = reinterpret_cast<int32_t*>(b + o_ri);
    d_item_slot = reinterpret_cast<int64_t*>(b + o_is);
    d_partial = reinterpret_cast<double*>(b + o_part);
    d_run_count = reinterpret_cast<unsigned*>(b + o_rc);
    d_flags = reinterpret_cast<unsigned*>(b + o_fl);
    cudaError_t e = cudaSuccess;
    auto up = [&](void* dst, const void* src, size_t n) {
        if (e == cudaSuccess && n) e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, stream);
    };
    up(d_runs, refs.data(), sizeof(BatchRunRef) * refs.size());
    up(d_items, items.data(), sizeof(BatchItem) * items.size());
    up(d_block_ptr, block_ptr.data(), sizeof(int32_t) * block_ptr.size());
    up(d_block_items, block_items.data(), sizeof(int32_t) * block_items.size());
    up(d_run_items, run_items.data(), sizeof(int32_t) * run_items.size());
    std::vector<int64_t> item_slot(items.size());
    for (size_t i = 0; i < items.size(); ++i) item_slot[i] = items[i].slot;
    up(d_item_slot, item_slot.data(), sizeof(int64_t) * item_slot.size());
    if (e == cudaSuccess) e = cudaMemsetAsync(d_run_count, 0, sizeof(unsigned) * (runs.size() + 1), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_flags, 0, sizeof(unsigned) * (size_t)(total_vals + 1), stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    for (int o = 0; o < 2; ++o)
        if (graph[o]) {
            cudaGraphExecDestroy(graph[o]);
            graph[o] = nullptr;
        }
    return cuda_status(e);
}

BatchParams musr_batch_s::params(int obj, const double* thetas, double* values) const {
    BatchParams p;
    p.runs = d_runs;
    p.items = d_items;
    p.block_ptr = d_block_ptr;
    p.block_items = d_block_items;
    p.run_items = d_run_items;
    p.item_slot = d_item_slot;
    p.thetas = thetas;
    p.obj = obj;
    p.partial = d_partial;
    p.run_count = d_run_count;
    p.flags = d_flags;
    p.values = values;
    return p;
}

int musr_batch_s::launch(int obj, const double* thetas, double* values, cudaStream_t st) const {
    if (n_items == 0) return MUSR_OK;
    const size_t smem = sizeof(HistConst) * (size_t)std::max(1, vmax);
    return cuda_status(launch_batch(sig, blocks, shape.threads, smem, st, params(obj, thetas, values)));
}

// Time a handful of launch shapes on the device and keep the fastest.
int musr_batch_s::tune(int obj, const double* thetas) {
    const BatchShape cands[] = {{256, 1, 4}, {256, 2, 4}, {256, 2, 16}, {256, 3, 4},
                                {128, 2, 8}, {128, 4, 8}, {128, 4, 32}, {64, 6, 16}};
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    BatchShape best_s = shape;
    for (const BatchShape& c : cands) {
        if (plan(c) != MUSR_OK) continue;
        if (launch(obj, thetas, d_values, stream) != MUSR_OK) continue;  // warm-up
        cudaEventRecord(a, stream);
        for (int r = 0; r < 3; ++r) launch(obj, thetas, d_values, stream);
        cudaEventRecord(b, stream);
        if (cudaEventSynchronize(b) != cudaSuccess) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best) {
            best = ms;
            best_s = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    tuned = true;
    return plan(best_s);
}

extern "C" {

int musr_batch_create(const musr_run* runs, int32_t n_runs, const int32_t* max_vec, musr_batch* out) {
    if (!runs || n_runs <= 0 || !max_vec || !out) return MUSR_EINVAL;
    *out = nullptr;
    for (int r = 0; r < n_runs; ++r) {
        if (!runs[r]) return MUSR_EINVAL;
        if (runs[r]->F > 0) return MUSR_ENOTSUP;  // function values are formed per host call
        if (max_vec[r] < 1 || max_vec[r] > kBatchMaxVec) return MUSR_ENOTSUP;
        if (r && runs[r]->sig != runs[0]->sig) return MUSR_ENOTSUP;
        if (runs[r]->device != runs[0]->device) return MUSR_EINVAL;
    }
    musr_batch_s* B = new (std::nothrow) musr_batch_s();
    if (!B) return MUSR_ENOMEM;
    B->device = runs[0]->device;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != B->device) cudaSetDevice(B->device);
    cudaDeviceGetAttribute(&B->sms, cudaDevAttrMultiProcessorCount, B->device);
    B->runs.assign(runs, runs + n_runs);
    B->max_vec.assign(max_vec, max_vec + n_runs);
    B->sig = runs[0]->sig;
    for (int r = 0; r < n_runs; ++r) {
        B->theta_off.push_back(B->total_theta);
        B->val_off.push_back(B->total_vals);
        B->total_theta += (int64_t)max_vec[r] * runs[r]->P;
        B->total_vals += max_vec[r];
        B->vmax = std::max(B->vmax, (int)max_vec[r]);
    }
    int st = cuda_status(cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking));
    if (st == MUSR_OK) st = cuda_status(cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking));
    if (st == MUSR_OK &&
        cudaMallocHost(&B->h_pinned, sizeof(double) * (size_t)(B->total_theta + B->total_vals + 2)) != cudaSuccess)
        st = MUSR_ENOMEM;
    if (st == MUSR_OK) {
        B->h_thetas = static_cast<double*>(B->h_pinned);
        B->h_values = B->h_thetas + B->total_theta + 1;
        if (cudaMalloc(&B->io, sizeof(double) * (size_t)(B->total_theta + B->total_vals + 2)) != cudaSuccess) {
            B->io = nullptr;
            st = MUSR_ENOMEM;
        } else {
            B->d_thetas = static_cast<double*>(B->io);
            B->d_values = B->d_thetas + B->total_theta + 1;
        }
    }
    if (st == MUSR_OK) st = B->plan(BatchShape());
    if (cur != B->device) cudaSetDevice(cur);
    if (st != MUSR_OK) {
        delete B;
        return st;
    }
    *out = B;
    return MUSR_OK;
}

int musr_batch_destroy(musr_batch batch) {
    if (!batch) return MUSR_OK;
    cudaStreamSynchronize(batch->stream);
    delete batch;
    return MUSR_OK;
}

int musr_batch_eval_device(musr_batch B, int obj, const double* thetas_dev, double* values_dev) {
    if (!B || !thetas_dev || !values_dev) return MUSR_EINVAL;
    if (obj != MUSR_CHI2 && obj != MUSR_POISSON) return MUSR_EINVAL;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != B->device) cudaSetDevice(B->device);
    int st = MUSR_OK;
    if (!B->tuned) st = B->tune(obj, thetas_dev);
    if (st == MUSR_OK) st = B->launch(obj, thetas_dev, values_dev, B->stream);
    if (cur != B->device) cudaSetDevice(cur);
    return st;
}

int musr_batch_eval(musr_batch B, int obj, const double* thetas, const int32_t* n_vec, double* values) {
    if (!B || !thetas || !values) return MUSR_EINVAL;
    if (obj != MUSR_CHI2 && obj != MUSR_POISSON) return MUSR_EINVAL;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != B->device) cudaSetDevice(B->device);
    // gather the caller's vectors into the plan's fixed slots (unused slots
    // repeat the run's last given vector so every slot holds a valid theta)
    int64_t src = 0;
    int st = MUSR_OK;
    for (size_t r = 0; r < B->runs.size() && st == MUSR_OK; ++r) {
        const int P = B->runs[r]->P;
        const int nv = n_vec ? n_vec[r] : B->max_vec[r];
        if (nv < 1 || nv > B->max_vec[r]) {
            st = MUSR_EINVAL;
            break;
        }
        for (int v = 0; v < B->max_vec[r]; ++v) {
            const double* th = thetas + src + (int64_t)std::min(v, nv - 1) * P;
            for (int j = 0; j < P; ++j)
                if (!isfinite(th[j])) st = MUSR_ENONFINITE;
            memcpy(B->h_thetas + B->theta_off[r] + (int64_t)v * P, th, sizeof(double) * P);
        }
        src += (int64_t)nv * P;
    }
    cudaError_t e = cudaSuccess;
    if (st == MUSR_OK && !B->tuned) {
        e = cudaMemcpyAsync(B->d_thetas, B->h_thetas, sizeof(double) * B->total_theta,
                            cudaMemcpyHostToDevice, B->stream);
        st = cuda_status(e);
        if (st == MUSR_OK) st = B->tune(obj, B->d_thetas);
    }
    if (st == MUSR_OK && !B->graph[obj]) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemcpyAsync(B->d_thetas, B->h_thetas, sizeof(double) * B->total_theta,
                            cudaMemcpyHostToDevice, B->cap_stream);
            B->launch(obj, B->d_thetas, B->d_values, B->cap_stream);
            cudaMemcpyAsync(B->h_values, B->d_values, sizeof(double) * B->total_vals,
                            cudaMemcpyDeviceToHost, B->cap_stream);
            e = cudaStreamEndCapture(B->cap_stream, &g);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&B->graph[obj], g, 0);
        if (g) cudaGraphDestroy(g);
        st = cuda_status(e);
    }
    if (st == MUSR_OK) st = cuda_status(cudaGraphLaunch(B->graph[obj], B->stream));
    if (st == MUSR_OK) st = cuda_status(cudaStreamSynchronize(B->stream));
    if (st == MUSR_OK) {
        int64_t o = 0;
        for (size_t r = 0; r < B->runs.size(); ++r) {
            const int nv = n_vec ? n_vec[r] : B->max_vec[r];
            memcpy(values + o, B->h_values + B->val_off[r], sizeof(double) * nv);
            o += nv;
        }
    }
    if (cur != B->device) cudaSetDevice(cur);
    return st;
}

int musr_chi2_batch(const musr_run* runs, int32_t n_runs, int obj, const double* thetas,
                    const int32_t* n_vec, double* values) {
    if (!runs || n_runs < 0 || !thetas || !n_vec || !values) return MUSR_EINVAL;
    if (n_runs == 0) return MUSR_OK;
    musr_batch B = nullptr;
    int st = musr_batch_create(runs, n_runs, n_vec, &B);
    if (st == MUSR_OK) {
        B->tuned = true;  // one-shot: keep the default shape, skip tuning
        st = musr_batch_eval(B, obj, thetas, n_vec, values);
    }
    musr_batch_destroy(B);
    return st;
}

}  // extern "C"

namespace musr {

// Central-difference gradient over the free parameters from one batched launch
// per kBatchMaxVec vectors: theta and theta +- h_j e_j (and +- 2 h_j e_j for
// order 4).  A parameter whose stencil meets a non-finite value (a deviance
// step past N = 0) has its step quartered, up to three times; h_abs keeps
// the reduced steps.  The launches use one fixed shape (no autotuning), so
// a fit's differences, and so its path, are the same in every process.
int batch_fd_gradient(musr_run run, int obj, const double* theta, const std::vector<int>& fidx, double* h_abs,
                      int order, double* value, double* grad, double* hdiag) {
    const int P = run->P;
    const int nf = (int)fidx.size();
    const int per = order == 4 ? 4 : 2;
    if (!run->fd_batch) {
        int32_t mv = std::min(1 + 4 * nf, kBatchMaxVec);  // room for either order
        musr_run r = run;
        int st = musr_batch_create(&r, 1, &mv, &run->fd_batch);
        if (st != MUSR_OK) return st;
        run->fd_batch->tuned = true;  // the default shape, in every process
        run->fd_batch_vec = mv;
    }
    musr_batch B = run->fd_batch;
    const int cap = run->fd_batch_vec;
    static const double kOffsets[4] = {1.0, -1.0, 2.0, -2.0};
    memset(grad, 0, sizeof(double) * P);
    std::vector<int> todo(nf);
    for (int a = 0; a < nf; ++a) todo[a] = a;
    for (int attempt = 0; attempt < 4 && !todo.empty(); ++attempt) {
        // vector 0 is theta (first attempt); then per parameter to do +h, -h [, +2h, -2h]
        const int first = attempt == 0 ? 1 : 0;
        const int nv_total = first + per * (int)todo.size();
        std::vector<double> vecs((size_t)nv_total * P), vals(nv_total);
        for (int v = 0; v < nv_total; ++v) memcpy(vecs.data() + (size_t)v * P, theta, sizeof(double) * P);
        for (size_t i = 0; i < todo.size(); ++i)
            for (int u = 0; u < per; ++u)
                vecs[(size_t)(first + per * i + u) * P + fidx[todo[i]]] += kOffsets[u] * h_abs[todo[i]];
        for (int v0 = 0; v0 < nv_total; v0 += cap) {
            const int32_t nv = std::min(cap, nv_total - v0);
            int st = musr_batch_eval(B, obj, vecs.data() + (size_t)v0 * P, &nv, vals.data() + v0);
            if (st != MUSR_OK) return st;
        }
        if (first) {
            *value = vals[0];
            if (!isfinite(vals[0])) return MUSR_EDOMAIN;
        }
        std::vector<int> again;
        for (size_t i = 0; i < todo.size(); ++i) {
            const int a = todo[i];
            const double* f = vals.data() + first + per * i;  // f(+h), f(-h) [, f(+2h), f(-2h)]
            bool ok = true;
            for (int u = 0; u < per; ++u) ok = ok && isfinite(f[u]);
            if (!ok) {
                h_abs[a] *= 0.25;
                again.push_back(a);
                continue;
            }
            const double h = h_abs[a];
            if (order == 4) {
                // fourth-order central differences: truncation error O(h^4)
                grad[fidx[a]] = (8.0 * (f[0] - f[1]) - (f[2] - f[3])) / (12.0 * h);
                if (hdiag) hdiag[fidx[a]] = (16.0 * (f[0] + f[1]) - (f[2] + f[3]) - 30.0 * *value) / (12.0 * h * h);
            } else {
                grad[fidx[a]] = (f[0] - f[1]) / (2.0 * h);
                if (hdiag) hdiag[fidx[a]] = (f[0] - 2.0 * *value + f[1]) / (h * h);
            }
        }
        todo.swap(again);
    }
    return todo.empty() ? MUSR_OK : MUSR_EDOMAIN;
}

}  // namespace musr
