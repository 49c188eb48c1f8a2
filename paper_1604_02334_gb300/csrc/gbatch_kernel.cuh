// Batched value + gradient (+ Gauss-Newton matrix) for many runs, one
// parameter vector each, in ONE launch: the evaluation under a lockstep fit of
// many runs (musr_fit_batch), where a single run's launch would be dominated
// by its fixed cost (launch, staging, the grid-wide reduction).
//
// Work is cut into items (run, histogram, first bin, rows) scheduled onto
// persistent blocks by a host LPT schedule, as in the value-only batch kernel.
// Per item the block stages the histogram's constants, evaluates its rows with
// the objective kernel's per-bin code (adjoint modes), reduces the per-role
// accumulators (FP32 warp sums, FP64 across warps) into an item partial, and
// takes a per-run ticket.  The run's last item sums the run's item partials
// per histogram in a fixed order (shared memory) and maps them to theta
// through the run's CSR table, so every output is bitwise repeatable.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <queue>
#include <vector>

#include "eval_kernel.cuh"
#include "musr.h"
#include "musr_internal.h"
#include "run_impl.h"

namespace musr {

struct GRunRef {
    const float* data;
    const int64_t* hist_off;
    const int32_t* hist_nbins;
    const int32_t* role_theta;
    const int32_t* csr_ptr;
    const int32_t* csr_src;
    const int32_t* csr_row;  // Gauss-Newton: output index of each map row (null: row = output)
    const float* etab;  // lifetime factor at every chunk start
    RunConst rc;
    double t0, dt;
    int32_t P, K, n_out, n_rows;
    int64_t theta_off, out_off;
    int32_t hist_ptr_off;  // into hist_item_ptr: K + 1 offsets into run_items
};

struct GItem {
    int32_t run, hist, start, rows;
};

// One item as the kernel takes it, in each block's schedule order: everything
// its staging and rows need, so a block fetches an item with one contiguous
// copy (issued while the previous item is evaluated) instead of a chain of
// dependent loads through the run tables.
struct __align__(16) GWork {
    RunConst rc;
    const float* hdata;  // the histogram's counts
    const float* etab;   // the run's lifetime table
    int64_t theta_off;   // the run's parameter vector in the launch's thetas
    int32_t item, run, start, rows, M;
    float dtf, t0f;
    int32_t rt[2 * kMaxRoles];  // the histogram's role -> theta row
};
static_assert(sizeof(GWork) % 16 == 0, "GWork is copied in 16-byte pieces");

struct GParams {
    const GRunRef* runs;
    const GWork* works;  // by block: works[block_ptr[b] .. block_ptr[b + 1])
    const int32_t* block_ptr;
    const int32_t* run_items;      // per run, its items by (histogram, first bin)
    const int32_t* hist_item_ptr;  // per run, K + 1 offsets into run_items
    const int32_t* run_nitems;
    const double* thetas;
    const uint8_t* active;  // per run, or null (all)
    int obj;
    double* partial;  // [n_items][NACC]
    unsigned* run_count;
    unsigned* flags;  // per run
    double* out;
    int32_t* status;  // per run
};

template <int NE, int NG, int NS, int KT, int MODE>
__global__ void __launch_bounds__(kMaxThreads, MODE == kGrad ? 3 : 1) gbatch_kernel(const __grid_constant__ GParams p) {
    constexpr int NOSC = NE + NG + NS;
    constexpr int R = 2 + 4 * NOSC + NS + 2 * KT;
    constexpr int NACC = MODE == kGrad ? 1 + R : 1 + R + R * (R + 1) / 2;
    constexpr int NPART = stage_parts<NE, NG, NS, KT>();
    constexpr int G = kBinsPerThread;
    extern __shared__ double hsum[];  // the run's per-histogram sums, K x NACC
    __shared__ HistConst hc;
    __shared__ float red[kMaxWarps][NACC];
    __shared__ int s_last;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int stripe = blockDim.x * G;

    // item pipeline: wk / wth / wact hold item j's descriptor, theta entries
    // and active flag in buffer (j - w0) & 1; item j + 1's descriptor is
    // copied while item j's rows run, its theta entries while item j reduces
    __shared__ GWork wk[2];
    __shared__ double wth[2][2 * kMaxRoles];
    __shared__ int wact[2];
    constexpr int kWorkPieces = (int)(sizeof(GWork) / 16);
    const int w0 = p.block_ptr[blockIdx.x], w1 = p.block_ptr[blockIdx.x + 1];
    auto fetch_work = [&](int j, int buf) {
        if ((int)threadIdx.x < kWorkPieces)
            cp_async16(reinterpret_cast<uint4*>(&wk[buf]) + threadIdx.x,
                       reinterpret_cast<const uint4*>(p.works + j) + threadIdx.x);
    };
    // after wk[buf] is complete and visible: its theta entries and active flag
    auto fetch_theta = [&](int buf) {
        const int t = (int)threadIdx.x;
        if (t < 2 * kMaxRoles) {
            const int i = wk[buf].rt[t];
            if (i >= 0) cp_async8(&wth[buf][t], p.thetas + wk[buf].theta_off + i);
            else wth[buf][t] = 0.0;
        } else if (t == 2 * kMaxRoles) {
            wact[buf] = p.active ? (int)p.active[wk[buf].run] : 1;
        }
    };
    if (w0 < w1) {
        fetch_work(w0, 0);
        cp_async_wait_all();
        __syncthreads();
        fetch_theta(0);
        cp_async_wait_all();
    }

    for (int it = w0; it < w1; ++it) {
        const int cur = (it - w0) & 1, nxt = cur ^ 1;
        cp_async_wait_all();  // this thread's copies of item it's theta entries
        __syncthreads();  // item it's buffers complete; the previous item is done with hc / red / hsum
        const GWork& W = wk[cur];
        const bool act = wact[cur] != 0;  // uniform over the block
        if (it + 1 < w1) fetch_work(it + 1, nxt);
        const int item_idx = W.item, run = W.run;
        const int M = W.M;
        const float* hdata = W.hdata;
        int n0 = W.start + (int)threadIdx.x * G;

        // first row's loads in flight while the constants are staged
        float d[G];
        float E0 = 0.f;
        if (act && n0 < M) {
            E0 = __ldg(W.etab + (n0 >> 3));
            const float4* src = reinterpret_cast<const float4*>(hdata + n0);
            const float4 a = __ldg(src), b = __ldg(src + 1);
            d[0] = a.x; d[1] = a.y; d[2] = a.z; d[3] = a.w;
            d[4] = b.x; d[5] = b.y; d[6] = b.z; d[7] = b.w;
        } else {
#pragma unroll
            for (int g = 0; g < G; ++g) d[g] = 0.f;
        }
        if (act) {
            for (int part = warp; part < NPART; part += nwarps)
                stage_part<NE, NG, NS, KT>(part, ThetaGathered{wth[cur]}, W.rc, hc, stripe, lane);
        }
        __syncthreads();

        float acc[NACC];
#pragma unroll
        for (int a = 0; a < NACC; ++a) acc[a] = 0.f;
        bool bad = false;
        const float dtf = W.dtf, t0f = W.t0f;
        const int rows = act ? W.rows : 0;
        {
            GqCarry<NOSC> carry;
            carry.valid = false;
            GnAcc<R> gnacc;
            gnacc.zero();
            for (int row = 0; row < rows; ++row) {
                const int n1 = n0 + stripe;
                float dn[G];
                float En = 0.f;
                if (row + 1 < rows && n1 < M) {
                    const float4* src = reinterpret_cast<const float4*>(hdata + n1);
                    const float4 a = __ldg(src), b = __ldg(src + 1);
                    dn[0] = a.x; dn[1] = a.y; dn[2] = a.z; dn[3] = a.w;
                    dn[4] = b.x; dn[5] = b.y; dn[6] = b.z; dn[7] = b.w;
                    En = __ldg(W.etab + (n1 >> 3));
                } else {
#pragma unroll
                    for (int g = 0; g < G; ++g) dn[g] = 0.f;
                }
                if (n0 < M)
                    eval_chunk<NE, NG, NS, KT, MODE, NACC>(hc, n0, M, d, E0, p.obj, dtf, t0f, acc, bad, nullptr, &carry,
                                                           &gnacc);
#pragma unroll
                for (int g = 0; g < G; ++g) d[g] = dn[g];
                E0 = En;
                n0 = n1;
            }
            if constexpr (MODE == kGN) gn_scatter(gnacc, acc);
        }
        // the next item's theta entries, once its descriptor is in (they
        // arrive while this item reduces)
        if (it + 1 < w1) {
            cp_async_wait_all();
            __syncthreads();
            fetch_theta(nxt);
        }
        if (!act) continue;
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
        if (threadIdx.x == 0 && any_bad) atomicOr(&p.flags[run], 1u);
        for (int a = threadIdx.x; a < NACC; a += blockDim.x) {
            double s = 0.0;
            for (int w = 0; w < nwarps; ++w) s += (double)red[w][a];
            // the histogram's role factor of this accumulator (see eval_chunk)
            p.partial[(size_t)item_idx * NACC + a] = a > 0 ? s * (double)acc_factor<NE, NG, NS, KT, MODE>(hc, a) : s;
        }
        // the barrier orders the block's partials before thread 0's ticket, a
        // release (and, for the run's last item, an acquire of the others')
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned prev;
            asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;"
                         : "=r"(prev)
                         : "l"(p.run_count + run)
                         : "memory");
            s_last = prev == (unsigned)p.run_nitems[run] - 1u;
        }
        __syncthreads();
        if (!s_last) continue;
        const GRunRef& Rr = p.runs[run];
        // the run's last item: per-histogram sums in item order, then theta via the CSR
        const int32_t* hptr = p.hist_item_ptr + Rr.hist_ptr_off;
        for (int q = threadIdx.x; q < Rr.K * NACC; q += blockDim.x) {
            const int kk = q / NACC, a = q % NACC;
            const int j1 = hptr[kk + 1];
            double s = 0.0;
            int j = hptr[kk];
            for (; j + 4 <= j1; j += 4) {
                // four partials in flight, added in order
                double x[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) x[u] = __ldcg(p.partial + (size_t)p.run_items[j + u] * NACC + a);
#pragma unroll
                for (int u = 0; u < 4; ++u) s += x[u];
            }
            for (; j < j1; ++j) s += __ldcg(p.partial + (size_t)p.run_items[j] * NACC + a);
            hsum[q] = s;
        }
        __syncthreads();
        double* out = p.out + Rr.out_off;
        if (Rr.csr_row) {
            // outputs without a map row are 0 (the buffer's other layouts,
            // of other modes, may have left anything there)
            for (int o = threadIdx.x; o < Rr.n_out; o += blockDim.x) out[o] = 0.0;
            __syncthreads();
        }
        const int n_rows = Rr.csr_row ? Rr.n_rows : Rr.n_out;
        for (int r = threadIdx.x; r < n_rows; r += blockDim.x) {
            const int o = Rr.csr_row ? Rr.csr_row[r] : r;
            // Gauss-Newton entries: the rows carry H[i][j], i <= j; the sum is
            // stored at [i][j] and [j][i]
            int om = -1;
            if (MODE == kGN && o > Rr.P) {
                const int oh = o - 1 - Rr.P, i = oh / Rr.P, j = oh - i * Rr.P;
                if (i < j) om = 1 + Rr.P + j * Rr.P + i;
            }
            double s = 0.0;
            const int e = Rr.csr_ptr[r + 1];
            for (int j = Rr.csr_ptr[r]; j < e; ++j) s += hsum[Rr.csr_src[j]];
            out[o] = s;
            if (om >= 0) out[om] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned f = atomicExch(&p.flags[run], 0u);
            if (!isfinite(out[0])) f |= 2u;
            if (p.status) p.status[run] = (int32_t)f;
            p.run_count[run] = 0u;
        }
    }
}

template <int NE, int NG, int NS, int KT, int MODE>
cudaError_t launch_gbatch_sig(int blocks, int threads, size_t smem, cudaStream_t st, const GParams& p) {
    auto kern = gbatch_kernel<NE, NG, NS, KT, MODE>;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes < smem) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if ((int)smem > optin - (int)fa.sharedSizeBytes) return cudaErrorInvalidValue;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
    }
    kern<<<blocks, threads, smem, st>>>(p);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_gbatch_mode(const Signature& s, int blocks, int threads, size_t smem, cudaStream_t st,
                               const GParams& p) {
#define MUSR_CASE(NE, NG, NS, KT)                             \
    if (s.ne == NE && s.ng == NG && s.ns == NS && s.kt == KT) \
        return launch_gbatch_sig<NE, NG, NS, KT, MODE>(blocks, threads, smem, st, p);
    MUSR_FOR_EACH_SIGNATURE(MUSR_CASE)
#undef MUSR_CASE
    return cudaErrorInvalidValue;
}

}  // namespace musr
