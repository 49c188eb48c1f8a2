// BF16 tensor-core GEMM (tcgen05 / TMEM / TMA, sm_103a) and the small MLP of
// the learned start proposer built on it.
//
// GEMM: C[M x N] = A[M x K] . B[N x K]^T (both operands K-major, row-major in
// memory), FP32 accumulation in tensor memory, fused epilogue
//     C = act(C + bias)  -> FP32 and / or BF16 outputs.
// One CTA computes one 128 x 128 output tile with 128 threads:
//   warp 0 lane 0   TMA producer: 64-wide K slices of A and B, 128-byte swizzle,
//                   into a 4-stage ring guarded by mbarriers (full / empty);
//   warp 1 lane 0   MMA issuer: four tcgen05.mma (K = 16 each) per slice into a
//                   128 x 128 FP32 accumulator in TMEM; tcgen05.commit frees the
//                   slice and finally signals the epilogue;
//   all 4 warps     epilogue: tcgen05.ld of their 32 accumulator rows.
// Every mbarrier wait is bounded: on time-out the kernel records an error
// flag, stops issuing work, waits (bounded) for its own copies and frees TMEM.
// Sizes: M, N multiples of 128 and K a multiple of 64 (callers pad).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "musr.h"
#include "musr_internal.h"

namespace musr {
namespace {

constexpr int kTileM = 128, kTileN = 128, kTileK = 64, kStages = 4;
constexpr int kTileBytes = kTileM * kTileK * 2;  // 16 KB per operand per stage
constexpr uint32_t kTmemCols = 128;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait (about a second at worst); false and an error flag on time-out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned* err) {
    for (uint32_t i = 0; i < (1u << 22); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 32) __nanosleep(128);
    }
    atomicOr(err, 1u);
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major tile of 128-byte rows with the
// 128-byte swizzle (8-row atoms of 1024 bytes).
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* p) {
    const uint64_t addr = smem_u32(p);
    uint64_t d = (addr >> 4) & 0x3FFFull;       // start address
    d |= (uint64_t)1 << 16;                      // leading byte offset (unused when swizzled)
    d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                      // descriptor version
    d |= (uint64_t)2 << 61;                      // 128-byte swizzle
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: BF16 x BF16 -> FP32, both
// operands K-major, M x N tile.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4)                      // D format: F32
           | (1u << 7)                    // A format: BF16
           | (1u << 10)                   // B format: BF16
           | ((uint32_t)(n >> 3) << 17)   // N / 8
           | ((uint32_t)(m >> 4) << 24);  // M / 16
}

struct GemmArgs {
    int M, N, K;
    const float* bias;   // [N] or null
    int relu;
    float* out_f32;      // [M x ldc] or null
    __nv_bfloat16* out_bf16;  // [M x ldc] or null
    int ldc;
    unsigned* err;       // device error flag
    float* partial;      // split-K: [gridDim.z][M][N] raw FP32 tiles (bias / ReLU by the reduce kernel), or null
};

__global__ void __launch_bounds__(128, 1) gemm_tn_bf16_kernel(const __grid_constant__ CUtensorMap map_a,
                                                              const __grid_constant__ CUtensorMap map_b,
                                                              const GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned operand ring
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = base;
    unsigned char* sB = base + kStages * kTileBytes;
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kTileM, n0 = blockIdx.x * kTileN;
    // split-K: this CTA's contiguous range of K tiles (the host keeps every range non-empty)
    const int KT_all = g.K / kTileK;
    const int per = (KT_all + (int)gridDim.z - 1) / (int)gridDim.z;
    const int kt_base = (int)blockIdx.z * per;
    const int KT = min(per, KT_all - kt_base);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---- producer ----
        for (int kt = 0; kt < KT; ++kt) {
            const int s = kt % kStages;
            if (kt >= kStages && !mbar_wait(&empty[s], ((kt / kStages) - 1) & 1, g.err)) {
                s_abort = 1;
                break;
            }
            if (*(volatile int*)&s_abort) break;
            mbar_expect_tx(&full[s], 2 * kTileBytes);
            tma_load_2d(sA + s * kTileBytes, &map_a, (kt_base + kt) * kTileK, m0, &full[s]);
            tma_load_2d(sB + s * kTileBytes, &map_b, (kt_base + kt) * kTileK, n0, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        const uint32_t idesc = idesc_bf16(kTileM, kTileN);
        int kt = 0;
        for (; kt < KT; ++kt) {
            const int s = kt % kStages;
            if (!mbar_wait(&full[s], (kt / kStages) & 1, g.err)) {
                s_abort = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t da = smem_desc_sw128(sA + s * kTileBytes);
            const uint64_t db = smem_desc_sw128(sB + s * kTileBytes);
#pragma unroll
            for (int kk = 0; kk < kTileK / 16; ++kk) {
                const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                // advance 16 BF16 = 32 bytes along K inside the swizzled rows
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da + 2ull * kk), "l"(db + 2ull * kk), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&done))
                     : "memory");
    }
    __syncwarp();

    // ---- epilogue: 4 warps x 32 accumulator rows ----
    const bool ok = mbar_wait(&done, 0, g.err);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = m0 + warp * 32 + lane;
    if (ok && !s_abort) {
        for (int c0 = 0; c0 < kTileN; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float v[16];
            if (g.partial) {
                // split-K: the raw slice sum, bias and ReLU after the slices are added
                if (row < g.M) {
                    float4* dst = reinterpret_cast<float4*>(
                        g.partial + ((size_t)blockIdx.z * g.M + row) * g.N + n0 + c0);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        dst[i] = make_float4(__uint_as_float(r[4 * i]), __uint_as_float(r[4 * i + 1]),
                                             __uint_as_float(r[4 * i + 2]), __uint_as_float(r[4 * i + 3]));
                }
                continue;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                v[i] = __uint_as_float(r[i]);
                if (g.bias) v[i] += g.bias[n0 + c0 + i];
                if (g.relu) v[i] = fmaxf(v[i], 0.f);
            }
            if (row < g.M) {
                if (g.out_f32) {
                    float4* dst = reinterpret_cast<float4*>(g.out_f32 + (size_t)row * g.ldc + n0 + c0);
#pragma unroll
                    for (int i = 0; i < 4; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                }
                if (g.out_bf16) {
                    __nv_bfloat162 h[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
                    uint4* dst = reinterpret_cast<uint4*>(g.out_bf16 + (size_t)row * g.ldc + n0 + c0);
                    dst[0] = *reinterpret_cast<uint4*>(&h[0]);
                    dst[1] = *reinterpret_cast<uint4*>(&h[4]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0 && s_abort) {
        // let in-flight copies land before the block (and its shared memory) goes
        for (int s = 0; s < kStages; ++s) (void)mbar_try_wait(&full[s], 0);
    }
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// split-K: out = act(sum over slices in slice order + bias), four columns per thread
__global__ void splitk_reduce_kernel(const float* __restrict__ part, int splits, int M, int N,
                                     const float* __restrict__ bias, int relu, float* __restrict__ out_f32,
                                     __nv_bfloat16* __restrict__ out_bf16, int ldc) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // index of a group of 4 columns
    const int64_t n4 = (int64_t)M * (N / 4);
    if (q >= n4) return;
    const int row = (int)(q / (N / 4)), col = (int)(q % (N / 4)) * 4;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int z = 0; z < splits; ++z) {
        const float4 v = *reinterpret_cast<const float4*>(part + ((size_t)z * M + row) * N + col);
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
    }
    float v[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (bias) v[i] += bias[col + i];
        if (relu) v[i] = fmaxf(v[i], 0.f);
    }
    if (out_f32) *reinterpret_cast<float4*>(out_f32 + (size_t)row * ldc + col) = make_float4(v[0], v[1], v[2], v[3]);
    if (out_bf16) {
        __nv_bfloat162 h0 = __floats2bfloat162_rn(v[0], v[1]), h1 = __floats2bfloat162_rn(v[2], v[3]);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t*>(&h0);
        u.y = *reinterpret_cast<uint32_t*>(&h1);
        *reinterpret_cast<uint2*>(out_bf16 + (size_t)row * ldc + col) = u;
    }
}

// ---- host: tensor maps through the driver entry point ----
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// rows x cols BF16 row-major (cols contiguous), box 64 cols x 128 rows, 128B swizzle
bool make_map(CUtensorMap* m, const void* ptr, uint64_t rows, uint64_t cols) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kTileK, (cuuint32_t)kTileM};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// C = act(A . B^T + bias); see the file header.  err_dev: device unsigned flag.
int gemm_tn_bf16(const void* A, const void* B, int M, int N, int K, const float* bias, int relu, float* out_f32,
                 void* out_bf16, int ldc, unsigned* err_dev, cudaStream_t st, float* ws, size_t ws_floats) {
    if (M <= 0 || N <= 0 || K <= 0 || M % kTileM || N % kTileN || K % kTileK || ldc < N || (ldc % 8)) return MUSR_EINVAL;
    if (((uintptr_t)A & 15) || ((uintptr_t)B & 15)) return MUSR_EINVAL;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, (uint64_t)M, (uint64_t)K) || !make_map(&mb, B, (uint64_t)N, (uint64_t)K)) return MUSR_ECUDA;
    GemmArgs g;
    g.M = M;
    g.N = N;
    g.K = K;
    g.bias = bias;
    g.relu = relu;
    g.out_f32 = out_f32;
    g.out_bf16 = static_cast<__nv_bfloat16*>(out_bf16);
    g.ldc = ldc;
    g.err = err_dev;
    g.partial = nullptr;
    const size_t smem = 2 * (size_t)kStages * kTileBytes + 1024;
    static std::once_flag once;
    std::call_once(once, [smem] {
        cudaFuncSetAttribute(gemm_tn_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    // too few output tiles to fill the GPU: split K over CTAs (deterministic slice-order reduction)
    const int tiles = (N / kTileN) * (M / kTileM), KT = K / kTileK;
    int splits = 1;
    if (ws && tiles < 76 && KT >= 4) {
        splits = std::min(std::min(32, KT), std::max(1, 152 / tiles));
        while (splits > 1 && (size_t)splits * M * N > ws_floats) --splits;
        const int per = (KT + splits - 1) / splits;
        splits = (KT + per - 1) / per;  // every slice non-empty
    }
    if (splits > 1) g.partial = ws;
    dim3 grid(N / kTileN, M / kTileM, splits);
    gemm_tn_bf16_kernel<<<grid, 128, smem, st>>>(ma, mb, g);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && splits > 1) {
        const int64_t n4 = (int64_t)M * (N / 4);
        splitk_reduce_kernel<<<(unsigned)((n4 + 255) / 256), 256, 0, st>>>(ws, splits, M, N, bias, relu, out_f32,
                                                                          static_cast<__nv_bfloat16*>(out_bf16), ldc);
        e = cudaGetLastError();
    }
    return cuda_status(e);
}

}  // namespace musr

extern "C" int musr_gemm_bf16(const void* a_dev, const void* b_dev, int32_t m, int32_t n, int32_t k,
                              const float* bias_dev, int32_t relu, float* out_f32_dev, void* out_bf16_dev,
                              int32_t ldc, float* ws_dev, int64_t ws_floats, uint32_t* err_dev, void* stream) {
    if (!a_dev || !b_dev || !err_dev || (!out_f32_dev && !out_bf16_dev) || ws_floats < 0 ||
        (ws_dev && (reinterpret_cast<uintptr_t>(ws_dev) & 15)))
        return MUSR_EINVAL;
    return musr::gemm_tn_bf16(a_dev, b_dev, m, n, k, bias_dev, relu, out_f32_dev, out_bf16_dev, ldc, err_dev,
                              static_cast<cudaStream_t>(stream), ws_dev, ws_dev ? (size_t)ws_floats : 0);
}

// ===========================================================================
// The proposer MLP: n_in -> n_hid (x n_hidden_layers, ReLU) -> n_out, BF16
// weights and activations on the tensor cores, FP32 master weights, Adam.
// Weights are stored [out x in] row-major, so a layer is C = X . W^T (the
// GEMM above); the backward pass forms dW = dZ^T . X and dX = dZ . W from
// transposed BF16 copies.  The last layer is padded to 128 outputs.
// ===========================================================================
namespace musr {
namespace {

__global__ void f32_to_bf16_kernel(const float* __restrict__ x, float scale, __nv_bfloat16* __restrict__ y,
                                   int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i] * scale);
}

// [rows x cols] -> [cols x rows], BF16, 32 x 32 tiles through shared memory
__global__ void transpose_bf16_kernel(const __nv_bfloat16* __restrict__ x, __nv_bfloat16* __restrict__ y, int rows,
                                      int cols) {
    __shared__ __nv_bfloat16 t[32][34];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[i][threadIdx.x] = x[(size_t)r * cols + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) y[(size_t)c * rows + r] = t[threadIdx.x][i];
    }
}

// dY = 2 (Y - T) / (B n_out) on the n_out valid columns (0 on padding), FP32
// and BF16; per-block partial sums of (Y - T)^2.
__global__ void mse_grad_kernel(const float* __restrict__ y, const float* __restrict__ t, int B, int n_out,
                                int n_pad, float* __restrict__ dy, __nv_bfloat16* __restrict__ dyb,
                                float* __restrict__ part) {
    __shared__ float red[256];
    float s = 0.f;
    const float c = 2.f / ((float)B * (float)n_out);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B * n_pad; i += gridDim.x * blockDim.x) {
        const int r = i / n_pad, j = i % n_pad;
        float g = 0.f;
        if (j < n_out) {
            const float e = y[i] - t[(size_t)r * n_out + j];
            s += e * e;
            g = c * e;
        }
        dy[i] = g;
        dyb[i] = __float2bfloat16_rn(g);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// dZ = dH * (H > 0) (ReLU), FP32 and BF16
__global__ void relu_back_kernel(const float* __restrict__ dh, const __nv_bfloat16* __restrict__ h, int64_t n,
                                 float* __restrict__ dz, __nv_bfloat16* __restrict__ dzb) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float g = __bfloat162float(h[i]) > 0.f ? dh[i] : 0.f;
        dz[i] = g;
        dzb[i] = __float2bfloat16_rn(g);
    }
}

// db[j] = sum_r dz[r, j] (fixed order over rows)
__global__ void colsum_kernel(const float* __restrict__ dz, int rows, int cols, float* __restrict__ db) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += dz[(size_t)r * cols + j];
    db[j] = s;
}

// Adam on FP32 master values, BF16 copy refreshed
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, __nv_bfloat16* __restrict__ pb, int64_t n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        p[i] = pi;
        if (pb) pb[i] = __float2bfloat16_rn(pi);
    }
}

int blocks_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 8); }

}  // namespace
}  // namespace musr

struct musr_mlp_s {
    int n_in = 0, n_hid = 0, n_hl = 0, n_out = 0, n_out_pad = 0, max_b = 0, L = 0;
    float in_scale = 1.f;
    std::vector<int> din, dout;  // per layer (dout padded for the last)
    void* arena = nullptr;
    // per layer
    std::vector<float*> W, b, gW, gb, mW, vW, mb, vb;
    std::vector<__nv_bfloat16*> Wb, WTb;
    // activations
    __nv_bfloat16 *X = nullptr, *XT = nullptr;
    std::vector<__nv_bfloat16*> H, HT;  // hidden outputs (BF16) and transposes
    float *Y = nullptr, *dY = nullptr, *dH = nullptr, *dZ = nullptr, *loss_part = nullptr;
    __nv_bfloat16 *dYb = nullptr, *dZb = nullptr, *dZT = nullptr;
    unsigned* err = nullptr;
    float* ws = nullptr;  // split-K partial tiles: at most 152 tiles of 128 x 128 FP32
    int64_t n_params = 0;
    int step = 0;
    cudaStream_t stream = nullptr;
};

namespace {
using namespace musr;

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// split-K only runs with fewer than 76 output tiles and at most 152 / tiles slices
constexpr size_t kSplitWsFloats = (size_t)152 * 128 * 128;

int mlp_forward(musr_mlp m, const float* x, int B, cudaStream_t st) {
    const int64_t nx = (int64_t)B * m->n_in;
    f32_to_bf16_kernel<<<blocks_for(nx), 256, 0, st>>>(x, m->in_scale, m->X, nx);
    const __nv_bfloat16* in = m->X;
    for (int l = 0; l < m->L; ++l) {
        const bool last = l == m->L - 1;
        const int rc = gemm_tn_bf16(in, m->Wb[l], B, m->dout[l], m->din[l], m->b[l], last ? 0 : 1,
                                    last ? m->Y : nullptr, last ? nullptr : m->H[l], m->dout[l], m->err, st,
                                    m->ws, kSplitWsFloats);
        if (rc != MUSR_OK) return rc;
        in = last ? nullptr : m->H[l];
    }
    return cuda_status(cudaGetLastError());
}

void transpose(const __nv_bfloat16* x, __nv_bfloat16* y, int rows, int cols, cudaStream_t st) {
    dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
    transpose_bf16_kernel<<<grid, block, 0, st>>>(x, y, rows, cols);
}

int mlp_backward(musr_mlp m, const float* x, const float* t, int B, float* loss, cudaStream_t st) {
    int rc = mlp_forward(m, x, B, st);
    if (rc != MUSR_OK) return rc;
    const int nb = std::min(blocks_for((int64_t)B * m->n_out_pad), 512);
    mse_grad_kernel<<<nb, 256, 0, st>>>(m->Y, t, B, m->n_out, m->n_out_pad, m->dY, m->dYb, m->loss_part);
    for (int l = m->L - 1; l >= 0; --l) {
        const int o = m->dout[l], i = m->din[l];
        const float* dz = l == m->L - 1 ? m->dY : m->dZ;
        const __nv_bfloat16* dzb = l == m->L - 1 ? m->dYb : m->dZb;
        const __nv_bfloat16* act = l == 0 ? m->X : m->H[l - 1];
        __nv_bfloat16* actT = l == 0 ? m->XT : m->HT[l - 1];
        // dW = dZ^T . act  (M = o, N = i, K = B)
        transpose(dzb, m->dZT, B, o, st);
        transpose(act, actT, B, i, st);
        rc = gemm_tn_bf16(m->dZT, actT, o, i, B, nullptr, 0, m->gW[l], nullptr, i, m->err, st, m->ws,
                          kSplitWsFloats);
        if (rc != MUSR_OK) return rc;
        colsum_kernel<<<(o + 127) / 128, 128, 0, st>>>(dz, B, o, m->gb[l]);
        if (l > 0) {
            // dH = dZ . W  (M = B, N = i, K = o), then the ReLU of layer l - 1
            rc = gemm_tn_bf16(dzb, m->WTb[l], B, i, o, nullptr, 0, m->dH, nullptr, i, m->err, st, m->ws,
                              kSplitWsFloats);
            if (rc != MUSR_OK) return rc;
            const int64_t n = (int64_t)B * i;
            relu_back_kernel<<<blocks_for(n), 256, 0, st>>>(m->dH, m->H[l - 1], n, m->dZ, m->dZb);
        }
    }
    if (loss) {
        std::vector<float> part(nb);
        cudaError_t e = cudaMemcpyAsync(part.data(), m->loss_part, sizeof(float) * nb, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_status(e);
        double s = 0.0;
        for (float v : part) s += v;
        *loss = (float)(s / ((double)B * m->n_out));
    }
    return cuda_status(cudaGetLastError());
}

int mlp_adam(musr_mlp m, float lr, float b1, float b2, float eps, cudaStream_t st) {
    m->step++;
    const float c1 = 1.f / (1.f - powf(b1, (float)m->step)), c2 = 1.f / (1.f - powf(b2, (float)m->step));
    for (int l = 0; l < m->L; ++l) {
        const int64_t nw = (int64_t)m->dout[l] * m->din[l];
        adam_kernel<<<blocks_for(nw), 256, 0, st>>>(m->W[l], m->gW[l], m->mW[l], m->vW[l], m->Wb[l], nw, lr, b1, b2,
                                                    eps, c1, c2);
        adam_kernel<<<blocks_for(m->dout[l]), 256, 0, st>>>(m->b[l], m->gb[l], m->mb[l], m->vb[l], nullptr,
                                                            m->dout[l], lr, b1, b2, eps, c1, c2);
        if (l > 0) transpose(m->Wb[l], m->WTb[l], m->dout[l], m->din[l], st);
    }
    return cuda_status(cudaGetLastError());
}

int mlp_upload(musr_mlp m, const float* host) {
    // host: per layer W [dout_logical x din] then b [dout_logical]
    size_t o = 0;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < m->L && e == cudaSuccess; ++l) {
        const int ol = l == m->L - 1 ? m->n_out : m->dout[l];
        std::vector<float> w((size_t)m->dout[l] * m->din[l], 0.f), bb(m->dout[l], 0.f);
        memcpy(w.data(), host + o, sizeof(float) * (size_t)ol * m->din[l]);
        o += (size_t)ol * m->din[l];
        memcpy(bb.data(), host + o, sizeof(float) * ol);
        o += ol;
        e = cudaMemcpy(m->W[l], w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(m->b[l], bb.data(), sizeof(float) * bb.size(), cudaMemcpyHostToDevice);
        const int64_t nw = (int64_t)w.size();
        if (e == cudaSuccess) {
            f32_to_bf16_kernel<<<blocks_for(nw), 256, 0, m->stream>>>(m->W[l], 1.f, m->Wb[l], nw);
            if (l > 0) transpose(m->Wb[l], m->WTb[l], m->dout[l], m->din[l], m->stream);
            e = cudaStreamSynchronize(m->stream);
        }
    }
    return cuda_status(e);
}

int mlp_download(musr_mlp m, float* host, int grads) {
    size_t o = 0;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < m->L && e == cudaSuccess; ++l) {
        const int ol = l == m->L - 1 ? m->n_out : m->dout[l];
        e = cudaMemcpy(host + o, grads ? m->gW[l] : m->W[l], sizeof(float) * (size_t)ol * m->din[l],
                       cudaMemcpyDeviceToHost);
        o += (size_t)ol * m->din[l];
        if (e == cudaSuccess)
            e = cudaMemcpy(host + o, grads ? m->gb[l] : m->b[l], sizeof(float) * ol, cudaMemcpyDeviceToHost);
        o += ol;
    }
    return cuda_status(e);
}

}  // namespace

extern "C" {

int musr_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_hidden_layers, int32_t n_out, int32_t max_batch,
                    float in_scale, uint64_t seed, musr_mlp* out) {
    if (!out || n_in <= 0 || n_in % 128 || n_hidden <= 0 || n_hidden % 128 || n_hidden_layers < 1 || n_out <= 0 ||
        n_out > 128 || max_batch <= 0 || max_batch % 128)
        return MUSR_EINVAL;
    *out = nullptr;
    musr_mlp m = new (std::nothrow) musr_mlp_s();
    if (!m) return MUSR_ENOMEM;
    m->n_in = n_in;
    m->n_hid = n_hidden;
    m->n_hl = n_hidden_layers;
    m->n_out = n_out;
    m->n_out_pad = 128;
    m->max_b = max_batch;
    m->in_scale = in_scale;
    m->L = n_hidden_layers + 1;
    for (int l = 0; l < m->L; ++l) {
        m->din.push_back(l == 0 ? n_in : n_hidden);
        m->dout.push_back(l == m->L - 1 ? m->n_out_pad : n_hidden);
    }
    // one arena: parameters, Adam moments, gradients, BF16 copies, activations
    size_t sz = 0;
    std::vector<size_t> offs;
    auto take = [&](size_t bytes) {
        offs.push_back(sz);
        sz += al256(bytes);
    };
    for (int l = 0; l < m->L; ++l) {
        const size_t nw = (size_t)m->dout[l] * m->din[l], nb = m->dout[l];
        for (int k = 0; k < 3; ++k) take(4 * nw);  // W, mW, vW
        take(4 * nw);                              // gW
        for (int k = 0; k < 4; ++k) take(4 * nb);  // b, mb, vb, gb
        take(2 * nw);                              // Wb
        take(2 * nw);                              // WTb
    }
    const size_t B = max_batch, mx = std::max(n_in, n_hidden);
    take(2 * B * n_in);  // X
    take(2 * B * n_in);  // XT
    for (int l = 0; l < n_hidden_layers; ++l) {
        take(2 * B * n_hidden);  // H
        take(2 * B * n_hidden);  // HT
    }
    take(4 * B * 128);      // Y
    take(4 * B * 128);      // dY
    take(2 * B * 128);      // dYb
    take(4 * B * mx);       // dH
    take(4 * B * mx);       // dZ
    take(2 * B * mx);       // dZb
    take(2 * B * mx);       // dZT
    take(4 * 1024);         // loss partials
    take(16);               // err
    take(4 * kSplitWsFloats);  // split-K workspace
    int st = MUSR_OK;
    if (cudaMalloc(&m->arena, sz) != cudaSuccess) {
        m->arena = nullptr;
        st = MUSR_ENOMEM;
    }
    // zeroed and finished before any stream of the network touches the arena
    if (st == MUSR_OK) st = cuda_status(cudaMemset(m->arena, 0, sz));
    if (st == MUSR_OK) st = cuda_status(cudaDeviceSynchronize());
    if (st == MUSR_OK) st = cuda_status(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking));
    if (st != MUSR_OK) {
        musr_mlp_destroy(m);
        return st;
    }
    char* a = static_cast<char*>(m->arena);
    size_t q = 0;
    auto nxt = [&]() { return a + offs[q++]; };
    for (int l = 0; l < m->L; ++l) {
        m->W.push_back((float*)nxt());
        m->mW.push_back((float*)nxt());
        m->vW.push_back((float*)nxt());
        m->gW.push_back((float*)nxt());
        m->b.push_back((float*)nxt());
        m->mb.push_back((float*)nxt());
        m->vb.push_back((float*)nxt());
        m->gb.push_back((float*)nxt());
        m->Wb.push_back((__nv_bfloat16*)nxt());
        m->WTb.push_back((__nv_bfloat16*)nxt());
    }
    m->X = (__nv_bfloat16*)nxt();
    m->XT = (__nv_bfloat16*)nxt();
    for (int l = 0; l < n_hidden_layers; ++l) {
        m->H.push_back((__nv_bfloat16*)nxt());
        m->HT.push_back((__nv_bfloat16*)nxt());
    }
    m->Y = (float*)nxt();
    m->dY = (float*)nxt();
    m->dYb = (__nv_bfloat16*)nxt();
    m->dH = (float*)nxt();
    m->dZ = (float*)nxt();
    m->dZb = (__nv_bfloat16*)nxt();
    m->dZT = (__nv_bfloat16*)nxt();
    m->loss_part = (float*)nxt();
    m->err = (unsigned*)nxt();
    m->ws = (float*)nxt();
    // He-uniform initialisation from a splitmix64 stream (host), zero biases
    m->n_params = 0;
    for (int l = 0; l < m->L; ++l) {
        const int ol = l == m->L - 1 ? n_out : m->dout[l];
        m->n_params += (int64_t)ol * m->din[l] + ol;
    }
    std::vector<float> init(m->n_params, 0.f);
    uint64_t sm = seed;
    auto next = [&]() {
        uint64_t z = (sm += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    size_t o = 0;
    for (int l = 0; l < m->L; ++l) {
        const int ol = l == m->L - 1 ? n_out : m->dout[l];
        const float lim = sqrtf(6.f / (float)m->din[l]) * (l == m->L - 1 ? 0.1f : 1.f);
        for (int64_t i = 0; i < (int64_t)ol * m->din[l]; ++i)
            init[o++] = lim * (2.f * (float)((next() >> 11) * (1.0 / 9007199254740992.0)) - 1.f);
        o += ol;
    }
    st = mlp_upload(m, init.data());
    if (st != MUSR_OK) {
        musr_mlp_destroy(m);
        return st;
    }
    *out = m;
    return MUSR_OK;
}

int musr_mlp_destroy(musr_mlp m) {
    if (!m) return MUSR_OK;
    if (m->stream) cudaStreamSynchronize(m->stream);
    if (m->arena) cudaFree(m->arena);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
    return MUSR_OK;
}

int musr_mlp_n_params(musr_mlp m, int64_t* n) {
    if (!m || !n) return MUSR_EINVAL;
    *n = m->n_params;
    return MUSR_OK;
}

int musr_mlp_set_params(musr_mlp m, const float* host) {
    if (!m || !host) return MUSR_EINVAL;
    return mlp_upload(m, host);
}

int musr_mlp_get_params(musr_mlp m, float* host) {
    if (!m || !host) return MUSR_EINVAL;
    return mlp_download(m, host, 0);
}

int musr_mlp_get_grads(musr_mlp m, float* host) {
    if (!m || !host) return MUSR_EINVAL;
    return mlp_download(m, host, 1);
}

static int mlp_check(musr_mlp m, int32_t batch) {
    if (!m || batch <= 0 || batch > m->max_b || batch % 128) return MUSR_EINVAL;
    return MUSR_OK;
}

static int mlp_err(musr_mlp m, cudaStream_t st) {
    unsigned e = 0;
    cudaError_t c = cudaMemcpyAsync(&e, m->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (c == cudaSuccess) c = cudaStreamSynchronize(st);
    if (c != cudaSuccess) return cuda_status(c);
    return e ? MUSR_ETIMEOUT : MUSR_OK;
}

int musr_mlp_get_activation(musr_mlp m, int32_t layer, int32_t batch, float* host) {
    int st = mlp_check(m, batch);
    if (st != MUSR_OK || !host || layer < 0 || layer > m->L) return st != MUSR_OK ? st : MUSR_EINVAL;
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (layer == m->L) {
        e = cudaMemcpy2D(host, sizeof(float) * m->n_out, m->Y, sizeof(float) * m->n_out_pad, sizeof(float) * m->n_out,
                         batch, cudaMemcpyDeviceToHost);
        return cuda_status(e);
    }
    const int w = layer == 0 ? m->n_in : m->n_hid;
    std::vector<__nv_bfloat16> tmp((size_t)batch * w);
    e = cudaMemcpy(tmp.data(), layer == 0 ? m->X : m->H[layer - 1], tmp.size() * sizeof(__nv_bfloat16),
                   cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    for (size_t i = 0; i < tmp.size(); ++i) host[i] = __bfloat162float(tmp[i]);
    return MUSR_OK;
}

int musr_mlp_forward(musr_mlp m, const float* x_dev, int32_t batch, float* y_dev, void* stream) {
    int st = mlp_check(m, batch);
    if (st != MUSR_OK || !x_dev || !y_dev) return st != MUSR_OK ? st : MUSR_EINVAL;
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : m->stream;
    st = mlp_forward(m, x_dev, batch, s);
    if (st == MUSR_OK)
        st = cuda_status(cudaMemcpy2DAsync(y_dev, sizeof(float) * m->n_out, m->Y, sizeof(float) * m->n_out_pad,
                                           sizeof(float) * m->n_out, batch, cudaMemcpyDeviceToDevice, s));
    return st == MUSR_OK ? mlp_err(m, s) : st;
}

int musr_mlp_backward(musr_mlp m, const float* x_dev, const float* t_dev, int32_t batch, float* loss,
                      void* stream) {
    int st = mlp_check(m, batch);
    if (st != MUSR_OK || !x_dev || !t_dev) return st != MUSR_OK ? st : MUSR_EINVAL;
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : m->stream;
    st = mlp_backward(m, x_dev, t_dev, batch, loss, s);
    return st == MUSR_OK ? mlp_err(m, s) : st;
}

int musr_mlp_adam(musr_mlp m, float lr, float beta1, float beta2, float eps, void* stream) {
    if (!m) return MUSR_EINVAL;
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : m->stream;
    return mlp_adam(m, lr, beta1, beta2, eps, s);
}

int musr_mlp_train_step(musr_mlp m, const float* x_dev, const float* t_dev, int32_t batch, float lr, float* loss,
                        void* stream) {
    int st = musr_mlp_backward(m, x_dev, t_dev, batch, loss, stream);
    if (st == MUSR_OK) st = musr_mlp_adam(m, lr, 0.9f, 0.999f, 1e-8f, stream);
    return st;
}

}  // extern "C"
