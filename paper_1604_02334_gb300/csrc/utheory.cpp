// User-defined theory functions (Sec. 4.2.1): the asymmetry A_k(t) of Eq. 1
// given as a C expression over t, the parameter array p, the histogram's map
// row m and a function array f, compiled at run time with NVRTC into a kernel
// that evaluates the Eq. 3 / Eq. 4 objective of many parameter vectors in one
// launch.  The expression may call the predefined muSR functions of the
// paper's listing (se, ge, sg, stg) and tf, written here from their
// definitions, and the CUDA math functions.  Arithmetic is FP64 (the phase
// reaches hundreds of radians and the user expression is arbitrary).
//
// The generated kernel: one block per (tile of 2048 bins of a histogram,
// parameter vector), bins strided over the block's threads (coalesced),
// FP64 warp-shuffle and block sums into a partial per (vector, tile); a
// second small kernel adds each vector's partials in tile order, so values
// are bitwise repeatable.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>
#include <string.h>

#include <algorithm>
#include <cctype>
#include <cmath>
#include <functional>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "musr.h"
#include "musr_internal.h"
#include "run_impl.h"

using musr::cuda_status;

namespace musr {
int uth_eval_host(musr_utheory th, musr_run run, int obj, const double* thetas, const double* funcs, int n_vec,
                  double* values);
int uth_tangent_host(musr_utheory th, musr_run run, int obj, const double* theta, const double* funcs,
                     const std::vector<int>& dirs, double* grad_dirs);
}  // namespace musr

namespace {

// NVRTC entry points, resolved once from the toolkit's shared library
struct Nvrtc {
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    bool ok = false;
};

Nvrtc& nvrtc() {
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                               "/usr/local/cuda/lib64/libnvrtc.so"};
        void* h = nullptr;
        for (const char* nm : names)
            if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) return;
        n.create = reinterpret_cast<decltype(n.create)>(dlsym(h, "nvrtcCreateProgram"));
        n.compile = reinterpret_cast<decltype(n.compile)>(dlsym(h, "nvrtcCompileProgram"));
        n.log_size = reinterpret_cast<decltype(n.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
        n.log = reinterpret_cast<decltype(n.log)>(dlsym(h, "nvrtcGetProgramLog"));
        n.cubin_size = reinterpret_cast<decltype(n.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
        n.cubin = reinterpret_cast<decltype(n.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
        n.destroy = reinterpret_cast<decltype(n.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
        n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy;
    });
    return n;
}

thread_local std::string g_last_log;  // compile log of this thread's last failed musr_utheory_create

constexpr int kUTileBins = 2048;
constexpr int kUThreads = 256;

// An expression stays an expression: no statements, blocks, preprocessor,
// strings or assignments can be smuggled into the generated kernel.
bool expression_ok(const char* e) {
    if (!e) return false;
    size_t n = strlen(e);
    if (n == 0 || n > 8192) return false;
    int depth_p = 0, depth_b = 0;
    for (size_t i = 0; i < n; ++i) {
        const char c = e[i];
        const bool ok = (c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z') || (c >= '0' && c <= '9') || c == '_' ||
                        c == '.' || c == '+' || c == '-' || c == '*' || c == '/' || c == '(' || c == ')' ||
                        c == '[' || c == ']' || c == ',' || c == ' ' || c == '\t' || c == '\n';
        if (!ok) return false;
        depth_p += c == '(' ? 1 : c == ')' ? -1 : 0;
        depth_b += c == '[' ? 1 : c == ']' ? -1 : 0;
        if (depth_p < 0 || depth_b < 0) return false;
    }
    return depth_p == 0 && depth_b == 0;
}

// Floating literals of an FP32 expression get an f suffix, so that C's usual
// conversions keep its arithmetic in FP32 (integer literals stay int).
std::string to_fp32_literals(const std::string& e) {
    std::string out;
    size_t i = 0;
    while (i < e.size()) {
        const char c = e[i];
        const bool ident_before = i > 0 && (isalnum((unsigned char)e[i - 1]) || e[i - 1] == '_');
        if ((isdigit((unsigned char)c) || (c == '.' && i + 1 < e.size() && isdigit((unsigned char)e[i + 1]))) &&
            !ident_before) {
            size_t j = i;
            bool is_float = false;
            while (j < e.size() && (isdigit((unsigned char)e[j]) || e[j] == '.')) {
                if (e[j] == '.') is_float = true;
                ++j;
            }
            if (j < e.size() && (e[j] == 'e' || e[j] == 'E')) {
                size_t k = j + 1;
                if (k < e.size() && (e[k] == '+' || e[k] == '-')) ++k;
                if (k < e.size() && isdigit((unsigned char)e[k])) {
                    is_float = true;
                    j = k;
                    while (j < e.size() && isdigit((unsigned char)e[j])) ++j;
                }
            }
            out.append(e, i, j - i);
            if (is_float && !(j < e.size() && (e[j] == 'f' || e[j] == 'F'))) out.push_back('f');
            i = j;
        } else {
            out.push_back(c);
            ++i;
        }
    }
    return out;
}

// the kernel source around the user's expression; fp32: expression, model and
// objective in FP32 (per-thread partial sums, FP64 across threads), the
// precession phase of tf() in FP64 from the exact time
std::string kernel_source(const std::string& expr_in, bool fp32) {
    const std::string expr = fp32 ? to_fp32_literals(expr_in) : expr_in;
    std::string s = fp32 ? "typedef float real;\n#define MUSR_FP32 1\n" : "typedef double real;\n#define MUSR_FP32 0\n";
    s += R"SRC(
struct UParams {
    const float* data;
    const long long* hist_off;
    const int* hist_nbins;
    const int* map;
    const double* thetas;
    const double* funcs;
    double* partial;
    unsigned* flags;
    double t0, dt, inv_tau;
    int map_width, P, F, K, tph, n_tiles, obj;
};
// Forward-mode derivatives: a dual number carries a value and its derivative
// along one parameter; the expression compiled with dual parameters gives
// dN/dtheta_j exactly (up to rounding).
struct D {
    real v, d;
    __device__ D() : v(0), d(0) {}
    __device__ D(real a, real b) : v(a), d(b) {}
};
__device__ __forceinline__ real val(real x) { return x; }
__device__ __forceinline__ real val(D x) { return x.v; }
__device__ __forceinline__ D operator+(D a, D b) { return D(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ D operator+(D a, real b) { return D(a.v + b, a.d); }
__device__ __forceinline__ D operator+(real a, D b) { return D(a + b.v, b.d); }
__device__ __forceinline__ D operator-(D a, D b) { return D(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ D operator-(D a, real b) { return D(a.v - b, a.d); }
__device__ __forceinline__ D operator-(real a, D b) { return D(a - b.v, -b.d); }
__device__ __forceinline__ D operator-(D a) { return D(-a.v, -a.d); }
__device__ __forceinline__ D operator+(D a) { return a; }
__device__ __forceinline__ D operator*(D a, D b) { return D(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ D operator*(D a, real b) { return D(a.v * b, a.d * b); }
__device__ __forceinline__ D operator*(real a, D b) { return D(a * b.v, a * b.d); }
__device__ __forceinline__ D operator/(D a, D b) { return D(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
__device__ __forceinline__ D operator/(D a, real b) { return D(a.v / b, a.d / b); }
__device__ __forceinline__ D operator/(real a, D b) { return D(a / b.v, -a * b.d / (b.v * b.v)); }
__device__ __forceinline__ D operator+(D a, int b) { return a + (real)b; }
__device__ __forceinline__ D operator+(int a, D b) { return (real)a + b; }
__device__ __forceinline__ D operator-(D a, int b) { return a - (real)b; }
__device__ __forceinline__ D operator-(int a, D b) { return (real)a - b; }
__device__ __forceinline__ D operator*(D a, int b) { return a * (real)b; }
__device__ __forceinline__ D operator*(int a, D b) { return (real)a * b; }
__device__ __forceinline__ D operator/(D a, int b) { return a / (real)b; }
__device__ __forceinline__ D operator/(int a, D b) { return (real)a / b; }
__device__ __forceinline__ D exp(D a) { const real e = exp(a.v); return D(e, e * a.d); }
__device__ __forceinline__ D log(D a) { return D(log(a.v), a.d / a.v); }
__device__ __forceinline__ D sqrt(D a) { const real r = sqrt(a.v); return D(r, a.d / (2 * r)); }
__device__ __forceinline__ D cos(D a) { return D(cos(a.v), -sin(a.v) * a.d); }
__device__ __forceinline__ D sin(D a) { return D(sin(a.v), cos(a.v) * a.d); }
__device__ __forceinline__ D tan(D a) { const real q = tan(a.v); return D(q, (1 + q * q) * a.d); }
__device__ __forceinline__ D tanh(D a) { const real q = tanh(a.v); return D(q, (1 - q * q) * a.d); }
__device__ __forceinline__ D cosh(D a) { return D(cosh(a.v), sinh(a.v) * a.d); }
__device__ __forceinline__ D sinh(D a) { return D(sinh(a.v), cosh(a.v) * a.d); }
__device__ __forceinline__ D atan(D a) { return D(atan(a.v), a.d / (1 + a.v * a.v)); }
__device__ __forceinline__ D fabs(D a) { return a.v < 0 ? -a : a; }
__device__ __forceinline__ D pow(D a, real b) {
    const real q = pow(a.v, b);
    return D(q, a.v != 0 ? b * q / a.v * a.d : (b == 1 ? a.d : (real)0));
}
__device__ __forceinline__ D pow(D a, D b) {
    const real q = pow(a.v, b.v);
    return D(q, a.v > 0 ? q * (b.d * log(a.v) + b.v * a.d / a.v) : (real)0);
}
__device__ __forceinline__ D pow(real a, D b) { const real q = pow(a, b.v); return D(q, q * log(a) * b.d); }
__device__ __forceinline__ D pow(D a, int b) { return pow(a, (real)b); }
// the time: FP32 or FP64 value for the expression, the exact FP64 value for phases
struct TT {
    real f;
    double x;
    __device__ operator real() const { return f; }
};
// the predefined muSR functions of the user-function language (Sec. 4.2.1),
// from their definitions: se exponential, ge stretched exponential (1 where
// lambda t <= 0), sg Gaussian, stg static Gaussian Kubo-Toyabe
template <class L> __device__ __forceinline__ auto se(TT t, L lambda) { return exp(-(lambda * (real)t)); }
template <class L, class B> __device__ __forceinline__ auto ge(TT t, L lambda, B beta) {
    const auto x = lambda * (real)t;
    decltype(exp(-pow(x, beta))) one{};
    one = one + (real)1;
    return val(x) > 0 ? exp(-pow(x, beta)) : one;
}
template <class S> __device__ __forceinline__ auto sg(TT t, S sigma) {
    const auto x = sigma * (real)t;
    return exp(-(real)0.5 * (x * x));
}
template <class S> __device__ __forceinline__ auto stg(TT t, S sigma) {
    const auto x2 = (sigma * (real)t) * (sigma * (real)t);
    return (real)1 / (real)3 + (real)2 / (real)3 * ((real)1 - x2) * exp(-(real)0.5 * x2);
}
// transverse field precession: cos(2 pi gamma_mu B t + phi), B in G, t in us,
// phi in rad; the phase is formed in FP64 from the exact time and reduced to
// [-pi, pi] before the (FP32 in the FP32 variant) cosine
__device__ __forceinline__ double tf_phase(double t, double phi, double field) {
    const double ph = 6.283185307179586476925 * 0.013554 * field * t + phi;
    return ph - 6.283185307179586476925 * rint(ph * 0.15915494309189533577);
}
__device__ __forceinline__ real tf(TT t, real phi, real field) {
    return cos((real)tf_phase(t.x, (double)phi, (double)field));
}
__device__ __forceinline__ D tf(TT t, D phi, D field) {
    const real ph = (real)tf_phase(t.x, (double)phi.v, (double)field.v);
    const real w = (real)(6.283185307179586476925 * 0.013554) * (real)t;
    return D(cos(ph), -sin(ph) * (phi.d + w * field.d));
}
__device__ __forceinline__ D tf(TT t, real phi, D field) { return tf(t, D(phi, 0), field); }
__device__ __forceinline__ D tf(TT t, D phi, real field) { return tf(t, phi, D(field, 0)); }
__device__ __forceinline__ real lift(int x) { return (real)x; }
__device__ __forceinline__ real lift(real x) { return x; }
__device__ __forceinline__ D lift(D x) { return x; }
template <class P, class B> __device__ __forceinline__ auto tf(TT t, P phi, B field) {
    return tf(t, lift(phi), lift(field));
}
// parameter access: plain values, or duals seeded along parameter `dir`
// (an index outside p, m or f marks the bin bad instead of reading out of bounds)
struct PVal {
    const double* p;
    int n;
    bool* bad;
    __device__ real operator[](int i) const {
        if ((unsigned)i < (unsigned)n) return (real)p[i];
        *bad = true;
        return 0;
    }
};
struct PTan {
    const double* p;
    int n, dir;
    bool* bad;
    __device__ D operator[](int i) const {
        if ((unsigned)i < (unsigned)n) return D((real)p[i], i == dir ? (real)1 : (real)0);
        *bad = true;
        return D(0, 0);
    }
};
struct MVal {
    const int* m;
    int n;
    bool* bad;
    __device__ int operator[](int i) const {
        if ((unsigned)i < (unsigned)n) return m[i];
        *bad = true;
        return 0;
    }
};
struct FVal {
    const double* f;
    int n;
    bool* bad;
    __device__ real operator[](int i) const {
        if ((unsigned)i < (unsigned)n) return (real)f[i];
        *bad = true;
        return 0;
    }
};
template <class PA>
__device__ __forceinline__ auto user_asymmetry(TT t, const PA& p, const MVal& m, const FVal& f) {
    return (
)SRC";
    s += expr;
    s += R"SRC(
    );
}
// objective term of one bin and its derivative with respect to N (Eq. 3 / Eq. 4);
// the deviance as N h(r), h(r) = (1 + r) log1p(r) - r, r = (d - N) / N
__device__ __forceinline__ real obj_term(int obj, real dv, real N, bool& bad, real& dobj) {
    if (obj == 0) {
        const real w = (real)1 / (dv > (real)1 ? dv : (real)1);
        const real r = dv - N;
        dobj = (real)-2 * r * w;
        return r * r * w;
    }
    if (dv > 0) {
        if (!(N > 0)) {
            bad = true;
            dobj = 0;
            return 0;
        }
        const real r = (dv - N) / N;
        real h;
        if (MUSR_FP32 && fabs(r) < (real)0.125) {
            h = r * (real)(-1.0 / 72.0) + (real)(1.0 / 56.0);
            h = h * r - (real)(1.0 / 42.0);
            h = h * r + (real)(1.0 / 30.0);
            h = h * r - (real)(1.0 / 20.0);
            h = h * r + (real)(1.0 / 12.0);
            h = h * r - (real)(1.0 / 6.0);
            h = h * r + (real)0.5;
            h = h * r * r;
        } else {
            const real u = log1p(r);
            h = (1 + r) * u - r;
        }
        dobj = (real)2 * ((real)1 - dv / N);
        return (real)2 * N * h;
    }
    if (!(N >= 0)) bad = true;
    dobj = 2;
    return (real)2 * N;
}
extern "C" __global__ void __launch_bounds__(256) musr_user_objective(const UParams u) {
    __shared__ double red[8];
    __shared__ unsigned bad_s;
    const int tile = blockIdx.x, v = blockIdx.y;
    const int k = tile / u.tph;
    const int start = (tile - k * u.tph) * 2048;
    const int M = u.hist_nbins[k];
    bool bad = false;
    const PVal p{u.thetas + (size_t)v * u.P, u.P, &bad};
    const FVal f{u.funcs ? u.funcs + (size_t)v * u.F : nullptr, u.funcs ? u.F : 0, &bad};
    const MVal m{u.map + (size_t)k * u.map_width, u.map_width, &bad};
    const float* d = u.data + u.hist_off[k];
    const real n0 = p[m[0]], bkg = p[m[1]];
    const real inv_tau = (real)u.inv_tau;
    if (threadIdx.x == 0) bad_s = 0u;
    __syncthreads();
    real part = 0;  // at most 8 bins per thread per tile
    const int end = min(M, start + 2048);
    for (int n = start + (int)threadIdx.x; n < end; n += blockDim.x) {
        const double tx = u.t0 + (double)n * u.dt;
        const TT t{(real)tx, tx};
        const real N = n0 * exp(-(real)t * inv_tau) * ((real)1 + user_asymmetry(t, p, m, f)) + bkg;
        real dobj;
        part += obj_term(u.obj, (real)d[n], N, bad, dobj);
        if (!isfinite(N)) bad = true;
    }
    double acc = (double)part;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    if (bad) atomicOr(&bad_s, 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        u.partial[(size_t)v * u.n_tiles + tile] = s;
        if (bad_s) atomicOr(&u.flags[v], 1u);
    }
}
// d obj / d theta_j for the parameters dir_param[blockIdx.y] at one vector:
// sum over bins of (d obj / d N) (d N / d theta_j), N by forward-mode duals
extern "C" __global__ void __launch_bounds__(256) musr_user_tangent(const UParams u, const int* dir_param) {
    __shared__ double red[8];
    const int tile = blockIdx.x, dir = blockIdx.y;
    const int k = tile / u.tph;
    const int start = (tile - k * u.tph) * 2048;
    const int M = u.hist_nbins[k];
    bool bad = false;
    const PTan p{u.thetas, u.P, dir_param[dir], &bad};
    const FVal f{u.funcs, u.funcs ? u.F : 0, &bad};
    const MVal m{u.map + (size_t)k * u.map_width, u.map_width, &bad};
    const float* d = u.data + u.hist_off[k];
    const D n0 = p[m[0]], bkg = p[m[1]];
    const real inv_tau = (real)u.inv_tau;
    real part = 0;
    const int end = min(M, start + 2048);
    for (int n = start + (int)threadIdx.x; n < end; n += blockDim.x) {
        const double tx = u.t0 + (double)n * u.dt;
        const TT t{(real)tx, tx};
        const D N = n0 * exp(-(real)t * inv_tau) * ((real)1 + user_asymmetry(t, p, m, f)) + bkg;
        real dobj;
        obj_term(u.obj, (real)d[n], N.v, bad, dobj);
        part += dobj * N.d;
    }
    double acc = bad ? __longlong_as_double(0x7ff8000000000000LL) : (double)part;  // NaN marks a bad index
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        u.partial[(size_t)dir * u.n_tiles + tile] = s;
    }
}
// per vector, the tiles' partials in tile order
extern "C" __global__ void musr_user_sum(const double* partial, int n_tiles, int n_vec, unsigned* flags,
                                         double* values) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_vec) return;
    double s = 0.0;
    for (int i = 0; i < n_tiles; ++i) s += partial[(size_t)v * n_tiles + i];
    values[v] = flags[v] ? __longlong_as_double(0x7ff0000000000000LL) : s;
    flags[v] = 0u;
}
)SRC";
    return s;
}

}  // namespace

struct UParamsHost {  // the generated kernel's parameter block, same layout
    const float* data;
    const long long* hist_off;
    const int* hist_nbins;
    const int* map;
    const double* thetas;
    const double* funcs;
    double* partial;
    unsigned* flags;
    double t0, dt, inv_tau;
    int map_width, P, F, K, tph, n_tiles, obj;
};

struct musr_utheory_s {
    std::string expr, log;
    int n_funcs = 0;
    bool fp32 = false;
    int device = 0;
    cudaLibrary_t lib = nullptr;
    cudaKernel_t k_obj = nullptr, k_sum = nullptr, k_tan = nullptr;
    // scratch (grown on demand)
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    void* h_pinned = nullptr;
    size_t h_bytes = 0;
    cudaStream_t stream = nullptr;
    ~musr_utheory_s() {
        if (stream) cudaStreamSynchronize(stream);
        if (scratch) cudaFree(scratch);
        if (h_pinned) cudaFreeHost(h_pinned);
        if (lib) cudaLibraryUnload(lib);
        if (stream) cudaStreamDestroy(stream);
    }
};

namespace {

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// Evaluate obj for n_vec parameter vectors (device arrays); values_dev [n_vec].
int uth_launch(musr_utheory th, musr_run run, int obj, const double* thetas_dev, const double* funcs_dev, int n_vec,
               double* partial, unsigned* flags, double* values_dev, cudaStream_t st) {
    if (run->K == 0) return cuda_status(cudaMemsetAsync(values_dev, 0, sizeof(double) * n_vec, st));
    int64_t max_bins = 1;
    for (int k = 0; k < run->K; ++k) max_bins = std::max<int64_t>(max_bins, run->n_bins[k]);
    UParamsHost u;
    memset(&u, 0, sizeof(u));
    u.data = run->d_data;
    u.hist_off = reinterpret_cast<const long long*>(run->d_hist_off);
    u.hist_nbins = run->d_hist_nbins;
    u.map = run->d_map;
    u.thetas = thetas_dev;
    u.funcs = funcs_dev;
    u.partial = partial;
    u.flags = flags;
    u.t0 = run->t0;
    u.dt = run->dt;
    u.inv_tau = 1.0 / run->tau;
    u.map_width = run->W;
    u.P = run->P;
    u.F = th->n_funcs;
    u.K = run->K;
    u.tph = (int)((max_bins + kUTileBins - 1) / kUTileBins);
    u.n_tiles = u.K * u.tph;
    u.obj = obj;
    void* args[] = {&u};
    cudaError_t e = cudaLaunchKernel((const void*)th->k_obj, dim3(u.n_tiles, n_vec), dim3(kUThreads), args, 0, st);
    if (e != cudaSuccess) return cuda_status(e);
    int n_tiles = u.n_tiles;
    void* args2[] = {&partial, &n_tiles, &n_vec, &flags, &values_dev};
    e = cudaLaunchKernel((const void*)th->k_sum, dim3((n_vec + 127) / 128), dim3(128), args2, 0, st);
    return cuda_status(e);
}

int uth_reserve(musr_utheory th, musr_run run, int n_vec, size_t* o_theta, size_t* o_funcs, size_t* o_part,
                size_t* o_flags, size_t* o_vals, size_t* total, size_t* o_dirs = nullptr) {
    int64_t max_bins = 1;
    for (int k = 0; k < run->K; ++k) max_bins = std::max<int64_t>(max_bins, run->n_bins[k]);
    const size_t n_tiles = (size_t)std::max(run->K, 1) * ((max_bins + kUTileBins - 1) / kUTileBins);
    size_t o = 0;
    *o_theta = o;
    o += al256(sizeof(double) * (size_t)n_vec * run->P);
    *o_funcs = o;
    o += al256(sizeof(double) * (size_t)n_vec * std::max(th->n_funcs, 1));
    *o_part = o;
    o += al256(sizeof(double) * (size_t)n_vec * n_tiles);
    *o_flags = o;
    o += al256(sizeof(unsigned) * (size_t)n_vec);
    *o_vals = o;
    o += al256(sizeof(double) * (size_t)n_vec);
    if (o_dirs) *o_dirs = o;
    o += al256(sizeof(int32_t) * (size_t)n_vec);
    *total = o;
    if (o > th->scratch_bytes) {
        if (th->scratch) cudaFree(th->scratch);
        th->scratch = nullptr;
        th->scratch_bytes = 0;
        if (cudaMalloc(&th->scratch, o) != cudaSuccess) {
            th->scratch = nullptr;
            return MUSR_ENOMEM;
        }
        th->scratch_bytes = o;
        // zeroed on the handle's (non-blocking) stream, ahead of the launches that read the flags
        if (cudaMemsetAsync(th->scratch, 0, o, th->stream) != cudaSuccess) return MUSR_ECUDA;
    }
    if (o > th->h_bytes) {
        if (th->h_pinned) cudaFreeHost(th->h_pinned);
        th->h_pinned = nullptr;
        th->h_bytes = 0;
        if (cudaMallocHost(&th->h_pinned, o) != cudaSuccess) {
            th->h_pinned = nullptr;
            return MUSR_ENOMEM;
        }
        th->h_bytes = o;
    }
    return MUSR_OK;
}

}  // namespace

namespace musr {

// Host parameter vectors in, host values out (value = +inf where the deviance
// has no likelihood); one launch pair for all vectors.
int uth_eval_host(musr_utheory th, musr_run run, int obj, const double* thetas, const double* funcs, int n_vec,
                  double* values) {
    size_t ot, of, op, ofl, ov, total;
    int st = uth_reserve(th, run, n_vec, &ot, &of, &op, &ofl, &ov, &total);
    if (st != MUSR_OK) return st;
    char* d = static_cast<char*>(th->scratch);
    char* h = static_cast<char*>(th->h_pinned);
    memcpy(h + ot, thetas, sizeof(double) * (size_t)n_vec * run->P);
    if (funcs && th->n_funcs > 0) memcpy(h + of, funcs, sizeof(double) * (size_t)n_vec * th->n_funcs);
    cudaError_t e = cudaStreamSynchronize(run->stream);  // the run's data are in place
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d + ot, h + ot, sizeof(double) * (size_t)n_vec * run->P, cudaMemcpyHostToDevice,
                            th->stream);
    if (e == cudaSuccess && funcs && th->n_funcs > 0)
        e = cudaMemcpyAsync(d + of, h + of, sizeof(double) * (size_t)n_vec * th->n_funcs, cudaMemcpyHostToDevice,
                            th->stream);
    // the scratch layout depends on n_vec: this call's flag slots may hold an
    // earlier call's partial sums
    if (e == cudaSuccess) e = cudaMemsetAsync(d + ofl, 0, sizeof(unsigned) * (size_t)n_vec, th->stream);
    st = cuda_status(e);
    if (st == MUSR_OK)
        st = uth_launch(th, run, obj, reinterpret_cast<double*>(d + ot),
                        (funcs && th->n_funcs > 0) ? reinterpret_cast<double*>(d + of) : nullptr, n_vec,
                        reinterpret_cast<double*>(d + op), reinterpret_cast<unsigned*>(d + ofl),
                        reinterpret_cast<double*>(d + ov), th->stream);
    if (st == MUSR_OK)
        st = cuda_status(cudaMemcpyAsync(h + ov, d + ov, sizeof(double) * n_vec, cudaMemcpyDeviceToHost, th->stream));
    if (st == MUSR_OK) st = cuda_status(cudaStreamSynchronize(th->stream));
    if (st == MUSR_OK) memcpy(values, h + ov, sizeof(double) * n_vec);
    return st;
}

// d obj / d theta_j for the n_dirs parameter indices dirs[], by forward-mode
// duals: one launch over (tile, direction) and the fixed-order tile sums.
int uth_tangent_host(musr_utheory th, musr_run run, int obj, const double* theta, const double* funcs,
                     const std::vector<int>& dirs, double* grad_dirs) {
    const int nd = (int)dirs.size();
    if (nd == 0) return MUSR_OK;
    size_t ot, of, op, ofl, ov, od, total;
    int st = uth_reserve(th, run, std::max(nd, 1), &ot, &of, &op, &ofl, &ov, &total, &od);
    if (st != MUSR_OK) return st;
    if (run->K == 0) {
        for (int i = 0; i < nd; ++i) grad_dirs[i] = 0.0;
        return MUSR_OK;
    }
    char* d = static_cast<char*>(th->scratch);
    char* h = static_cast<char*>(th->h_pinned);
    memcpy(h + ot, theta, sizeof(double) * run->P);
    if (funcs && th->n_funcs > 0) memcpy(h + of, funcs, sizeof(double) * th->n_funcs);
    memcpy(h + od, dirs.data(), sizeof(int32_t) * nd);
    cudaError_t e = cudaStreamSynchronize(run->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d + ot, h + ot, sizeof(double) * run->P, cudaMemcpyHostToDevice, th->stream);
    if (e == cudaSuccess && funcs && th->n_funcs > 0)
        e = cudaMemcpyAsync(d + of, h + of, sizeof(double) * th->n_funcs, cudaMemcpyHostToDevice, th->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d + od, h + od, sizeof(int32_t) * nd, cudaMemcpyHostToDevice, th->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d + ofl, 0, sizeof(unsigned) * nd, th->stream);
    st = cuda_status(e);
    if (st != MUSR_OK) return st;
    int64_t max_bins = 1;
    for (int k = 0; k < run->K; ++k) max_bins = std::max<int64_t>(max_bins, run->n_bins[k]);
    UParamsHost u;
    memset(&u, 0, sizeof(u));
    u.data = run->d_data;
    u.hist_off = reinterpret_cast<const long long*>(run->d_hist_off);
    u.hist_nbins = run->d_hist_nbins;
    u.map = run->d_map;
    u.thetas = reinterpret_cast<double*>(d + ot);
    u.funcs = (funcs && th->n_funcs > 0) ? reinterpret_cast<double*>(d + of) : nullptr;
    u.partial = reinterpret_cast<double*>(d + op);
    u.flags = reinterpret_cast<unsigned*>(d + ofl);
    u.t0 = run->t0;
    u.dt = run->dt;
    u.inv_tau = 1.0 / run->tau;
    u.map_width = run->W;
    u.P = run->P;
    u.F = th->n_funcs;
    u.K = run->K;
    u.tph = (int)((max_bins + kUTileBins - 1) / kUTileBins);
    u.n_tiles = u.K * u.tph;
    u.obj = obj;
    const int* dirs_dev = reinterpret_cast<const int*>(d + od);
    void* args[] = {&u, (void*)&dirs_dev};
    e = cudaLaunchKernel((const void*)th->k_tan, dim3(u.n_tiles, nd), dim3(kUThreads), args, 0, th->stream);
    if (e == cudaSuccess) {
        double* part = u.partial;
        int n_tiles = u.n_tiles, n_vec = nd;
        unsigned* fl = u.flags;
        double* vals = reinterpret_cast<double*>(d + ov);
        void* args2[] = {&part, &n_tiles, &n_vec, &fl, &vals};
        e = cudaLaunchKernel((const void*)th->k_sum, dim3((nd + 127) / 128), dim3(128), args2, 0, th->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h + ov, d + ov, sizeof(double) * nd, cudaMemcpyDeviceToHost, th->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(th->stream);
    st = cuda_status(e);
    if (st == MUSR_OK) memcpy(grad_dirs, h + ov, sizeof(double) * nd);
    return st;
}

}  // namespace musr

int fit_bfgs_generic(int P, double* theta, const std::vector<int>& fidx, const musr_fit_opts& o, bool fd,
                     const std::function<int(const double*, double*, double*)>& value_grad,
                     const std::function<int(const double*, double*, double*, double*)>& start,
                     musr_fit_result* out);

namespace {

// value, central-difference gradient and (if hd) the diagonal second
// differences over the free entries, from one launch of 1 + 2 n_free vectors
int uth_fd(musr_utheory th, musr_run run, int obj, const double* theta, const double* funcs,
           const std::vector<int>& fidx, double rel_h, double* value, double* grad, double* hd) {
    const int P = run->P, nf = (int)fidx.size(), nv = 1 + 2 * nf;
    std::vector<double> vecs((size_t)nv * P), vals(nv), fv, h(nf);
    for (int v = 0; v < nv; ++v) memcpy(vecs.data() + (size_t)v * P, theta, sizeof(double) * P);
    for (int a = 0; a < nf; ++a) {
        const int j = fidx[a];
        h[a] = rel_h * std::max(std::fabs(theta[j]), 1.0);
        vecs[(size_t)(1 + 2 * a) * P + j] += h[a];
        vecs[(size_t)(2 + 2 * a) * P + j] -= h[a];
    }
    if (funcs && th->n_funcs > 0)
        for (int v = 0; v < nv; ++v) fv.insert(fv.end(), funcs, funcs + th->n_funcs);
    const int st = musr::uth_eval_host(th, run, obj, vecs.data(), fv.empty() ? nullptr : fv.data(), nv, vals.data());
    if (st != MUSR_OK) return st;
    *value = vals[0];
    if (!std::isfinite(vals[0])) return MUSR_EDOMAIN;
    memset(grad, 0, sizeof(double) * P);
    for (int a = 0; a < nf; ++a) {
        const double fp = vals[1 + 2 * a], fm = vals[2 + 2 * a];
        if (!std::isfinite(fp) || !std::isfinite(fm)) return MUSR_EDOMAIN;
        grad[fidx[a]] = (fp - fm) / (2.0 * h[a]);
        if (hd) hd[fidx[a]] = (fp - 2.0 * vals[0] + fm) / (h[a] * h[a]);
    }
    return MUSR_OK;
}

// value and forward-mode gradient over the free entries (two launches)
int uth_exact(musr_utheory th, musr_run run, int obj, const double* theta, const double* funcs,
              const std::vector<int>& fidx, double* value, double* grad) {
    int st = musr::uth_eval_host(th, run, obj, theta, funcs, 1, value);
    if (st != MUSR_OK) return st;
    if (!std::isfinite(*value)) return MUSR_EDOMAIN;
    std::vector<double> gd(fidx.size());
    st = musr::uth_tangent_host(th, run, obj, theta, funcs, fidx, gd.data());
    if (st != MUSR_OK) return st;
    memset(grad, 0, sizeof(double) * run->P);
    for (size_t a = 0; a < fidx.size(); ++a) {
        if (!std::isfinite(gd[a])) return MUSR_ENONFINITE;  // an index outside p, m or f
        grad[fidx[a]] = gd[a];
    }
    return MUSR_OK;
}

bool run_ok_for(musr_utheory th, musr_run run) {
    return th && run && run->device == th->device;
}

}  // namespace

extern "C" {

int musr_utheory_destroy(musr_utheory th) {
    delete th;
    return MUSR_OK;
}

const char* musr_utheory_log(musr_utheory th) { return th ? th->log.c_str() : g_last_log.c_str(); }

int musr_utheory_create(const char* expr, int32_t n_funcs, int32_t dtype, musr_utheory* out) {
    if (!out) return MUSR_EINVAL;
    *out = nullptr;
    if (!expression_ok(expr) || n_funcs < 0 || (dtype != MUSR_F32 && dtype != MUSR_F64)) return MUSR_EINVAL;
    Nvrtc& nv = nvrtc();
    if (!nv.ok) return MUSR_ENOTSUP;
    musr_utheory th = new (std::nothrow) musr_utheory_s();
    if (!th) return MUSR_ENOMEM;
    th->expr = expr;
    th->n_funcs = n_funcs;
    th->fp32 = dtype == MUSR_F32;
    cudaGetDevice(&th->device);
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, th->device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, th->device);
    const std::string src = kernel_source(th->expr, th->fp32);
    nvrtcProgram prog = nullptr;
    if (nv.create(&prog, src.c_str(), "musr_user_theory.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        delete th;
        return MUSR_ENOMEM;
    }
    const std::string arch = "--gpu-architecture=sm_" + std::to_string(major) + std::to_string(minor);
    const char* opts[] = {arch.c_str(), "--std=c++17", "-default-device"};
    const nvrtcResult cr = nv.compile(prog, 3, opts);
    size_t ls = 0;
    nv.log_size(prog, &ls);
    if (ls > 1) {
        th->log.resize(ls);
        nv.log(prog, &th->log[0]);
        th->log.resize(strlen(th->log.c_str()));
    }
    int st = MUSR_OK;
    std::vector<char> cubin;
    if (cr != NVRTC_SUCCESS) {
        st = MUSR_EINVAL;
    } else {
        size_t cs = 0;
        if (nv.cubin_size(prog, &cs) != NVRTC_SUCCESS || cs == 0) st = MUSR_ENOTSUP;
        if (st == MUSR_OK) {
            cubin.resize(cs);
            if (nv.cubin(prog, cubin.data()) != NVRTC_SUCCESS) st = MUSR_ENOTSUP;
        }
    }
    nv.destroy(&prog);
    if (st == MUSR_OK)
        st = cuda_status(cudaLibraryLoadData(&th->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0));
    if (st == MUSR_OK) st = cuda_status(cudaLibraryGetKernel(&th->k_obj, th->lib, "musr_user_objective"));
    if (st == MUSR_OK) st = cuda_status(cudaLibraryGetKernel(&th->k_sum, th->lib, "musr_user_sum"));
    if (st == MUSR_OK) st = cuda_status(cudaLibraryGetKernel(&th->k_tan, th->lib, "musr_user_tangent"));
    if (st == MUSR_OK) st = cuda_status(cudaStreamCreateWithFlags(&th->stream, cudaStreamNonBlocking));
    if (st != MUSR_OK && st != MUSR_EINVAL) {
        delete th;
        return st;
    }
    if (st == MUSR_EINVAL) {
        // a failed compile returns no handle; its log stays readable through
        // musr_utheory_log(NULL) on this thread until the next failure
        g_last_log = th->log;
        delete th;
        return st;
    }
    *out = th;
    return MUSR_OK;
}

int musr_utheory_eval(musr_utheory th, musr_run run, int obj, const double* thetas, const double* funcs,
                      int32_t n_vec, double* values) {
    if (!run_ok_for(th, run) || n_vec < 0 || (n_vec > 0 && (!thetas || !values))) return MUSR_EINVAL;
    if (run->F > 0) return MUSR_ENOTSUP;  // the expression takes its function array per call
    if (obj != MUSR_CHI2 && obj != MUSR_POISSON) return MUSR_EINVAL;
    if (th->n_funcs > 0 && n_vec > 0 && !funcs) return MUSR_EINVAL;
    if (n_vec == 0) return MUSR_OK;
    for (int64_t i = 0; i < (int64_t)n_vec * run->P; ++i)
        if (!std::isfinite(thetas[i])) return MUSR_ENONFINITE;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != th->device) cudaSetDevice(th->device);
    const int st = musr::uth_eval_host(th, run, obj, thetas, funcs, n_vec, values);
    if (cur != th->device) cudaSetDevice(cur);
    return st;
}

int musr_utheory_grad(musr_utheory th, musr_run run, int obj, const double* theta, const double* funcs,
                      const uint8_t* free_mask, double rel_h, double* value, double* grad) {
    if (!run_ok_for(th, run) || !theta || !value || !grad) return MUSR_EINVAL;
    if (run->F > 0) return MUSR_ENOTSUP;
    if (obj != MUSR_CHI2 && obj != MUSR_POISSON) return MUSR_EINVAL;
    if (th->n_funcs > 0 && !funcs) return MUSR_EINVAL;
    for (int j = 0; j < run->P; ++j)
        if (!std::isfinite(theta[j])) return MUSR_ENONFINITE;
    std::vector<int> fidx;
    for (int j = 0; j < run->P; ++j)
        if (!free_mask || free_mask[j]) fidx.push_back(j);
    if (rel_h > 0.0) return uth_fd(th, run, obj, theta, funcs, fidx, rel_h, value, grad, nullptr);
    return uth_exact(th, run, obj, theta, funcs, fidx, value, grad);
}

int musr_utheory_fit(musr_utheory th, musr_run run, int obj, double* theta, const double* funcs,
                     const uint8_t* free_mask, const musr_fit_opts* opts, musr_fit_result* out) {
    if (!run_ok_for(th, run) || !theta || !out) return MUSR_EINVAL;
    if (run->F > 0) return MUSR_ENOTSUP;
    if (obj != MUSR_CHI2 && obj != MUSR_POISSON) return MUSR_EINVAL;
    if (th->n_funcs > 0 && !funcs) return MUSR_EINVAL;
    musr_fit_opts o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.max_iter <= 0) o.max_iter = 500;
    if (!(o.edm_tol > 0.0)) o.edm_tol = 1e-8;
    if (!(o.fd_rel_h > 0.0)) o.fd_rel_h = 1e-4;
    std::vector<int> fidx;
    for (int j = 0; j < run->P; ++j)
        if (!free_mask || free_mask[j]) fidx.push_back(j);
    int evals = 0;
    auto vg = [&](const double* th_, double* f, double* g) {
        ++evals;
        return uth_exact(th, run, obj, th_, funcs, fidx, f, g);
    };
    auto start = [&](const double* th_, double* f, double* g, double* hd) {
        ++evals;
        return uth_fd(th, run, obj, th_, funcs, fidx, o.fd_rel_h, f, g, hd);
    };
    musr_fit_result r = *out;
    r.n_free = (int32_t)fidx.size();
    r.ndf = (double)(run->total_bins - (int64_t)fidx.size());
    const int st = fit_bfgs_generic(run->P, theta, fidx, o, false, vg, start, &r);
    r.n_evals = evals;
    r.status = st;
    *out = r;
    return st;
}

}  // extern "C"
