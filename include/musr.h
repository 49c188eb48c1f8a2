/*
 * musr.h -- C ABI of the GB300 muSR fit-objective library (libmusr.so).
 *
 * The library evaluates, on one GPU, the objective a muSR fit minimises:
 *
 *   theory   (Sec. 4.1, Eq. 1)  N_k(t) = N0_k exp(-t/tau_mu) [1 + A_k(t)] + Nbkg_k,
 *                               t = t0 + n * dt for bin n of histogram k;
 *   chi2     (Sec. 4.1, Eq. 3)  sum_k sum_n (d - N)^2 / max(d, 1);
 *   deviance (Sec. 4.1, Eq. 4)  2 sum_k sum_n [(N - d) + d ln(d / N)]  (2N where d = 0),
 *
 * over every bin of every histogram, for a parameter vector theta addressed
 * through a per-histogram map (Sec. 4.1 Eq. 2; the parameter / map arrays of
 * Sec. 4.2.1).  A_k(t) is a sum of components built from the predefined muSR
 * relaxation functions of Sec. 4.2.1 and the precession of Sec. 4.3 Eq. 5:
 *
 *   MUSR_TF_EXP          a exp(-lambda t)        cos(2 pi gamma (B + B2) t + phi)
 *   MUSR_TF_GAUSS        a exp(-(sigma t)^2 / 2) cos(2 pi gamma (B + B2) t + phi)
 *   MUSR_KT_STATIC_GAUSS a [1/3 + 2/3 (1 - (D t)^2) exp(-(D t)^2 / 2)]
 *   MUSR_TF_STRETCHED    a ge(t, lambda, beta)   cos(2 pi gamma (B + B2) t + phi),
 *                        ge = exp(-(lambda t)^beta) where lambda t > 0, 1 elsewhere
 *                        (the stretched exponential; a negative base has no
 *                        real power, so lambda t <= 0 is read as 1)
 *
 * Conventions shared by every entry point:
 *   - Every function returns MUSR_OK (0) or a negative status; none aborts.
 *   - Host buffers belong to the caller.  musr_create_run copies the data
 *     once (Sec. 4.2: data sets are uploaded once and reused for the whole
 *     fit) and keeps no caller pointer afterwards.
 *   - Host-pointer entry points are synchronous: results are in the caller's
 *     buffers when they return.  Entry points named *_device are
 *     asynchronous on the stream given (NULL = the run's own stream).
 *   - One run handle may be used by one host thread at a time, and calls on
 *     one run must not overlap on the GPU (they share the run's scratch).
 *   - Units: t in microseconds, fields in gauss, gamma in MHz/G, phases in
 *     radians, rates in 1/us.
 *   - Limits: map_width <= 32, at most 2 precession components (TF_EXP,
 *     TF_GAUSS or TF_STRETCHED, of which at most one TF_STRETCHED) and at most
 *     one KT_STATIC_GAUSS per run, at most 2^24 bins per histogram, at most
 *     4096 parameters.  Other layouts return MUSR_ENOTSUP.
 */
#ifndef MUSR_H
#define MUSR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MUSR_GAMMA_MU_MHZ_PER_G 0.013554 /* gamma_mu / 2 pi */
#define MUSR_TAU_MU_US 2.197             /* muon lifetime */

/* status codes */
enum {
    MUSR_OK = 0,
    MUSR_EINVAL = -1,     /* bad argument or layout */
    MUSR_ENOMEM = -2,     /* device or host allocation failed */
    MUSR_ECUDA = -3,      /* a CUDA call failed (no device, launch error ...) */
    MUSR_ENONFINITE = -4, /* theta holds NaN or Inf, or a result is not finite */
    MUSR_EDOMAIN = -5,    /* deviance: a bin has N < 0, or N = 0 with d > 0 */
    MUSR_ETIMEOUT = -6,   /* a bounded device wait ran out */
    MUSR_ENOCONV = -7,    /* the minimiser stopped without meeting its tolerance */
    MUSR_ENOTSUP = -8     /* layout outside the supported limits */
};

/* theory component kinds */
enum { MUSR_TF_EXP = 0, MUSR_TF_GAUSS = 1, MUSR_KT_STATIC_GAUSS = 2, MUSR_TF_STRETCHED = 3 };
/* objectives */
enum { MUSR_CHI2 = 0, MUSR_POISSON = 1 };
/* data element types */
enum { MUSR_F32 = 0, MUSR_F64 = 1 };
/* evaluation modes of musr_chi2_grad_device */
enum { MUSR_VALUE = 0, MUSR_VALUE_GRAD = 1, MUSR_VALUE_GRAD_GN = 2 };

/*
 * One theory component.  Each field is a COLUMN of the histogram's map row
 * (not a theta index); -1 means "not used" (the quantity is 0).
 *   amp    amplitude a
 *   rate   lambda (TF_EXP, TF_STRETCHED), sigma (TF_GAUSS) or Delta
 *          (KT_STATIC_GAUSS)
 *   field  field B of the precession (TF only)
 *   field2 a second field added to B, e.g. a line splitting dB (TF only)
 *   phase  phase phi in radians (TF only)
 *   beta   stretching exponent beta (TF_STRETCHED only; ignored otherwise)
 */
typedef struct {
    int32_t kind, amp, rate, field, field2, phase, beta;
} musr_component;

/*
 * Run description (Sec. 4.1 Eq. 1-2).
 *   n_hist, n_bins   K histograms with n_bins[k] bins each (uneven allowed).
 *   t0_us, dt_us     time grid t = t0 + n dt (Eq. 1 has t0 = 0).
 *   tau_us, gamma    muon lifetime and gamma_mu / 2 pi (MUSR_* defaults).
 *   n_params         length P of theta.
 *   map_width, map   K x map_width int32 row-major; map[k][c] is an index
 *                    into theta, -1 (constant 0) or -2 - j for entry j of
 *                    the function array.  Column 0 is N0 and column 1 is
 *                    Nbkg of histogram k.
 *   n_comp, comp     the components of A_k(t); the same list for every
 *                    histogram, each histogram reading its own map row.
 *   data_dtype, data counts d, histogram-major, concatenated (sum n_bins
 *                    values), MUSR_F32 or MUSR_F64.  The device keeps FP32
 *                    (counts are exact in FP32 below 2^24).  May be NULL for
 *                    a run used only to evaluate the model.
 *   data_on_device   nonzero if data is a device pointer (copied D2D).
 *   stream           cudaStream_t the run works on; NULL = the library
 *                    creates one for the run.
 *   n_funcs, funcs   the function array of Sec. 4.2.1 (n_funcs may be 0 and
 *                    funcs NULL): funcs[j] is an expression over p[i]
 *                    (theta entries, 0-based), numeric literals, + - * / ^
 *                    ( ) and exp log sqrt sin cos tan atan abs pow, whose
 *                    value a map entry -2 - j stands for.  The library copies
 *                    and compiles them at create (MUSR_EINVAL on a syntax
 *                    error or an index outside theta) and evaluates them on
 *                    the host per call, gradients and Gauss-Newton matrices
 *                    by the chain rule through their exact derivatives.  Runs
 *                    with functions serve the host-pointer entry points
 *                    (musr_chi2, musr_chi2_grad, musr_model, musr_fit,
 *                    musr_fit_multistart); the device, batched, generator,
 *                    proposer, user-theory and central-difference paths
 *                    return MUSR_ENOTSUP for them.  A function value that is
 *                    not finite gives MUSR_ENONFINITE.
 */
typedef struct {
    int32_t n_hist;
    const int64_t* n_bins;
    double t0_us, dt_us, tau_us, gamma_mhz_per_g;
    int32_t n_params, map_width;
    const int32_t* map;
    int32_t n_comp;
    const musr_component* comp;
    int32_t data_dtype;
    const void* data;
    int32_t data_on_device;
    void* stream;
    int32_t n_funcs;
    const char* const* funcs;
} musr_run_desc;

typedef struct musr_run_s* musr_run;

/*
 * One function-array expression (the syntax of musr_run_desc.funcs) at a
 * host parameter vector theta[n_params]: *value, and grad[n_params] (may be
 * NULL) its exact derivatives (forward mode; 0 for entries it does not read).
 * MUSR_EINVAL for a syntax error or an index outside theta, MUSR_ENONFINITE
 * for a value that is not finite.  Host only; needs no GPU.
 */
int musr_function_eval(const char* expr, int32_t n_params, const double* theta, double* value, double* grad);

/* Create a run: validates the layout, uploads the data once (Sec. 4.2) and
 * allocates the run's device scratch.  *out receives the handle. */
int musr_create_run(const musr_run_desc* desc, musr_run* out);

/* Release a run and everything it owns.  NULL is allowed. */
int musr_destroy_run(musr_run run);

/* Number of parameters P / total bins of a run (for marshalling). */
int musr_run_info(musr_run run, int32_t* n_params, int64_t* total_bins, int32_t* n_hist);

/* Replace the run's data (same layout) without re-planning.  Host or device
 * pointer as in the description; FP32 or FP64. */
int musr_set_data(musr_run run, int32_t data_dtype, const void* data, int32_t data_on_device);

/* Objective value (Eq. 3 if obj == MUSR_CHI2, Eq. 4 if MUSR_POISSON) at the
 * host FP64 vector theta[P].  Synchronous.  MUSR_EDOMAIN for an invalid
 * Poisson mean (value set to +inf), MUSR_ENONFINITE for non-finite theta. */
int musr_chi2(musr_run run, int obj, const double* theta, double* value);

/* Value, gradient d obj / d theta (grad[P], may be NULL) and Gauss-Newton
 * matrix gn[P*P] row-major (may be NULL), computed in one adjoint pass.
 * GN weights: 2 / max(d, 1) for chi2, 2 / N (Fisher scoring) for the
 * deviance.  Synchronous, host buffers. */
int musr_chi2_grad(musr_run run, int obj, const double* theta, double* value, double* grad,
                   double* gn);

/* Device variant: theta_dev[P] FP64 on the device; out_dev receives
 * [value, grad[P] (mode >= 1), gn[P*P] (mode == 2)] FP64; status_dev (may be
 * NULL) receives an int32 bit set: 1 = deviance domain error, 2 = non-finite
 * value.  Asynchronous on stream (NULL = run stream). */
int musr_chi2_grad_device(musr_run run, int obj, int mode, const double* theta_dev,
                          double* out_dev, int32_t* status_dev, void* stream);

/* Queued variant: theta[P] is a HOST FP64 vector, read during the call and
 * passed by value inside the launch (the caller may reuse it on return);
 * out_dev / status_dev / stream as for musr_chi2_grad_device, results in
 * stream order.  Because theta cannot change after the call, a queued
 * evaluation's parameter staging and bin loop (Eq. 1, Eq. 3 / Eq. 4 and their
 * adjoint) may run while the previous kernel in the stream finishes; its
 * additions into the run's reduction buffers and its results wait for that
 * kernel.  Runs of equal-length histograms are split into fewer, longer
 * blocks here than in the other entries (queued launches overlap, so fewer
 * blocks cost less), so results agree with theirs to FP32 rounding, not bit
 * for bit; repeated queued calls are bitwise equal.  MUSR_ENONFINITE for
 * non-finite theta, MUSR_ENOTSUP with a function array or more than 256
 * parameters.  Evaluations of one run queued on different streams must be
 * ordered by the caller (one reduction buffer per run). */
int musr_chi2_grad_async(musr_run run, int obj, int mode, const double* theta, double* out_dev,
                         int32_t* status_dev, void* stream);

/* Model N for every bin (FP32, histogram-major, total_bins values) into a
 * host (out_on_device == 0) or device buffer. */
int musr_model(musr_run run, const double* theta, float* out, int32_t out_on_device);

/*
 * Batched evaluation (many runs x many parameter vectors in one persistent
 * launch under a CUDA graph).  runs[r] has n_vec[r] parameter vectors of its
 * own length P_r, stored consecutively in thetas (run 0's vectors first);
 * values receives sum n_vec values in the same order.  The one-shot form
 * plans, evaluates and frees; musr_batch_* keep the plan for repeated use.
 */
int musr_chi2_batch(const musr_run* runs, int32_t n_runs, int obj, const double* thetas,
                    const int32_t* n_vec, double* values);

typedef struct musr_batch_s* musr_batch;
/* Plan a batch over runs[n_runs] with at most max_vec[r] vectors per run.
 * The runs must outlive the plan. */
int musr_batch_create(const musr_run* runs, int32_t n_runs, const int32_t* max_vec,
                      musr_batch* out);
int musr_batch_destroy(musr_batch batch);
/* Host-pointer evaluation with a plan (synchronous). */
int musr_batch_eval(musr_batch batch, int obj, const double* thetas, const int32_t* n_vec,
                    double* values);
/* Device-pointer evaluation with a plan: thetas_dev as above, on the device,
 * with every run's vector count fixed at its max_vec; values_dev FP64 on the
 * device.  Asynchronous on the plan's stream. */
int musr_batch_eval_device(musr_batch batch, int obj, const double* thetas_dev,
                           double* values_dev);

/*
 * Synthetic data.  (The paper fits measured histograms; the learned start
 * proposer is trained on histograms generated from the theory of Eq. 1.)
 *
 * musr_poisson_sample: counts_dev[i] ~ Poisson(mu_dev[i]) for n FP32 means on
 * the device.  Random numbers: Philox4x32-10 keyed by seed, counter (attempt,
 * i low, i high, 0xffffffff).  Inversion below mean 12, Hormann's PTRS above.
 * Asynchronous on stream.
 *
 * musr_generate: for n_samples parameter vectors thetas_dev (FP64, n_samples x
 * P, device) of the run's layout, the theory summed over groups of `rebin`
 * consecutive bins (the last group of a histogram may be short), a Poisson
 * count drawn for every group (counter (attempt, group, histogram,
 * sample_offset + sample)), written to out_dev as FP32 counts, or log(1 + count)
 * if log1p_out != 0; layout sample-major, then histogram, then group
 * (sum_k ceil(n_bins[k] / rebin) values per sample).  mu_dev (may be NULL)
 * receives the group means in the same layout.  The run's data are not used.
 * Asynchronous on stream (NULL = run stream).
 */
int musr_poisson_sample(const float* mu_dev, int64_t n, uint64_t seed, int32_t* counts_dev, void* stream);
int musr_generate(musr_run run, const double* thetas_dev, int32_t n_samples, int32_t rebin, uint64_t seed,
                  uint64_t sample_offset, int32_t log1p_out, float* out_dev, float* mu_dev, void* stream);

/*
 * BF16 tensor-core GEMM (the learned start proposer's dense layers; the paper
 * has no neural component).  C = act(A . B^T + bias): A [m x k] and B [n x k]
 * BF16 row-major on the device (16-byte aligned), FP32 accumulation, bias [n]
 * FP32 or NULL, relu != 0 applies max(., 0); results to out_f32 and / or
 * out_bf16 ([m x ldc] row-major, ldc >= n, ldc % 8 == 0).  m and n must be
 * multiples of 128 and k of 64 (MUSR_EINVAL otherwise).  ws_dev (FP32, device,
 * 16-byte aligned, ws_floats elements, may be NULL): scratch for split-K; when
 * the product has fewer than 76 output tiles of 128 x 128 and k >= 256, K is cut
 * into up to min(32, 152 / tiles) slices that fit in ws_floats (m * n floats a
 * slice; 152 * 128 * 128 always suffices), each slice's partial tile is written
 * there and a second kernel adds the slices in slice order (deterministic), then
 * bias and ReLU.  NULL or too small: one CTA per output tile.  err_dev: a
 * device uint32 the kernel ORs 1 into if a bounded internal wait times out.
 * Asynchronous on stream.
 */
int musr_gemm_bf16(const void* a_dev, const void* b_dev, int32_t m, int32_t n, int32_t k,
                   const float* bias_dev, int32_t relu, float* out_f32_dev, void* out_bf16_dev,
                   int32_t ldc, float* ws_dev, int64_t ws_floats, uint32_t* err_dev, void* stream);

/*
 * Learned start proposer: an MLP n_in -> n_hidden (x n_hidden_layers, ReLU)
 * -> n_out on the BF16 tensor cores (musr_gemm_bf16), FP32 master weights,
 * Adam.  Inputs are FP32 [batch x n_in] on the device, multiplied by in_scale
 * and rounded to BF16; outputs FP32 [batch x n_out].  Requirements: n_in % 128
 * == 0, n_hidden % 128 == 0, n_out <= 128, batch % 128 == 0 and batch <=
 * max_batch.  Parameters are exchanged as one FP32 host vector: for every
 * layer W [out x in] row-major then b [out].  Weights start He-uniform from a
 * splitmix64 stream of seed.  Forward / backward / train_step are synchronous
 * with respect to the returned loss and report MUSR_ETIMEOUT if a bounded
 * wait inside a GEMM timed out.
 *   musr_mlp_backward: forward, MSE loss mean((y - t)^2) (t FP32 [batch x
 *   n_out], device) into *loss (may be NULL), gradients kept internally
 *   (musr_mlp_get_grads); musr_mlp_adam applies one Adam step to them;
 *   musr_mlp_train_step = backward + Adam(lr, 0.9, 0.999, 1e-8).
 */
typedef struct musr_mlp_s* musr_mlp;
int musr_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_hidden_layers, int32_t n_out, int32_t max_batch,
                    float in_scale, uint64_t seed, musr_mlp* out);
int musr_mlp_destroy(musr_mlp mlp);
int musr_mlp_n_params(musr_mlp mlp, int64_t* n);
int musr_mlp_set_params(musr_mlp mlp, const float* host);
int musr_mlp_get_params(musr_mlp mlp, float* host);
int musr_mlp_get_grads(musr_mlp mlp, float* host);
int musr_mlp_forward(musr_mlp mlp, const float* x_dev, int32_t batch, float* y_dev, void* stream);
/* Activations of the last forward pass (or the forward inside the last
 * backward) to host FP32: layer 0 = the BF16 scaled input [batch x n_in],
 * 1..n_hidden_layers = the BF16 hidden outputs [batch x n_hidden],
 * n_hidden_layers + 1 = the FP32 output [batch x n_out]. */
int musr_mlp_get_activation(musr_mlp mlp, int32_t layer, int32_t batch, float* host);
int musr_mlp_backward(musr_mlp mlp, const float* x_dev, const float* t_dev, int32_t batch, float* loss,
                      void* stream);
int musr_mlp_adam(musr_mlp mlp, float lr, float beta1, float beta2, float eps, void* stream);
int musr_mlp_train_step(musr_mlp mlp, const float* x_dev, const float* t_dev, int32_t batch, float lr, float* loss,
                        void* stream);

/* Fit options and result (the host minimiser that replaces Minuit2's role,
 * Sec. 4.1). */
enum {
    MUSR_FIT_LM = 0,      /* Levenberg-Marquardt on the adjoint GN matrix */
    MUSR_FIT_BFGS = 1,    /* quasi-Newton (BFGS) on the adjoint gradient */
    MUSR_FIT_BFGS_FD = 2  /* BFGS on central differences from the batched kernel */
};
typedef struct {
    int32_t method;   /* MUSR_FIT_* */
    int32_t max_iter; /* <= 0: 500 */
    double edm_tol;   /* <= 0: 1e-8; stop when 1/2 g^T H^-1 g < edm_tol */
    double mu0;       /* <= 0: 1e-3; initial LM damping */
    double fd_rel_h;  /* MUSR_FIT_BFGS_FD steps: > 0 second-order central
                         differences with a fixed relative step
                         fd_rel_h * max(|theta_j|, 1); <= 0 (default)
                         fourth-order central differences with a step of two
                         standard errors of each parameter, from two passes
                         of second differences at the start (the FP32 value
                         noise enters the gradient divided by the step); a
                         step whose stencil meets a non-finite value is
                         quartered (up to three times) */
} musr_fit_opts;

typedef struct {
    double value;   /* objective at the returned theta */
    double ndf;     /* total bins - free parameters */
    double edm;     /* estimated distance to the minimum at exit */
    double mu;      /* final LM damping */
    int32_t iters;  /* minimiser iterations */
    int32_t n_evals;/* objective / adjoint launches */
    int32_t status; /* MUSR_OK or MUSR_ENOCONV / another error */
    int32_t n_free;
    double* cov;    /* caller buffer n_free x n_free (2 H^-1) or NULL */
} musr_fit_result;

/* Minimise obj over the parameters with free_mask[j] != 0 (NULL = all),
 * starting from theta_inout, which receives the result.  opts may be NULL
 * (defaults).  The return value equals out->status. */
int musr_fit(musr_run run, int obj, double* theta_inout, const uint8_t* free_mask,
             const musr_fit_opts* opts, musr_fit_result* out);

/*
 * Fit with a caller-supplied evaluation (histogram-sharded runs).  Every
 * objective sum of Sec. 4.1 (Eq. 3, Eq. 4) and its derivatives are sums over
 * histograms, so a run split by histogram over several GPUs (the multi-GPU
 * extension the paper's Sec. 6 names as future work) evaluates its shard on
 * each GPU and adds the shards' sums; this entry point drives the same
 * Levenberg-Marquardt (opts->method MUSR_FIT_LM) or BFGS (MUSR_FIT_BFGS)
 * steps as musr_fit, each evaluation a call of `eval`.  Called with the same
 * arguments on every rank, and with evaluations that return the same combined
 * sums on every rank, every rank takes the same steps and returns the same
 * theta.  Host only: the call itself makes no CUDA call.
 *   eval(user, mode, theta, value, grad, gn): at theta[n_params], *value,
 *            and for mode MUSR_VALUE_GRAD grad[n_params], for
 *            MUSR_VALUE_GRAD_GN also gn[n_params^2] (row-major); returns
 *            MUSR_OK, MUSR_EDOMAIN (the deviance has no likelihood there: a
 *            rejected step), or any other status, which ends the fit with it.
 *   n_bins_total  bins of the whole run (for ndf).
 *   theta_inout, free_mask, opts, out   as for musr_fit (MUSR_FIT_BFGS_FD
 *            returns MUSR_ENOTSUP).
 */
typedef int (*musr_eval_fn)(void* user, int mode, const double* theta, double* value, double* grad, double* gn);
int musr_fit_eval(int32_t n_params, int64_t n_bins_total, musr_eval_fn eval, void* user, double* theta_inout,
                  const uint8_t* free_mask, const musr_fit_opts* opts, musr_fit_result* out);

/*
 * Batched adjoint evaluation: value + gradient (and the GN matrix) of many
 * runs, one parameter vector each, in ONE launch (Eq. 3 / Eq. 4 and their
 * derivatives as for musr_chi2_grad; the same run may appear several times,
 * e.g. once per start point).  All runs must use the same component kinds and
 * device and have at least one histogram (MUSR_EINVAL otherwise); histograms
 * without bins are allowed.  with_gn != 0 prepares MUSR_VALUE_GRAD_GN (P <= 1024 per run) as
 * well as MUSR_VALUE_GRAD.  The handle refers to the runs (they must outlive
 * it) and owns its own tables, buffers and stream; launch shapes are tuned by
 * timing a few candidates on the first evaluation of each mode.
 *   thetas   concatenated parameter vectors, run r at sum_{q<r} P_q (FP64).
 *   out      concatenated outputs, run r at sum_{q<r} n_q with n_q = 1 + P_q
 *            (MUSR_VALUE_GRAD) or 1 + P_q + P_q^2 (MUSR_VALUE_GRAD_GN),
 *            laid out as musr_chi2_grad's value, grad, gn.
 *   active   NULL or one byte per run: runs with 0 are skipped (outputs and
 *            flags untouched).
 *   flags    NULL or one int32 per run: bit 0 deviance domain error (value
 *            meaningless), bit 1 non-finite value.
 * musr_gbatch_eval: host buffers, synchronous.  musr_gbatch_eval_device: device
 * buffers (thetas_dev, out_dev, flags_dev may be NULL), all runs, asynchronous
 * on stream (NULL = the handle's stream; the first call of a mode tunes and
 * synchronises).
 */
typedef struct musr_gbatch_s* musr_gbatch;
int musr_gbatch_create(const musr_run* runs, int32_t n_runs, int32_t with_gn, musr_gbatch* out);
int musr_gbatch_destroy(musr_gbatch batch);
int musr_gbatch_eval(musr_gbatch batch, int obj, int mode, const double* thetas, const uint8_t* active, double* out,
                     int32_t* flags);
int musr_gbatch_eval_device(musr_gbatch batch, int obj, int mode, const double* thetas_dev, double* out_dev,
                            int32_t* flags_dev, void* stream);

/* Levenberg-Marquardt fits of every run of a batch (created with with_gn) in
 * lockstep: one batched launch per iteration evaluates the trial points of
 * all unfinished runs; each run follows exactly musr_fit's LM rules and stops
 * on its own.  thetas: concatenated start vectors, replaced by the results;
 * free_masks: NULL (all free) or concatenated per-run masks; opts->method
 * MUSR_FIT_LM (each run follows musr_fit's LM rules; the batch needs with_gn)
 * or MUSR_FIT_BFGS (each run follows musr_fit's BFGS rules on the batched
 * value + gradient, one launch per round of line-search trials, the start's
 * Hessian diagonal from the GN matrix when the batch has it); others
 * MUSR_ENOTSUP; results: one per run (cov: caller buffer n_free x n_free or
 * NULL).  Returns MUSR_OK or the first run's non-OK status. */
int musr_fit_batch(musr_gbatch batch, int obj, double* thetas, const uint8_t* free_masks, const musr_fit_opts* opts,
                   musr_fit_result* results);

/* Multi-start fits of many runs in lockstep: every (run, start) pair is one
 * entry of an internal batch fitted by musr_fit_batch; per run the fit with
 * the smallest finite objective is kept.  starts: per run n_starts x P_r,
 * concatenated over runs; free_masks: NULL or concatenated per-run masks;
 * thetas_out: concatenated results; results: one per run (iters and n_evals
 * summed over its starts; cov, if given, is filled with NaN: not computed). */
int musr_fit_multistart_batch(const musr_run* runs, int32_t n_runs, int obj, const double* starts, int32_t n_starts,
                              const uint8_t* free_masks, const musr_fit_opts* opts, double* thetas_out,
                              musr_fit_result* results);

/* Plain multi-start fit: musr_fit from each of the n_starts rows of starts
 * (n_starts x n_params, FP64 host) in order; theta_out and out receive the
 * fit with the smallest finite objective (ties: the earliest).  Returns that
 * fit's status, or the first error if no fit gave a finite objective.
 * out->iters and out->n_evals are summed over all starts. */
int musr_fit_multistart(musr_run run, int obj, const double* starts, int32_t n_starts, const uint8_t* free_mask,
                        const musr_fit_opts* opts, double* theta_out, musr_fit_result* out);

/*
 * Learned start proposer (no counterpart in the paper, which starts every fit
 * from the user's values): an MLP (musr_mlp_*) maps standardised log counts
 * summed over groups of `rebin` bins (musr_proposer_features) to the parameters
 * with lo_j < hi_j, each scaled to [-1, 1] over [lo_j, hi_j].  It trains on
 * histograms that musr_generate draws from the layout run for parameter
 * vectors uniform in the box [lo, hi] (parameters with lo_j == hi_j held at
 * lo_j), fresh samples every step, all on the device.
 *   layout     a run whose layout (histograms, bins, time grid, map,
 *              components) the proposer serves; its data are not used.  It
 *              must outlive the proposer.
 *   lo, hi     FP64 host [n_params]; hi_j >= lo_j; at most 128 with hi > lo.
 *   opts       NULL or zeros for the defaults: rebin 64, n_hidden 512,
 *              n_hidden_layers 3, batch 512, in_scale 1 (a factor on the
 *              standardised features), seed 1, box_margin 0.25 (the
 *              learned-start fits fall back when a learned parameter ends
 *              outside [lo - m (hi - lo), hi + m (hi - lo)]; a very large
 *              value turns the check off).
 * The features must number <= 2^20 after padding to a multiple of 128.
 */
typedef struct musr_proposer_s* musr_proposer;
typedef struct {
    int32_t rebin;
    int32_t n_hidden;
    int32_t n_hidden_layers;
    int32_t batch;        /* training batch, multiple of 128 */
    float in_scale;
    uint64_t seed;
    float box_margin;
} musr_proposer_opts;
int musr_proposer_create(musr_run layout, const double* lo, const double* hi, const musr_proposer_opts* opts,
                         musr_proposer* out);
int musr_proposer_destroy(musr_proposer prop);
/* The proposer's network (owned by the proposer), e.g. to save or load it. */
int musr_proposer_mlp(musr_proposer prop, musr_mlp* out);
/* The training inputs: n parameter vectors (FP64 device [n x n_params]) for
 * sample indices offset .. offset + n - 1, learned entries lo_j + (hi_j -
 * lo_j) u with u in (0, 1) of 53 random bits from Philox4x32-10 (counter
 * (index low, index high, q / 2, 0xfffffffe), key (seed low ^ 0x0A5F00D1,
 * seed high), q the learned entry's rank; words 2h, 2h + 1 of the block give
 * entry q = 2 (q / 2) + h as ((w0 >> 5) 2^26 + (w1 >> 6) + 1/2) 2^-53), other
 * entries lo_j; targets_dev (FP32 [n x n_learned] or NULL) = 2u - 1.
 * Training step s draws indices s * batch .. (s + 1) * batch - 1 and their
 * histograms by musr_generate with the same seed and sample_offset s * batch
 * (counts, turned into features as musr_proposer_features does).
 * Asynchronous on stream (NULL = the proposer's). */
int musr_proposer_sample(musr_proposer prop, int32_t n, uint64_t offset, double* thetas_dev, float* targets_dev,
                         void* stream);
/* The network's input rows for n_runs runs (the layout's histogram and bin
 * counts), FP32 device [n_runs x n_features]: with c_kg the data counts
 * summed over group g of rebin bins of histogram k (musr_generate's order)
 * and C_k = sum_g c_kg, features f = 0 .. G-1 are
 * (log(1 + c_kg) - log(1 + C_k) - mu_f) * inv_sigma_f and features G + k are
 * (log(1 + C_k) - mu_f) * inv_sigma_f, G = sum_k ceil(n_bins[k] / rebin).
 * mu, inv_sigma: the standardisation (musr_proposer_get_norm).  Synchronous;
 * stream is unused. */
int musr_proposer_features(musr_proposer prop, const musr_run* runs, int32_t n_runs, float* out_dev, void* stream);
/* n_features (G + n_hist), n_learned (entries with hi > lo) and the network's
 * input width (n_features rounded up to a multiple of 128, zero-padded). */
int musr_proposer_info(musr_proposer prop, int32_t* n_features, int32_t* n_learned, int32_t* n_inputs);
/* The feature standardisation, FP32 host [n_features] each: mu_f and
 * 1 / max(sd_f, 1e-3) of the unstandardised features over 16 generated
 * batches of sample indices from 2^62 (estimated at the first call that needs
 * it); set_norm replaces it (e.g. with a saved one). */
int musr_proposer_get_norm(musr_proposer prop, float* mu, float* inv_sigma);
int musr_proposer_set_norm(musr_proposer prop, const float* mu, const float* inv_sigma);
/* n_steps Adam steps on fresh generated batches, learning rate decaying
 * geometrically from lr_start to lr_end; losses (NULL or n_steps floats)
 * receive the per-step MSE.  Successive calls continue the sample stream. */
int musr_proposer_train(musr_proposer prop, int32_t n_steps, float lr_start, float lr_end, float* losses);
/* Proposals for n_runs runs with the layout's histograms and bin counts
 * (MUSR_EINVAL otherwise), from each run's data: thetas_out FP64 host
 * [n_runs x n_params], learned entries clamped to [lo, hi], others lo. */
int musr_proposer_propose(musr_proposer prop, const musr_run* runs, int32_t n_runs, double* thetas_out);
/* Learned-start fit: propose, then musr_fit from the proposal.  If that fit
 * fails, ends with value / ndf > chi2ndf_max, or ends with a learned
 * parameter outside the box widened by box_margin (a basin the proposer was
 * not trained on, e.g. two precession lines that traded places), the
 * fallback follows in two stages, each keeping the better result:
 * (1) musr_fit_multistart from the n_fallback rows of fallback_starts shrunk
 * 8 times about their mean and centred on the proposal (entries the rows do
 * not scan take the proposal's value, scanned ones are searched finely around
 * it), at most 100 iterations per start, the first start that converges
 * within chi2ndf_max and the box ending the stage; (2) if that gave no such
 * fit, musr_fit_multistart from the rows as given (the plain fit).  *used_fallback (may be NULL): 0, or the last
 * stage run (1 or 2).  out->iters and out->n_evals count every fit made. */
int musr_fit_learned(musr_proposer prop, musr_run run, int obj, const uint8_t* free_mask, const musr_fit_opts* opts,
                     double chi2ndf_max, const double* fallback_starts, int32_t n_fallback, double* theta_out,
                     musr_fit_result* out, int32_t* used_fallback);
/* Learned-start fits of every run of a batch (musr_gbatch_create with
 * with_gn, runs of the proposer's layout): one network pass proposes all
 * starts, musr_fit_batch fits them in lockstep, and the runs whose fit fails,
 * ends above chi2ndf_max or leaves the widened box are refitted by
 * musr_fit_multistart_batch in the same two stages as musr_fit_learned from
 * their fallback starts (per run n_fallback x P_r, concatenated), keeping the
 * better result.  thetas_out, results, used_fallback (NULL or one int32):
 * one per run. */
int musr_fit_learned_batch(musr_proposer prop, musr_gbatch batch, int obj, const uint8_t* free_masks,
                           const musr_fit_opts* opts, double chi2ndf_max, const double* fallback_starts,
                           int32_t n_fallback, double* thetas_out, musr_fit_result* results, int32_t* used_fallback);

/*
 * User-defined theory functions (Sec. 4.2.1): the asymmetry A_k(t) of Eq. 1 as
 * a C expression, compiled at run time with NVRTC (loaded from the CUDA
 * toolkit; MUSR_ENOTSUP if it is missing) into a kernel that evaluates
 * N_k(t) = p[m[0]] e^{-t/tau} (1 + A_k(t)) + p[m[1]] and the Eq. 3 / Eq. 4
 * objective for many parameter vectors in one launch.
 *   dtype    MUSR_F64: everything in FP64 (as the paper's kernels);
 *            MUSR_F32: the expression, model and objective in FP32 (floating
 *            literals of the expression are taken as float), per-thread
 *            partial sums of at most 8 bins, FP64 beyond; tf() keeps its phase
 *            in FP64 from the exact time, so precession phases should be formed
 *            with tf (a phase written out in the expression is FP32).
 *            Relative accuracy of the objective ~1e-6 (FP32) / ~1e-12 (FP64).
 * An index outside p (n_params), m (map_width) or f (n_funcs) makes the
 * value +inf (the gradient MUSR_ENONFINITE) instead of reading out of bounds.
 *   expr     an expression (no statements) over: t (us, double); p (the
 *            parameter vector, double[]); m (the histogram's map row of the run
 *            descriptor, int[]: m[0] N0, m[1] background, the rest free for the
 *            expression); f (the function array, double[n_funcs], supplied per
 *            vector); numeric literals; + - * / ( ) [ ] ,; the CUDA math
 *            functions (exp, cos, sin, pow, sqrt, log, ...) and the muSR
 *            functions se(t, lambda) = exp(-lambda t), ge(t, lambda, beta) =
 *            exp(-(lambda t)^beta), sg(t, sigma) = exp(-(sigma t)^2 / 2),
 *            stg(t, sigma) = 1/3 + 2/3 (1 - (sigma t)^2) exp(-(sigma t)^2 / 2),
 *            tf(t, phi, B) = cos(2 pi 0.013554 B t + phi) (B in G, phi in rad).
 *            Characters outside [A-Za-z0-9_. +-*()/[],] are rejected
 *            (MUSR_EINVAL); a compile error returns MUSR_EINVAL and no
 *            handle; musr_utheory_log(NULL) then returns the compiler's log
 *            (per thread, until the next failure); musr_utheory_log(th) the
 *            log of a successful compile (warnings).
 * The run supplies histograms, bins, time grid, data and map rows; its
 * component table is not used.  Every call below is synchronous.
 *   musr_utheory_eval: values[v] (host) of obj for the n_vec host vectors
 *     thetas [n_vec x n_params] and funcs [n_vec x n_funcs] (NULL if
 *     n_funcs == 0); +inf where the deviance has no likelihood.
 *   musr_utheory_grad: value and gradient over the free entries: rel_h > 0
 *     central differences with step rel_h max(|theta_j|, 1) (one launch of
 *     1 + 2 n_free vectors); rel_h <= 0 forward-mode derivatives of the
 *     expression (dual numbers along each free parameter, one launch over
 *     histogram tiles x free parameters), exact up to rounding.
 *   musr_utheory_fit: BFGS on the forward-mode gradients, the start's Hessian
 *     diagonal from central second differences (opts->method and fd_rel_h
 *     set only that start's step); results as musr_fit.
 */
typedef struct musr_utheory_s* musr_utheory;
int musr_utheory_create(const char* expr, int32_t n_funcs, int32_t dtype, musr_utheory* out);
int musr_utheory_destroy(musr_utheory th);
const char* musr_utheory_log(musr_utheory th);
int musr_utheory_eval(musr_utheory th, musr_run run, int obj, const double* thetas, const double* funcs,
                      int32_t n_vec, double* values);
int musr_utheory_grad(musr_utheory th, musr_run run, int obj, const double* theta, const double* funcs,
                      const uint8_t* free_mask, double rel_h, double* value, double* grad);
int musr_utheory_fit(musr_utheory th, musr_run run, int obj, double* theta_inout, const double* funcs,
                     const uint8_t* free_mask, const musr_fit_opts* opts, musr_fit_result* out);

/* Message for a status code (static string). */
const char* musr_strerror(int code);

/* Library version string. */
const char* musr_version(void);

/*
 * Allocation-free evaluation.  (No counterpart in the paper: an interface
 * addition of this library.)  For callers that cannot call cudaMalloc --
 * e.g. code running while another framework owns the device memory pool, or
 * acquisition software that forbids allocation once it runs -- this entry
 * point evaluates the objective (mode MUSR_VALUE) or the objective and its
 * gradient (MUSR_VALUE_GRAD) without allocating anything: all scratch lives
 * in one static device array of MUSR_NOALLOC_SCRATCH_BYTES inside the
 * library.  The CUDA driver reserves that array on a device when it loads
 * the code of this entry point there, which with lazy module loading (the
 * default) happens during the first call on that device; from then on the
 * device holds it until the process ends.  Callers that start while another
 * framework may take the device memory therefore make one call at start-up.
 *   desc        layout as for musr_create_run; data must be FP32 on the device
 *               (data_on_device != 0, data_dtype == MUSR_F32); desc->stream
 *               is ignored.
 *   theta_dev   FP64 [n_params] on the device.
 *   out_dev     FP64 on the device: [value] or [value, grad[n_params]].
 *   status_dev  int32 on the device or NULL (bit 1: deviance domain error).
 *   stream      cudaStream_t; the call is asynchronous on it.
 * Limits: n_hist <= MUSR_NOALLOC_MAX_HIST, n_params <= MUSR_NOALLOC_MAX_PARAMS,
 * and the padded histograms plus tables must fit the scratch array (about 8e6
 * bins); anything larger returns MUSR_ENOTSUP, as do other modes or FP64 data.
 * Every call shares the one array and rewrites it, so calls whose work
 * overlaps on the GPU (different streams or host threads) race and must be
 * serialised by the caller.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress).  Each call uploads its
 * small tables from a host buffer the next call rewrites (pageable
 * cudaMemcpyAsync, which may block the host briefly); a call made while
 * `stream` is being captured into a graph returns MUSR_ENOTSUP.
 */
#define MUSR_NOALLOC_SCRATCH_BYTES (32u << 20)
#define MUSR_NOALLOC_MAX_HIST 64
#define MUSR_NOALLOC_MAX_PARAMS 256
int musr_chi2_grad_noalloc(const musr_run_desc* desc, int obj, int mode, const double* theta_dev,
                           double* out_dev, int32_t* status_dev, void* stream);

/* Name of the CUDA error behind the most recent MUSR_ECUDA / MUSR_ENOMEM
 * returned on the calling host thread ("none" if there was none). */
const char* musr_last_cuda_error(void);

/*
 * Measured pipe throughputs of the current device.  (No counterpart in the
 * paper: the objective kernels are bound by the FP32 and SFU pipes, Sec. 4.2.2
 * states none, and this call measures both so that fractions of peak are
 * fractions of what the GPU does.)  Each rate comes from a probe kernel that
 * keeps 16 independent chains of one operation per thread over four waves of
 * fully occupied SMs, best of five launches timed with CUDA events.
 *   rates    FP64 [n_rates >= MUSR_RATE_COUNT], thread-level operations per
 *            second, indexed by the MUSR_RATE_* constants: FP32 FMA (scalar),
 *            FP32 FMA issued as packed pairs (each pair counts two), and the
 *            SFU approximations ex2, sin, cos, rcp, lg2 (one PTX instruction
 *            each).
 * Allocates 4 bytes of device memory and a stream for the duration of the
 * call; returns MUSR_EINVAL for a short array, MUSR_ECUDA on a CUDA error.
 */
enum {
    MUSR_RATE_FFMA = 0,
    MUSR_RATE_FFMA2 = 1,
    MUSR_RATE_EX2 = 2,
    MUSR_RATE_SIN = 3,
    MUSR_RATE_COS = 4,
    MUSR_RATE_RCP = 5,
    MUSR_RATE_LG2 = 6,
    MUSR_RATE_COUNT = 7
};
int musr_pipe_rates(double* rates, int32_t n_rates);

#ifdef __cplusplus
}
#endif

#endif /* MUSR_H */
