/*
 * Plain FP64 CPU oracle for the muSR fit objective.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU library computes.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header or constant with the CUDA library: every formula
 * here is written directly from the paper.
 *
 *   Sec. 4.1, Eq. 1  N^j(t) = N0^j exp(-t/tau_mu) [1 + A^j(p, t)] + Nbkg^j,
 *                    t = n * dt  (n = 0, 1, 2, ...; a start offset t0 is
 *                    allowed, t = t0 + n * dt, with t0 = 0 reproducing Eq. 1)
 *   Sec. 4.1, Eq. 2  per-histogram parameter set {N0, Nbkg, p}; the map array
 *                    of Sec. 4.2.1 gives the indirect addressing from a
 *                    histogram's slots to the global parameter vector.
 *   Sec. 4.1, Eq. 3  chi2 = sum_j sum_n (d - N)^2 / d_err^2, d_err^2 = d;
 *                    reading: d_err^2 = max(d, 1) so that empty bins are
 *                    defined.
 *   Sec. 4.1, Eq. 4  L = 2 sum_j sum_n [(N - d) + d ln(d / N)]; reading: the
 *                    log term sits inside the bracket (Poisson deviance,
 *                    -2 ln of the likelihood ratio), it is minimised, and a
 *                    bin with d = 0 contributes 2N.
 *   Sec. 4.2.1       theories are built from predefined relaxation functions
 *                    common in muSR (the exponential and Gaussian ones among
 *                    them); the four used here, from their standard
 *                    definitions, lambda and sigma rates in 1/us:
 *                    exponential          exp(-lambda t)
 *                    Gaussian             exp(-(sigma t)^2 / 2)
 *                    static Gaussian Kubo-Toyabe (zero field)
 *                                         1/3 + 2/3 (1 - (sigma t)^2) exp(-(sigma t)^2 / 2)
 *                    stretched exponential exp(-(lambda t)^beta); reading: 1
 *                                         where lambda t <= 0 (a negative
 *                                         base has no real power)
 *   Sec. 4.3, Eq. 5  A = A0 exp(-(sigma t)^2 / 2) cos(gamma_mu B t + phi);
 *                    the precession factor is cos(2 pi gamma B t + phi) with
 *                    gamma in MHz/G, t in us, phi in radians.
 *
 * Component kinds (columns are indices into the histogram's map row; a map
 * entry of -1 stands for the constant 0):
 *   0  TF_EXP   a * se(t, rate) * cos(2 pi gamma (B + B2) t + phi)
 *   1  TF_GAUSS a * sg(t, rate) * cos(2 pi gamma (B + B2) t + phi)
 *   2  KT_SG    a * stg(t, rate)
 *   3  TF_GE    a * ge(t, rate, beta) * cos(2 pi gamma (B + B2) t + phi)
 *
 * Every sum over bins uses Neumaier-compensated FP64 summation, so the value
 * returned is the exact sum of the FP64 per-bin terms to within a few ulp.
 *
 * Gradients: analytic chain rule (Sec. 4.1 objectives differentiated by
 * hand) and, independently, FP64 central finite differences.  The
 * Gauss-Newton matrix is H = sum c J J^T with c = 2 / max(d, 1) for chi2 and
 * c = 2 / N (expected information, Fisher scoring) for the deviance.
 *
 * The fit is a Levenberg-Marquardt minimiser (the paper drives the same
 * objective with Minuit2, Sec. 4.1) over the free parameters.
 *
 * Parity status: every function here is pinned by closed forms, invariants,
 * library routines or brute force in tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_ENONFINITE -4
#define ORC_EDOMAIN -5
#define ORC_ENOCONV -7

#define ORC_TF_EXP 0
#define ORC_TF_GAUSS 1
#define ORC_KT_SG 2
#define ORC_TF_GE 3

#define ORC_CHI2 0
#define ORC_POISSON 1

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* Neumaier compensated summation                                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    double s, c;
} orc_acc;

static void acc_add(orc_acc* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double acc_val(const orc_acc* a) { return a->s + a->c; }

/* ------------------------------------------------------------------------ */
/* Layout                                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n_hist;
    const int64_t* n_bins;
    double t0, dt, tau, gamma;
    int n_params, map_width;
    const int32_t* map;
    int n_comp;
    const int32_t* comp; /* n_comp x 7: kind, amp, rate, field, field2, phase, beta */
} orc_layout;

static int64_t hist_offset(const orc_layout* L, int k) {
    int64_t off = 0;
    for (int j = 0; j < k; ++j) off += L->n_bins[j];
    return off;
}

static int64_t total_bins(const orc_layout* L) { return hist_offset(L, L->n_hist); }

/* theta index of map column col for histogram k, or -1 */
static int map_index(const orc_layout* L, int k, int col) {
    if (col < 0) return -1;
    return L->map[(int64_t)k * L->map_width + col];
}

static double map_value(const orc_layout* L, const double* theta, int k, int col) {
    int i = map_index(L, k, col);
    return i < 0 ? 0.0 : theta[i];
}

static int check_layout(const orc_layout* L) {
    if (L->n_hist < 0 || L->n_params < 0 || L->map_width < 2 || L->n_comp < 0) return ORC_EINVAL;
    if (!(L->dt > 0.0) || !(L->tau > 0.0)) return ORC_EINVAL;
    for (int k = 0; k < L->n_hist; ++k) {
        if (L->n_bins[k] < 0) return ORC_EINVAL;
        for (int c = 0; c < L->map_width; ++c) {
            int i = L->map[(int64_t)k * L->map_width + c];
            if (i < -1 || i >= L->n_params) return ORC_EINVAL;
        }
    }
    for (int c = 0; c < L->n_comp; ++c) {
        const int32_t* d = L->comp + 7 * c;
        if (d[0] < 0 || d[0] > 3) return ORC_EINVAL;
        for (int s = 1; s < 7; ++s)
            if (d[s] < -1 || d[s] >= L->map_width) return ORC_EINVAL;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Relaxation functions of the component kinds (Sec. 4.2.1, Eq. 5), in the  */
/* order of the kinds                                                        */
/* ------------------------------------------------------------------------ */
/* TF_EXP: exponential relaxation */
static double relax_exponential(double t, double lambda) { return exp(-lambda * t); }

/* TF_GAUSS: Gaussian relaxation (Eq. 5) */
static double relax_gaussian(double t, double sigma) {
    double st = sigma * t;
    return exp(-0.5 * st * st);
}

/* KT_SG: static Gaussian Kubo-Toyabe function in zero field; -> 1/3 at large t */
static double kubo_toyabe_static_gaussian(double t, double sigma) {
    double x = (sigma * t) * (sigma * t);
    return 1.0 / 3.0 + (2.0 / 3.0) * (1.0 - x) * exp(-0.5 * x);
}

/* TF_GE: stretched exponential; l t <= 0 gives 1 (a negative base has no real power) */
static double relax_stretched(double t, double lambda, double beta) {
    double x = lambda * t;
    return x > 0.0 ? exp(-pow(x, beta)) : 1.0;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 theory at one bin, plus its derivative with respect to every map    */
/* column of the histogram (dcol may be NULL).                              */
/* ------------------------------------------------------------------------ */
static double theory_bin(const orc_layout* L, const double* theta, int k, double t, double* dcol) {
    double n0 = map_value(L, theta, k, 0);
    double bkg = map_value(L, theta, k, 1);
    double life = exp(-t / L->tau);
    double asym = 0.0;
    /* dA/d(column value) accumulated per column */
    double* dA = NULL;
    double dA_local[64];
    if (dcol) {
        dA = dA_local;
        for (int c = 0; c < L->map_width; ++c) dA[c] = 0.0;
    }
    for (int c = 0; c < L->n_comp; ++c) {
        const int32_t* d = L->comp + 7 * c;
        int kind = d[0];
        double a = map_value(L, theta, k, d[1]);
        double rate = map_value(L, theta, k, d[2]);
        if (kind == ORC_KT_SG) {
            double g = kubo_toyabe_static_gaussian(t, rate);
            asym += a * g;
            if (dA) {
                if (d[1] >= 0) dA[d[1]] += g;
                if (d[2] >= 0) {
                    /* d stg / d sigma = (2/3) sigma t^2 ((sigma t)^2 - 3) exp(-(sigma t)^2/2) */
                    double x = (rate * t) * (rate * t);
                    dA[d[2]] += a * (2.0 / 3.0) * rate * t * t * (x - 3.0) * exp(-0.5 * x);
                }
            }
            continue;
        }
        double field = map_value(L, theta, k, d[3]) + map_value(L, theta, k, d[4]);
        double phi = map_value(L, theta, k, d[5]);
        double arg = 2.0 * ORC_PI * L->gamma * field * t + phi;
        double cs = cos(arg), sn = sin(arg);
        double env, denv_drate, denv_dbeta = 0.0;
        if (kind == ORC_TF_EXP) {
            env = relax_exponential(t, rate);
            denv_drate = -t * env;
        } else if (kind == ORC_TF_GAUSS) {
            env = relax_gaussian(t, rate);
            denv_drate = -rate * t * t * env;
        } else {
            /* d/dl exp(-(l t)^b) = -b t (l t)^(b-1) exp(-(l t)^b);
               d/db exp(-(l t)^b) = -(l t)^b ln(l t) exp(-(l t)^b); both 0 where l t <= 0 */
            double beta = map_value(L, theta, k, d[6]);
            double x = rate * t;
            env = relax_stretched(t, rate, beta);
            denv_drate = x > 0.0 ? -beta * t * pow(x, beta - 1.0) * env : 0.0;
            denv_dbeta = x > 0.0 ? -pow(x, beta) * log(x) * env : 0.0;
        }
        asym += a * env * cs;
        if (dA) {
            if (d[1] >= 0) dA[d[1]] += env * cs;
            if (d[2] >= 0) dA[d[2]] += a * denv_drate * cs;
            if (kind == ORC_TF_GE && d[6] >= 0) dA[d[6]] += a * denv_dbeta * cs;
            double dphase = -a * env * sn;
            if (d[3] >= 0) dA[d[3]] += dphase * 2.0 * ORC_PI * L->gamma * t;
            if (d[4] >= 0) dA[d[4]] += dphase * 2.0 * ORC_PI * L->gamma * t;
            if (d[5] >= 0) dA[d[5]] += dphase;
        }
    }
    double n = n0 * life * (1.0 + asym) + bkg;
    if (dcol) {
        for (int c = 0; c < L->map_width; ++c) dcol[c] = n0 * life * dA[c];
        dcol[0] += life * (1.0 + asym);
        dcol[1] += 1.0;
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Per-bin objective terms (Eq. 3 and Eq. 4)                                 */
/* ------------------------------------------------------------------------ */
static double chi2_term(double d, double n) {
    double var = d > 1.0 ? d : 1.0;
    double r = d - n;
    return r * r / var;
}

/* returns 0 on success, ORC_EDOMAIN when the Poisson mean is invalid */
static int deviance_term(double d, double n, double* out) {
    if (n < 0.0 || (n == 0.0 && d > 0.0) || !(n == n)) return ORC_EDOMAIN;
    if (d == 0.0) {
        *out = 2.0 * n;
        return 0;
    }
    *out = 2.0 * ((n - d) + d * log(d / n));
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Public entry points                                                       */
/* ------------------------------------------------------------------------ */
#define LAYOUT_ARGS                                                                         \
    int n_hist, const int64_t *n_bins, double t0, double dt, double tau, double gamma,     \
        int n_params, int map_width, const int32_t *map, int n_comp, const int32_t *comp
#define MAKE_LAYOUT                                                                          \
    orc_layout L = {n_hist, n_bins, t0, dt, tau, gamma, n_params, map_width, map, n_comp, comp}

int orc_model(LAYOUT_ARGS, const double* theta, double* out) {
    MAKE_LAYOUT;
    int st = check_layout(&L);
    if (st) return st;
    if (L.map_width > 64) return ORC_EINVAL;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < L.n_hist; ++k) {
        int64_t off = hist_offset(&L, k);
        for (int64_t i = 0; i < L.n_bins[k]; ++i)
            out[off + i] = theory_bin(&L, theta, k, L.t0 + (double)i * L.dt, NULL);
    }
    return ORC_OK;
}

static int objective_impl(const orc_layout* L, const double* data, const double* theta, int obj,
                          double* value) {
    int status = ORC_OK;
    double* hsum = (double*)calloc((size_t)(L->n_hist > 0 ? L->n_hist : 1), sizeof(double));
    int* hst = (int*)calloc((size_t)(L->n_hist > 0 ? L->n_hist : 1), sizeof(int));
    if (!hsum || !hst) {
        free(hsum);
        free(hst);
        return ORC_ENOMEM;
    }
#pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < L->n_hist; ++k) {
        int64_t off = hist_offset(L, k);
        orc_acc a = {0.0, 0.0};
        for (int64_t i = 0; i < L->n_bins[k]; ++i) {
            double n = theory_bin(L, theta, k, L->t0 + (double)i * L->dt, NULL);
            double d = data[off + i];
            if (obj == ORC_CHI2) {
                acc_add(&a, chi2_term(d, n));
            } else {
                double term;
                if (deviance_term(d, n, &term)) {
                    hst[k] = ORC_EDOMAIN;
                    break;
                }
                acc_add(&a, term);
            }
        }
        hsum[k] = acc_val(&a);
    }
    orc_acc tot = {0.0, 0.0};
    for (int k = 0; k < L->n_hist; ++k) {
        if (hst[k]) status = hst[k];
        acc_add(&tot, hsum[k]);
    }
    free(hsum);
    free(hst);
    *value = status ? INFINITY : acc_val(&tot);
    return status;
}

int orc_objective(LAYOUT_ARGS, const double* data, const double* theta, int obj, double* value) {
    MAKE_LAYOUT;
    int st = check_layout(&L);
    if (st) return st;
    if (L.map_width > 64 || (obj != ORC_CHI2 && obj != ORC_POISSON)) return ORC_EINVAL;
    for (int j = 0; j < L.n_params; ++j)
        if (!isfinite(theta[j])) return ORC_ENONFINITE;
    return objective_impl(&L, data, theta, obj, value);
}

/*
 * Analytic gradient and Gauss-Newton matrix over the full parameter vector.
 * grad: n_params, gn: n_params x n_params row-major (either may be NULL).
 */
static int gradient_impl(const orc_layout* L, const double* data, const double* theta, int obj,
                         double* value, double* grad, double* gn) {
    int P = L->n_params, W = L->map_width, K = L->n_hist;
    int status = ORC_OK;
    size_t per = 1 + (size_t)P + (gn ? (size_t)P * P : 0);
    /* per-histogram compensated accumulators: value, grad[P], gn[P*P] */
    orc_acc* acc = (orc_acc*)calloc((size_t)(K > 0 ? K : 1) * per, sizeof(orc_acc));
    int* hst = (int*)calloc((size_t)(K > 0 ? K : 1), sizeof(int));
    if (!acc || !hst) {
        free(acc);
        free(hst);
        return ORC_ENOMEM;
    }
#pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < K; ++k) {
        orc_acc* a = acc + (size_t)k * per;
        int64_t off = hist_offset(L, k);
        double dcol[64];
        int idx[64];
        for (int c = 0; c < W; ++c) idx[c] = map_index(L, k, c);
        for (int64_t i = 0; i < L->n_bins[k]; ++i) {
            double t = L->t0 + (double)i * L->dt;
            double n = theory_bin(L, theta, k, t, dcol);
            double d = data[off + i];
            double term, wg, wh;
            if (obj == ORC_CHI2) {
                double var = d > 1.0 ? d : 1.0;
                term = (d - n) * (d - n) / var;
                wg = -2.0 * (d - n) / var; /* d term / d N */
                wh = 2.0 / var;
            } else {
                if (deviance_term(d, n, &term)) {
                    hst[k] = ORC_EDOMAIN;
                    break;
                }
                wg = 2.0 * (1.0 - d / n); /* d/dN of 2[(N-d) + d ln(d/N)] */
                wh = 2.0 / n;
            }
            acc_add(&a[0], term);
            /* chain rule through the map: dN/dtheta_j = sum over columns mapped to j */
            for (int c = 0; c < W; ++c) {
                if (idx[c] < 0) continue;
                if (grad) acc_add(&a[1 + idx[c]], wg * dcol[c]);
            }
            if (gn) {
                for (int c1 = 0; c1 < W; ++c1) {
                    if (idx[c1] < 0) continue;
                    for (int c2 = 0; c2 < W; ++c2) {
                        if (idx[c2] < 0) continue;
                        acc_add(&a[1 + P + (size_t)idx[c1] * P + idx[c2]], wh * dcol[c1] * dcol[c2]);
                    }
                }
            }
        }
    }
    orc_acc tot = {0.0, 0.0};
    for (int k = 0; k < K; ++k) {
        if (hst[k]) status = hst[k];
        acc_add(&tot, acc_val(&acc[(size_t)k * per]));
    }
    if (value) *value = status ? INFINITY : acc_val(&tot);
    if (grad) {
        for (int j = 0; j < P; ++j) {
            orc_acc s = {0.0, 0.0};
            for (int k = 0; k < K; ++k) acc_add(&s, acc_val(&acc[(size_t)k * per + 1 + j]));
            grad[j] = acc_val(&s);
        }
    }
    if (gn) {
        for (size_t e = 0; e < (size_t)P * P; ++e) {
            orc_acc s = {0.0, 0.0};
            for (int k = 0; k < K; ++k) acc_add(&s, acc_val(&acc[(size_t)k * per + 1 + P + e]));
            gn[e] = acc_val(&s);
        }
    }
    free(acc);
    free(hst);
    return status;
}

int orc_gradient(LAYOUT_ARGS, const double* data, const double* theta, int obj, double* value,
                 double* grad, double* gn) {
    MAKE_LAYOUT;
    int st = check_layout(&L);
    if (st) return st;
    if (L.map_width > 32 || (obj != ORC_CHI2 && obj != ORC_POISSON)) return ORC_EINVAL;
    for (int j = 0; j < L.n_params; ++j)
        if (!isfinite(theta[j])) return ORC_ENONFINITE;
    return gradient_impl(&L, data, theta, obj, value, grad, gn);
}

/* FP64 central finite differences, h_j = rel_h * max(|theta_j|, 1). */
int orc_gradient_fd(LAYOUT_ARGS, const double* data, const double* theta, int obj, double rel_h,
                    double* grad) {
    MAKE_LAYOUT;
    int st = check_layout(&L);
    if (st) return st;
    if (L.map_width > 64) return ORC_EINVAL;
    double* th = (double*)malloc(sizeof(double) * (size_t)(L.n_params > 0 ? L.n_params : 1));
    if (!th) return ORC_ENOMEM;
    memcpy(th, theta, sizeof(double) * (size_t)L.n_params);
    for (int j = 0; j < L.n_params; ++j) {
        double h = rel_h * (fabs(theta[j]) > 1.0 ? fabs(theta[j]) : 1.0);
        double fp, fm;
        th[j] = theta[j] + h;
        st = objective_impl(&L, data, th, obj, &fp);
        if (st) break;
        th[j] = theta[j] - h;
        st = objective_impl(&L, data, th, obj, &fm);
        if (st) break;
        th[j] = theta[j];
        grad[j] = (fp - fm) / (2.0 * h);
    }
    free(th);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Levenberg-Marquardt fit                                                   */
/* ------------------------------------------------------------------------ */

/* Cholesky solve of the n x n SPD system A x = b (A row-major, overwritten). */
static int cholesky_solve(double* A, double* b, int n) {
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0.0)) return -1;
        double ljj = sqrt(s);
        A[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double v = A[i * n + j];
            for (int k = 0; k < j; ++k) v -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = v / ljj;
        }
    }
    for (int i = 0; i < n; ++i) {
        double v = b[i];
        for (int k = 0; k < i; ++k) v -= A[i * n + k] * b[k];
        b[i] = v / A[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double v = b[i];
        for (int k = i + 1; k < n; ++k) v -= A[k * n + i] * b[k];
        b[i] = v / A[i * n + i];
    }
    return 0;
}

/*
 * stats (out, 8 doubles): [0] objective at the minimum, [1] ndf = bins - free,
 * [2] iterations, [3] objective evaluations, [4] EDM, [5] final damping,
 * [6] status, [7] 0.
 * cov (out, n_free x n_free or NULL): 2 H^-1 over the free parameters.
 */
int orc_fit(LAYOUT_ARGS, const double* data, int obj, double* theta, const uint8_t* free_mask,
            int max_iter, double edm_tol, double* stats, double* cov) {
    MAKE_LAYOUT;
    int st = check_layout(&L);
    if (st) return st;
    int P = L.n_params;
    int nf = 0;
    int fidx[512];
    for (int j = 0; j < P; ++j)
        if (free_mask[j]) {
            if (nf >= 512) return ORC_EINVAL;
            fidx[nf++] = j;
        }
    double* g = (double*)malloc(sizeof(double) * (size_t)P);
    double* H = (double*)malloc(sizeof(double) * (size_t)P * P);
    double* A = (double*)malloc(sizeof(double) * (size_t)nf * nf + 8);
    double* b = (double*)malloc(sizeof(double) * (size_t)nf + 8);
    double* trial = (double*)malloc(sizeof(double) * (size_t)P);
    if (!g || !H || !A || !b || !trial) {
        free(g); free(H); free(A); free(b); free(trial);
        return ORC_ENOMEM;
    }
    double f;
    int evals = 0, it = 0;
    double mu = 1e-3, edm = INFINITY;
    st = gradient_impl(&L, data, theta, obj, &f, g, H);
    ++evals;
    int result = ORC_ENOCONV;
    if (st) result = st;
    while (!st && it < max_iter) {
        ++it;
        /* EDM = 1/2 g^T H^-1 g over the free block */
        for (int a = 0; a < nf; ++a) {
            b[a] = -g[fidx[a]];
            for (int c = 0; c < nf; ++c) A[a * nf + c] = H[fidx[a] * P + fidx[c]];
        }
        if (cholesky_solve(A, b, nf) == 0) {
            double e = 0.0;
            for (int a = 0; a < nf; ++a) e -= 0.5 * g[fidx[a]] * b[a];
            edm = e;
            if (edm < edm_tol) {
                result = ORC_OK;
                break;
            }
        }
        /* damped step */
        for (int a = 0; a < nf; ++a) {
            b[a] = -g[fidx[a]];
            for (int c = 0; c < nf; ++c) A[a * nf + c] = H[fidx[a] * P + fidx[c]];
            A[a * nf + a] *= (1.0 + mu);
        }
        if (cholesky_solve(A, b, nf) != 0) {
            mu *= 10.0;
            if (mu > 1e20) break;
            continue;
        }
        memcpy(trial, theta, sizeof(double) * (size_t)P);
        for (int a = 0; a < nf; ++a) trial[fidx[a]] += b[a];
        double ft;
        int s2 = objective_impl(&L, data, trial, obj, &ft);
        ++evals;
        if (s2 == ORC_OK && ft < f) {
            double rel = (f - ft) / (fabs(f) > 1e-300 ? fabs(f) : 1e-300);
            memcpy(theta, trial, sizeof(double) * (size_t)P);
            st = gradient_impl(&L, data, theta, obj, &f, g, H);
            ++evals;
            mu = mu * 0.1 > 1e-12 ? mu * 0.1 : 1e-12;
            if (rel < 1e-15) {
                result = ORC_OK;
                break;
            }
        } else {
            mu *= 10.0;
            if (mu > 1e20) break;
        }
    }
    if (st) result = st;
    int64_t nb = total_bins(&L);
    stats[0] = f;
    stats[1] = (double)(nb - nf);
    stats[2] = it;
    stats[3] = evals;
    stats[4] = edm;
    stats[5] = mu;
    stats[6] = result;
    stats[7] = 0.0;
    if (cov && !st) {
        /* 2 H^-1 column by column */
        for (int c = 0; c < nf; ++c) {
            for (int a = 0; a < nf; ++a) {
                for (int e = 0; e < nf; ++e) A[a * nf + e] = H[fidx[a] * P + fidx[e]];
                b[a] = (a == c) ? 2.0 : 0.0;
            }
            if (cholesky_solve(A, b, nf) != 0) {
                for (int a = 0; a < nf; ++a) cov[a * nf + c] = NAN;
            } else {
                for (int a = 0; a < nf; ++a) cov[a * nf + c] = b[a];
            }
        }
    }
    free(g); free(H); free(A); free(b); free(trial);
    return result;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Thread count of the following parallel regions (n <= 0: leave unchanged). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ======================================================================== */
/* Synthetic-data generator: Philox4x32-10 and a Poisson sampler             */
/* ======================================================================== */
/*
 * Random numbers come from the counter-based generator Philox4x32-10
 * (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC 2011): ten rounds of two 32x32->64 multiplications with the round
 * multipliers 0xD2511F53 / 0xCD9E8D57, the key bumped by the Weyl constants
 * 0x9E3779B9 / 0xBB67AE85 between rounds.
 *
 * Poisson variates: inversion by sequential search for mean < 12, and the
 * transformed-rejection sampler PTRS of Hormann (1993, "The transformed
 * rejection method for generating Poisson random variables") above.  The
 * acceptance test of PTRS compares log(V * alpha^-1 / (a / us^2 + b)) with the
 * log-probability log p(k; mu); for k >= 10 the latter is written with
 * Stirling's series in the cancellation-free form
 *     log p = -mu h(y) + 1/2 log1p(y) - 1/2 log(2 pi mu) - 1/(12 n) + 1/(360 n^3),
 *     n = k + 1, y = (n - mu) / mu, h(y) = (1 + y) log1p(y) - y,
 * so that it can be evaluated in FP32 at any mean.
 *
 * The sampler's floating-point decisions are taken in FP32, in the operation
 * order of the GPU sampler, with logarithm and exponential built from IEEE
 * basic operations (below), so both produce the same integers.  This file is
 * compiled with -ffp-contract=off; fused multiply-adds appear only as fmaf().
 */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

/* uniform in (0, 1): ((r >> 9) + 1/2) * 2^-23, exact in FP32, never 0 or 1 */
static float u01(uint32_t r) { return ((float)(r >> 9) + 0.5f) * 1.1920928955078125e-07f; }

static float f_from_bits(uint32_t b) {
    float f;
    memcpy(&f, &b, 4);
    return f;
}
static uint32_t bits_from_f(float f) {
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
}

/* natural log of a positive normal float: x = m 2^e, m in [sqrt(1/2), sqrt(2)),
 * log m = 2 atanh(s), s = (m - 1)/(m + 1), series to s^9 */
static float s_log(float x) {
    const uint32_t b = bits_from_f(x);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float m = f_from_bits((b & 0x7fffffu) | 0x3f800000u);
    if (m > 1.41421356f) {
        m = m * 0.5f;
        e = e + 1;
    }
    const float s = (m - 1.0f) / (m + 1.0f);
    const float s2 = s * s;
    float p = fmaf(s2, 0.111111111f, 0.142857143f);
    p = fmaf(s2, p, 0.2f);
    p = fmaf(s2, p, 0.333333333f);
    p = p * s2;
    const float two_s = s + s;
    const float lm = fmaf(two_s, p, two_s);
    const float fe = (float)e;
    return fmaf(fe, 0.693145752f, fmaf(fe, 1.42860677e-06f, lm));
}

/* exp(x) for x in [-88, 0]: 2^(x log2 e) = 2^n 2^f, 2^f = e^(f ln 2) by a
 * 10-term Taylor polynomial, 2^n applied to the exponent bits */
static float s_exp(float x) {
    const float y = x * 1.44269504f;
    const float n = floorf(y);
    const float t = (y - n) * 0.693147181f;
    float p = fmaf(t, 0.1f, 1.0f);
    p = fmaf(t * 0.111111111f, p, 1.0f);
    p = fmaf(t * 0.125f, p, 1.0f);
    p = fmaf(t * 0.142857143f, p, 1.0f);
    p = fmaf(t * 0.166666667f, p, 1.0f);
    p = fmaf(t * 0.2f, p, 1.0f);
    p = fmaf(t * 0.25f, p, 1.0f);
    p = fmaf(t * 0.333333333f, p, 1.0f);
    p = fmaf(t * 0.5f, p, 1.0f);
    p = fmaf(t, p, 1.0f);
    const int ni = (int)n;
    if (ni < -126) return 0.0f;
    return f_from_bits(bits_from_f(p) + (uint32_t)(ni * (1 << 23)));
}

/* (1 + y) log1p(y) - y */
static float s_h(float y) {
    if (fabsf(y) < 0.125f) {
        float h = fmaf(y, -1.0f / 72.0f, 1.0f / 56.0f);
        h = fmaf(y, h, -1.0f / 42.0f);
        h = fmaf(y, h, 1.0f / 30.0f);
        h = fmaf(y, h, -1.0f / 20.0f);
        h = fmaf(y, h, 1.0f / 12.0f);
        h = fmaf(y, h, -1.0f / 6.0f);
        h = fmaf(y, h, 0.5f);
        return h * y * y;
    }
    const float u = s_log(1.0f + y);
    return fmaf(y, u, u - y);
}

/* log p(k; mu) for k >= 0, mu >= 12 */
static float s_log_pmf(int k, float mu, float log_mu) {
    if (k < 10) {
        float lf = 0.0f;
        for (int i = 2; i <= k; ++i) lf = lf + s_log((float)i);
        return fmaf((float)k, log_mu, -mu) - lf;
    }
    const float n = (float)(k + 1);
    const float y = (n - mu) / mu;
    const float l1p = s_log(1.0f + y);
    const float rn = 1.0f / n;
    float v = -(mu * s_h(y));
    v = fmaf(0.5f, l1p, v);
    v = v - 0.5f * s_log(6.28318531f * mu);
    v = v - rn * 0.0833333333f;
    v = fmaf(rn * rn * rn, 0.00277777778f, v);
    return v;
}

/* Poisson variate for mean mu; ctr[1..3] identify the draw, ctr[0] counts
 * the Philox blocks it consumes. */
int32_t orc_poisson_one(float mu, const uint32_t key[2], uint32_t c1, uint32_t c2, uint32_t c3) {
    if (!(mu > 0.0f)) return 0;
    uint32_t ctr[4] = {0u, c1, c2, c3}, r[4];
    if (mu < 12.0f) {
        orc_philox4x32_10(ctr, key, r);
        const float u = u01(r[0]);
        float p = s_exp(-mu);
        float F = p;
        int32_t k = 0;
        while (u > F && k < 1000) {
            k = k + 1;
            p = (p * mu) / (float)k;
            F = F + p;
        }
        return k;
    }
    const float slam = sqrtf(mu);
    const float log_mu = s_log(mu);
    const float b = fmaf(2.53f, slam, 0.931f);
    const float a = fmaf(0.02483f, b, -0.059f);
    const float inv_alpha = 1.1239f + 1.1328f / (b - 3.4f);
    const float vr = 0.9277f - 3.6224f / (b - 2.0f);
    for (uint32_t it = 0; it < 64u; ++it) {
        ctr[0] = it;
        orc_philox4x32_10(ctr, key, r);
        const float U = u01(r[0]) - 0.5f;
        const float V = u01(r[1]);
        const float us = 0.5f - fabsf(U);
        const float kf = floorf(fmaf((a + a) / us + b, U, mu + 0.43f));
        if (us >= 0.07f && V <= vr) return (int32_t)kf;
        if (kf < 0.0f || (us < 0.013f && V > us)) continue;
        const float lhs = s_log((V * inv_alpha) / (a / (us * us) + b));
        if (lhs <= s_log_pmf((int)kf, mu, log_mu)) return (int32_t)kf;
    }
    return (int32_t)floorf(mu + 0.5f);
}

/* counts[i] for means mu[i]: draw i uses counter words (i lo, i hi, 0xffffffff) */
void orc_poisson(const float* mu, int64_t n, uint64_t seed, int32_t* counts) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        counts[i] = orc_poisson_one(mu[i], key, (uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0xffffffffu);
}

/* Rebinned means of the Eq. 1 theory: for each parameter vector s, histogram
 * k and group j, the sum of N over bins [j rebin, min((j+1) rebin, M_k)).
 * out: n_samples x sum_k ceil(M_k / rebin), FP64. */
int orc_rebinned_mean(LAYOUT_ARGS, const double* thetas, int n_samples, int rebin, double* out) {
    MAKE_LAYOUT;
    int st = check_layout(&L);
    if (st) return st;
    if (rebin < 1 || L.map_width > 64) return ORC_EINVAL;
    int64_t per = 0;
    for (int k = 0; k < L.n_hist; ++k) per += (L.n_bins[k] + rebin - 1) / rebin;
#pragma omp parallel for schedule(dynamic)
    for (int s = 0; s < n_samples; ++s) {
        const double* th = thetas + (int64_t)s * L.n_params;
        int64_t o = (int64_t)s * per;
        for (int k = 0; k < L.n_hist; ++k) {
            const int64_t M = L.n_bins[k];
            for (int64_t j0 = 0; j0 < M; j0 += rebin) {
                orc_acc a = {0.0, 0.0};
                for (int64_t i = j0; i < j0 + rebin && i < M; ++i)
                    acc_add(&a, theory_bin(&L, th, k, L.t0 + (double)i * L.dt, NULL));
                out[o++] = acc_val(&a);
            }
        }
    }
    return ORC_OK;
}

/* Training parameter vectors of the learned start proposer: entries with
 * hi > lo (ranked q = 0, 1, ... in index order) drawn as lo + (hi - lo) u,
 * u = ((w_a >> 5) 2^26 + (w_b >> 6) + 1/2) 2^-53 from the Philox4x32-10
 * block of counter (index low, index high, q / 2, 0xfffffffe) under key
 * (seed low ^ 0x0A5F00D1, seed high), words (0, 1) for even q and (2, 3) for
 * odd q; other entries lo.  targets (or NULL) = 2u - 1 as float. */
void orc_sample_thetas(const double* lo, const double* hi, int P, int64_t n, uint64_t seed, uint64_t offset,
                       double* thetas, float* targets) {
    int n_learned = 0;
    for (int j = 0; j < P; ++j) n_learned += hi[j] > lo[j];
    for (int64_t s = 0; s < n; ++s) {
        const uint64_t id = offset + (uint64_t)s;
        double* th = thetas + s * P;
        int q = 0;
        for (int j = 0; j < P; ++j) {
            th[j] = lo[j];
            if (!(hi[j] > lo[j])) continue;
            const uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), (uint32_t)(q / 2), 0xfffffffeu};
            const uint32_t key[2] = {(uint32_t)seed ^ 0x0A5F00D1u, (uint32_t)(seed >> 32)};
            uint32_t w[4];
            orc_philox4x32_10(ctr, key, w);
            const uint32_t wa = w[2 * (q % 2)], wb = w[2 * (q % 2) + 1];
            const double u = ((double)(wa >> 5) * 67108864.0 + (double)(wb >> 6) + 0.5) * (1.0 / 9007199254740992.0);
            th[j] = lo[j] + (hi[j] - lo[j]) * u;
            if (targets) targets[s * n_learned + q] = (float)(2.0 * u - 1.0);
            ++q;
        }
    }
}
