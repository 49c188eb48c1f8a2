// Host minimiser driving the GPU objective (the role Minuit2 plays in the
// paper, Sec. 4.1): Levenberg-Marquardt on the Gauss-Newton matrix that the
// adjoint kernel returns, or BFGS on the adjoint (or central-difference)
// gradient.  All linear algebra is FP64 on the host; each iteration costs one
// kernel launch (value + gradient + GN at the trial point) and one small copy
// back.
#include <math.h>
#include <string.h>

#include <cmath>

#include <algorithm>
#include <functional>
#include <vector>

#include "musr.h"
#include "musr_internal.h"
#include "run_impl.h"

namespace musr {
int gbatch_eval_host(musr_gbatch b, int obj, int mode, const double* thetas, const uint8_t* active, double* out,
                     int32_t* flags);
const double* gbatch_host_out(musr_gbatch b);
int64_t gbatch_out_offset(musr_gbatch b, int mode, int r);
int64_t gbatch_theta_offset(musr_gbatch b, int r);
int gbatch_has_gn(musr_gbatch b);
int gbatch_n_runs(musr_gbatch b);
musr_run gbatch_run(musr_gbatch b, int r);
// Central-difference gradient (and, if hdiag != NULL, the diagonal second
// differences) of the objective over the free entries, one batched launch.
// Central differences of the objective along every free parameter fidx[a]
// with absolute steps h_abs[a] (order 2: +-h; order 4: +-h, +-2h), in one
// batched launch (batch.cu); hdiag (or NULL) receives the second differences.
int batch_fd_gradient(musr_run run, int obj, const double* theta, const std::vector<int>& fidx, double* h_abs,
                      int order, double* value, double* grad, double* hdiag);
}

using namespace musr;

namespace {

// Dot product of x[0..m) and y[0..m) with four independent partial sums (the
// multiply-add chains of a plain loop would wait on one another).
inline double dot4(const double* x, const double* y, int m) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int k = 0;
    for (; k + 4 <= m; k += 4) {
        s0 += x[k] * y[k];
        s1 += x[k + 1] * y[k + 1];
        s2 += x[k + 2] * y[k + 2];
        s3 += x[k + 3] * y[k + 3];
    }
    for (; k < m; ++k) s0 += x[k] * y[k];
    return (s0 + s1) + (s2 + s3);
}

// Cholesky factor A = L L^T of an n x n SPD matrix in place (row-major; L in
// the lower triangle, the strict upper triangle is left as it was); false if A
// is not positive definite.  Right-looking: once column j is scaled, every
// later row is updated by a contiguous multiply-add over its lower part (no
// reduction chains, so the loops vectorise).
bool cholesky_factor(std::vector<double>& A, int n) {
    std::vector<double> c(n);
    for (int j = 0; j < n; ++j) {
        double* Aj = A.data() + (size_t)j * n;
        const double s = Aj[j];
        if (!(s > 0.0)) return false;
        const double l = sqrt(s), il = 1.0 / l;
        Aj[j] = l;
        for (int k = j + 1; k < n; ++k) c[k] = (A[(size_t)k * n + j] *= il);
        for (int i = j + 1; i < n; ++i) {
            double* Ai = A.data() + (size_t)i * n;
            const double f = c[i];
            for (int k = j + 1; k <= i; ++k) Ai[k] -= f * c[k];
        }
    }
    return true;
}

// Solve L L^T x = b with the factor of cholesky_factor (b overwritten):
// forward by row dot products, backward by column updates.
void cholesky_back(const std::vector<double>& A, std::vector<double>& b, int n) {
    for (int i = 0; i < n; ++i) b[i] = (b[i] - dot4(A.data() + (size_t)i * n, b.data(), i)) / A[(size_t)i * n + i];
    for (int i = n - 1; i >= 0; --i) {
        const double xi = (b[i] /= A[(size_t)i * n + i]);
        const double* Ai = A.data() + (size_t)i * n;
        for (int k = 0; k < i; ++k) b[k] -= Ai[k] * xi;
    }
}

// Solve L L^T X = B for the n x m right-hand sides B (row-major, n rows of m)
// with the factor of cholesky_factor: every step updates whole rows of B.
void cholesky_back_rows(const std::vector<double>& A, std::vector<double>& B, int n, int m) {
    for (int i = 0; i < n; ++i) {
        double* Bi = B.data() + (size_t)i * m;
        const double* Ai = A.data() + (size_t)i * n;
        for (int k = 0; k < i; ++k) {
            const double f = Ai[k];
            const double* Bk = B.data() + (size_t)k * m;
            for (int c = 0; c < m; ++c) Bi[c] -= f * Bk[c];
        }
        const double il = 1.0 / Ai[i];
        for (int c = 0; c < m; ++c) Bi[c] *= il;
    }
    for (int i = n - 1; i >= 0; --i) {
        double* Bi = B.data() + (size_t)i * m;
        const double il = 1.0 / A[(size_t)i * n + i];
        for (int c = 0; c < m; ++c) Bi[c] *= il;
        const double* Ai = A.data() + (size_t)i * n;
        for (int k = 0; k < i; ++k) {
            const double f = Ai[k];
            double* Bk = B.data() + (size_t)k * m;
            for (int c = 0; c < m; ++c) Bk[c] -= f * Bi[c];
        }
    }
}

// Cholesky solve of the n x n SPD system A x = b (A overwritten).
bool cholesky_solve(std::vector<double>& A, std::vector<double>& b, int n) {
    if (!cholesky_factor(A, n)) return false;
    cholesky_back(A, b, n);
    return true;
}

struct Evaluator {
    musr_run run;
    int obj;
    int P;
    std::vector<double> buf;
    int evals = 0;
    // value (+grad, +GN) at theta; returns MUSR_OK, MUSR_EDOMAIN (value = inf) or an error
    int operator()(const double* theta, int mode, double* value, double* grad, double* gn) {
        buf.resize((size_t)run->n_out[mode] + 1);
        int32_t flags = 0;
        ++evals;
        // results read straight from the run's pinned buffer where it holds them
        // (no function array): one copy of the P x P matrix, not two
        const double* o = buf.data();
        int st = run->eval_host(obj, mode, theta, buf.data(), &flags, &o);
        if (st != MUSR_OK) return st;
        *value = (flags & 1) ? INFINITY : o[0];
        if (grad && mode >= kGrad) memcpy(grad, o + 1, sizeof(double) * P);
        if (gn && mode == kGN) memcpy(gn, o + 1 + P, sizeof(double) * P * P);
        if (flags & 1) return MUSR_EDOMAIN;
        return isfinite(*value) ? MUSR_OK : MUSR_ENONFINITE;
    }
};

// EDM = 1/2 g^T H^-1 g over the free block (inf if H is not positive definite).
double edm_of(const std::vector<double>& g, const std::vector<double>& H, const std::vector<int>& fidx,
              int P, std::vector<double>& A, std::vector<double>& b) {
    const int nf = (int)fidx.size();
    for (int a = 0; a < nf; ++a) {
        b[a] = -g[fidx[a]];
        for (int c = 0; c < nf; ++c) A[(size_t)a * nf + c] = H[(size_t)fidx[a] * P + fidx[c]];
    }
    if (!cholesky_solve(A, b, nf)) return INFINITY;
    double e = 0.0;
    for (int a = 0; a < nf; ++a) e -= 0.5 * g[fidx[a]] * b[a];
    return e;
}

// Relative resolution of objective values computed with FP32 evaluation and
// FP64 accumulation: below it, value comparisons are decided by rounding.
constexpr double kValueNoise = 1e-6;

// The adjoint gradient of an FP32 evaluation resolves the EDM only down to a
// floor that grows with the number of bins (~2e-8 at 4e6 bins).  When a step
// below the value resolution no longer lowers the EDM and the EDM is within
// this factor of the tolerance (distance to the minimum ~3e-4 of the
// parameter errors for the default 1e-8), the fit has converged as far as
// the arithmetic allows.
constexpr double kEdmResolution = 10.0;

// Central-difference fits with automatic steps: fourth-order differences
// with a step of kFdStepSigma standard errors along each free parameter (from
// second differences at the start).  The FP32 value noise enters the gradient
// divided by the step (a parameter's distance to the minimum is ~ noise /
// (2 kFdStepSigma) of its error, noise = the value's rounding noise), so the
// step must be of the parameter's own scale or larger; at that scale
// second-order differences would carry a truncation error of ~1e-3 of the
// errors on correlated, curved directions, fourth-order ones ~(h / L)^4 with
// the curvature length L ~ 30 errors.  They stop after kFdStallSteps
// successive accepted steps that each move every free parameter by less
// than kFdStallSigma of its standard error.
constexpr double kFdStepSigma = 2.0;
constexpr double kFdStallSigma = 1e-4;
constexpr int kFdStallSteps = 3;

}  // namespace

// One run's Levenberg-Marquardt iteration as a state machine, so that a single
// fit (musr_fit) and many fits in lockstep (musr_fit_batch) share one
// definition: next() proposes a trial point (or reports the fit finished),
// observe() takes the objective, gradient and GN matrix at that point.
struct LmStepper {
    int P = 0, nf = 0;
    std::vector<int> fidx;
    musr_fit_opts o{};
    std::vector<double> theta, g, H, gt, Ht, trial, A, b;
    double f = 0.0, mu = 0.0, edm = INFINITY, pred = 0.0;
    int it = 0, result = MUSR_ENOCONV;
    bool done = false;

    void init(int P_, const std::vector<int>& fidx_, const musr_fit_opts& o_, const double* th) {
        P = P_;
        fidx = fidx_;
        nf = (int)fidx.size();
        o = o_;
        theta.assign(th, th + P);
        g.assign(P, 0.0);
        gt.assign(P, 0.0);
        trial.assign(P, 0.0);
        H.assign((size_t)P * P, 0.0);
        Ht.assign((size_t)P * P, 0.0);
        A.assign((size_t)nf * nf, 0.0);
        b.assign(nf, 0.0);
        mu = o.mu0;
    }
    // the evaluation at the start point (g and H filled by the caller)
    void start(double f0) {
        f = f0;
        edm = edm_of(g, H, fidx, P, A, b);
    }
    // true: evaluate at `trial` (into gt / Ht) and call observe(); false: finished
    bool next() {
        while (!done) {
            if (it >= o.max_iter) {
                done = true;
                break;
            }
            ++it;
            if (edm < o.edm_tol) {
                result = MUSR_OK;
                done = true;
                break;
            }
            for (int a = 0; a < nf; ++a) {
                b[a] = -g[fidx[a]];
                for (int c = 0; c < nf; ++c) A[(size_t)a * nf + c] = H[(size_t)fidx[a] * P + fidx[c]];
                A[(size_t)a * nf + a] *= (1.0 + mu);
            }
            if (!cholesky_solve(A, b, nf)) {
                mu *= 10.0;
                if (mu > 1e20) done = true;
                continue;
            }
            // predicted decrease of the quadratic model
            pred = 0.0;
            for (int a = 0; a < nf; ++a) {
                double hb = 0.0;
                for (int c = 0; c < nf; ++c) hb += H[(size_t)fidx[a] * P + fidx[c]] * b[c];
                pred -= g[fidx[a]] * b[a] + 0.5 * b[a] * hb;
            }
            memcpy(trial.data(), theta.data(), sizeof(double) * P);
            for (int a = 0; a < nf; ++a) trial[fidx[a]] += b[a];
            return true;
        }
        return false;
    }
    // s2: MUSR_OK, MUSR_EDOMAIN or MUSR_ENONFINITE (other errors end the fit upstream)
    void observe(int s2, double ft) {
        bool accept = false, at_resolution = false;
        double edm_t = INFINITY;
        if (s2 == MUSR_OK) {
            const double noise = kValueNoise * fabs(f);
            if (ft < f) {
                accept = true;
            } else if (pred < noise && ft - f < noise) {
                // the change is below the value resolution: let the gradient decide
                edm_t = edm_of(gt, Ht, fidx, P, A, b);
                accept = edm_t < edm;
                at_resolution = !accept && edm < kEdmResolution * o.edm_tol;
            }
        }
        if (at_resolution) {
            result = MUSR_OK;
            done = true;
            return;
        }
        if (accept) {
            const double rel = (f - ft) / std::max(fabs(f), 1e-300);
            theta.swap(trial);
            f = ft;
            g.swap(gt);
            H.swap(Ht);
            edm = std::isfinite(edm_t) ? edm_t : edm_of(g, H, fidx, P, A, b);
            mu = std::max(mu * 0.1, 1e-12);
            if (rel >= 0.0 && rel < 1e-15 && edm < 1e3 * o.edm_tol) {
                result = MUSR_OK;
                done = true;
            }
        } else {
            mu *= 10.0;
            if (mu > 1e20) done = true;
        }
    }
    void finish(double* theta_out, musr_fit_result* out) {
        memcpy(theta_out, theta.data(), sizeof(double) * P);
        out->value = f;
        out->edm = edm;
        out->mu = mu;
        out->iters = it;
        if (out->cov) {
            // covariance 2 H^-1 over the free block: one factorisation, the nf
            // right-hand sides of 2 I solved together
            for (int a = 0; a < nf; ++a)
                for (int e = 0; e < nf; ++e) A[(size_t)a * nf + e] = H[(size_t)fidx[a] * P + fidx[e]];
            const bool ok = cholesky_factor(A, nf);
            std::vector<double> X((size_t)nf * nf, 0.0);
            for (int a = 0; a < nf; ++a) X[(size_t)a * nf + a] = 2.0;
            if (ok) cholesky_back_rows(A, X, nf, nf);
            for (size_t q = 0; q < X.size(); ++q) out->cov[q] = ok ? X[q] : NAN;
        }
    }
};

namespace {

int fit_lm(Evaluator& ev, double* theta, const std::vector<int>& fidx, const musr_fit_opts& o,
           musr_fit_result* out) {
    LmStepper lm;
    lm.init(ev.P, fidx, o, theta);
    double f;
    int st = ev(theta, kGN, &f, lm.g.data(), lm.H.data());
    if (st != MUSR_OK) return st;
    lm.start(f);
    while (lm.next()) {
        double ft;
        const int s2 = ev(lm.trial.data(), kGN, &ft, lm.gt.data(), lm.Ht.data());
        if (s2 != MUSR_OK && s2 != MUSR_EDOMAIN && s2 != MUSR_ENONFINITE) return s2;
        lm.observe(s2, ft);
    }
    lm.finish(theta, out);
    return lm.result;
}

}  // namespace

// One run's BFGS iteration as a state machine (like LmStepper), shared by a
// single fit and many fits in lockstep: next() proposes the point at which the
// value and gradient are needed next (a line-search trial), observe() takes
// them.  The inverse-Hessian estimate starts from the diagonal preconditioner
// 1 / H_jj when the start supplies the Hessian diagonal (the parameters'
// scales differ by 1e5).  fd: the gradient is a central difference, whose
// value noise rules out the EDM test (see observe()).
struct BfgsStepper {
    int P = 0, nf = 0;
    std::vector<int> fidx;
    musr_fit_opts o{};
    bool fd = false;
    std::vector<double> theta, g, gt, x, Hi, d, hi0, inv_sig;
    double f = 0.0, edm = INFINITY, slope = 0.0, step = 1.0;
    int it = 0, result = MUSR_ENOCONV, stall = 0, ls = 0;
    bool done = false, in_ls = false;

    void init(int P_, const std::vector<int>& fidx_, const musr_fit_opts& o_, const double* th, bool fd_) {
        P = P_;
        fidx = fidx_;
        nf = (int)fidx.size();
        o = o_;
        fd = fd_;
        theta.assign(th, th + P);
        g.assign(P, 0.0);
        gt.assign(P, 0.0);
        x.assign(P, 0.0);
        Hi.assign((size_t)nf * nf, 0.0);
        d.assign(nf, 0.0);
        hi0.assign(nf, 0.0);
        inv_sig.assign(nf, 0.0);
    }
    // after the start evaluation (value f0, gradient in g); hd: Hessian diagonal or null
    void start(double f0, const double* hd) {
        f = f0;
        double gnorm = 0.0;
        for (int a = 0; a < nf; ++a) gnorm += g[fidx[a]] * g[fidx[a]];
        gnorm = sqrt(gnorm);
        for (int a = 0; a < nf; ++a) {
            const double h = hd ? hd[fidx[a]] : 0.0;
            hi0[a] = (h > 0.0 && std::isfinite(h)) ? 1.0 / h : 1.0 / std::max(gnorm, 1.0);
            Hi[(size_t)a * nf + a] = hi0[a];
            inv_sig[a] = 1.0 / sqrt(2.0 * hi0[a]);  // standard error sqrt(2 / H_jj)
        }
    }
    void set_trial() {
        memcpy(x.data(), theta.data(), sizeof(double) * P);
        for (int a = 0; a < nf; ++a) x[fidx[a]] += step * d[a];
    }
    // true: evaluate value and gradient at x (into gt) and call observe()
    bool next() {
        while (!done) {
            if (in_ls) return true;
            if (it >= o.max_iter) {
                done = true;
                break;
            }
            ++it;
            for (int a = 0; a < nf; ++a) {
                double v = 0.0;
                for (int c = 0; c < nf; ++c) v -= Hi[(size_t)a * nf + c] * g[fidx[c]];
                d[a] = v;
            }
            slope = 0.0;
            for (int a = 0; a < nf; ++a) slope += g[fidx[a]] * d[a];
            edm = -0.5 * slope;
            if (edm < o.edm_tol) {
                result = MUSR_OK;
                done = true;
                break;
            }
            if (slope >= 0.0) {  // not a descent direction: reset to the preconditioner
                for (int a = 0; a < nf; ++a)
                    for (int c = 0; c < nf; ++c) Hi[(size_t)a * nf + c] = a == c ? hi0[a] : 0.0;
                continue;
            }
            step = 1.0;
            ls = 0;
            set_trial();
            in_ls = true;
            return true;
        }
        return false;
    }
    // st: MUSR_OK, MUSR_EDOMAIN or MUSR_ENONFINITE (other errors end the fit upstream)
    void observe(int st, double fn) {
        bool ok = st == MUSR_OK && fn <= f + 1e-4 * step * slope;
        if (!ok && st == MUSR_OK && -step * slope < kValueNoise * fabs(f) && fn - f < kValueNoise * fabs(f)) {
            // below the value resolution: accept if the gradient shrinks in the Hi metric
            double e_new = 0.0;
            for (int a = 0; a < nf; ++a) {
                double v = 0.0;
                for (int c = 0; c < nf; ++c) v += Hi[(size_t)a * nf + c] * gt[fidx[c]];
                e_new += 0.5 * gt[fidx[a]] * v;
            }
            ok = e_new < edm;
        }
        if (!ok) {
            step *= 0.5;
            if (++ls >= 40) {  // no acceptable step along d
                // a central-difference fit whose last steps were already below
                // its stall size has reached the resolution of its gradient
                if (fd && stall > 0) result = MUSR_OK;
                done = true;
                in_ls = false;
                return;
            }
            set_trial();
            return;
        }
        in_ls = false;
        const double rel = (f - fn) / std::max(fabs(f), 1e-300);
        std::vector<double> sv(nf), yv(nf);
        double sy = 0.0;
        for (int a = 0; a < nf; ++a) {
            sv[a] = step * d[a];
            yv[a] = gt[fidx[a]] - g[fidx[a]];
            sy += sv[a] * yv[a];
        }
        theta.swap(x);
        f = fn;
        g.swap(gt);
        if (sy > 1e-300) {
            // Hi <- (I - rho s y^T) Hi (I - rho y s^T) + rho s s^T
            const double rho = 1.0 / sy;
            std::vector<double> Hy(nf, 0.0);
            for (int a = 0; a < nf; ++a)
                for (int c = 0; c < nf; ++c) Hy[a] += Hi[(size_t)a * nf + c] * yv[c];
            double yHy = 0.0;
            for (int a = 0; a < nf; ++a) yHy += yv[a] * Hy[a];
            for (int a = 0; a < nf; ++a)
                for (int c = 0; c < nf; ++c)
                    Hi[(size_t)a * nf + c] += (1.0 + rho * yHy) * rho * sv[a] * sv[c] -
                                              rho * (Hy[a] * sv[c] + sv[a] * Hy[c]);
        }
        if (rel >= 0.0 && rel < 1e-15 && it > 1) {
            result = MUSR_OK;
            done = true;
            return;
        }
        // central differences carry the FP32 value noise into the gradient, so
        // the EDM test cannot pass; that fit stops once kFdStallSteps
        // successive steps each moved every parameter by less than
        // kFdStallSigma of its standard error
        if (fd) {
            double smax = 0.0;
            for (int a = 0; a < nf; ++a) smax = std::max(smax, fabs(sv[a]) * inv_sig[a]);
            stall = smax < kFdStallSigma ? stall + 1 : 0;
            if (stall >= kFdStallSteps) {
                result = MUSR_OK;
                done = true;
            }
        }
    }
    void finish(double* theta_out, musr_fit_result* out) const {
        memcpy(theta_out, theta.data(), sizeof(double) * P);
        out->value = f;
        out->edm = edm;
        out->mu = 0.0;
        out->iters = it;
        if (out->cov)
            for (size_t e = 0; e < (size_t)nf * nf; ++e) out->cov[e] = 2.0 * Hi[e];
    }
};

// BFGS over the free entries for any objective: value_grad(theta, f, g) gives
// the value and gradient, start(theta, f, g, hd) also the Hessian diagonal hd
// (zero where unknown).
int fit_bfgs_generic(int P, double* theta, const std::vector<int>& fidx, const musr_fit_opts& o, bool fd,
                     const std::function<int(const double*, double*, double*)>& value_grad,
                     const std::function<int(const double*, double*, double*, double*)>& start,
                     musr_fit_result* out) {
    BfgsStepper b;
    b.init(P, fidx, o, theta, fd);
    std::vector<double> hd(P, 0.0);
    double f;
    int st = start(theta, &f, b.g.data(), hd.data());
    if (st != MUSR_OK) return st;
    b.start(f, hd.data());
    while (b.next()) {
        double fn;
        st = value_grad(b.x.data(), &fn, b.gt.data());
        if (st != MUSR_OK && st != MUSR_EDOMAIN && st != MUSR_ENONFINITE) return st;
        b.observe(st, fn);
    }
    b.finish(theta, out);
    return b.result;
}

namespace {

// fd: 0 adjoint gradient; 1 second-order central differences with relative
// steps rel_h; 2 fourth-order central differences with steps of kFdStepSigma
// standard errors, found by two passes of second differences at the start
// (the first with relative steps rel_h, the second with steps from the
// first's curvature)
int fit_bfgs(Evaluator& ev, double* theta, const std::vector<int>& fidx, const musr_fit_opts& o, int fd,
             double rel_h, musr_fit_result* out) {
    const int P = ev.P;
    const int nf = (int)fidx.size();
    std::vector<double> h(nf);
    for (int a = 0; a < nf; ++a) h[a] = rel_h * fmax(fabs(theta[fidx[a]]), 1.0);
    auto value_grad = [&](const double* th, double* f, double* gr) -> int {
        if (fd) {
            ++ev.evals;
            return batch_fd_gradient(ev.run, ev.obj, th, fidx, h.data(), fd == 2 ? 4 : 2, f, gr, nullptr);
        }
        return ev(th, kGrad, f, gr, nullptr);
    };
    // start: the Hessian diagonal from the adjoint kernel's Gauss-Newton matrix,
    // or from the second differences of the same central-difference launch
    auto start = [&](const double* th, double* f, double* gr, double* hd) -> int {
        if (fd) {
            ++ev.evals;
            int st = batch_fd_gradient(ev.run, ev.obj, th, fidx, h.data(), 2, f, gr, hd);
            for (int pass = 0; fd == 2 && pass < 2 && st == MUSR_OK; ++pass) {
                for (int a = 0; a < nf; ++a) {
                    const double c = hd[fidx[a]];
                    if (c > 0.0 && std::isfinite(c)) h[a] = kFdStepSigma * sqrt(2.0 / c);
                }
                if (pass == 1) break;  // the second pass's curvature sets the steps
                ++ev.evals;
                st = batch_fd_gradient(ev.run, ev.obj, th, fidx, h.data(), 4, f, gr, hd);
            }
            return st;
        }
        if (ev.run->Pk <= musr::kMaxGnParams) {
            std::vector<double> H((size_t)P * P);
            const int st = ev(th, kGN, f, gr, H.data());
            for (int j = 0; j < P; ++j) hd[j] = H[(size_t)j * P + j];
            return st;
        }
        return value_grad(th, f, gr);
    };
    return fit_bfgs_generic(P, theta, fidx, o, fd != 0, value_grad, start, out);
}

}  // namespace

extern "C" int musr_fit(musr_run run, int obj, double* theta, const uint8_t* free_mask,
                        const musr_fit_opts* opts, musr_fit_result* out) {
    if (!run || !theta || !out) return MUSR_EINVAL;
    if (obj != MUSR_CHI2 && obj != MUSR_POISSON) return MUSR_EINVAL;
    musr_fit_opts o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.max_iter <= 0) o.max_iter = 500;
    if (!(o.edm_tol > 0.0)) o.edm_tol = 1e-8;
    if (!(o.mu0 > 0.0)) o.mu0 = 1e-3;
    const int fd_mode = o.fd_rel_h > 0.0 ? 1 : 2;  // fixed relative steps, or steps of the standard errors
    if (!(o.fd_rel_h > 0.0)) o.fd_rel_h = 1e-4;
    if (o.method < MUSR_FIT_LM || o.method > MUSR_FIT_BFGS_FD) return MUSR_EINVAL;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != run->device) cudaSetDevice(run->device);
    std::vector<int> fidx;
    for (int j = 0; j < run->P; ++j)
        if (!free_mask || free_mask[j]) fidx.push_back(j);
    Evaluator ev{run, obj, run->P, {}, 0};
    musr_fit_result r = *out;
    r.n_free = (int32_t)fidx.size();
    r.ndf = (double)(run->total_bins - (int64_t)fidx.size());
    int method = o.method;
    if (method == MUSR_FIT_LM && run->Pk > musr::kMaxGnParams) method = MUSR_FIT_BFGS;
    int st;
    if (method == MUSR_FIT_LM) st = fit_lm(ev, theta, fidx, o, &r);
    else st = fit_bfgs(ev, theta, fidx, o, method == MUSR_FIT_BFGS_FD ? fd_mode : 0, o.fd_rel_h, &r);
    r.n_evals = ev.evals;
    r.status = st;
    *out = r;
    if (cur != run->device) cudaSetDevice(cur);
    return st;
}

// Fits whose objective is evaluated by the caller (musr_fit_eval): the same
// Levenberg-Marquardt and BFGS steppers as musr_fit, with every evaluation a
// call of `eval`.  A histogram-sharded run evaluates its shard on each GPU
// and combines the shards' sums before returning them, so every rank takes
// the same steps.
extern "C" int musr_fit_eval(int32_t n_params, int64_t n_bins_total, musr_eval_fn eval, void* user,
                             double* theta, const uint8_t* free_mask, const musr_fit_opts* opts,
                             musr_fit_result* out) {
    if (n_params <= 0 || !eval || !theta || !out) return MUSR_EINVAL;
    musr_fit_opts o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.max_iter <= 0) o.max_iter = 500;
    if (!(o.edm_tol > 0.0)) o.edm_tol = 1e-8;
    if (!(o.mu0 > 0.0)) o.mu0 = 1e-3;
    if (o.method != MUSR_FIT_LM && o.method != MUSR_FIT_BFGS) return o.method == MUSR_FIT_BFGS_FD ? MUSR_ENOTSUP
                                                                                                : MUSR_EINVAL;
    for (int j = 0; j < n_params; ++j)
        if (!std::isfinite(theta[j])) return MUSR_ENONFINITE;
    const int P = n_params;
    std::vector<int> fidx;
    for (int j = 0; j < P; ++j)
        if (!free_mask || free_mask[j]) fidx.push_back(j);
    int evals = 0;
    // value (+ gradient, + GN matrix) at th; a domain error reads as value +inf
    auto call = [&](const double* th, int mode, double* f, double* g, double* H) -> int {
        ++evals;
        const int st = eval(user, mode, th, f, g, H);
        if (st == MUSR_EDOMAIN) *f = INFINITY;
        if (st == MUSR_OK && !std::isfinite(*f)) return MUSR_ENONFINITE;
        return st;
    };
    musr_fit_result r = *out;
    r.n_free = (int32_t)fidx.size();
    r.ndf = (double)(n_bins_total - (int64_t)fidx.size());
    int st;
    if (o.method == MUSR_FIT_LM) {
        LmStepper lm;
        lm.init(P, fidx, o, theta);
        double f;
        st = call(theta, MUSR_VALUE_GRAD_GN, &f, lm.g.data(), lm.H.data());
        if (st == MUSR_OK) {
            lm.start(f);
            while (lm.next()) {
                double ft;
                const int s2 = call(lm.trial.data(), MUSR_VALUE_GRAD_GN, &ft, lm.gt.data(), lm.Ht.data());
                if (s2 != MUSR_OK && s2 != MUSR_EDOMAIN && s2 != MUSR_ENONFINITE) {
                    st = s2;
                    break;
                }
                lm.observe(s2, ft);
            }
            if (st == MUSR_OK) {
                lm.finish(theta, &r);
                st = lm.result;
            }
        }
    } else {
        std::vector<double> H((size_t)P * P);
        auto value_grad = [&](const double* th, double* f, double* g) -> int {
            return call(th, MUSR_VALUE_GRAD, f, g, nullptr);
        };
        auto start = [&](const double* th, double* f, double* g, double* hd) -> int {
            const int s0 = call(th, MUSR_VALUE_GRAD_GN, f, g, H.data());
            for (int j = 0; j < P; ++j) hd[j] = H[(size_t)j * P + j];
            return s0;
        };
        st = fit_bfgs_generic(P, theta, fidx, o, false, value_grad, start, &r);
    }
    r.n_evals = evals;
    r.status = st;
    *out = r;
    return st;
}

extern "C" int musr_fit_multistart(musr_run run, int obj, const double* starts, int32_t n_starts,
                                   const uint8_t* free_mask, const musr_fit_opts* opts, double* theta_out,
                                   musr_fit_result* out) {
    if (!run || !starts || n_starts <= 0 || !theta_out || !out) return MUSR_EINVAL;
    const int P = run->P;
    int nf = 0;
    for (int j = 0; j < P; ++j) nf += (!free_mask || free_mask[j]) ? 1 : 0;
    std::vector<double> th(P), cov(out->cov ? (size_t)nf * nf : 0), best_cov(cov.size());
    musr_fit_result best;
    memset(&best, 0, sizeof(best));
    bool have = false;
    int first_err = MUSR_OK;
    int32_t iters = 0, evals = 0;
    for (int s = 0; s < n_starts; ++s) {
        std::copy(starts + (size_t)s * P, starts + (size_t)(s + 1) * P, th.begin());
        musr_fit_result r;
        memset(&r, 0, sizeof(r));
        r.cov = cov.empty() ? nullptr : cov.data();
        const int st = musr_fit(run, obj, th.data(), free_mask, opts, &r);
        iters += r.iters;
        evals += r.n_evals;
        const bool ok = (st == MUSR_OK || st == MUSR_ENOCONV) && std::isfinite(r.value);
        if (!ok) {
            if (first_err == MUSR_OK) first_err = st != MUSR_OK ? st : MUSR_ENONFINITE;
            if (st == MUSR_ECUDA || st == MUSR_ETIMEOUT) return st;
            continue;
        }
        if (!have || r.value < best.value) {
            have = true;
            best = r;
            std::copy(th.begin(), th.end(), theta_out);
            best_cov.swap(cov);
            if (!cov.empty() || !best_cov.empty()) cov.resize(best_cov.size());
        }
    }
    if (!have) {
        out->status = first_err;
        out->iters = iters;
        out->n_evals = evals;
        return first_err;
    }
    double* user_cov = out->cov;
    *out = best;
    out->cov = user_cov;
    if (user_cov) std::copy(best_cov.begin(), best_cov.end(), user_cov);
    out->iters = iters;
    out->n_evals = evals;
    return best.status;
}

// BFGS fits of every run of a batch in lockstep: the start evaluation gives
// the Hessian diagonal (Gauss-Newton mode when the batch has it), then one
// batched value + gradient launch per round of line-search trials.
// group / accept: as for the lockstep LM (fit_batch_impl)
static int fit_batch_bfgs(musr_gbatch b, int obj, double* thetas, const uint8_t* free_masks,
                          const musr_fit_opts& o, musr_fit_result* results, const std::vector<int>* group = nullptr,
                          const std::function<bool(int, const double*, double)>* accept = nullptr) {
    const int n = gbatch_n_runs(b);
    std::vector<BfgsStepper> bf(n);
    std::vector<int32_t> flags(n, 0), evals(n, 1);
    std::vector<uint8_t> active(n, 1);
    std::vector<int> status(n, MUSR_OK);
    int64_t total_theta = 0;
    for (int r = 0; r < n; ++r) total_theta += gbatch_run(b, r)->P;
    for (int64_t i = 0; i < total_theta; ++i)
        if (!std::isfinite(thetas[i])) return MUSR_ENONFINITE;
    std::vector<double> work(thetas, thetas + total_theta);
    for (int r = 0; r < n; ++r) {
        const musr_run run = gbatch_run(b, r);
        const int64_t to = gbatch_theta_offset(b, r);
        std::vector<int> fidx;
        for (int j = 0; j < run->P; ++j)
            if (!free_masks || free_masks[to + j]) fidx.push_back(j);
        bf[r].init(run->P, fidx, o, thetas + to, false);
    }
    const int start_mode = gbatch_has_gn(b) ? kGN : kGrad;
    int st = gbatch_eval_host(b, obj, start_mode, work.data(), nullptr, nullptr, flags.data());
    if (st != MUSR_OK) return st;
#pragma omp parallel for schedule(dynamic, 1) if (n >= 8)
    for (int r = 0; r < n; ++r) {
        const musr_run run = gbatch_run(b, r);
        const int P = run->P;
        const double* src = gbatch_host_out(b) + gbatch_out_offset(b, start_mode, r);
        if ((flags[r] & 1) || !std::isfinite(src[0])) {
            status[r] = (flags[r] & 1) ? MUSR_EDOMAIN : MUSR_ENONFINITE;
            bf[r].done = true;
            continue;
        }
        memcpy(bf[r].g.data(), src + 1, sizeof(double) * P);
        std::vector<double> hd(P, 0.0);
        if (start_mode == kGN)
            for (int j = 0; j < P; ++j) hd[j] = src[1 + P + (size_t)j * P + j];
        bf[r].start(src[0], hd.data());
    }
    std::vector<uint8_t> seen_done(n, 0);
    for (;;) {
#pragma omp parallel for schedule(dynamic, 1) if (n >= 8)
        for (int r = 0; r < n; ++r) {
            active[r] = (status[r] == MUSR_OK && bf[r].next()) ? 1 : 0;
            if (active[r]) {
                memcpy(work.data() + gbatch_theta_offset(b, r), bf[r].x.data(), sizeof(double) * bf[r].P);
                ++evals[r];
            }
        }
        if (group && accept) {
            for (int r = 0; r < n; ++r) {
                if (active[r] || seen_done[r]) continue;
                seen_done[r] = 1;
                if (status[r] != MUSR_OK || bf[r].result != MUSR_OK || !(*accept)(r, bf[r].theta.data(), bf[r].f))
                    continue;
                for (int q = 0; q < n; ++q)
                    if (q != r && (*group)[q] == (*group)[r] && !bf[q].done) {
                        bf[q].done = true;
                        active[q] = 0;
                    }
            }
        }
        int n_active = 0;
        for (int r = 0; r < n; ++r) n_active += active[r];
        if (n_active == 0) break;
        st = gbatch_eval_host(b, obj, kGrad, work.data(), active.data(), nullptr, flags.data());
        if (st != MUSR_OK) return st;
#pragma omp parallel for schedule(dynamic, 1) if (n_active >= 8)
        for (int r = 0; r < n; ++r) {
            if (!active[r]) continue;
            const int P = bf[r].P;
            const double* src = gbatch_host_out(b) + gbatch_out_offset(b, kGrad, r);
            const double fn = (flags[r] & 1) ? INFINITY : src[0];
            memcpy(bf[r].gt.data(), src + 1, sizeof(double) * P);
            const int s2 = (flags[r] & 1) ? MUSR_EDOMAIN : (std::isfinite(fn) ? MUSR_OK : MUSR_ENONFINITE);
            bf[r].observe(s2, fn);
        }
    }
    int worst = MUSR_OK;
    for (int r = 0; r < n; ++r) {
        const musr_run run = gbatch_run(b, r);
        musr_fit_result& res = results[r];
        double* cov = res.cov;
        memset(&res, 0, sizeof(res));
        res.cov = cov;
        res.n_free = bf[r].nf;
        res.ndf = (double)(run->total_bins - (int64_t)bf[r].nf);
        if (status[r] == MUSR_OK) {
            bf[r].finish(thetas + gbatch_theta_offset(b, r), &res);
            res.status = bf[r].result;
        } else {
            res.value = INFINITY;
            res.status = status[r];
        }
        res.n_evals = evals[r];
        if (res.status != MUSR_OK && worst == MUSR_OK) worst = res.status;
    }
    return worst;
}

namespace {

// The lockstep fit of every entry of a batch.  group / accept (both null, or
// both set): when entry r's LM fit converges and accept(r, theta, value)
// holds, the other entries of group[r] still running stop where they are
// (status MUSR_ENOCONV).
int fit_batch_impl(musr_gbatch b, int obj, double* thetas, const uint8_t* free_masks, const musr_fit_opts* opts,
                   musr_fit_result* results, const std::vector<int>* group,
                   const std::function<bool(int, const double*, double)>* accept) {
    if (!b || !thetas || !results) return MUSR_EINVAL;
    if (obj != MUSR_CHI2 && obj != MUSR_POISSON) return MUSR_EINVAL;
    musr_fit_opts o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.max_iter <= 0) o.max_iter = 500;
    if (!(o.edm_tol > 0.0)) o.edm_tol = 1e-8;
    if (!(o.mu0 > 0.0)) o.mu0 = 1e-3;
    if (o.method == MUSR_FIT_BFGS) return fit_batch_bfgs(b, obj, thetas, free_masks, o, results, group, accept);
    if (o.method != MUSR_FIT_LM) return MUSR_ENOTSUP;
    if (!gbatch_has_gn(b)) return MUSR_EINVAL;
    const int n = gbatch_n_runs(b);
    std::vector<LmStepper> lm(n);
    std::vector<int32_t> flags(n, 0), evals(n, 1);
    std::vector<uint8_t> active(n, 1);
    int64_t total_theta = 0;
    for (int r = 0; r < n; ++r) total_theta += gbatch_run(b, r)->P;
    for (int64_t i = 0; i < total_theta; ++i)
        if (!std::isfinite(thetas[i])) return MUSR_ENONFINITE;
    std::vector<double> work(thetas, thetas + total_theta);
    for (int r = 0; r < n; ++r) {
        const musr_run run = gbatch_run(b, r);
        const int64_t to = gbatch_theta_offset(b, r);
        std::vector<int> fidx;
        for (int j = 0; j < run->P; ++j)
            if (!free_masks || free_masks[to + j]) fidx.push_back(j);
        lm[r].init(run->P, fidx, o, thetas + to);
    }
    // start: value, gradient and GN matrix of every run at its start point
    int st = gbatch_eval_host(b, obj, kGN, work.data(), nullptr, nullptr, flags.data());
    if (st != MUSR_OK) return st;
    std::vector<int> status(n, MUSR_OK);
    auto take = [&](int r, double* f, double* g, double* H) -> int {
        const musr_run run = gbatch_run(b, r);
        const int P = run->P;
        const double* src = gbatch_host_out(b) + gbatch_out_offset(b, kGN, r);
        *f = (flags[r] & 1) ? INFINITY : src[0];
        memcpy(g, src + 1, sizeof(double) * P);
        memcpy(H, src + 1 + P, sizeof(double) * P * P);
        if (flags[r] & 1) return MUSR_EDOMAIN;
        return std::isfinite(*f) ? MUSR_OK : MUSR_ENONFINITE;
    };
    // every run's LM step is independent: spread them over the host cores
#pragma omp parallel for schedule(dynamic, 1) if (n >= 8)
    for (int r = 0; r < n; ++r) {
        double f;
        status[r] = take(r, &f, lm[r].g.data(), lm[r].H.data());
        if (status[r] == MUSR_OK) lm[r].start(f);
        else lm[r].done = true;
    }
    std::vector<uint8_t> seen_done(n, 0);
    for (;;) {
#pragma omp parallel for schedule(dynamic, 1) if (n >= 8)
        for (int r = 0; r < n; ++r) {
            active[r] = (status[r] == MUSR_OK && lm[r].next()) ? 1 : 0;
            if (active[r]) {
                memcpy(work.data() + gbatch_theta_offset(b, r), lm[r].trial.data(), sizeof(double) * lm[r].P);
                ++evals[r];
            }
        }
        if (group && accept) {
            // a converged entry the caller accepts stops the rest of its group
            for (int r = 0; r < n; ++r) {
                if (active[r] || seen_done[r]) continue;
                seen_done[r] = 1;
                if (status[r] != MUSR_OK || lm[r].result != MUSR_OK || !(*accept)(r, lm[r].theta.data(), lm[r].f))
                    continue;
                for (int q = 0; q < n; ++q)
                    if (q != r && (*group)[q] == (*group)[r] && !lm[q].done) {
                        lm[q].done = true;
                        active[q] = 0;
                    }
            }
        }
        int n_active = 0;
        for (int r = 0; r < n; ++r) n_active += active[r];
        if (n_active == 0) break;
        st = gbatch_eval_host(b, obj, kGN, work.data(), active.data(), nullptr, flags.data());
        if (st != MUSR_OK) return st;
#pragma omp parallel for schedule(dynamic, 1) if (n_active >= 8)
        for (int r = 0; r < n; ++r) {
            if (!active[r]) continue;
            double ft;
            const int s2 = take(r, &ft, lm[r].gt.data(), lm[r].Ht.data());
            lm[r].observe(s2, ft);
        }
    }
    int worst = MUSR_OK;
    for (int r = 0; r < n; ++r) {
        const musr_run run = gbatch_run(b, r);
        musr_fit_result& res = results[r];
        double* cov = res.cov;
        memset(&res, 0, sizeof(res));
        res.cov = cov;
        res.n_free = lm[r].nf;
        res.ndf = (double)(run->total_bins - (int64_t)lm[r].nf);
        if (status[r] == MUSR_OK) {
            lm[r].finish(thetas + gbatch_theta_offset(b, r), &res);
            res.status = lm[r].result;
        } else {
            res.value = INFINITY;
            res.status = status[r];
        }
        res.n_evals = evals[r];
        if (res.status != MUSR_OK && worst == MUSR_OK) worst = res.status;
    }
    return worst;
}

}  // namespace

extern "C" int musr_fit_batch(musr_gbatch b, int obj, double* thetas, const uint8_t* free_masks,
                              const musr_fit_opts* opts, musr_fit_result* results) {
    return fit_batch_impl(b, obj, thetas, free_masks, opts, results, nullptr, nullptr);
}

extern "C" int musr_fit_multistart_batch(const musr_run* runs, int32_t n_runs, int obj, const double* starts,
                                         int32_t n_starts, const uint8_t* free_masks, const musr_fit_opts* opts,
                                         double* thetas_out, musr_fit_result* results) {
    return musr::fit_multistart_batch_accept(runs, n_runs, obj, starts, n_starts, free_masks, opts, nullptr,
                                             thetas_out, results);
}

// musr_fit_multistart_batch; with accept, the first converged start
// of run r that accept(r, theta, value) takes ends r's other starts and is r's
// result.
int musr::fit_multistart_batch_accept(const musr_run* runs, int n_runs, int obj, const double* starts, int n_starts,
                                      const uint8_t* free_masks, const musr_fit_opts* opts,
                                      const std::function<bool(int, const double*, double)>* accept,
                                      double* thetas_out, musr_fit_result* results) {
    if (!runs || n_runs <= 0 || !starts || n_starts <= 0 || !thetas_out || !results) return MUSR_EINVAL;
    // entry e = (run r, start s), e = r * n_starts + s
    std::vector<musr_run> entries;
    std::vector<int64_t> toff(n_runs + 1, 0);
    for (int r = 0; r < n_runs; ++r) {
        if (!runs[r]) return MUSR_EINVAL;
        toff[r + 1] = toff[r] + runs[r]->P;
        for (int s = 0; s < n_starts; ++s) entries.push_back(runs[r]);
    }
    std::vector<double> th;
    std::vector<uint8_t> fm;
    for (int r = 0; r < n_runs; ++r) {
        const int P = runs[r]->P;
        const double* st = starts + toff[r] * n_starts;
        th.insert(th.end(), st, st + (size_t)P * n_starts);
        for (int s = 0; s < n_starts; ++s) {
            if (free_masks) fm.insert(fm.end(), free_masks + toff[r], free_masks + toff[r] + P);
            else fm.insert(fm.end(), (size_t)P, (uint8_t)1);
        }
    }
    musr_gbatch b = nullptr;
    int st = musr_gbatch_create(entries.data(), (int32_t)entries.size(), 1, &b);
    if (st != MUSR_OK) return st;
    std::vector<musr_fit_result> res(entries.size());
    for (auto& x : res) memset(&x, 0, sizeof(x));
    std::vector<int> group(entries.size());
    for (size_t e = 0; e < entries.size(); ++e) group[e] = (int)(e / n_starts);
    std::vector<uint8_t> taken(entries.size(), 0);
    std::function<bool(int, const double*, double)> on_converged = [&](int e, const double* theta, double f) {
        if (!(*accept)(group[e], theta, f)) return false;
        taken[e] = 1;
        return true;
    };
    st = fit_batch_impl(b, obj, th.data(), fm.data(), opts, res.data(), accept ? &group : nullptr,
                        accept ? &on_converged : nullptr);
    musr_gbatch_destroy(b);
    if (st != MUSR_OK && st != MUSR_ENOCONV && st != MUSR_EDOMAIN && st != MUSR_ENONFINITE) return st;
    int worst = MUSR_OK;
    int64_t e_off = 0;
    for (int r = 0; r < n_runs; ++r) {
        const int P = runs[r]->P;
        int best = -1;
        int32_t iters = 0, evals = 0;
        for (int s = 0; s < n_starts; ++s) {
            const musr_fit_result& x = res[(size_t)r * n_starts + s];
            iters += x.iters;
            evals += x.n_evals;
            const bool ok = (x.status == MUSR_OK || x.status == MUSR_ENOCONV) && std::isfinite(x.value);
            if (ok && (best < 0 || x.value < res[(size_t)r * n_starts + best].value)) best = s;
        }
        for (int s = 0; s < n_starts; ++s)
            if (taken[(size_t)r * n_starts + s]) best = s;  // the accepted start ends the run's search
        double* cov = results[r].cov;
        if (best < 0) {
            memset(&results[r], 0, sizeof(musr_fit_result));
            results[r].cov = cov;
            results[r].value = INFINITY;
            results[r].status = res[(size_t)r * n_starts].status != MUSR_OK ? res[(size_t)r * n_starts].status
                                                                             : MUSR_ENONFINITE;
            memcpy(thetas_out + toff[r], starts + toff[r] * n_starts, sizeof(double) * P);
        } else {
            results[r] = res[(size_t)r * n_starts + best];
            results[r].cov = cov;  // the covariance is not kept for batched starts
            if (cov)
                for (int i = 0; i < results[r].n_free * results[r].n_free; ++i) cov[i] = NAN;
            memcpy(thetas_out + toff[r], th.data() + e_off + (size_t)best * P, sizeof(double) * P);
        }
        results[r].iters = iters;
        results[r].n_evals = evals;
        if (results[r].status != MUSR_OK && worst == MUSR_OK) worst = results[r].status;
        e_off += (int64_t)P * n_starts;
    }
    return worst;
}
