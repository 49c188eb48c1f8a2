// Batched evaluation entry points (placeholder until the persistent batched
// kernel lands): evaluates each vector with the single-run kernel.
#include <math.h>
#include <string.h>

#include <vector>

#include "musr.h"
#include "musr_internal.h"
#include "run_impl.h"

namespace musr {

int batch_fd_gradient(musr_run run, int obj, const double* theta, const std::vector<int>& fidx,
                      double rel_h, double* value, double* grad) {
    const int P = run->P;
    std::vector<double> th(theta, theta + P);
    int32_t flags = 0;
    int st = run->eval_host(obj, kValue, theta, value, &flags);
    if (st != MUSR_OK) return st;
    if (flags & 1) {
        *value = INFINITY;
        return MUSR_EDOMAIN;
    }
    memset(grad, 0, sizeof(double) * P);
    for (int j : fidx) {
        const double h = rel_h * fmax(fabs(theta[j]), 1.0);
        double fp, fm;
        th[j] = theta[j] + h;
        st = run->eval_host(obj, kValue, th.data(), &fp, &flags);
        if (st != MUSR_OK) return st;
        if (flags & 1) return MUSR_EDOMAIN;
        th[j] = theta[j] - h;
        st = run->eval_host(obj, kValue, th.data(), &fm, &flags);
        if (st != MUSR_OK) return st;
        if (flags & 1) return MUSR_EDOMAIN;
        th[j] = theta[j];
        grad[j] = (fp - fm) / (2.0 * h);
    }
    return MUSR_OK;
}

}  // namespace musr

extern "C" {

int musr_chi2_batch(const musr_run* runs, int32_t n_runs, int obj, const double* thetas,
                    const int32_t* n_vec, double* values) {
    if (!runs || n_runs < 0 || !thetas || !n_vec || !values) return MUSR_EINVAL;
    size_t to = 0, vo = 0;
    for (int r = 0; r < n_runs; ++r) {
        for (int v = 0; v < n_vec[r]; ++v) {
            int st = musr_chi2(runs[r], obj, thetas + to, values + vo);
            if (st != MUSR_OK && st != MUSR_EDOMAIN) return st;
            to += runs[r]->P;
            ++vo;
        }
    }
    return MUSR_OK;
}

int musr_batch_create(const musr_run*, int32_t, const int32_t*, musr_batch* out) {
    if (out) *out = nullptr;
    return MUSR_ENOTSUP;
}
int musr_batch_destroy(musr_batch) { return MUSR_OK; }
int musr_batch_eval(musr_batch, int, const double*, const int32_t*, double*) { return MUSR_ENOTSUP; }
int musr_batch_eval_device(musr_batch, int, const double*, double*) { return MUSR_ENOTSUP; }

}  // extern "C"
