// The function array of Sec. 4.2.1: values the theory reads that are
// functions of the parameters (Musrfit precomputes them before each
// evaluation and hands them to the kernel next to the parameter array).
//
// A run may declare n_funcs functions, each an arithmetic expression over
// p[i] (theta entries), numeric literals, + - * / ^ ( ) and the functions
// exp log sqrt sin cos tan atan abs pow.  They are compiled here once into a
// postfix program and evaluated on the host per call, with forward-mode
// derivatives (value and derivative along one parameter) for the chain rule
// of the gradient and Gauss-Newton matrix.  The kernels never see the
// expressions: they read the function values as extra parameter slots.
#include <ctype.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "run_impl.h"

namespace musr {
namespace {

enum Op { kConst, kParam, kAdd, kSub, kMul, kDiv, kNeg, kPow, kExp, kLog, kSqrt, kSin, kCos, kTan, kAtan, kAbs };

struct Parser {
    const char* s;
    int P;
    std::vector<HostExpr::Ins>& code;
    std::vector<int>& refs;
    bool ok = true;

    void ws() {
        while (*s == ' ' || *s == '\t' || *s == '\n' || *s == '\r') ++s;
    }
    bool eat(char c) {
        ws();
        if (*s != c) return false;
        ++s;
        return true;
    }
    void emit(int op, double c = 0.0, int i = 0) { code.push_back(HostExpr::Ins{op, i, c}); }

    void expr() {
        term();
        for (;;) {
            if (eat('+')) {
                term();
                emit(kAdd);
            } else if (eat('-')) {
                term();
                emit(kSub);
            } else {
                return;
            }
        }
    }
    void term() {
        unary();
        for (;;) {
            if (eat('*')) {
                unary();
                emit(kMul);
            } else if (eat('/')) {
                unary();
                emit(kDiv);
            } else {
                return;
            }
        }
    }
    void unary() {
        if (eat('-')) {
            unary();
            emit(kNeg);
        } else if (eat('+')) {
            unary();
        } else {
            power();
        }
    }
    // a ^ b binds tighter than unary minus on its left and is right-associative
    void power() {
        primary();
        if (eat('^')) {
            unary();
            emit(kPow);
        }
    }
    void primary() {
        ws();
        if (!ok) return;
        if (isdigit((unsigned char)*s) || *s == '.') {
            char* end = nullptr;
            const double v = strtod(s, &end);
            if (end == s) {
                ok = false;
                return;
            }
            s = end;
            emit(kConst, v);
            return;
        }
        if (eat('(')) {
            expr();
            if (!eat(')')) ok = false;
            return;
        }
        if (isalpha((unsigned char)*s)) {
            const char* b = s;
            while (isalnum((unsigned char)*s) || *s == '_') ++s;
            const std::string name(b, s);
            if (name == "p") {
                if (!eat('[')) {
                    ok = false;
                    return;
                }
                ws();
                char* end = nullptr;
                const long i = strtol(s, &end, 10);
                if (end == s || i < 0 || i >= P) {
                    ok = false;
                    return;
                }
                s = end;
                if (!eat(']')) {
                    ok = false;
                    return;
                }
                emit(kParam, 0.0, (int)i);
                if (std::find(refs.begin(), refs.end(), (int)i) == refs.end()) refs.push_back((int)i);
                return;
            }
            static const struct {
                const char* n;
                int op, args;
            } fns[] = {{"exp", kExp, 1}, {"log", kLog, 1}, {"sqrt", kSqrt, 1}, {"sin", kSin, 1},
                       {"cos", kCos, 1}, {"tan", kTan, 1}, {"atan", kAtan, 1}, {"abs", kAbs, 1},
                       {"fabs", kAbs, 1}, {"pow", kPow, 2}};
            for (const auto& f : fns) {
                if (name != f.n) continue;
                if (!eat('(')) {
                    ok = false;
                    return;
                }
                expr();
                if (f.args == 2 && !eat(',')) {
                    ok = false;
                    return;
                }
                if (f.args == 2) expr();
                if (!eat(')')) {
                    ok = false;
                    return;
                }
                emit(f.op);
                return;
            }
        }
        ok = false;
    }
};

}  // namespace

int compile_host_expr(const char* text, int P, HostExpr& out) {
    out = HostExpr{};
    if (!text) return MUSR_EINVAL;
    Parser ps{text, P, out.code, out.refs};
    ps.expr();
    ps.ws();
    if (!ps.ok || *ps.s != '\0' || out.code.empty()) return MUSR_EINVAL;
    // the stack depth the program needs (every op is checked for its operands)
    int depth = 0, peak = 0;
    for (const auto& in : out.code) {
        const int pops = (in.op == kConst || in.op == kParam) ? 0 : (in.op >= kAdd && in.op <= kDiv) || in.op == kPow ? 2 : 1;
        if (depth < pops) return MUSR_EINVAL;
        depth += 1 - pops;
        peak = std::max(peak, depth);
    }
    if (depth != 1) return MUSR_EINVAL;
    out.depth = peak;
    std::sort(out.refs.begin(), out.refs.end());
    return MUSR_OK;
}

// Value of the expression at theta and, if dvar >= 0, its derivative with
// respect to theta[dvar] (forward mode: every stack entry is a value and a
// derivative).
double eval_host_expr(const HostExpr& e, const double* theta, int dvar, double* deriv) {
    std::vector<double> v(e.depth + 1), d(e.depth + 1);
    int n = 0;
    for (const auto& in : e.code) {
        switch (in.op) {
            case kConst: v[n] = in.c; d[n] = 0.0; ++n; break;
            case kParam: v[n] = theta[in.i]; d[n] = in.i == dvar ? 1.0 : 0.0; ++n; break;
            case kNeg: v[n - 1] = -v[n - 1]; d[n - 1] = -d[n - 1]; break;
            case kExp: v[n - 1] = exp(v[n - 1]); d[n - 1] *= v[n - 1]; break;
            case kLog: d[n - 1] /= v[n - 1]; v[n - 1] = log(v[n - 1]); break;
            case kSqrt: v[n - 1] = sqrt(v[n - 1]); d[n - 1] = d[n - 1] / (2.0 * v[n - 1]); break;
            case kSin: d[n - 1] *= cos(v[n - 1]); v[n - 1] = sin(v[n - 1]); break;
            case kCos: d[n - 1] *= -sin(v[n - 1]); v[n - 1] = cos(v[n - 1]); break;
            case kTan: { const double c = cos(v[n - 1]); d[n - 1] /= c * c; v[n - 1] = tan(v[n - 1]); break; }
            case kAtan: d[n - 1] /= 1.0 + v[n - 1] * v[n - 1]; v[n - 1] = atan(v[n - 1]); break;
            case kAbs: if (v[n - 1] < 0.0) { v[n - 1] = -v[n - 1]; d[n - 1] = -d[n - 1]; } break;
            default: {
                const double a = v[n - 2], da = d[n - 2], b = v[n - 1], db = d[n - 1];
                double r = 0.0, dr = 0.0;
                if (in.op == kAdd) { r = a + b; dr = da + db; }
                else if (in.op == kSub) { r = a - b; dr = da - db; }
                else if (in.op == kMul) { r = a * b; dr = da * b + a * db; }
                else if (in.op == kDiv) { r = a / b; dr = (da - r * db) / b; }
                else {  // a^b: b a^(b-1) da + a^b ln(a) db (the log term only where b varies)
                    r = pow(a, b);
                    dr = (da != 0.0 ? b * pow(a, b - 1.0) * da : 0.0) + (db != 0.0 ? r * log(a) * db : 0.0);
                }
                --n;
                v[n - 1] = r;
                d[n - 1] = dr;
            }
        }
    }
    if (deriv) *deriv = d[0];
    return v[0];
}

}  // namespace musr

extern "C" int musr_function_eval(const char* expr, int32_t n_params, const double* theta, double* value,
                                  double* grad) {
    if (!expr || n_params < 0 || (n_params > 0 && !theta) || !value) return MUSR_EINVAL;
    musr::HostExpr e;
    if (musr::compile_host_expr(expr, n_params, e) != MUSR_OK) return MUSR_EINVAL;
    *value = musr::eval_host_expr(e, theta, -1, nullptr);
    if (grad) {
        for (int j = 0; j < n_params; ++j) grad[j] = 0.0;
        for (int r : e.refs) musr::eval_host_expr(e, theta, r, &grad[r]);
    }
    return isfinite(*value) ? MUSR_OK : MUSR_ENONFINITE;
}
