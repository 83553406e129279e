// opcount.cpp -- op-counting build of the oracle.  TEST / MEASUREMENT
// INFRASTRUCTURE ONLY (the benchmark's FP64 roofline takes its algorithmic
// flop count from it); it shares nothing with the CUDA path.
//
// oracle.c is compiled as C++ with every `double` replaced by a value type
// that counts the arithmetic done on it: additions and subtractions,
// multiplications, divisions, square roots, minima and maxima, comparisons,
// absolute values and the transcendental functions (exp, log, pow, tanh,
// cosh, cbrt) separately.  Unary minus and copies are free.  oc_stage runs
// one stage of or_stage (serially) and returns the counts.
#include <float.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>

namespace {
enum { OC_ADD, OC_MUL, OC_DIV, OC_SQRT, OC_MINMAX, OC_CMP, OC_ABS, OC_TRANSC, OC_N };
unsigned long long g_ops[OC_N];
}  // namespace

struct cdouble {
    double v;
    cdouble() = default;
    constexpr cdouble(double x) : v(x) {}
    constexpr cdouble(int x) : v(x) {}
    constexpr cdouble(long x) : v(double(x)) {}
    constexpr cdouble(unsigned long x) : v(double(x)) {}
    explicit operator int() const { return int(v); }
    explicit operator long() const { return long(v); }
    explicit operator bool() const { return v != 0.0; }
    cdouble& operator+=(cdouble b) { ++g_ops[OC_ADD]; v += b.v; return *this; }
    cdouble& operator-=(cdouble b) { ++g_ops[OC_ADD]; v -= b.v; return *this; }
    cdouble& operator*=(cdouble b) { ++g_ops[OC_MUL]; v *= b.v; return *this; }
    cdouble& operator/=(cdouble b) { ++g_ops[OC_DIV]; v /= b.v; return *this; }
};
static inline cdouble operator-(cdouble a) { return cdouble(-a.v); }
static inline cdouble operator+(cdouble a) { return a; }
#define OC_BIN(op, cls)                                                                        \
    static inline cdouble operator op(cdouble a, cdouble b) { ++g_ops[cls]; return cdouble(a.v op b.v); } \
    static inline cdouble operator op(cdouble a, double b) { ++g_ops[cls]; return cdouble(a.v op b); }    \
    static inline cdouble operator op(double a, cdouble b) { ++g_ops[cls]; return cdouble(a op b.v); }    \
    static inline cdouble operator op(cdouble a, int b) { ++g_ops[cls]; return cdouble(a.v op b); }       \
    static inline cdouble operator op(int a, cdouble b) { ++g_ops[cls]; return cdouble(a op b.v); }
OC_BIN(+, OC_ADD)
OC_BIN(-, OC_ADD)
OC_BIN(*, OC_MUL)
OC_BIN(/, OC_DIV)
#define OC_CMP(op)                                                                             \
    static inline bool operator op(cdouble a, cdouble b) { ++g_ops[OC_CMP]; return a.v op b.v; } \
    static inline bool operator op(cdouble a, double b) { ++g_ops[OC_CMP]; return a.v op b; }    \
    static inline bool operator op(double a, cdouble b) { ++g_ops[OC_CMP]; return a op b.v; }    \
    static inline bool operator op(cdouble a, int b) { ++g_ops[OC_CMP]; return a.v op b; }       \
    static inline bool operator op(int a, cdouble b) { ++g_ops[OC_CMP]; return a op b.v; }
OC_CMP(<)
OC_CMP(>)
OC_CMP(<=)
OC_CMP(>=)
OC_CMP(==)
OC_CMP(!=)
static inline bool operator!(cdouble a) { return a.v == 0.0; }
static inline cdouble fabs(cdouble a) { ++g_ops[OC_ABS]; return cdouble(std::fabs(a.v)); }
static inline cdouble sqrt(cdouble a) { ++g_ops[OC_SQRT]; return cdouble(std::sqrt(a.v)); }
static inline cdouble fmin(cdouble a, cdouble b) { ++g_ops[OC_MINMAX]; return cdouble(std::fmin(a.v, b.v)); }
static inline cdouble fmax(cdouble a, cdouble b) { ++g_ops[OC_MINMAX]; return cdouble(std::fmax(a.v, b.v)); }
static inline cdouble exp(cdouble a) { ++g_ops[OC_TRANSC]; return cdouble(std::exp(a.v)); }
static inline cdouble log(cdouble a) { ++g_ops[OC_TRANSC]; return cdouble(std::log(a.v)); }
static inline cdouble pow(cdouble a, cdouble b) { ++g_ops[OC_TRANSC]; return cdouble(std::pow(a.v, b.v)); }
static inline cdouble tanh(cdouble a) { ++g_ops[OC_TRANSC]; return cdouble(std::tanh(a.v)); }
static inline cdouble cosh(cdouble a) { ++g_ops[OC_TRANSC]; return cdouble(std::cosh(a.v)); }
static inline cdouble cbrt(cdouble a) { ++g_ops[OC_TRANSC]; return cdouble(std::cbrt(a.v)); }
static inline bool isfinite(cdouble a) { return std::isfinite(a.v); }

#define double cdouble
#include "oracle.c"
#undef double

// one stage of the oracle on the whole grid with the arithmetic counted;
// counts[8] receives add/sub, mul, div, sqrt, min/max, compare, abs,
// transcendental
extern "C" int oc_stage(const void* P, int k, double dt, const double* q0, const double* qprev, double* qout,
                        unsigned long long* counts)
{
    memset(g_ops, 0, sizeof g_ops);
    const int st = or_stage(static_cast<const or_params*>(P), k, cdouble(dt), reinterpret_cast<const cdouble*>(q0),
                            reinterpret_cast<const cdouble*>(qprev), reinterpret_cast<cdouble*>(qout), NULL, NULL);
    for (int i = 0; i < OC_N; ++i) counts[i] = g_ops[i];
    return st;
}

// the boundary and primitive update alone (box_fill over the box or_stage
// fills for the whole grid): the part of a stage that the oracle does by
// bisection rather than by the closed form
extern "C" int oc_box_fill(const void* Pv, const double* q, unsigned long long* counts)
{
    const or_params* P = static_cast<const or_params*>(Pv);
    int blo[3], bhi[3];
    for (int d = 0; d < 3; ++d) {
        blo[d] = d < P->ndim ? -2 : 0;
        bhi[d] = d < P->ndim ? P->n[d] + 2 : 1;
    }
    box_t B;
    memset(&B, 0, sizeof(B));
    memset(g_ops, 0, sizeof g_ops);
    const int st = box_fill(P, reinterpret_cast<const cdouble*>(q), &B, blo, bhi);
    for (int i = 0; i < OC_N; ++i) counts[i] = g_ops[i];
    box_free(&B);
    return st;
}
