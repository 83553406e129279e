// fv_device.cuh -- device-side data structures and the per-cell / per-face
// arithmetic of the All-Mach THINC-TDU stage (Jiao, Schmidt & Adams,
// arXiv 2304.00140).  Templated on the arithmetic type R: double for the
// FP64 form, float for the mixed form (FP64 conserved registers and an FP64
// core in the primitive recovery, FP32 everywhere else, pressure carried as
// an offset p' = p - p_ref).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tfv {

constexpr int MAXC = 4;
// closures (compile-time kernel parameter): stiffened / ideal gas (App. A.1),
// Peng-Robinson (App. A.2.1), barotropic liquid-vapour + gases (Sec. 2.2)
constexpr int CL_SG = 0, CL_PR = 1, CL_BARO = 2;
constexpr int ERR_NONPHYS = 1;
constexpr int ERR_NONCONV = 2;
constexpr int ERR_TIMEOUT = 4;   // a bounded wait in a kernel gave up
// boundary kind of a block side shared with the neighbouring block of a grid
// split into slabs (internal; the public kinds are 0..3)
constexpr int BC_HALO = 4;

// Per-case geometry, copied to the device once at init.
struct CaseDesc {
    int n[3];            // interior cells (1 in unused dims)
    int g[3];            // ghosted extents: n + 4 in active dims, 1 otherwise
    int gp;              // row pitch of the primitive arrays: g[0] rounded up to 4 (16-byte rows for TMA)
    long long qoff;      // first cell of this case in the conserved arrays
    long long poff;      // first cell of this case in the primitive arrays
    double dx[3], idx[3];
    float fdx[3], fidx[3];   // float copies for the FP32 arithmetic
    int bc[3][2];
    int inflow;          // x-low side is an inflow disc
    double in_yc, in_zc, in_r2, in_T;
    double in_u0[3];
    double in_Y[MAXC];
    long long in_uoff;   // offset of this case's [3][nz][ny] inflow velocity, -1 = use in_u0
    long long in_ustride;   // component stride of that array (ny nz of the whole grid)
    int org[3];          // index of the case's first cell in the whole grid (a slab of a split grid; else 0)
};

// Constants of the arithmetic in the working precision R (a double and a
// float copy are kept so the FP32 arithmetic never converts at run time).
template <typename R>
struct ConstT {
    R Pk[MAXC];          // p_ref + pinf_k
    R gm1cv[MAXC], igamma[MAXC], gcv[MAXC], cv[MAXC], q[MAXC], pinf[MAXC], pother[MAXC];
    R p_ref, beta, thinc_eps, thinc_gamma, tb, icb, itb;
    R thr_ducros, thr_gas, eps_ducros, d3p_coef, sigma, grad_eps;
    R gm1_lo[MAXC], gpi_hi[MAXC], gpi_lo[MAXC];   // gamma-1 (lo part) and gamma pinf + p_ref as float-float
    R gm1_hi[MAXC];
    R Po[MAXC];          // pinf of the other pressure class + p_ref
    R mu[MAXC], kc[MAXC];   // viscosity and conductivity per component (Eq. 2-2)
    R grav[3];              // body force per unit mass (Eq. 2-2 Q)
    R icvmin;               // 1 / smallest component cv (diffusive step limit)
    // barotropic closure (Sec. 2.2): R T_ref per gas (0 for the liquid);
    // saturated liquid / vapour densities, p_sat - p_ref, 1/c_L^2, 1/c_M^2
    R brt[MAXC];
    R b_rsl, b_rsv, b_pso, b_icl2, b_icm2, thr_vap;
    R b_hcl2, b_irsl;       // c_L^2 / 2 and 1 / rho_sat,liq (the recovery's divisions as products)
};

struct CompDev {
    double gamma, pinf, cv, q;
    double gm1cv;        // (gamma - 1) cv
    double gcv;          // gamma cv
    double igamma;       // 1 / gamma
    double pother;       // pinf of the other pressure class (see prim recovery)
    int classA;          // 1 if pinf == the larger class pressure
};

// Peng-Robinson constants (Eq. A.2.1): per species b_k, 1/M_k, cv_k; per
// species pair A_ab = 0.457236 (R Tc_ab)^2 / pc_ab, c_ab (acentric term) and
// 1/sqrt(Tc_ab).  Always used in FP64.
template <typename F>
struct PRConstT {
    F b[MAXC], iM[MAXC], cv[MAXC];
    F A[MAXC][MAXC], cc[MAXC][MAXC], isqTc[MAXC][MAXC];
};
using PRConst = PRConstT<double>;

// Scheme constants, passed by value to every kernel (kernel-parameter bank).
struct DevParams {
    int ndim, ncomp, nv, nprim, liquid;
    int iles, thinc, lim_vel, lim_scalar;
    int csf, aux_rc, aux_al, i_rho, i_c, i_al;
    int visc, grav;      // viscous / heat-flux terms on; gravity source on
    int hf;              // CSF curvature from the height function (Sec. 3.5 option)
    int capj;            // surface tension as a capillary pressure jump in the Riemann solver
    int i_kap;           // primitive-array field of the cell curvature (capillary jump)
    int i_mu, i_kc;      // primitive-array fields of the mixture viscosity and conductivity
    double beta, thinc_eps, thinc_gamma, tb, icb, itb;
    double thr_ducros, thr_gas, eps_ducros, d3p_coef;
    double sigma, grad_eps;
    double p_ref;        // pressure offset (0 in the FP64 form)
    int single_class;    // every component shares one pinf
    CompDev c[MAXC];
    double Pk[MAXC];     // p_ref + pinf_k
    long long ntot_q;    // interior cells of all cases (field stride of q)
    long long ntot_p;    // ghosted cells of all cases (field stride of primitives)
    ConstT<double> kd;
    ConstT<float> kf;
    int pr;              // every component is Peng-Robinson
    int baro;            // barotropic closure (Sec. 2.2)
    int i_av;            // primitive-array field of the vapour volume fraction (barotropic)
    PRConst prc;
    PRConstT<float> prcf;  // FP32 copy (the mixed form's face TDU)
};

template <typename R> __device__ __forceinline__ const ConstT<R>& K(const DevParams& P);
template <> __device__ __forceinline__ const ConstT<double>& K<double>(const DevParams& P) { return P.kd; }
template <> __device__ __forceinline__ const ConstT<float>& K<float>(const DevParams& P) { return P.kf; }
template <typename R> __device__ __forceinline__ R pick(double d, float f);
template <> __device__ __forceinline__ double pick<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float pick<float>(double, float f) { return f; }

// ---------------------------------------------------------------- helpers
template <typename R> __device__ __forceinline__ R clip01(R x) { return x < R(0) ? R(0) : (x > R(1) ? R(1) : x); }
// FP64 tests on the bit patterns (integer instructions, which leave the slow
// FP64 pipe to the arithmetic): the patterns of non-negative doubles order
// like their values, a pattern that is negative as a 64-bit integer is a
// negative double, and above infinity's pattern lie the NaNs
constexpr long long DSIGN = (long long)0x8000000000000000ull, DINF = 0x7ff0000000000000ll,
                    DONE = 0x3ff0000000000000ll;
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
// x > 0 (false for NaN)
__device__ __forceinline__ bool gt0(double x) { const long long b = dbits(x); return b > 0 && b <= DINF; }
__device__ __forceinline__ bool gt0(float x) { return x > 0.0f; }
// clip to [0, 1] with NaN passed through, as the generic form does
template <> __device__ __forceinline__ double clip01<double>(double x)
{
    const long long b = dbits(x), a = b & ~DSIGN;
    if (a > DINF) return x;
    return b < 0 ? 0.0 : (b > DONE ? 1.0 : x);
}
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double sq_rt(double x) { return sqrt(x); }
__device__ __forceinline__ float sq_rt(float x) { return sqrtf(x); }
__device__ __forceinline__ double ex(double x) { return exp(x); }
__device__ __forceinline__ float ex(float x) { return __expf(x); }
// Division and reciprocal: IEEE in double (the FP64 form matches the oracle
// to rounding), the hardware approximation in float (a couple of ulp, well
// inside the FP32 form's accuracy; every float denominator here is far below
// 2^126).
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double frcp(double a) { return 1.0 / a; }
__device__ __forceinline__ float frcp(float a) { return __fdividef(1.0f, a); }

// ------------------------------------------------ compensated FP32 registers
// The mixed form keeps the conserved LSRK registers as float-float pairs
// (float2: hi + lo, about 48 significant bits, 8 bytes like FP64), so that
// its arithmetic never touches the FP64 pipe.  Error-free transformations
// (Knuth two-sum, Dekker/FMA two-product).
__device__ __forceinline__ float2 ff_two_sum(float a, float b)
{
    const float s = a + b, bb = s - a;
    return make_float2(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ float2 ff_fast(float a, float b)
{
    const float s = a + b;
    return make_float2(s, b - (s - a));
}
__device__ __forceinline__ float2 ff_add_f(float2 a, float b)
{
    const float2 s = ff_two_sum(a.x, b);
    return ff_fast(s.x, s.y + a.y);
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b)
{
    const float2 s = ff_two_sum(a.x, b.x);
    return ff_fast(s.x, s.y + (a.y + b.y));
}
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b)
{
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
    return ff_fast(p, e);
}
__host__ __device__ inline float2 ff_from_double(double x)
{
    const float hi = float(x);
    return make_float2(hi, float(x - double(hi)));
}

template <typename T> struct IsFF { static constexpr bool value = false; };
template <> struct IsFF<float2> { static constexpr bool value = true; };

// conserved register value in the working precision R
__device__ __forceinline__ double qv_d(double x) { return x; }
__device__ __forceinline__ double qv_d(float2 x) { return double(x.x) + double(x.y); }
template <typename R> __device__ __forceinline__ R qv(double x) { return R(x); }
template <typename R> __device__ __forceinline__ R qv(float2 x) { return R(x.x + x.y); }

// Packed FP32 pairs: one FADD2 / FMUL2 / FFMA2 instruction does the same
// IEEE round-to-nearest operation on two independent values (here the left
// and right states of a face), halving the issue slots of symmetric code.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Reciprocals of N (<= 3) pressures with one division:
// 1/P_k = prod_{j != k} P_j / prod_j P_j (products stay far from overflow).
template <int N, typename R>
__device__ __forceinline__ void recips(const R* P, R* iP)
{
    if (N == 1) { iP[0] = frcp(P[0]); return; }
    R pre[N], acc = R(1);
#pragma unroll
    for (int k = 0; k < N; ++k) { pre[k] = acc; acc *= P[k]; }
    R inv = frcp(acc), suf = R(1);
#pragma unroll
    for (int k = N - 1; k >= 0; --k) { iP[k] = pre[k] * suf * inv; suf *= P[k]; }
}


// ------------------------------------------------------- Peng-Robinson
constexpr double PR_RU = 8.314462618;
constexpr double SQRT2 = 1.4142135623730951;

template <int NC, typename F = double>
struct PRMix {
    F X[NC], M, iM, b, cvig;   // mole fractions, molar mass and its reciprocal, covolume, ideal-gas cv
};

// PR constants in the working precision
template <typename F> __device__ __forceinline__ const PRConstT<F>& prk(const DevParams& P);
template <> __device__ __forceinline__ const PRConstT<double>& prk<double>(const DevParams& P) { return P.prc; }
template <> __device__ __forceinline__ const PRConstT<float>& prk<float>(const DevParams& P) { return P.prcf; }

// math of the working precision (the CUDA library functions of each type)
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_cbrt(double x) { return cbrt(x); }
__device__ __forceinline__ float m_cbrt(float x) { return cbrtf(x); }
__device__ __forceinline__ double m_acos(double x) { return acos(x); }
__device__ __forceinline__ float m_acos(float x) { return acosf(x); }
__device__ __forceinline__ double m_cos(double x) { return cos(x); }
__device__ __forceinline__ float m_cos(float x) { return cosf(x); }

template <int NC, typename F = double>
__device__ __forceinline__ void pr_mix(const DevParams& P, const F* Y, PRMix<NC, F>& m)
{
    const PRConstT<F>& K = prk<F>(P);
    F s = F(0), cv = F(0);
#pragma unroll
    for (int k = 0; k < NC; ++k) { s += Y[k] * K.iM[k]; cv += Y[k] * K.cv[k]; }
    m.M = F(1) / s;
    m.iM = s;
    m.cvig = cv;
    m.b = F(0);
#pragma unroll
    for (int k = 0; k < NC; ++k) { m.X[k] = Y[k] * K.iM[k] * m.M; m.b += m.X[k] * K.b[k]; }
}

// a(T) = sum_ab X_a X_b A_ab (1 + c_ab (1 - sqrt(T/Tc_ab)))^2 and its first two T derivatives
template <int NC, typename F = double>
__device__ __forceinline__ void pr_a(const DevParams& P, const PRMix<NC, F>& m, F T, F& a, F& da, F& d2a)
{
    const PRConstT<F>& K = prk<F>(P);
    const F isT = rsq(T), sT = T * isT, iT = isT * isT;
    a = da = d2a = F(0);
#pragma unroll
    for (int i = 0; i < NC; ++i)
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            const F xx = m.X[i] * m.X[j], A = K.A[i][j], c = K.cc[i][j], iq = K.isqTc[i][j];
            const F g = F(1) + c * (F(1) - sT * iq);
            a += xx * A * g * g;
            da -= xx * A * c * g * iq * isT;
            d2a += xx * F(0.5) * A * c * iT * iq * (c * iq + g * isT);
        }
}

template <typename F> __device__ __forceinline__ F pr_cubic(F c2, F c1, F c0, F Z) { return ((Z + c2) * Z + c1) * Z + c0; }

// log((v + (1 - sqrt2) b) / (v + (1 + sqrt2) b)): as written in FP64; in FP32
// as log1p(-2 sqrt2 b / (v + (1 + sqrt2) b)), the same value without the
// cancellation of a ratio near 1 (gas-like states, v >> b)
__device__ __forceinline__ double pr_logratio(double v, double b)
{
    return log((v + (1.0 - SQRT2) * b) / (v + (1.0 + SQRT2) * b));
}
__device__ __forceinline__ float pr_logratio(float v, float b)
{
    return log1pf(-2.0f * float(SQRT2) * b / (v + (1.0f + float(SQRT2)) * b));
}

// Gibbs-energy departure of root Z (up to terms common to all roots)
__device__ __forceinline__ double pr_gdep(double Z, double A, double B)
{
    return Z - 1.0 - log(Z - B) - A / (2.0 * SQRT2 * B) * log((Z + (1.0 + SQRT2) * B) / (Z + (1.0 - SQRT2) * B));
}
__device__ __forceinline__ float pr_gdep(float Z, float A, float B)
{
    const float s2 = float(SQRT2);
    return Z - 1.0f - logf(Z - B) - A / (2.0f * s2 * B) * log1pf(2.0f * s2 * B / (Z + (1.0f - s2) * B));
}

// TDU with the PR closure: (p, T, Y) -> rho, e, c.  Roots of the cubic in Z
// in closed form (Cardano / trigonometric), polished by Newton; of several
// roots above B the one of lowest Gibbs energy is taken.  FP64, or FP32 for
// the mixed form's face states (the App. B Newton inversion stays FP64).
template <int NC, typename F = double>
__device__ __forceinline__ bool pr_tdu(const DevParams& P, F p, F T, const F* Y, F& rho, F& e, F& c)
{
    if (!(T > F(0)) || !(p > F(0))) return false;
    PRMix<NC, F> m;
    pr_mix<NC, F>(P, Y, m);
    F a, da, d2a;
    pr_a<NC, F>(P, m, T, a, da, d2a);
    // (divisions cost several instructions each, on the FP64 pipe in the
    // FP64 form: constant ones are products, and the others share
    // reciprocals where the formulas allow)
    const F RU = F(PR_RU);
    const F RT = RU * T, iRT = F(1) / RT;
    const F A = a * p * iRT * iRT, B = m.b * p * iRT;
    const F third = F(1.0 / 3.0), i27 = F(1.0 / 27.0);
    const F c2 = -(F(1) - B), c1 = A - F(3) * B * B - F(2) * B, c0 = -(A * B - B * B - B * B * B);
    const F sh = c2 * third;
    const F pp = c1 - c2 * sh;
    const F qq = (F(2) * i27) * c2 * c2 * c2 - c2 * c1 * third + c0;
    const F D = F(0.25) * qq * qq + pp * pp * pp * i27;
    F Z[3];
    int nr;
    if (D > F(0)) {
        const F sD = sq_rt(D);
        Z[0] = m_cbrt(F(-0.5) * qq + sD) + m_cbrt(F(-0.5) * qq - sD) - sh;
        nr = 1;
    } else {
        const F r = sq_rt(fmax(-pp * third, F(0)));
        const F cosphi = (r > F(0)) ? fmin(F(1), fmax(F(-1), F(-0.5) * qq / (r * r * r))) : F(1);
        const F phi = m_acos(cosphi);
        const F tpi = F(2) * F(3.141592653589793);
        Z[0] = F(2) * r * m_cos(phi * third) - sh;
        Z[1] = F(2) * r * m_cos((phi - tpi) * third) - sh;
        Z[2] = F(2) * r * m_cos((phi + tpi) * third) - sh;
        nr = 3;
    }
    F best = F(-1), gbest = F(sizeof(F) == 8 ? 1e300 : 1e30);
    for (int i = 0; i < nr; ++i) {
        F z = Z[i];
#pragma unroll
        for (int it = 0; it < 2; ++it) {
            const F f = pr_cubic(c2, c1, c0, z), df = (F(3) * z + F(2) * c2) * z + c1;
            if (df != F(0)) z -= f / df;
        }
        if (!(z > B)) continue;
        const F g = (nr == 1) ? F(0) : pr_gdep(z, A, B);
        if (g < gbest) { gbest = g; best = z; }
    }
    if (!(best > B)) return false;
    const F v = best * RT / p, iv = F(1) / v;
    const F c2k = F(2) * F(SQRT2) * m.b * m.M;
    F k2;
    if constexpr (sizeof(F) == 8) {
        // log((v + (1 - sqrt2) b) / den) and k2 = L / c2k over one reciprocal
        const F den = v + (F(1) + F(SQRT2)) * m.b, r = F(1) / (den * c2k);
        k2 = log((v + (F(1) - F(SQRT2)) * m.b) * (c2k * r)) * (den * r);
    } else {
        k2 = pr_logratio(v, m.b) / c2k;
    }
    rho = m.M * iv;
    e = m.cvig * T + (a - T * da) * k2;
    const F cv = m.cvig - T * d2a * k2;
    const F dd = v * v + F(2) * m.b * v - m.b * m.b;
    const F i1 = F(1) / (v - m.b), i2 = F(1) / dd;
    const F dpdT = RU * i1 - da * i2;
    const F dpdv = -RT * i1 * i1 + a * (F(2) * v + F(2) * m.b) * i2 * i2;
    // v^2 / M and 1 / rho^2 = v^2 / M^2 from 1 / M
    const F v2iM = v * v * m.iM;
    const F c2s = -v2iM * dpdv + T * dpdT * dpdT * (v2iM * m.iM) / cv;
    c = sq_rt(c2s);
    return c2s > F(0) && cv > F(0);
}

// Primitive recovery with the PR closure (App. B): Newton on T for
// e(T, v) = e at fixed molar volume v = M/rho, started from the previous T
// (T0; an ideal-gas estimate when T0 is not usable), steps limited to a
// factor 5, at most 50 iterations; then p explicit from Eq. A.2.1.  Newton
// converges quadratically, so once a step is below 3e-7 T the next one would
// be below ~1e-13 T: the iteration stops there, and a(T) at the new T is the
// first-order Taylor value a + a' dT (second-order term ~(dT/T)^2 ~ 1e-13).
template <int NC>
__device__ __forceinline__ int pr_invert(const DevParams& P, double rho, double e, const double* Y, double T0,
                                         double& p, double& T, double irho)
{
    // divisions on the FP64 pipe cost several instructions each: 1/rho comes
    // from the caller, and the log ratio and k2 share one reciprocal
    PRMix<NC> m;
    pr_mix<NC>(P, Y, m);
    const double v = m.M * irho;
    if (!(v > m.b) || !isfinite(e)) return ERR_NONPHYS;
    const double den = v + (1.0 + SQRT2) * m.b, c2 = 2.0 * SQRT2 * m.b * m.M;
    const double r = 1.0 / (den * c2);
    const double L = log((v + (1.0 - SQRT2) * m.b) * (c2 * r));
    const double k2 = L * (den * r);
    double t = (T0 > 1.0 && T0 < 1e5) ? T0 : (e > 0.0 ? e / m.cvig : 300.0);
    double a, da, d2a;
    bool conv = false;
    for (int it = 0; it < 50; ++it) {
        pr_a<NC>(P, m, t, a, da, d2a);
        const double f = m.cvig * t + (a - t * da) * k2 - e;
        const double df = m.cvig - t * d2a * k2;
        double tn = t - f / df;
        tn = fmin(fmax(tn, 0.2 * t), 5.0 * t);
        const double dt = tn - t;
        if (fabs(dt) <= 3e-7 * t) {
            a += da * dt;
            t = tn;
            conv = true;
            break;
        }
        t = tn;
    }
    T = t;
    if (!conv) pr_a<NC>(P, m, t, a, da, d2a);
    // RU t / (v - b) - a / (v^2 + 2 b v - b^2) over one division
    const double d1 = v - m.b, d2 = v * v + 2.0 * m.b * v - m.b * m.b;
    p = (PR_RU * t * d2 - a * d1) / (d1 * d2);
    if (!conv) return ERR_NONCONV;
    return isfinite(p) ? 0 : ERR_NONPHYS;
}

// FP32 Newton on the same residual as pr_invert, from T0 to |dT| <= 1e-6 T
// (at most 8 steps): the starting temperature of the FP64 Newton in the
// mixed form, which then usually stops after one step.  Returns T0 when a
// step leaves the physical range.
template <int NC>
__device__ __forceinline__ float pr_predict_T(const DevParams& P, float rho, float e, const float* Y, float T0)
{
    PRMix<NC, float> m;
    pr_mix<NC, float>(P, Y, m);
    const float v = m.M / rho;
    if (!(v > m.b) || !(T0 > 1.0f && T0 < 1e5f)) return T0;
    const float k2 = pr_logratio(v, m.b) / (2.0f * float(SQRT2) * m.b * m.M);
    float t = T0;
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {
        float a, da, d2a;
        pr_a<NC, float>(P, m, t, a, da, d2a);
        const float f = m.cvig * t + (a - t * da) * k2 - e;
        const float df = m.cvig - t * d2a * k2;
        float tn = t - fdiv(f, df);
        tn = fminf(fmaxf(tn, 0.2f * t), 5.0f * t);
        if (!(tn > 1.0f && tn < 1e5f)) return T0;
        const bool done = fabsf(tn - t) <= 1e-6f * t;
        t = tn;
        if (done) break;
    }
    return t;
}

// ------------------------------------------------------------ closure
// Thermodynamic-dependent update (Eq. 3-5/3-6, App. B): from the face
// pressure offset pp = p - p_ref, temperature T and the NC-1 tracked mass
// fractions, the stiffened-gas / ideal-gas mixture in p-T equilibrium
// (App. A.1) gives
//   1/rho = T sum_k Y_k (gamma_k-1) cv_k / (p + pinf_k)
//   e     = cp T - p / rho + sum_k Y_k q_k,     cp = sum_k Y_k gamma_k cv_k
//   1/(rho c^2) = sum_k alpha_k / (gamma_k (p + pinf_k))   (Wood)
// Returns false for a non-physical input (T <= 0, p + pinf_k <= 0 for a
// present component, NaN).
template <int NC, typename R>
__device__ __forceinline__ bool baro_tdu(const DevParams& P, R pp, const R* Y, R& rho, R& c);

template <int NC, typename R, int CL>
__device__ __forceinline__ bool tdu(const DevParams& P, R pp, R T, const R* Yt, R& rho, R& e, R& c)
{
    R Y[NC], s = R(0);
#pragma unroll
    for (int k = 0; k < NC - 1; ++k) { Y[k] = clip01(Yt[k]); s += Y[k]; }
    Y[NC - 1] = clip01(R(1) - s);
    const ConstT<R>& Kc = K<R>(P);
    if constexpr (CL == CL_PR) {
        // the face state's PR closure in the working precision
        return pr_tdu<NC, R>(P, Kc.p_ref + pp, T, Y, rho, e, c);
    }
    if constexpr (CL == CL_BARO) {
        e = T;   // the energy is passive: the T slot carries e
        return baro_tdu<NC, R>(P, pp, Y, rho, c);
    }
    R Pk[NC], iP[NC];
    bool ok = T > R(0);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        Pk[k] = Kc.Pk[k] + pp;
        if (Y[k] > R(0)) ok = ok && (Pk[k] > R(0)); else Pk[k] = R(1);
    }
    recips<NC, R>(Pk, iP);
    R v = R(0), w = R(0), cp = R(0), eq = R(0);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        R a = Y[k] * Kc.gm1cv[k] * iP[k];
        v += a;
        w += a * iP[k] * Kc.igamma[k];
        cp += Y[k] * Kc.gcv[k];
        eq += Y[k] * Kc.q[k];
    }
    v *= T;
    w *= T;
    rho = frcp(v);
    e = cp * T - (Kc.p_ref + pp) * v + eq;
    c = v * rsq(w);
    return ok && (v > R(0)) && (w > R(0));
}

// The stiffened/ideal-gas TDU of tdu() for both sides of a face, stopped
// before its divisions: v = 1/rho, w = 1/(rho c)^2 (Wood), cp, eq per side,
// so that the flux takes rho c = w^{-1/2} for the impedances and one
// reciprocal and one energy for the upwind side only.  In FP64 the pressure
// reciprocals of both sides share one division (their product stays far
// below overflow; in FP32 each side keeps its own).
template <typename R> struct SGSide { R v, w, cp, eq; };

template <int NC, typename R>
__device__ __forceinline__ bool tdu_sg_pair(const DevParams& P, R ppL, R TL, const R* YtL, R ppR, R TR,
                                            const R* YtR, SGSide<R>& L, SGSide<R>& Rs)
{
    const ConstT<R>& Kc = K<R>(P);
    if constexpr (sizeof(R) == 4) {
        // both sides at once in packed pairs (.x left, .y right), the scalar
        // form's operations in its order
        float2 Y[NC], Pk[NC], iP[NC];
        float2 s = f2(0.0f);
#pragma unroll
        for (int k = 0; k < NC - 1; ++k) {
            Y[k] = f2(clip01(YtL[k]), clip01(YtR[k]));
            s = k == 0 ? Y[k] : add2(s, Y[k]);
        }
        Y[NC - 1] = f2(clip01(1.0f - s.x), clip01(1.0f - s.y));
        bool ok = TL > 0.0f && TR > 0.0f;
        const float2 pp = f2(ppL, ppR);
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            Pk[k] = add2(f2(Kc.Pk[k]), pp);
            if (Y[k].x > 0.0f) ok = ok && (Pk[k].x > 0.0f); else Pk[k].x = 1.0f;
            if (Y[k].y > 0.0f) ok = ok && (Pk[k].y > 0.0f); else Pk[k].y = 1.0f;
        }
        // 1/P_k = prod_{j != k} P_j / prod_j P_j, as recips() forms it
        if (NC == 1) {
            iP[0] = f2(frcp(Pk[0].x), frcp(Pk[0].y));
        } else {
            float2 pre[NC], acc = Pk[0];
#pragma unroll
            for (int k = 1; k < NC; ++k) { pre[k] = acc; acc = mul2(acc, Pk[k]); }
            const float2 inv = f2(frcp(acc.x), frcp(acc.y));
            float2 suf = Pk[NC - 1];
            iP[NC - 1] = mul2(pre[NC - 1], inv);
#pragma unroll
            for (int k = NC - 2; k >= 1; --k) { iP[k] = mul2(mul2(pre[k], suf), inv); suf = mul2(suf, Pk[k]); }
            iP[0] = mul2(suf, inv);
        }
        float2 v, w, cp, eq;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const float2 a = mul2(mul2(Y[k], f2(Kc.gm1cv[k])), iP[k]);
            if (k == 0) {
                v = a;
                w = mul2(mul2(a, iP[k]), f2(Kc.igamma[k]));
                cp = mul2(Y[k], f2(Kc.gcv[k]));
                eq = mul2(Y[k], f2(Kc.q[k]));
            } else {
                v = add2(v, a);
                w = fma2(mul2(a, iP[k]), f2(Kc.igamma[k]), w);
                cp = fma2(Y[k], f2(Kc.gcv[k]), cp);
                eq = fma2(Y[k], f2(Kc.q[k]), eq);
            }
        }
        const float2 T2 = f2(TL, TR);
        v = mul2(v, T2);
        w = mul2(w, T2);
        L.v = v.x; Rs.v = v.y;
        L.w = w.x; Rs.w = w.y;
        L.cp = cp.x; Rs.cp = cp.y;
        L.eq = eq.x; Rs.eq = eq.y;
        return ok && v.x > 0.0f && v.y > 0.0f && w.x > 0.0f && w.y > 0.0f;
    }
    R Y[2][NC], Pk[2 * NC], iP[2 * NC];
    const R pp[2] = {ppL, ppR}, T[2] = {TL, TR};
    const R* Yt[2] = {YtL, YtR};
    bool ok = gt0(TL) && gt0(TR);
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
        R s = R(0);
#pragma unroll
        for (int k = 0; k < NC - 1; ++k) { Y[sd][k] = clip01(Yt[sd][k]); s += Y[sd][k]; }
        Y[sd][NC - 1] = clip01(R(1) - s);
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            R& pk = Pk[sd * NC + k];
            pk = Kc.Pk[k] + pp[sd];
            if (gt0(Y[sd][k])) ok = ok && gt0(pk); else pk = R(1);
        }
    }
    if constexpr (sizeof(R) == 8) {
        recips<2 * NC, R>(Pk, iP);
    } else {
        recips<NC, R>(Pk, iP);
        recips<NC, R>(Pk + NC, iP + NC);
    }
    SGSide<R>* out[2] = {&L, &Rs};
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
        R v = R(0), w = R(0), cp = R(0), eq = R(0);
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const R a = Y[sd][k] * Kc.gm1cv[k] * iP[sd * NC + k];
            v += a;
            w += a * iP[sd * NC + k] * Kc.igamma[k];
            cp += Y[sd][k] * Kc.gcv[k];
            eq += Y[sd][k] * Kc.q[k];
        }
        out[sd]->v = v * T[sd];
        out[sd]->w = w * T[sd];
        out[sd]->cp = cp;
        out[sd]->eq = eq;
        ok = ok && gt0(out[sd]->v) && gt0(out[sd]->w);
    }
    return ok;
}

// Barotropic closure (Sec. 2.2) at the offset pressure pp = p - p_ref: the
// liquid-vapour phase density rho_LM = rho_sat,liq + (p - p_sat)/c^2 with
// c = c_L above p_sat (Eq. 2-3) and c_M^2 = p_sat/rho_sat,liq below (Eq. 2-4),
// gas densities p/(R T_ref) (Eq. 2-5); 1/rho = sum_k Y_k/rho_k and Wood's
// 1/(rho c^2) = rho sum_k Y_k/(rho_k^2 c_k^2), i.e. c = (1/rho)/sqrt(W) with
// W = Y_LM/(rho_LM^2 c_LM^2) + sum_gas Y_g R T_ref,g / p^2.
template <int NC, typename R>
__device__ __forceinline__ bool baro_tdu(const DevParams& P, R pp, const R* Y, R& rho, R& c)
{
    const ConstT<R>& Kc = K<R>(P);
    const R p = Kc.p_ref + pp;
    const R ic2 = (pp >= Kc.b_pso) ? Kc.b_icl2 : Kc.b_icm2;
    const R rlm = Kc.b_rsl + (pp - Kc.b_pso) * ic2;
    // 1/p and 1/rho_LM over one reciprocal (1 for a liquid-free state, where
    // rho_LM is not used)
    const R irp = frcp(p * rlm);
    const R ip = rlm * irp, ir = p * irp;
    R v = R(0), w = R(0);
    bool ok = gt0(p);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        if (k == P.liquid) {
            if (gt0(Y[k])) {
                ok = ok && gt0(rlm);
                v += Y[k] * ir;
                w += Y[k] * ir * ir * ic2;
            }
        } else {
            const R a = Y[k] * Kc.brt[k] * ip;
            v += a;
            w += a * ip;
        }
    }
    rho = frcp(v);
    c = v * rsq(w);
    return ok && gt0(v) && gt0(w);
}

// Vapour volume fraction of Eq. 2-7 (vapour share of the liquid-vapour phase
// capped at 0.995), that phase's volume fraction alpha_LM = rho Y_LM / rho_LM
// and the gas volume fraction sum_g Y_g rho R T_g / p (Eq. 2-6), from rho, Y, pp
template <int NC, typename R>
__device__ __forceinline__ R baro_vapour(const DevParams& P, R pp, R rho, const R* Yt, R* alm_out = nullptr,
                                         R* ag_out = nullptr)
{
    const ConstT<R>& Kc = K<R>(P);
    R Y[NC], s = R(0);
#pragma unroll
    for (int k = 0; k < NC - 1; ++k) { Y[k] = clip01(Yt[k]); s += Y[k]; }
    Y[NC - 1] = clip01(R(1) - s);
    const R ic2 = (pp >= Kc.b_pso) ? Kc.b_icl2 : Kc.b_icm2;
    const R rlm = Kc.b_rsl + (pp - Kc.b_pso) * ic2;
    R YL = R(0), ag = R(0);
    const R ip = frcp(Kc.p_ref + pp);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        if (k == P.liquid) YL = Y[k];
        else ag += Y[k] * rho * Kc.brt[k] * ip;
    }
    const R alm = fdiv(rho * YL, rlm);
    if (alm_out) *alm_out = alm;
    if (ag_out) *ag_out = ag;
    if (rlm >= Kc.b_rsl) return R(0);
    const R sh = fmin(R(0.995), fdiv(Kc.b_rsl - rlm, Kc.b_rsl - Kc.b_rsv));
    return alm * sh;
}

// Sound speed of a face state whose density came from the liquid-vapour
// THINC (Sec. 3.4 Remark 2): gas fractions from (p, rho, Y), the liquid-vapour
// phase takes the rest; false when that leaves no positive volume or density.
template <int NC, typename R>
__device__ __forceinline__ bool baro_sound_rho(const DevParams& P, R pp, R rho, const R* Yt, R& c)
{
    const ConstT<R>& Kc = K<R>(P);
    R Y[NC], s = R(0);
#pragma unroll
    for (int k = 0; k < NC - 1; ++k) { Y[k] = clip01(Yt[k]); s += Y[k]; }
    Y[NC - 1] = clip01(R(1) - s);
    const R p = Kc.p_ref + pp;
    const R ip = frcp(p);
    R ag = R(0), inv = R(0);
#pragma unroll
    for (int k = 0; k < NC; ++k)
        if (k != P.liquid && Y[k] > R(0)) {
            const R a = Y[k] * rho * Kc.brt[k] * ip;
            ag += a;
            inv += a * ip;
        }
    const R alm = R(1) - ag;
    const R YL = Y[P.liquid];
    if (YL > R(0)) {
        if (!(alm > R(0))) return false;
        const R rlm = fdiv(YL * rho, alm);
        if (!(rlm > R(0))) return false;
        const R ic2 = (rlm >= Kc.b_rsl) ? Kc.b_icl2 : Kc.b_icm2;
        inv += fdiv(alm * ic2, rlm);
    }
    if (!(inv > R(0))) return false;
    c = rsq(rho * inv);
    return true;
}

// Primitive recovery (App. B "T = f(e, rho, xi), then p"): for the SG/IG
// mixture with at most two distinct pinf (classes A and B) the p-T
// equilibrium is the quadratic
//   cv p^2 + b p + c = 0,  b = sum_k Y_k cv_k (E_k + pinf_other(k)),
//                          c = sum_k Y_k cv_k pinf_other(k) E_k,
//   E_k = gamma_k pinf_k - (gamma_k - 1) rho e
// whose larger root is the physical one; with one class present the root is
// p = -sum_k Y_k cv_k E_k / cv.  Then T = (rho e' + p) / (rho cp).  The E_k
// carry the p + pinf cancellation and are formed in FP64 (or compensated
// FP32 in the mixed form).
// Outputs w = (u_0..u_{ND-1}, p - p_ref, T, Y_0..Y_{NC-2}).
template <int ND, int NC, typename R, int CL, typename Q>
__device__ __forceinline__ int prim_recover(const DevParams& P, const Q* qc, R* w, R& rho_out, R& T_out,
                                            R& p_abs, double T0)
{
    const R rr = qv<R>(qc[0]);
    rho_out = rr;
    const R irho = frcp(rr);
    R ke = R(0);
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        const R m = qv<R>(qc[1 + d]);
        w[d] = m * irho;
        ke += R(0.5) * m * w[d];
    }
    R Y[NC], s = R(0);
#pragma unroll
    for (int k = 0; k < NC - 1; ++k) {
        Y[k] = clip01(qv<R>(qc[ND + 2 + k]) * irho);
        s += Y[k];
        w[ND + 2 + k] = Y[k];
    }
    Y[NC - 1] = clip01(R(1) - s);
    if constexpr (CL == CL_BARO) {
        // barotropic (Sec. 2.2), FP64 in both forms: with A = rho sum_g Y_g R T_ref,g
        // and B = Y_LM rho, 1/rho = Y_LM/rho_LM(p) + sum Y_g R T_g / p becomes
        // (p - A)(d + k p) = B p, k = 1/c^2, d = rho_sat,liq - p_sat k: the liquid
        // branch's positive root if it is >= p_sat, else (d = 0 below p_sat)
        // p = A + B p_sat / rho_sat,liq.  The energy is passive (T slot = e).
        // (divisions on the FP64 pipe cost several instructions each: one
        // reciprocal of rho, the constant ones as products)
        const ConstT<double>& Kd = P.kd;
        const double rho = qv_d(qc[0]), irho = 1.0 / rho;
        double ked = 0.0;
#pragma unroll
        for (int d = 0; d < ND; ++d) { const double m = qv_d(qc[1 + d]); ked += 0.5 * m * m; }
        const double e = (qv_d(qc[ND + 1]) - ked * irho) * irho;
        double A = 0.0, B = 0.0;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            if (k == P.liquid) B = double(Y[k]) * rho;
            else A += double(Y[k]) * rho * Kd.brt[k];
        }
        const double psat = Kd.b_pso + P.p_ref;
        double pd = A;
        if (B > 0.0) {
            const double kk = Kd.b_icl2, dd = Kd.b_rsl - psat * kk;
            const double b = dd - A * kk - B;
            const double disc = sqrt(b * b + 4.0 * kk * A * dd);
            pd = (b < 0.0) ? (disc - b) * Kd.b_hcl2 : ((A > 0.0) ? 2.0 * A * dd / (b + disc) : 0.0);
            if (!(pd >= psat)) pd = A + B * psat * Kd.b_irsl;
        }
        w[ND] = R(pd - P.p_ref);
        w[ND + 1] = R(e);
        T_out = R(e);
        p_abs = R(pd);
        // rho > 0, 0 < pd < inf, e finite (on the bit patterns)
        const long long pb = dbits(pd);
        return (gt0(rho) && pb > 0 && pb < DINF && (dbits(e) & ~DSIGN) < DINF) ? 0 : ERR_NONPHYS;
    }
    if constexpr (CL == CL_PR) {
        // Peng-Robinson: FP64 Newton in both forms; the mixed form starts it
        // from an FP32 Newton's temperature (FP32 arithmetic for the steps
        // that only approach the root, FP64 for the last)
        const double rho = qv_d(qc[0]), irho = 1.0 / rho;
        double ked = 0.0;
#pragma unroll
        for (int d = 0; d < ND; ++d) { const double m = qv_d(qc[1 + d]); ked += 0.5 * m * m; }
        const double e = (qv_d(qc[ND + 1]) - ked * irho) * irho;
        double Yd[NC], pd = 0.0, Td = 0.0;
#pragma unroll
        for (int k = 0; k < NC; ++k) Yd[k] = double(Y[k]);
        double Ts = T0;
        if constexpr (sizeof(R) == 4) {
            if (rho > 0.0 && isfinite(e)) Ts = double(pr_predict_T<NC>(P, float(rho), float(e), Y, float(T0)));
        }
        const int st = (rho > 0.0) ? pr_invert<NC>(P, rho, e, Yd, Ts, pd, Td, irho) : ERR_NONPHYS;
        w[ND] = R(pd - P.p_ref);
        w[ND + 1] = R(Td);
        T_out = R(Td);
        p_abs = R(pd);
        return st;
    }
    const ConstT<R>& Kc = K<R>(P);
    R cv = R(0), cp = R(0), b = R(0), cc = R(0), se = R(0), eq = R(0);
    R sA = R(0), sB = R(0);
#pragma unroll
    for (int k = 0; k < NC; ++k) eq += Y[k] * Kc.q[k];
    // The quadratic is solved directly for the offset p' = p - p_ref (so the
    // FP32 form keeps p' to its own relative precision): with
    //   E'_k = gamma_k pinf_k + p_ref - (gamma_k - 1) rho e'   (cancellation-prone)
    // and Po_k = pinf_other(k) + p_ref,
    //   cv p'^2 + b' p' + c' = 0,  b' = sum Y_k cv_k (E'_k + Po_k),  c' = sum Y_k cv_k Po_k E'_k.
    R rhoe_r;     // rho e' in the working precision (for T)
    R Ek[NC];
    if constexpr (IsFF<Q>::value) {
        // float-float registers: E'_k in compensated FP32, no FP64 instruction
        float2 rhoe = ff_add_f(qc[ND + 1], -(ke + rr * eq));
        rhoe_r = rhoe.x + rhoe.y;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const float2 t = ff_mul(rhoe, make_float2(-Kc.gm1_hi[k], -Kc.gm1_lo[k]));
            const float2 E = ff_add(t, make_float2(Kc.gpi_hi[k], Kc.gpi_lo[k]));
            Ek[k] = E.x + E.y;
        }
    } else {
        // FP64 registers: the one FP64 operation per component
        const double rhoe = qv_d(qc[ND + 1]) - double(ke) - double(rr) * double(eq);
        rhoe_r = R(rhoe);
#pragma unroll
        for (int k = 0; k < NC; ++k)
            Ek[k] = R(fma(-(P.c[k].gamma - 1.0), rhoe, P.c[k].gamma * P.c[k].pinf + P.p_ref));
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const R Yc = Y[k] * Kc.cv[k];
        cv += Yc;
        cp += Y[k] * Kc.gcv[k];
        b += Yc * (Ek[k] + Kc.Po[k]);
        cc += Yc * (Kc.Po[k] * Ek[k]);
        se += Yc * Ek[k];
        if (gt0(Y[k])) { if (P.c[k].classA) sA += Y[k]; else sB += Y[k]; }
    }
    R pp, T;     // p - p_ref, temperature
    const bool one = P.single_class || !gt0(sA) || !gt0(sB);
    if constexpr (sizeof(R) == 8) {
        // FP64: p' = Np / Dp and T = (rho e' + p) / (rho cp) over one
        // reciprocal, 1 / (Dp rho cp) (divisions cost several FP64-pipe
        // instructions each)
        R Np, Dp;
        if (one) {
            Np = -se;
            Dp = cv;
        } else {
            const R disc = b * b - R(4) * cv * cc;
            const R sq = sq_rt(fmax(disc, R(0)));
            const bool bpos = dbits(b) >= 0;
            Np = bpos ? R(-2) * cc : sq - b;
            Dp = bpos ? b + sq : R(2) * cv;
        }
        const R rcp = rr * cp, r = frcp(Dp * rcp);
        pp = Np * rcp * r;
        T = ((rhoe_r + Kc.p_ref) * Dp + Np) * r;
    } else {
        if (one) {
            pp = fdiv(-se, cv);
        } else {
            const R disc = b * b - R(4) * cv * cc;
            const R sq = sq_rt(disc > R(0) ? disc : R(0));
            pp = (b >= R(0)) ? fdiv(R(-2) * cc, b + sq) : fdiv(sq - b, R(2) * cv);
        }
        T = fdiv(rhoe_r + (Kc.p_ref + pp), rr * cp);
    }
    const R p = Kc.p_ref + pp;
    w[ND] = pp;
    w[ND + 1] = T;
    T_out = T;
    p_abs = p;
    bool ok = gt0(rr) && gt0(T) && gt0(cv);
#pragma unroll
    for (int k = 0; k < NC; ++k)
        if (gt0(Y[k])) ok = ok && gt0(Kc.Pk[k] + pp);
    return ok ? 0 : ERR_NONPHYS;
}

// ---------------------------------------------------------- reconstruction
// Sec. 3.3 / Table 4.2 limited slope term  f(r) * den  with r = num / den,
// written without the division for Minmod and Koren.
template <typename R>
__device__ __forceinline__ R limited(int id, R num, R den)
{
    // FP32, branch-free, the same values as the min/max form below in fewer
    // instructions (in FP64, where these operations run on the FP64 pipe,
    // the branch-free forms were 20% slower).
    if constexpr (sizeof(R) == 4) {
        // Minmod: the median of num, den and 0 (four min/max operations)
        if (id == 0) return fminf(fmaxf(num, fminf(den, 0.0f)), fmaxf(den, 0.0f));
        if (id == 1) {
            // Koren in den's orientation: with s = sign(den), num' = s num and
            // |den|, the slope term is s max(0, min(2 num', (|den| + 2 num')/3,
            // 2 |den|)) (a num of the other sign makes the minimum negative)
            const int sd = __float_as_int(den) & int(0x80000000u);
            const float ad = fabsf(den), sn = __int_as_float(__float_as_int(num) ^ sd);
            const float m = fmaxf(0.0f, fminf(2.0f * sn, fminf((ad + 2.0f * sn) * (1.0f / 3.0f), 2.0f * ad)));
            return __int_as_float(__float_as_int(m) ^ sd);
        }
    }
    if constexpr (sizeof(R) == 8) {
        // FP64: the selections on the bit patterns (integer instructions,
        // which leave the FP64 pipe to the arithmetic).  Patterns of
        // non-negative doubles order like the values; a pattern that is
        // negative as a 64-bit integer is a negative double.
        constexpr long long SGN = (long long)0x8000000000000000ull;
        const long long bn = __double_as_longlong(num), bd = __double_as_longlong(den);
        if (id == 0) {
            // Minmod: the smaller magnitude with den's sign, 0 for opposite signs
            const long long an = bn & ~SGN, ad = bd & ~SGN;
            return (bn ^ bd) < 0 ? R(0) : __longlong_as_double((an < ad ? an : ad) | (bd & SGN));
        }
        if (id == 1) {
            // Koren in den's orientation (num' = sign(den) num): 0 unless
            // num' > 0, else 2 min(num', (|den| + 2 num')/6, |den|) -- the
            // halves of the three candidates, so the doubling is exact
            const long long sd = bd & SGN;
            const long long sn = bn ^ sd, ad = bd & ~SGN;
            if (sn <= 0) return R(0);
            const double h = fma(2.0, __longlong_as_double(sn), __longlong_as_double(ad)) * (1.0 / 6.0);
            long long m = sn < ad ? sn : ad;
            const long long hb = __double_as_longlong(h);
            m = hb < m ? hb : m;
            const double mm = __longlong_as_double(m);
            return __longlong_as_double(__double_as_longlong(mm + mm) ^ sd);
        }
    }
    if (den == R(0)) return R(0);
    switch (id) {
    case 0: {  // Minmod  max(0, min(1, r))
        if (den > R(0)) return fmax(R(0), fmin(den, num));
        return fmin(R(0), fmax(den, num));
    }
    case 1: {  // Koren  max(0, min(2, 2r, (1 + 2r)/3))
        const R t = (den + R(2) * num) * R(1.0 / 3.0);
        if (den > R(0)) return fmax(R(0), fmin(R(2) * den, fmin(R(2) * num, t)));
        return fmin(R(0), fmax(R(2) * den, fmax(R(2) * num, t)));
    }
    default: {
        const R r = fdiv(num, den);
        R f;
        switch (id) {
        case 2: f = (r + fabs(r)) / (R(1) + fabs(r)); break;                        // van Leer
        case 3: f = (r + r * r) / (R(1) + r * r); break;                            // van Albada
        case 4: f = fmax(R(0), fmin(R(1), R(4) * r)); break;                        // Chakravarthy
        case 5: f = fmax(R(0), fmin(R(2), fmin(R(2) * r, R(0.5) * (R(1) + r)))); break;  // MC
        case 6: f = fmax(R(0), fmax(fmin(R(1), R(2) * r), fmin(r, R(2)))); break;     // Superbee
        default: f = R(0);
        }
        return f * den;
    }
    }
}

// MUSCL face values of the face between cells x2 and x3 (stencil x1..x4).
template <typename R>
__device__ __forceinline__ void muscl(int id, R x1, R x2, R x3, R x4, R& L, R& Rv)
{
    const R dc = x3 - x2;
    L = x2 + R(0.5) * limited(id, dc, x2 - x1);
    Rv = x3 - R(0.5) * limited(id, dc, x4 - x3);
}

template <typename R>
__device__ __forceinline__ bool eligible(R eps, R xm, R x, R xp)
{
    if constexpr (sizeof(R) == 8) {
        const long long b = dbits(x), p = dbits((x - xm) * (xp - x));
        return b > dbits(eps) && b < dbits(R(1) - eps) && p > 0 && p <= DINF;
    }
    return (x > eps) && (x < R(1) - eps) && ((x - xm) * (xp - x) > R(0));
}

// THINC (Eq. 3-3 for the left state of the face between the centre cell xc
// and xn, from (xp, xc, xn); Eq. 3-4 is the same profile read at the
// centre cell's other face).  jump normalised by max - min + gamma.
template <typename R>
__device__ __forceinline__ R thinc_side(const DevParams& P, R xa, R xc, R xb, bool left)
{
    const R mn = fmin(xa, xb), mx = fmax(xa, xb);
    const R th = (xb >= xa) ? R(1) : R(-1);
    const ConstT<R>& Kc = K<R>(P);
    const R gam = Kc.thinc_gamma;
    const R F = fdiv(xc - mn + gam, mx - mn + gam);
    const R E = (ex(th * Kc.beta * (R(2) * F - R(1))) * Kc.icb - R(1)) * Kc.itb;
    const R tb = Kc.tb;
    const R t = left ? fdiv(tb + E, R(1) + E * tb) : E;
    return mn + R(0.5) * (mx - mn) * (R(1) + th * t);
}

// --------------------------------------------------------------- face flux
// One face between cells 1 and 2 of the stencil w[0..3] (cells i-1..i+2 along
// direction d).  ws[s][v]: primitives (u, p', T, Y); rc[s]: (rho, c) of the
// cells for the App. D impedances; f: App. D switch (1 in plain mode).
// F receives (rho, rho u_0.., rho E, rho Y..) fluxes.  In the mixed form the
// constant p_ref is left out of the normal-momentum flux (it cancels in every
// cell's flux difference).
// LIM: limiter pair fixed at compile time ((velocity id << 4) | scalar id), or
// LIM_RUNTIME to read it from the parameters.
constexpr int LIM_RUNTIME = -1;
constexpr int LIM_TABLE42 = (1 << 4) | 0;   // Koren for velocities, Minmod for p, T, Y (Table 4.2)

// av4: vapour fractions of the four cells (barotropic closure), else unused.
// SW: the App. D switch fixed at compile time (0 off, 1 on) or -1 to read it
// from the parameters.
// CJ = 1: capJ is the capillary pressure jump J = sigma kappa_f
// (alpha_i+1 - alpha_i) of the Sec. 3.5 jump model, added to the pressure
// difference of u*; the face's u* is returned in *us_out when given.
template <int ND, int NC, typename R, int CL, int LIM, int SW = -1, int CJ = 0>
__device__ __forceinline__ bool face_flux(const DevParams& P, int d, const R (*ws)[ND + NC + 1], const R* rho4,
                                          const R* c4, int f, R* F, const R* av4 = nullptr, R capJ = R(0),
                                          R* us_out = nullptr)
{
    constexpr int NW = ND + NC + 1;
    constexpr int IP = ND, IT = ND + 1, IY = ND + 2;
    R WL[NW], WR[NW];
    const bool iles = SW < 0 ? P.iles != 0 : SW == 1;
    const bool smooth = iles && !f;
    if (smooth) {
#pragma unroll
        for (int v = 0; v < NW; ++v) {
            // Eq. D.1 for u, p, T; the 2nd-order mean for Y and for the
            // barotropic closure's internal energy
            const bool fourth = (v < IY) && !(CL == CL_BARO && v == IT);
            const R cval = fourth ? (R(7) * (ws[1][v] + ws[2][v]) - ws[0][v] - ws[3][v]) * R(1.0 / 12.0)
                                  : R(0.5) * (ws[1][v] + ws[2][v]);
            WL[v] = WR[v] = cval;
        }
    } else {
#pragma unroll
        for (int v = 0; v < NW; ++v) {
            const int lim = LIM >= 0 ? ((v < ND) ? (LIM >> 4) : (LIM & 15)) : ((v < ND) ? P.lim_vel : P.lim_scalar);
            muscl(lim, ws[0][v], ws[1][v], ws[2][v], ws[3][v], WL[v], WR[v]);
            if (v >= IY && P.thinc) {
                const R eps = K<R>(P).thinc_eps;
                if (eligible(eps, ws[0][v], ws[1][v], ws[2][v])) WL[v] = thinc_side(P, ws[0][v], ws[1][v], ws[2][v], true);
                if (eligible(eps, ws[1][v], ws[2][v], ws[3][v])) WR[v] = thinc_side(P, ws[1][v], ws[2][v], ws[3][v], false);
            }
        }
    }
    R rL = R(0), eL = R(0), cL = R(0), rR = R(0), eR = R(0), cR = R(0);
    bool ok;
    [[maybe_unused]] SGSide<R> sL, sR;
    if constexpr (CL == CL_SG) {
        ok = tdu_sg_pair<NC, R>(P, WL[IP], WL[IT], WL + IY, WR[IP], WR[IT], WR + IY, sL, sR);
    } else {
        ok = tdu<NC, R, CL>(P, WL[IP], WL[IT], WL + IY, rL, eL, cL);
        ok = tdu<NC, R, CL>(P, WR[IP], WR[IT], WR + IY, rR, eR, cR) && ok;
    }
    if constexpr (CL == CL_BARO) {
        // Sec. 3.4 Remarks 1-2: THINC of the cell densities where the vapour
        // fraction is eligible and the densities are monotone (the profile
        // needs the centre value between its neighbours), then the sound
        // speed from (p*, rho*, Y*)
        if (P.thinc && !smooth) {
            const R eps = K<R>(P).thinc_eps;
            R cs;
            if (eligible(eps, av4[0], av4[1], av4[2]) && (rho4[1] - rho4[0]) * (rho4[2] - rho4[1]) > R(0)) {
                const R t = thinc_side(P, rho4[0], rho4[1], rho4[2], true);
                if (baro_sound_rho<NC, R>(P, WL[IP], t, WL + IY, cs)) { rL = t; cL = cs; }
            }
            if (eligible(eps, av4[1], av4[2], av4[3]) && (rho4[2] - rho4[1]) * (rho4[3] - rho4[2]) > R(0)) {
                const R t = thinc_side(P, rho4[1], rho4[2], rho4[3], false);
                if (baro_sound_rho<NC, R>(P, WR[IP], t, WR + IY, cs)) { rR = t; cR = cs; }
            }
        }
    }
    // normal velocities by select: indexing with the run-time d would put WL
    // and WR in local memory
    R uL = WL[0], uR = WR[0];
    if (ND > 1 && d == 1) { uL = WL[1]; uR = WR[1]; }
    if (ND > 2 && d == 2) { uL = WL[ND > 2 ? 2 : 0]; uR = WR[ND > 2 ? 2 : 0]; }
    const R pL = WL[IP], pR = WR[IP];
    // u* = N / D.  FP64 stiffened gas: one reciprocal 1/(D v_up) gives both
    // rho* u* = N / (D v_up) and u* = (rho* u*) v_up (D > 0, so the upwind
    // side is the sign of N); otherwise the division and the upwind density
    R us, ps, N, D;
    bool smooth_us = false;
    R d3 = R(0);
    if (iles) {
        const R cm = fmax(c4[1], c4[2]);
        const R IL = (R(3) * rho4[1] + rho4[2]) * cm * R(0.25);
        const R IR = (rho4[1] + R(3) * rho4[2]) * cm * R(0.25);
        D = IL + IR;
        if (f) {
            N = CJ ? IL * uL + IR * uR + pL - pR + capJ : IL * uL + IR * uR + pL - pR;
            ps = R(0.5) * (pL + pR);
        } else {
            d3 = K<R>(P).d3p_coef * (ws[0][IP] - R(3) * ws[1][IP] + R(3) * ws[2][IP] - ws[3][IP]);
            if (CJ) d3 = d3 - capJ;
            N = uL * D - d3;
            smooth_us = true;
            ps = pL;
        }
    } else {
        ps = R(0.5) * (pL + pR);
        // impedances rho c: w^{-1/2} straight from the Wood sum (stiffened gas)
        R zL, zR;
        if constexpr (CL == CL_SG) { zL = rsq(sL.w); zR = rsq(sR.w); }
        else { zL = rL * cL; zR = rR * cR; }
        N = CJ ? zL * uL + zR * uR + pL - pR + capJ : zL * uL + zR * uR + pL - pR;
        D = zL + zR;
    }
    constexpr bool ONE_RCP = sizeof(R) == 8 && CL == CL_SG;
    if constexpr (!ONE_RCP) us = smooth_us ? uL - fdiv(d3, D) : fdiv(N, D);
    // upwind side (FP64: the sign bit; u* = -0 carries no mass, so either side gives the same flux)
    bool up;
    if constexpr (ONE_RCP) up = dbits(double(N)) >= 0;
    else up = sizeof(R) == 8 ? dbits(double(us)) >= 0 : us >= R(0);
    R Ws[NW];   // element-wise select keeps both sides in registers
#pragma unroll
    for (int v = 0; v < NW; ++v) Ws[v] = up ? WL[v] : WR[v];
    R rs, es, mflux;
    if constexpr (CL == CL_SG) {
        // density and internal energy of the upwind side only (as tdu() forms them)
        const R v_ = up ? sL.v : sR.v, cp_ = up ? sL.cp : sR.cp, eq_ = up ? sL.eq : sR.eq;
        if constexpr (ONE_RCP) {
            mflux = N * frcp(D * v_);
            us = mflux * v_;
        } else {
            rs = frcp(v_);
            mflux = us * rs;
        }
        es = cp_ * Ws[IT] - (K<R>(P).p_ref + Ws[IP]) * v_ + eq_;
    } else {
        rs = up ? rL : rR;
        es = up ? eL : eR;
        mflux = us * rs;
    }
    if (us_out) *us_out = us;
    R ke = R(0);
#pragma unroll
    for (int a = 0; a < ND; ++a) ke += R(0.5) * Ws[a] * Ws[a];
    F[0] = mflux;
#pragma unroll
    for (int a = 0; a < ND; ++a) F[1 + a] = mflux * Ws[a] + (a == d ? ps : R(0));
    F[1 + ND] = mflux * (es + ke) + (K<R>(P).p_ref + ps) * us;
#pragma unroll
    for (int k = 0; k < NC - 1; ++k) F[2 + ND + k] = mflux * Ws[IY + k];
    return ok;
}

}  // namespace tfv
