// Device-side building blocks of libxs: physical constants, the Faddeeva
// function w(z) = exp(-z^2) erfc(-iz) by tiers (Sec. 2.1.1), and small helpers.
//
// Faddeeva tiers.  H = Re w is needed to a relative accuracy of ~1e-7 (FP32) or
// ~1e-15 (FP64) everywhere, including the Gaussian-to-Lorentzian transition at
// small a where Re w is far smaller than |w|.  Each tier keeps the real part free
// of cancellation:
//   * |z| large: the asymptotic series of Eq. asywofz,
//       w ~ i/(sqrt(pi) z) * (1 + sum_{k>=1} (2k-1)!! (1/(2 z^2))^k),
//     truncated at K terms chosen per |z| band (bands measured against an
//     arbitrary-precision reference); with z = x + ia and 1/z = (x - ia)/|z|^2
//     the real part is (a Re p - x Im p)/(sqrt(pi)|z|^2) with both terms of one
//     sign, so it keeps its relative accuracy as a -> 0.
//   * |z| small: the exponentially convergent series behind Eq. algo916 /
//     algo916L (Zaghloul & Ali 2011).  Written with E_n^-+ = exp(-(nh -+ x)^2):
//       Re w = e^{-x^2} [K(a) cos 2ax + (2h/pi) sin(ax) sin(ax)/a] + (a h/pi) Sc
//       Im w = e^{-x^2} [-K(a) sin 2ax + (h/pi) sin(2ax)/a]       + (h/pi) Ss
//       Sc = sum_n (E_n^- + E_n^+)/(n^2h^2 + a^2),  Ss = sum_n nh (E_n^- - E_n^+)/(n^2h^2 + a^2)
//       K(a) = erfcx(a) - (2ah/pi) sum_n e^{-n^2h^2}/(n^2h^2 + a^2)   (per line, precomputed)
//     Every E_n is taken directly from its own small exponent (no recurrence
//     through e^{-x^2} e^{2nhx}, which would lose digits); only the n near x/h
//     (and, for small x, the first E_n^+) are summed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace xsd {

// CODATA 2018 (cgs) and the second radiation constant c2 as printed in Sec. 2.2.
constexpr double kB = 1.380649e-16;
constexpr double hP = 6.62607015e-27;
constexpr double cL = 2.99792458e10;
constexpr double amu = 1.66053906660e-24;
constexpr double c2 = 1.4387773;
constexpr double Tref = 296.0;
constexpr double bar_per_atm = 1.01325;
constexpr double PI = 3.14159265358979323846;
constexpr double SQRTPI = 1.77245385090551602730;
constexpr double INV_SQRTPI = 0.56418958354775628695;
constexpr double SQRT2 = 1.41421356237309504880;

// Scale applied to line strengths in the FP32 path so that partial sums of the
// cross-section (1e-35 .. 1e-12 cm^2) sit well inside the normal float range.
constexpr double MIXED_SCALE = 1208925819614629174706176.0; // 2^80
constexpr double MIXED_UNSCALE = 8.27180612553027674871e-25; // 2^-80

template <class R> struct vec4;
template <> struct vec4<float> { using type = float4; };
template <> struct vec4<double> { using type = double4_32a; };

// Per-precision Faddeeva tier table.
template <class R> struct Tier;
template <> struct Tier<float> {
    // The FP32 path evaluates w only through the wing forms (|z| >= 25, main
    // kernels), the polynomial in 1/|z|^2 (6 <= |z| < 25) and the series below
    // |z| = 6 (near kernels, w_series_tab); these are the series' parameters.
    static constexpr float z2_series = 64.0f;  // K(a) is precomputed for lines with a^2 below this
    static constexpr float h = 0.7f;           // series step (error ~1e-8 relative)
};
template <> struct Tier<double> {
    static constexpr double z2_fast = 1e300;   // no truncated fast form in double precision
    static constexpr double z2_fast_adj = 1e300;
    static constexpr double z2_far = 22500.0;  // |z| >= 150: K = 3
    static constexpr double z2_mid1 = 1600.0;  // |z| >= 40 : K = 5
    static constexpr double z2_mid2 = 100.0;   // |z| >= 10 : K = 12, below: series
    static constexpr double z2_series = 100.0;
    static constexpr int K1 = 3, K2 = 5, K3 = 12;
    static constexpr double h = 0.5;           // series step (error ~1e-17)
    static constexpr int nwin = 13;
    static constexpr double tcut = 6.5;
};

// Bounds-checked build (nvcc -DXS_CHECKED): index checks guard the kernels'
// global and shared accesses.  A failed check records its source line in this
// translation unit's device status word (the largest line wins) and the access is
// skipped, so a bad index never faults or traps; xs_check_status reads the words.
// In the normal build XS_CHECK(c) is the constant true and costs nothing.
#ifdef XS_CHECKED
static __device__ int g_xs_check_line = 0;
__device__ __forceinline__ bool xs_check(bool ok, int line)
{
    if (!ok) atomicMax(&g_xs_check_line, line);
    return ok;
}
#define XS_CHECK(c) ::xsd::xs_check((c), __LINE__)
// host accessor of this translation unit's word (read, then cleared if asked)
#define XS_CHECK_ACCESSOR(name)                                                                      \
    namespace xsi {                                                                                  \
    int check_status_##name(int clear)                                                               \
    {                                                                                                \
        int v = 0;                                                                                   \
        if (cudaMemcpyFromSymbol(&v, ::xsd::g_xs_check_line, sizeof(int)) != cudaSuccess) return -1; \
        if (clear) {                                                                                 \
            const int z = 0;                                                                         \
            if (cudaMemcpyToSymbol(::xsd::g_xs_check_line, &z, sizeof(int)) != cudaSuccess) return -1; \
        }                                                                                            \
        return v;                                                                                    \
    }                                                                                                \
    }
#else
#define XS_CHECK(c) true
#define XS_CHECK_ACCESSOR(name)                 \
    namespace xsi {                             \
    int check_status_##name(int) { return 0; } \
    }
#endif

__device__ __forceinline__ float rcp_fast(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp_fast(double x) { return 1.0 / x; }

// x = |d| c with d = dh + dl and c = ch + cl as unevaluated float pairs:
// returns x as a pair (xh, xl), xh = fl(|dh| ch).
__device__ __forceinline__ void scaled_pair(float dh, float dl, float ch, float cl, float* xh, float* xl)
{
    // renormalise d = dh + dl first (Fast2Sum, |dl| << |dh| or both tiny) so that
    // xh, which the asymptotic tiers use alone, carries all of d's leading bits
    float d = dh + dl;
    float e = (dh - d) + dl;
    float sgn = (d < 0.0f) ? -1.0f : 1.0f;
    d *= sgn;
    e *= sgn;
    float p = d * ch;
    *xh = p;
    *xl = fmaf(d, ch, -p) + fmaf(d, cl, e * ch);
}
__device__ __forceinline__ void scaled_pair(double dh, double, double ch, double, double* xh, double* xl)
{
    *xh = fabs(dh) * ch;
    *xl = 0.0;
}

__device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ int round_int(float v) { return __float2int_rn(v); }
__device__ __forceinline__ int round_int(double v) { return __double2int_rn(v); }

// accurate expf (a few ulp): the small-|z| tier is rare, and its exponent can reach ~40
__device__ __forceinline__ float exp_neg(float t2) { return expf(-t2); }
__device__ __forceinline__ double exp_neg(double t2) { return exp(-t2); }

__device__ __forceinline__ void sincos_r(float v, float* s, float* c) { sincosf(v, s, c); }
__device__ __forceinline__ void sincos_r(double v, double* s, double* c) { sincos(v, s, c); }
__device__ __forceinline__ float sin_r(float v) { return sinf(v); }
__device__ __forceinline__ double sin_r(double v) { return sin(v); }

// exp(-x^2) with x^2 split into hi + lo so the rounding of x*x does not enter.
__device__ __forceinline__ float exp_negsq(float x)
{
    float hi = x * x;
    float lo = fmaf(x, x, -hi);
    return expf(-hi) * (1.0f - lo);
}
__device__ __forceinline__ double exp_negsq(double x)
{
    double hi = x * x;
    double lo = fma(x, x, -hi);
    return exp(-hi) * (1.0 - lo);
}

// Asymptotic series (Eq. asywofz) with K correction terms; x >= 0, a >= 0,
// r = 1/(x^2 + a^2).  Returns w.
template <class R, int K>
__device__ __forceinline__ void w_asym(R x, R a, R r, R* wr, R* wi)
{
    // u = 1/(2 z^2) = conj(z)^2 r^2 / 2
    R hr2 = R(0.5) * r * r;
    R ur = (x - a) * (x + a) * hr2;
    R ui = R(-2) * a * x * hr2;
    R pr = R(1), pi = R(0);
#pragma unroll
    for (int k = K; k >= 1; --k) {
        R c = R(2 * k - 1);
        R tr = ur * pr - ui * pi;
        R ti = ur * pi + ui * pr;
        pr = R(1) + c * tr;
        pi = c * ti;
    }
    R s = r * R(INV_SQRTPI);
    *wr = (a * pr - x * pi) * s;
    *wi = (x * pr + a * pi) * s;
}

// Asymptotic series of w'(z) = dw/dz:  w' ~ -(2 i u / sqrt(pi)) (1 + sum_k (2k+1)!! u^k).
template <class R, int K>
__device__ __forceinline__ void dw_asym(R x, R a, R r, R* dr, R* di)
{
    R hr2 = R(0.5) * r * r;
    R ur = (x - a) * (x + a) * hr2;
    R ui = R(-2) * a * x * hr2;
    R pr = R(1), pi = R(0);
#pragma unroll
    for (int k = K; k >= 1; --k) {
        R c = R(2 * k + 1);
        R tr = ur * pr - ui * pi;
        R ti = ur * pi + ui * pr;
        pr = R(1) + c * tr;
        pi = c * ti;
    }
    // q = u p ; w' = -(2i/sqrt(pi)) q = (2/sqrt(pi)) (Im q - i Re q)
    R qr = ur * pr - ui * pi;
    R qi = ur * pi + ui * pr;
    *dr = R(2 * INV_SQRTPI) * qi;
    *di = R(-2 * INV_SQRTPI) * qr;
}

// Small-|z| series; x = xh + xl >= 0 (xl a small correction carrying the bits
// of x a single float cannot: exp(-x^2) has condition number 2x^2 in x),
// a >= 0, Kc = K(a) for this precision's step h.
template <class R>
__device__ __forceinline__ void w_series(R xh, R xl, R a, R Kc, R* wr, R* wi)
{
    const R x = xh;
    const R h = Tier<R>::h;
    const int nwin = Tier<R>::nwin;
    R sc = R(0), ss = R(0);
    int n0 = round_int(x / h);
    R a2 = a * a;
#pragma unroll 1
    for (int k = -nwin; k <= nwin; ++k) {
        int n = n0 + k;
        if (n < 1) continue;
        R nh = R(n) * h;
        R t = (nh - xh) - xl;
        R e = exp_neg(t * t);
        R d = rcp_fast(fma(nh, nh, a2));
        sc = fma(d, e, sc);
        ss = fma(nh * d, e, ss);
    }
#pragma unroll 1
    for (int n = 1; n <= 64; ++n) { // bounded even for non-finite x
        R nh = R(n) * h;
        R t = (nh + xh) + xl;
        if (!(t < Tier<R>::tcut)) break;
        R e = exp_neg(t * t);
        R d = rcp_fast(fma(nh, nh, a2));
        sc = fma(d, e, sc);
        ss = fma(-nh * d, e, ss);
    }
    R ex = exp_negsq(xh) * (R(1) - R(2) * xh * xl);
    R s2, c2v;
    sincos_r(R(2) * a * x, &s2, &c2v);
    R sax = sin_r(a * x);
    R sax_a = (a > R(0)) ? sax / a : x;
    R s2_a = (a > R(0)) ? s2 / a : R(2) * x;
    const R hpi = h * R(1.0 / PI);
    *wr = ex * (Kc * c2v + R(2) * hpi * sax * sax_a) + a * hpi * sc;
    *wi = ex * (-Kc * s2 + hpi * s2_a) + hpi * ss;
}

// Per-line table for w_series_tab (near kernels, |z| < 6 so n0 = round(x/h) <= 9):
// d[n + SER_OFF] = 1/(n^2 h^2 + a^2) for n = 1 .. SER_TAB - 1 - SER_OFF, and 0 for
// n <= 0 (terms that do not exist).
constexpr int SER_OFF = 6;  // n0 - 6 >= -6
constexpr int SER_TAB = 22; // n up to 9 + 6 = 15

__device__ __forceinline__ void series_table(float a, float* d)
{
    const float h = Tier<float>::h;
    const float a2 = a * a;
#pragma unroll 2
    for (int i = 0; i < SER_TAB; ++i) {
        const int n = i - SER_OFF;
        const float nh = (float)n * h;
        d[i] = (n >= 1) ? rcp_fast(fmaf(nh, nh, a2)) : 0.0f;
    }
}

// FP32 small-|z| series (near kernels, 0 <= x < 6.3) with the E_n^- taken by a
// two-way recurrence from the term nearest the peak, n0 = round(x/h), where
// t = n0 h - x = delta is small:
//   E_{n0+k} = E_{n0+k-1} e^{-2h delta} q^{2k-1},  E_{n0-k} = E_{n0-k+1} e^{+2h delta} q^{2k-1},
//   q = e^{-h^2};
// every factor has a small exponent, so no digits are lost to e^{-x^2} e^{2nhx}.
// E_n^+ = E_n^- e^{-4nhx} rides along.  Terms with |k| > 6 are below 1e-9 of the
// peak term.  The terms above and below the peak go as packed pairs, with the
// line's table of 1/(n^2 h^2 + a^2) (series_table).
__device__ __forceinline__ void w_series_tab(float xh, float xl, float a, float Kc, const float* dt, float* wr,
                                             float* wi)
{
    const float h = Tier<float>::h;
    // q^(2k-1), q = exp(-h^2) with h = 0.7f
    const float Q[6] = {0.61262643f, 0.22992550f, 0.08629359f, 0.03238694f, 0.012155180f, 0.0045619742f};
    const float x = xh;
    const int n0 = __float2int_rn(x * (1.0f / h));
    const float n0h = (float)n0 * h;
    const float delta = (n0h - xh) - xl;
    const float E0 = __expf(-delta * delta);
    const float2 f = make_float2(__expf(-2.0f * h * delta), __expf(2.0f * h * delta));
    const float R4 = __expf(-4.0f * h * x);
    const float2 g = make_float2(R4, rcp_fast(R4));
    const float Rn = __expf(-4.0f * h * x * (float)n0);
    if (!XS_CHECK(n0 >= 0 && n0 + 2 * SER_OFF < SER_TAB)) { // |z| < 6 keeps n0 <= 9
        *wr = 0.0f;
        *wi = 0.0f;
        return;
    }
    const float* d0 = dt + (n0 + SER_OFF);
    // centre term (d0[0] = 0 when n0 = 0)
    const float ep0 = E0 * Rn;
    const float dc = d0[0];
    float2 sc = make_float2(dc * (E0 + ep0), 0.0f);
    float2 ss = make_float2(n0h * dc * (E0 - ep0), 0.0f);
    float2 E = make_float2(E0, E0), R = make_float2(Rn, Rn), nh = make_float2(n0h, n0h);
    const float2 hstep = make_float2(h, -h);
#pragma unroll
    for (int k = 1; k <= 6; ++k) {
        E = __fmul2_rn(__fmul2_rn(E, f), make_float2(Q[k - 1], Q[k - 1])); // (E_{n0+k}, E_{n0-k})
        R = __fmul2_rn(R, g);
        nh = __fadd2_rn(nh, hstep);
        const float2 ep = __fmul2_rn(E, R);
        const float2 dd = make_float2(d0[k], d0[-k]);
        sc = __ffma2_rn(dd, __fadd2_rn(E, ep), sc);
        ss = __ffma2_rn(__fmul2_rn(nh, dd), __fadd2_rn(E, make_float2(-ep.x, -ep.y)), ss);
    }
    const float scs = sc.x + sc.y, sss = ss.x + ss.y;
    const float ex = exp_negsq(xh) * (1.0f - 2.0f * xh * xl);
    float sax, cax;
    sincosf(a * x, &sax, &cax);
    const float c2v = 1.0f - 2.0f * sax * sax; // cos 2ax
    const float s2 = 2.0f * sax * cax;         // sin 2ax
    const float sax_a = (a > 0.0f) ? sax * rcp_fast(a) : x;
    const float s2_a = 2.0f * sax_a * cax;
    const float hpi = h * (float)(1.0 / PI);
    *wr = ex * (Kc * c2v + 2.0f * hpi * sax * sax_a) + a * hpi * scs;
    *wi = ex * (-Kc * s2 + hpi * s2_a) + hpi * sss;
}

template <class R>
__device__ __forceinline__ void w_small(R x, R xl, R a, R Kc, const R*, R* wr, R* wi)
{
    w_series<R>(x, xl, a, Kc, wr, wi);
}

// w(x + ia) for any tier (the FP64 path); x = x + xl >= 0; dtab is not used.
template <class R>
__device__ __forceinline__ void faddeeva(R x, R xl, R a, R Kc, R* wr, R* wi, const R* dtab = nullptr)
{
    R z2 = fma(x, x, a * a);
    if (z2 >= Tier<R>::z2_mid2) {
        R r = rcp_fast(z2);
        if (z2 >= Tier<R>::z2_far)
            w_asym<R, Tier<R>::K1>(x, a, r, wr, wi);
        else if (z2 >= Tier<R>::z2_mid1)
            w_asym<R, Tier<R>::K2>(x, a, r, wr, wi);
        else
            w_asym<R, Tier<R>::K3>(x, a, r, wr, wi);
    } else {
        w_small<R>(x, xl, a, Kc, dtab, wr, wi);
    }
}

// w and w' for any tier; x = x + xl >= 0.
template <class R>
__device__ __forceinline__ void faddeeva_d(R x, R xl, R a, R Kc, R* wr, R* wi, R* dr, R* di, const R* dtab = nullptr)
{
    R z2 = fma(x, x, a * a);
    if (z2 >= Tier<R>::z2_mid2) {
        R r = rcp_fast(z2);
        if (z2 >= Tier<R>::z2_far) {
            w_asym<R, Tier<R>::K1>(x, a, r, wr, wi);
            dw_asym<R, Tier<R>::K1>(x, a, r, dr, di);
        } else if (z2 >= Tier<R>::z2_mid1) {
            w_asym<R, Tier<R>::K2>(x, a, r, wr, wi);
            dw_asym<R, Tier<R>::K2>(x, a, r, dr, di);
        } else {
            w_asym<R, Tier<R>::K3>(x, a, r, wr, wi);
            dw_asym<R, Tier<R>::K3>(x, a, r, dr, di);
        }
    } else {
        w_small<R>(x, xl, a, Kc, dtab, wr, wi);
        // w' = -2 z w + 2i/sqrt(pi)
        *dr = R(-2) * (x * *wr - a * *wi);
        *di = R(-2) * (x * *wi + a * *wr) + R(2 * INV_SQRTPI);
    }
}

// ------------------------------------------------------------------ wing polynomials
//
// The asymptotic series of Eq. asywofz, truncated after the term k = ASY_K, as a
// polynomial in u = 1/|z|^2 with per-line coefficients (FP32 near kernels,
// 6 <= |z| < 25).  Term k is c_k Re(i z^-(2k+1))/sqrt(pi) = c_k Im(z^(2k+1)) u^(2k+1)/sqrt(pi),
// c_k = (2k-1)!!/2^k.  Writing z^m = x alpha_m + i beta_m with alpha_m, beta_m
// homogeneous polynomials in r = |z|^2 and a (x^2 = r - a^2), multiplication by
// z^2 = (r - 2a^2) + 2iax gives
//   alpha_{m+2} = (r - 2a^2) alpha_m - 2a beta_m,   beta_{m+2} = (r - 2a^2) beta_m + 2a (r - a^2) alpha_m,
// alpha_1 = 1, beta_1 = a.  With beta_{2k+1} = a r^k sum_j q_kj t^j (t = a^2/r):
//   H = sum_n C_n u^(n+1),  C_n = (a/sqrt(pi)) sum_{k+j=n} c_k q_kj a^(2j).
// For the adjoint, Euler's relation for the homogeneous terms (degree -(2k+1))
// gives H + x H_x + a H_a = -sum_k 2k T_k, and differentiating a^(2j+1) u^p at
// fixed x gives
//   a H_a = sum_n E_n u^(n+1) - 2 a^2 sum_n (n+1) C_n u^(n+2),  E_n = (1/sqrt(pi)) sum_{k+j=n} (2j+1) c_k q_kj a^(2j+1).
// With ASY_K = 6 the truncation and FP32 rounding stay below 4e-7 of H for |z| >= 6.
// To keep every coefficient inside the FP32 range (a up to 25, scaled strengths
// up to ~1e13) the polynomials are written in v = ASY_S u (v < 1 for |z| >= 6):
// the table holds c_k q_kj / ASY_S^k and a^(2j) enters as (a^2/ASY_S)^j, so that
// H = u sum_n C'_n v^n with C'_n = C_n / ASY_S^n (a power of two: exact).
constexpr int ASY_K = 6;
constexpr int ASY_N = 2 * ASY_K + 1; // powers u^1 .. u^13
constexpr float ASY_S = 32.0f;

struct AsyTable {
    float cq[ASY_K + 1][ASY_K + 1]; // c_k q_kj / ASY_S^k (j <= k)
};

constexpr AsyTable make_asy_table()
{
    // integer coefficients b[s] of beta_m = sum_s b[s] r^s a^(m-2s) and c[s] of
    // alpha_m = sum_s c[s] r^s a^(m-1-2s), advanced m -> m + 2
    long long b[ASY_K + 2] = {}, c[ASY_K + 2] = {};
    b[0] = 1;
    c[0] = 1;
    AsyTable t{};
    double ck = 1.0;
    for (int k = 0; k <= ASY_K; ++k) {
        if (k > 0) {
            long long nb[ASY_K + 2] = {}, nc[ASY_K + 2] = {};
            for (int s = 0; s <= k; ++s) {
                const long long bs1 = s > 0 ? b[s - 1] : 0, cs1 = s > 0 ? c[s - 1] : 0;
                nc[s] = cs1 - 2 * c[s] - 2 * b[s];
                nb[s] = bs1 - 2 * b[s] + 2 * cs1 - 2 * c[s];
            }
            for (int s = 0; s <= k; ++s) {
                b[s] = nb[s];
                c[s] = nc[s];
            }
            ck *= (2.0 * k - 1.0) / 2.0;
        }
        // beta_{2k+1} = sum_s b[s] r^s a^(2k+1-2s) = a r^k sum_j b[k-j] t^j
        double sk = 1.0;
        for (int i = 0; i < k; ++i) sk /= (double)ASY_S;
        for (int j = 0; j <= k; ++j) t.cq[k][j] = (float)(ck * (double)b[k - j] * sk);
    }
    return t;
}

__constant__ const AsyTable ASY = make_asy_table();

// C'_n (n = 0 .. ASY_N - 1) of H = u sum_n C'_n v^n, times amp.
__device__ __forceinline__ void asy_coeffs(float a, float amp, float (&C)[ASY_N])
{
    const float a2 = a * a * (1.0f / ASY_S);
    float ap[ASY_K + 1]; // amp a^(2j+1) / sqrt(pi)
    ap[0] = amp * a * (float)INV_SQRTPI;
#pragma unroll
    for (int j = 1; j <= ASY_K; ++j) ap[j] = ap[j - 1] * a2;
#pragma unroll
    for (int n = 0; n < ASY_N; ++n) C[n] = 0.0f;
#pragma unroll
    for (int k = 0; k <= ASY_K; ++k)
#pragma unroll
        for (int j = 0; j <= k; ++j) C[k + j] = fmaf(ASY.cq[k][j], ap[j], C[k + j]);
}

// Adjoint: f_T = u sum_n F_n v^n and f_b = u sum_n G_n v^n (n = 0 .. ASY_N) for
// f_T = aS V0 + hT D_beta + nn D_gamma and f_b = D_gamma, with V0 = amp H,
// D_beta = -amp (H + x H_x + a H_a), D_gamma = amp a H_a.
__device__ __forceinline__ void asy_coeffs_adj(float a, float amp, float aS, float hT, float nn,
                                               float (&F)[ASY_N + 1], float (&G)[ASY_N + 1])
{
    const float a2 = a * a * (1.0f / ASY_S); // a^2 / ASY_S
    float ap[ASY_K + 1];
    ap[0] = amp * a * (float)INV_SQRTPI;
#pragma unroll
    for (int j = 1; j <= ASY_K; ++j) ap[j] = ap[j - 1] * a2;
    float C[ASY_N], D[ASY_N], E[ASY_N];
#pragma unroll
    for (int n = 0; n < ASY_N; ++n) {
        C[n] = 0.0f;
        D[n] = 0.0f;
        E[n] = 0.0f;
    }
#pragma unroll
    for (int k = 0; k <= ASY_K; ++k)
#pragma unroll
        for (int j = 0; j <= k; ++j) {
            const float v = ASY.cq[k][j] * ap[j];
            C[k + j] += v;
            D[k + j] = fmaf(2.0f * (float)k, v, D[k + j]);
            E[k + j] = fmaf(2.0f * (float)j + 1.0f, v, E[k + j]);
        }
    // coefficient of u v^n: V0: C'_n, D_beta: D'_n, D_gamma: E'_n - 2 (a^2/ASY_S) n C'_{n-1}
#pragma unroll
    for (int n = 0; n <= ASY_N; ++n) {
        const float cn = n < ASY_N ? C[n] : 0.0f;
        const float dn = n < ASY_N ? D[n] : 0.0f;
        const float en = n < ASY_N ? E[n] : 0.0f;
        const float gm = en - (n > 0 ? 2.0f * a2 * (float)n * C[n - 1] : 0.0f);
        G[n] = gm;
        F[n] = fmaf(aS, cn, fmaf(hT, dn, nn * gm));
    }
}

template <class R>
__device__ __noinline__ R voigt_H(R x, R xl, R a, R Kc, const R* dtab)
{
    R wr, wi;
    faddeeva<R>(x, xl, a, Kc, &wr, &wi, dtab);
    return wr;
}
template <class R>
__device__ __noinline__ void voigt_w_dw(R x, R xl, R a, R Kc, R* w4, const R* dtab)
{
    faddeeva_d<R>(x, xl, a, Kc, &w4[0], &w4[1], &w4[2], &w4[3], dtab);
}

} // namespace xsd
