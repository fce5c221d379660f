// Line-by-line cross-section on sm_103a: per-line/per-layer parameters, the
// direct line-profile sum (Eq. crosssec summed over lines, Sec. 3.1) and its
// reverse-mode adjoint.
//
// Work decomposition.  Lines are sorted by centre.  A CTA owns one strip of
// STRIP = 1024 consecutive grid points of one layer; each of its 4 warps owns
// 256 points (G = 8 per lane, lane-interleaved) and walks the strip's line window
// (all lines with an in-cut point in the strip, optionally split into K chunks
// across CTAs).  Lines are staged through shared memory 128 at a time and every
// warp reads them as broadcasts.  For each 32-line sub-tile a warp decides once
// whether all its points are inside every line's wing cut and at |z| >= 100;
// then the whole sub-tile runs the 5-FP32-op + 1-reciprocal Lorentz-wing form
// of the asymptotic Faddeeva series (the bulk of the work).  Otherwise each
// evaluation checks the cut by integer index and picks its Faddeeva tier.
//
// Precision (XS_PREC_MIXED): per-line scalars are formed in FP64 and rounded
// once; the line-centre offset nu_j - nu_hat is formed from FP64 offsets to the
// strip's reference point (hi + lo floats); Voigt values and sums are FP32, with
// the running sum per grid point kept as an FP32 (hi, lo) pair updated after
// every 32 lines (Fast2Sum).  XS_PREC_FP64 runs the same code in double.
#include <algorithm>
#include <type_traits>

#include "xs_device.cuh"
#include "xs_internal.h"

namespace xsd {

constexpr int LS_THREADS = 128;
constexpr int LS_WARPS = 4;
constexpr int LS_G = 8;
constexpr int LS_STRIP = LS_WARPS * 32 * LS_G; // 1024
// resident CTAs per SM the register budget targets (FP32: 96 registers; FP64 keeps more)
template <class R> struct MinBlocks { static constexpr int v = 5; };
template <> struct MinBlocks<double> { static constexpr int v = 3; };

// ------------------------------------------------------------------ K0: cut ranges

// For each line: first grid index with nu_j - nu_hat >= -W and last with
// nu_j - nu_hat <= W (double precision, boundary included).  Both are
// non-decreasing along a sorted line list.
__global__ void cut_range_kernel(const double* __restrict__ nu_hat, int64_t nl, const double* __restrict__ nu,
                                 int64_t N, double W, int2* __restrict__ jr)
{
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nl) return;
    double c = nu_hat[l];
    int64_t lo = 0, hi = N; // first j with nu[j] - c >= -W
    while (lo < hi) {
        int64_t m = (lo + hi) >> 1;
        if (nu[m] - c >= -W) hi = m; else lo = m + 1;
    }
    int64_t jlo = lo;
    lo = 0;
    hi = N; // first j with nu[j] - c > W
    while (lo < hi) {
        int64_t m = (lo + hi) >> 1;
        if (nu[m] - c > W) hi = m; else lo = m + 1;
    }
    jr[l] = make_int2((int)jlo, (int)(lo - 1));
}

__global__ void sorted_check_kernel(const double* __restrict__ nu_hat, int64_t nl, int* __restrict__ bad)
{
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l + 1 < nl && !(nu_hat[l] <= nu_hat[l + 1])) atomicOr(bad, 1);
}

__global__ void grid_check_kernel(const double* __restrict__ nu, int64_t N, int* __restrict__ bad)
{
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j + 1 < N && !(nu[j] < nu[j + 1])) atomicOr(bad, 1);
}

// ------------------------------------------------------------------ K1: line params

__global__ void layer_agg_init_kernel(float* agg, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) agg[i] = __int_as_float(0x7f800000); // +inf
}

// Per (layer, line), FP64 math rounded once to R:
//   rec1 = {G = gamma^2, Al = s gamma/pi, F1 = 1.5 B Al, F2 = -2 G B Al}   (B = 2 beta^2)
//   rec2 = {c = 1/(sqrt2 beta), a = gamma c, Av = s c / sqrt(pi), Kc = K(a)}
//   rec3 = {dlnS/dT, -n/T}                                                   (adjoint only)
// s = S(T) * scale.  Per layer: agg[2n] = min c, agg[2n+1] = min a.
// e^{-(k h)^2}, k = 1.., for the two series steps (h = 0.7f and h = 0.5)
__device__ const float KC_E32[10] = {0.612626433f, 0.140858427f, 0.0121551799f, 0.00039366915f, 4.78511947e-06f,
                                     2.18295906e-08f, 3.73757449e-11f, 2.40173736e-14f, 5.79232066e-18f,
                                     5.24289428e-22f};
__device__ const double KC_E64[13] = {0.77880078307140488, 0.36787944117144233, 0.10539922456186433,
                                      0.018315638888734179, 0.0019304541362277093, 0.00012340980408667956,
                                      4.7851173921290088e-06, 1.1253517471925912e-07, 1.6052280551856116e-09,
                                      1.3887943864964021e-11, 7.2877240958196922e-14, 2.3195228302435691e-16,
                                      4.4777324417183015e-19};

// K(a) = erfcx(a) - (2 a h/pi) sum_k e^{-(kh)^2} / ((kh)^2 + a^2), the per-line constant
// of the small-|z| series (see xs_device.cuh)
__device__ __forceinline__ float series_K(float a)
{
    const float h = Tier<float>::h;
    float s1 = 0.0f;
#pragma unroll
    for (int k = 1; k <= 10; ++k) {
        float kh = (float)k * h;
        s1 = fmaf(KC_E32[k - 1], rcp_fast(fmaf(kh, kh, a * a)), s1);
    }
    return erfcxf(a) - 2.0f * a * h * (float)(1.0 / PI) * s1;
}
__device__ __forceinline__ double series_K(double a)
{
    const double h = Tier<double>::h;
    double s1 = 0.0;
    for (int k = 1; k <= 13; ++k) {
        double kh = k * h;
        s1 += KC_E64[k - 1] / (kh * kh + a * a);
    }
    return erfcx(a) - 2.0 * a * h / PI * s1;
}

// Per (layer, line), rounded once to R:
//   rec1 = {G = gamma^2, Al = s gamma/pi, F1 = 1.5 B Al, F2 = -2 G B Al}   (B = 2 beta^2)
//   rec2 = {c = 1/(sqrt2 beta), a = gamma c, Av = s c / sqrt(pi), Kc = K(a)}
//   clo  = c - (R)c,  rec3 = {dlnS/dT, -n/T} (adjoint only)
// s = S(T) * scale.  The Boltzmann exponent of S (Eq. Slog) and c are formed in
// FP64 in both paths; in the FP32 path the factors that only need ~1e-7
// (stimulated emission, the width's temperature power, K(a)) use FP32.
// Per layer: agg[2n] = min c, agg[2n+1] = min a.
template <class R>
__global__ void line_params_kernel(const double* __restrict__ nu_hat, const double* __restrict__ ln_S0,
                                   const double* __restrict__ elower, const double* __restrict__ gamma_ref,
                                   const double* __restrict__ n_temp, int64_t nl, double mass, double qexp,
                                   const double* __restrict__ T, const double* __restrict__ P_bar, int layer0,
                                   double sb, double scale, typename vec4<R>::type* __restrict__ rec1,
                                   typename vec4<R>::type* __restrict__ rec2, R* __restrict__ clo,
                                   R* __restrict__ rec3, float* __restrict__ agg)
{
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int n = blockIdx.y;
    float cmin = __int_as_float(0x7f800000), amin = cmin;
    if (l < nl) {
        const double Tn = T[layer0 + n], Pn = P_bar[layer0 + n];
        const double nuh = nu_hat[l];
        const double lnTr = log(Tn / Tref);
        const double boltz = exp(ln_S0[l] - c2 * elower[l] * (1.0 / Tn - 1.0 / Tref) - qexp * lnTr);
        const double beta = sqrt(kB * Tn / (mass * amu)) * nuh / cL;
        const double c = 1.0 / (SQRT2 * beta);
        R stim, gam;
        if (std::is_same<R, float>::value) {
            const float u = (float)(c2 * nuh);
            stim = (R)(expm1f(-u / (float)Tn) / expm1f(-u / (float)Tref));
            gam = (R)((float)(sb * gamma_ref[l] * (Pn / bar_per_atm)) * expf(-(float)n_temp[l] * (float)lnTr));
        } else {
            stim = (R)(expm1(-c2 * nuh / Tn) / expm1(-c2 * nuh / Tref));
            gam = (R)(sb * gamma_ref[l] * exp(-n_temp[l] * lnTr) * (Pn / bar_per_atm));
        }
        const double s = boltz * scale * (double)stim;
        const R cr = (R)c;
        const R a = gam * cr;
        const R Al = (R)(s * (double)gam / PI);
        const R Av = (R)(s * c * INV_SQRTPI);
        const R B = R(1) / (cr * cr);
        const R G = gam * gam;
        const R Kc = (a * a < (R)Tier<R>::z2_series) ? series_K(a) : R(0);
        const size_t idx = (size_t)n * nl + l;
        typename vec4<R>::type v1, v2;
        v1.x = G;
        v1.y = Al;
        v1.z = R(1.5) * B * Al;
        v1.w = R(-2) * G * B * Al;
        v2.x = cr;
        v2.y = a;
        v2.z = Av;
        v2.w = Kc;
        rec1[idx] = v1;
        rec2[idx] = v2;
        clo[idx] = (R)(c - (double)cr); // the part of c the rounded value misses
        if (rec3) {
            const R Tr = (R)Tn;
            const R u = (R)(c2 * nuh) / Tr;
            const R dlnS = (R)(c2 * elower[l] / (Tn * Tn) - qexp / Tn) - (u / Tr) / (R)expm1((double)u);
            rec3[2 * idx] = dlnS;
            rec3[2 * idx + 1] = (R)(-n_temp[l]) / Tr;
        }
        cmin = (float)cr * (1.0f - 1e-6f);
        amin = (float)a * (1.0f - 1e-6f);
    }
    // block min then one atomic per block (positive floats order like their bits)
    for (int o = 16; o > 0; o >>= 1) {
        cmin = fminf(cmin, __shfl_xor_sync(0xffffffffu, cmin, o));
        amin = fminf(amin, __shfl_xor_sync(0xffffffffu, amin, o));
    }
    if ((threadIdx.x & 31) == 0 && cmin < __int_as_float(0x7f800000)) {
        atomicMin((int*)&agg[2 * (layer0 + n)], __float_as_int(cmin));
        atomicMin((int*)&agg[2 * (layer0 + n) + 1], __float_as_int(amin));
    }
}

// ------------------------------------------------------------------ K2: line sum

// Offsets: the FP32 path keeps nu relative to a reference point (the warp's
// middle grid point) as hi + lo floats; the FP64 path keeps absolute doubles.
template <class R> struct Off;
template <> struct Off<float> {
    __device__ static void make(double v, double ref, float* hi, float* lo)
    {
        double o = v - ref;
        *hi = (float)o;
        *lo = (float)(o - (double)*hi);
    }
    // (ohi - bhi) is exact when the point is near the line (Sterbenz); the lo parts ride along
    __device__ static void dnu2(float ohi, float olo, float bhi, float blo, float* dh, float* dl)
    {
        *dh = ohi - bhi;
        *dl = olo - blo;
    }
};
template <> struct Off<double> {
    __device__ static void make(double v, double, double* hi, float* lo)
    {
        *hi = v;
        *lo = 0.0f;
    }
    __device__ static void dnu2(double ohi, float, double bhi, float, double* dh, double* dl)
    {
        *dh = ohi - bhi;
        *dl = 0.0;
    }
};

__device__ __forceinline__ int64_t lb_jhi(const int2* jr, int64_t n, int v) // first l with jr[l].y >= v
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t m = (lo + hi) >> 1;
        if (jr[m].y >= v) hi = m; else lo = m + 1;
    }
    return lo;
}
__device__ __forceinline__ int64_t lb_jlo(const int2* jr, int64_t n, int v) // first l with jr[l].x > v
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t m = (lo + hi) >> 1;
        if (jr[m].x > v) hi = m; else lo = m + 1;
    }
    return lo;
}

// Line window of a strip (all lines with an in-cut point in [j0, jlast]) and
// the kc-th of ksplit equal parts of it, rounded to whole 32-line chunks.
// Lane 0 searches, the warp gets the result by shuffle.
__device__ __forceinline__ void strip_window(const int2* jrange, int64_t nl, int64_t j0, int64_t jlast, int ksplit,
                                             int kc, int64_t* cb, int64_t* ce)
{
    long long b = 0, e = 0;
    if ((threadIdx.x & 31) == 0) {
        int64_t bb = lb_jhi(jrange, nl, (int)j0);
        int64_t ee = lb_jlo(jrange, nl, (int)jlast);
        if (ee < bb) ee = bb;
        int64_t per = (ee - bb + ksplit - 1) / ksplit;
        per = (per + 31) & ~(int64_t)31;
        b = min64(ee, bb + per * kc);
        e = min64(ee, b + per);
    }
    *cb = __shfl_sync(0xffffffffu, b, 0);
    *ce = __shfl_sync(0xffffffffu, e, 0);
}

// Grid points of one warp: G per lane, lane-interleaved, offsets to the warp's
// middle point.  Returns false when the warp has no point in the grid.
template <class R>
struct WarpPoints {
    R ohi[LS_G];
    int jg[LS_G];
    int jw0, jw1; // first and last valid point of the warp
    R ow0, ow1;   // their offsets
    double ref;

    __device__ bool init(const double* nu, int64_t jbase, int64_t jlast, float* olo_s)
    {
        const int lane = threadIdx.x & 31;
        if (jbase > jlast) return false;
        ref = nu[min64(jlast, jbase + 16 * LS_G)];
#pragma unroll
        for (int g = 0; g < LS_G; ++g) {
            int64_t j = jbase + g * 32 + lane;
            jg[g] = (int)j;
            float lo;
            Off<R>::make(nu[min64(j, jlast)], ref, &ohi[g], &lo);
            olo_s[g * 32 + lane] = lo;
        }
        jw0 = (int)jbase;
        jw1 = (int)min64(jlast, jbase + 32 * LS_G - 1);
        ow0 = __shfl_sync(0xffffffffu, ohi[0], 0);
        int jl = jw1 - (int)jbase, gl = jl >> 5, ll = jl & 31;
        R v = ohi[0];
#pragma unroll
        for (int g = 0; g < LS_G; ++g)
            if (g == gl) v = ohi[g];
        ow1 = __shfl_sync(0xffffffffu, v, ll);
        return true;
    }
};

// Lower bound of |z| over the warp's points for lines [bf, bl] (offsets, sorted):
// true when every point is at |z|^2 >= z2 from every line.
__device__ __forceinline__ bool all_far(float bf, float bl, float ow0, float ow1, float cmin, float amin, float z2)
{
    float dist = fmaxf(fmaxf(bf - ow1, ow0 - bl), 0.0f);
    float xm = dist * cmin;
    return fmaf(xm, xm, amin * amin) >= z2;
}

template <class R>
struct LineTile {
    R bhi[32];
    float blo[32];
    R G[32], k0[32], f2[32];
    typename vec4<R>::type k[32]; // k1..k4 of the fast form
    typename vec4<R>::type r2[32];
    R clo[32];
    int2 jr[32];
    // the fast-form constants again, each duplicated so that one broadcast load
    // fills a register pair for the packed two-point FP32 instructions:
    float4 q0[32]; // (-b, -b, G, G)
    float4 q1[32]; // (k0, k0, k1, k1)
    float4 q2[32]; // (k2, k2, k3, k3)
    float4 q3[32]; // (k4, k4, F2, F2)
};

// Packed fast forms: two grid points per FP32 instruction (FADD2/FFMA2), one
// reciprocal each.  Only the FP32 path has them; the FP64 path never takes a
// fast branch.
template <class R>
__device__ __forceinline__ void fast_k1(const LineTile<R>&, const R (&)[LS_G], R (&)[LS_G])
{
}
template <class R>
__device__ __forceinline__ void fast_k2(const LineTile<R>&, const R (&)[LS_G], R (&)[LS_G])
{
}

__device__ __forceinline__ float2 f2lo(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 f2hi(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 rcp2(float2 v) { return make_float2(rcp_fast(v.x), rcp_fast(v.y)); }
// both reciprocals from one: 1/D1 = D2/(D1 D2), 1/D2 = D1/(D1 D2) (about 1.5 ulp);
// trades a second MUFU op for two FP32 multiplies.  D1 D2 stays in range in the fast
// forms (0.01 < D < 1e4 there).
__device__ __forceinline__ float2 rcp2_shared(float2 v)
{
    float r = rcp_fast(v.x * v.y);
    return __fmul2_rn(make_float2(v.y, v.x), make_float2(r, r));
}
// pairs 0 and 1 share one reciprocal, pairs 2 and 3 take one each: this balances
// the MUFU pipe (16 ops/clk/SM) against the FP32 pipe (128 lanes/clk/SM)
__device__ __forceinline__ float2 rcp2_mix(float2 v, int p) { return (p < 2) ? rcp2_shared(v) : rcp2(v); }

// K = 1: acc += rho (k0 + rho (k1 + rho F2)),  rho = 1/((o - b)^2 + G)
template <>
__device__ __forceinline__ void fast_k1<float>(const LineTile<float>& tl, const float (&ohi)[LS_G],
                                               float (&acc)[LS_G])
{
    float2 o2[LS_G / 2], a2[LS_G / 2];
#pragma unroll
    for (int p = 0; p < LS_G / 2; ++p) {
        o2[p] = make_float2(ohi[2 * p], ohi[2 * p + 1]);
        a2[p] = make_float2(acc[2 * p], acc[2 * p + 1]);
    }
#pragma unroll 4
    for (int i = 0; i < 32; ++i) {
        const float4 v0 = tl.q0[i], v1 = tl.q1[i], v3 = tl.q3[i];
        const float2 nb = f2lo(v0), G = f2hi(v0), k0 = f2lo(v1), k1 = f2hi(v1), f2 = f2hi(v3);
#pragma unroll
        for (int p = 0; p < LS_G / 2; ++p) {
            float2 d = __fadd2_rn(o2[p], nb);
            float2 rho = rcp2_mix(__ffma2_rn(d, d, G), p);
            float2 u = __ffma2_rn(__ffma2_rn(f2, rho, k1), rho, k0);
            a2[p] = __ffma2_rn(rho, u, a2[p]);
        }
    }
#pragma unroll
    for (int p = 0; p < LS_G / 2; ++p) {
        acc[2 * p] = a2[p].x;
        acc[2 * p + 1] = a2[p].y;
    }
}

// K = 2: acc += rho (k0 + rho (k1 + rho (k2 + rho (k3 + rho k4))))
template <>
__device__ __forceinline__ void fast_k2<float>(const LineTile<float>& tl, const float (&ohi)[LS_G],
                                               float (&acc)[LS_G])
{
    float2 o2[LS_G / 2], a2[LS_G / 2];
#pragma unroll
    for (int p = 0; p < LS_G / 2; ++p) {
        o2[p] = make_float2(ohi[2 * p], ohi[2 * p + 1]);
        a2[p] = make_float2(acc[2 * p], acc[2 * p + 1]);
    }
#pragma unroll 2
    for (int i = 0; i < 32; ++i) {
        const float4 v0 = tl.q0[i], v1 = tl.q1[i], v2 = tl.q2[i], v3 = tl.q3[i];
        const float2 nb = f2lo(v0), G = f2hi(v0), k0 = f2lo(v1), k1 = f2hi(v1), k2 = f2lo(v2), k3 = f2hi(v2),
                     k4 = f2lo(v3);
#pragma unroll
        for (int p = 0; p < LS_G / 2; ++p) {
            float2 d = __fadd2_rn(o2[p], nb);
            float2 rho = rcp2_mix(__ffma2_rn(d, d, G), p);
            float2 u = __ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(k4, rho, k3), rho, k2), rho, k1), rho, k0);
            a2[p] = __ffma2_rn(rho, u, a2[p]);
        }
    }
#pragma unroll
    for (int p = 0; p < LS_G / 2; ++p) {
        acc[2 * p] = a2[p].x;
        acc[2 * p + 1] = a2[p].y;
    }
}

// Fast form of a line's term from the asymptotic series with K = 2 (Eq. asywofz),
// written in rho = 1/(dnu^2 + gamma^2):  Av H = rho (k0 + rho (k1 + rho (k2 + rho (k3 + rho k4))))
// with k0 = s gamma/pi = Al, B = 2 beta^2, G = gamma^2 and
//   k1 = 1.5 B Al,  k2 = Al (3.75 B^2 - 2 G B),  k3 = -15 G B^2 Al,  k4 = 12 G^2 B^2 Al.
// From rec1 = {G, Al, F1 = 1.5 B Al, F2 = -2 G B Al} and c = 1/sqrt(B):
template <class R>
__device__ __forceinline__ void fast_coeffs(const typename vec4<R>::type& p1, R c, R* k0,
                                            typename vec4<R>::type* k)
{
    R B = rcp_fast(c * c);
    *k0 = p1.y;
    k->x = p1.z;
    k->y = fma(R(2.5) * B, p1.z, p1.w);
    k->z = R(7.5) * B * p1.w;
    k->w = R(-6) * p1.x * B * p1.w;
}

// one lane's line record as loaded from global memory
// ---- mixed chunks (FP32 only): per-line dispatch with packed arithmetic

// K = 2 form over lines [i0, i1) of the tile; when masked, each point only takes
// the lines whose cut range holds it.
__device__ __forceinline__ void k2_lines(const LineTile<float>& tl, int i0, int i1, const float2 (&o2)[LS_G / 2],
                                         float2 (&a2)[LS_G / 2], bool masked, const int (&jg)[LS_G])
{
    for (int i = i0; i < i1; ++i) {
        const float4 v0 = tl.q0[i], v1 = tl.q1[i], v2 = tl.q2[i], v3 = tl.q3[i];
        const float2 nb = f2lo(v0), G = f2hi(v0), k0 = f2lo(v1), k1 = f2hi(v1), k2 = f2lo(v2), k3 = f2hi(v2),
                     k4 = f2lo(v3);
        const int2 jr = tl.jr[i];
#pragma unroll
        for (int p = 0; p < LS_G / 2; ++p) {
            float2 d = __fadd2_rn(o2[p], nb);
            float2 rho = rcp2_mix(__ffma2_rn(d, d, G), p);
            float2 u = __ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(k4, rho, k3), rho, k2), rho, k1), rho, k0);
            if (masked) {
                rho.x = (jg[2 * p] >= jr.x && jg[2 * p] <= jr.y) ? rho.x : 0.0f;
                rho.y = (jg[2 * p + 1] >= jr.x && jg[2 * p + 1] <= jr.y) ? rho.y : 0.0f;
            }
            a2[p] = __ffma2_rn(rho, u, a2[p]);
        }
    }
}

// One line near the warp's points: the K = 5 form in rho (coefficients ctab[0..10],
// see k5_coeff) at every point with |z| >= 8, i.e. dnu^2 >= dthr2, and the small-|z|
// series (dtab, see w_series_rec) at the others.
__device__ __forceinline__ void near_line(const LineTile<float>& tl, int i, const float (&ohi)[LS_G],
                                          const float* olo, const float* ctab, const float* dtab,
                                          float2 (&a2)[LS_G / 2], const int (&jg)[LS_G])
{
    const int lane = threadIdx.x & 31;
    const float bh = tl.bhi[i], bl = tl.blo[i], G = tl.G[i], cl = tl.clo[i];
    const float4 p2 = tl.r2[i];
    const int2 jr = tl.jr[i];
    const float a = p2.y, c = p2.x;
    const float dthr2 = fmaxf(Tier<float>::z2_series - a * a, 0.0f) * rcp_fast(c * c);
    float dh[LS_G], dl[LS_G];
    float2 rho[LS_G / 2], u[LS_G / 2];
#pragma unroll
    for (int p = 0; p < LS_G / 2; ++p) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int g = 2 * p + q;
            dh[g] = ohi[g] - bh;
            dl[g] = olo[g * 32 + lane] - bl;
        }
        float2 d = __fadd2_rn(make_float2(dh[2 * p], dh[2 * p + 1]), make_float2(dl[2 * p], dl[2 * p + 1]));
        rho[p] = rcp2(__ffma2_rn(d, d, make_float2(G, G)));
        const float cc = ctab[10];
        u[p] = make_float2(cc, cc);
    }
#pragma unroll
    for (int n = 9; n >= 0; --n) {
        const float cc = ctab[n];
        const float2 c2 = make_float2(cc, cc);
#pragma unroll
        for (int p = 0; p < LS_G / 2; ++p) u[p] = __ffma2_rn(u[p], rho[p], c2);
    }
#pragma unroll
    for (int p = 0; p < LS_G / 2; ++p) {
        float2 v = __fmul2_rn(rho[p], u[p]);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int g = 2 * p + q;
            const float d = dh[g] + dl[g];
            const bool in = jg[g] >= jr.x && jg[g] <= jr.y;
            float add = (q == 0) ? v.x : v.y;
            if (!(in && d * d >= dthr2)) add = 0.0f;
            if (__any_sync(0xffffffffu, in && d * d < dthr2)) {
                if (in && d * d < dthr2) {
                    float x, xl;
                    scaled_pair(dh[g], dl[g], c, cl, &x, &xl);
                    add = p2.z * voigt_H_series(x, xl, a, p2.w, dtab);
                }
            }
            if (q == 0) a2[p].x += add; else a2[p].y += add;
        }
    }
}

// Whole mixed chunk: runs of lines that are far (|z| >= 25 at every point) and
// cover the warp go through the packed K = 2 loop; far lines that cover only part
// of the warp take it masked; the rest go through near_line.
__device__ __forceinline__ void mixed_chunk(const LineTile<float>& tl, const WarpPoints<float>& pts,
                                            const float* olo, float* ctab, float* dtab, float (&acc)[LS_G])
{
    const int lane = threadIdx.x & 31;
    // classify line `lane`
    const float bh = tl.bhi[lane];
    const float4 p2 = tl.r2[lane];
    const int2 jr = tl.jr[lane];
    const float dist = fmaxf(fmaxf(bh - pts.ow1, pts.ow0 - bh), 0.0f);
    const float xm = dist * p2.x;
    const bool far = fmaf(xm, xm, p2.y * p2.y) >= Tier<float>::z2_fast;
    const bool full = (jr.x <= pts.jw0) && (jr.y >= pts.jw1);
    const unsigned fm = __ballot_sync(0xffffffffu, far && full);
    const unsigned em = __ballot_sync(0xffffffffu, far && !full);

    float2 o2[LS_G / 2], a2[LS_G / 2];
#pragma unroll
    for (int p = 0; p < LS_G / 2; ++p) {
        o2[p] = make_float2(pts.ohi[2 * p], pts.ohi[2 * p + 1]);
        a2[p] = make_float2(acc[2 * p], acc[2 * p + 1]);
    }
    int i = 0;
    while (i < 32) {
        const unsigned rest = fm >> i;
        if (rest & 1u) {
            const unsigned zeros = ~rest;
            const int j = (zeros == 0u) ? 32 : i + __ffs(zeros) - 1;
            k2_lines(tl, i, j, o2, a2, false, pts.jg);
            i = j;
        } else if ((em >> i) & 1u) {
            k2_lines(tl, i, i + 1, o2, a2, true, pts.jg);
            ++i;
        } else {
            // per-line tables shared by the warp
            const float4 q = tl.r2[i];
            const float hn = (float)(lane + 1) * Tier<float>::h;
            __syncwarp();
            dtab[lane] = rcp_fast(fmaf(hn, hn, q.y * q.y));
            if (lane < 11) ctab[lane] = k5_coeff(lane, tl.k0[i], rcp_fast(q.x * q.x), tl.G[i]);
            __syncwarp();
            near_line(tl, i, pts.ohi, olo, ctab, dtab, a2, pts.jg);
            ++i;
        }
    }
#pragma unroll
    for (int p = 0; p < LS_G / 2; ++p) {
        acc[2 * p] = a2[p].x;
        acc[2 * p + 1] = a2[p].y;
    }
}

template <class R>
__device__ __forceinline__ void mixed_chunk_dispatch(const LineTile<R>&, const WarpPoints<R>&, const float*, float*,
                                                     float*, R (&)[LS_G])
{
}
template <>
__device__ __forceinline__ void mixed_chunk_dispatch<float>(const LineTile<float>& tl, const WarpPoints<float>& pts,
                                                            const float* olo, float* ctab, float* dtab,
                                                            float (&acc)[LS_G])
{
    mixed_chunk(tl, pts, olo, ctab, dtab, acc);
}

template <class R>
struct LineRec {
    double nu;
    typename vec4<R>::type p1, p2;
    R cl;
    int2 jr;

    __device__ void load(const double* nu_hat, const int2* jrange, const typename vec4<R>::type* rec1,
                         const typename vec4<R>::type* rec2, const R* clo, int64_t l, int64_t ce)
    {
        if (l < ce) {
            nu = nu_hat[l];
            p1 = rec1[l];
            p2 = rec2[l];
            cl = clo[l];
            jr = jrange[l];
        } else {
            // padding: the chunk's last line with zero amplitude keeps every
            // sub-tile test and offset that of real lines
            nu = nu_hat[ce - 1];
            jr = jrange[ce - 1];
            p1.x = R(1); p1.y = R(0); p1.z = R(0); p1.w = R(0);
            p2.x = R(1); p2.y = R(1); p2.z = R(0); p2.w = R(0);
            cl = R(0);
        }
    }
};

template <class R, bool FAST>
__global__ void __launch_bounds__(LS_THREADS, MinBlocks<R>::v) linesum_kernel(
    const double* __restrict__ nu_hat, const int2* __restrict__ jrange,
    const typename vec4<R>::type* __restrict__ rec1, const typename vec4<R>::type* __restrict__ rec2,
    const R* __restrict__ clo, const float* __restrict__ agg, const double* __restrict__ nu, int64_t N, int64_t nl,
    int layer0, int ksplit, double unscale, void* __restrict__ sigma, int sigma_is_float, double* __restrict__ partial,
    int L_total)
{
    using R4 = typename vec4<R>::type;
    __shared__ LineTile<R> tiles[LS_WARPS];
    __shared__ float olo_s[LS_WARPS][32 * LS_G];
    __shared__ R dtab_s[LS_WARPS][32];
    __shared__ float ctab_s[LS_WARPS][12];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int strip = blockIdx.x, nloc = blockIdx.y, kc = blockIdx.z;
    const int64_t j0 = (int64_t)strip * LS_STRIP;
    const int64_t jlast = min64(N - 1, j0 + LS_STRIP - 1);
    LineTile<R>& tl = tiles[w];
    float* olo = olo_s[w];
    R* dtab = dtab_s[w];
    float* ctab = ctab_s[w];

    WarpPoints<R> pts;
    if (!pts.init(nu, j0 + (int64_t)w * (32 * LS_G), jlast, olo)) return;
    int64_t cb, ce;
    strip_window(jrange, nl, j0, jlast, ksplit, kc, &cb, &ce);
    const int layer = layer0 + nloc;
    const float cmin = agg[2 * layer], amin = agg[2 * layer + 1];
    const size_t lay = (size_t)nloc * nl; // records hold the current layer chunk
    const R4* r1g = rec1 + lay;
    const R4* r2g = rec2 + lay;
    const R* clg = clo + lay;

    R acc[LS_G], shi[LS_G], slo[LS_G];
#pragma unroll
    for (int g = 0; g < LS_G; ++g) {
        acc[g] = R(0);
        shi[g] = R(0);
        slo[g] = R(0);
    }
    LineRec<R> nx;
    if (cb < ce) nx.load(nu_hat, jrange, r1g, r2g, clg, cb + lane, ce);

    for (int64_t t0 = cb; t0 < ce; t0 += 32) {
        {
            R bh;
            float bl;
            Off<R>::make(nx.nu, pts.ref, &bh, &bl);
            tl.bhi[lane] = bh;
            tl.blo[lane] = bl;
            R k0;
            R4 kk;
            fast_coeffs<R>(nx.p1, nx.p2.x, &k0, &kk);
            tl.G[lane] = nx.p1.x;
            tl.k0[lane] = k0;
            tl.f2[lane] = nx.p1.w;
            tl.k[lane] = kk;
            tl.r2[lane] = nx.p2;
            tl.clo[lane] = nx.cl;
            tl.jr[lane] = nx.jr;
            if (FAST) {
                const float nbf = -(float)bh, Gf = (float)nx.p1.x;
                tl.q0[lane] = make_float4(nbf, nbf, Gf, Gf);
                tl.q1[lane] = make_float4((float)k0, (float)k0, (float)kk.x, (float)kk.x);
                tl.q2[lane] = make_float4((float)kk.y, (float)kk.y, (float)kk.z, (float)kk.z);
                tl.q3[lane] = make_float4((float)kk.w, (float)kk.w, (float)nx.p1.w, (float)nx.p1.w);
            }
        }
        __syncwarp();
        if (t0 + 32 < ce) nx.load(nu_hat, jrange, r1g, r2g, clg, t0 + 32 + lane, ce); // in flight meanwhile

        // chunk class: 2 = every (line, point) at |z| >= 100 (K = 1 form),
        // 1 = at |z| >= 25 (K = 2 form), 0 = mixed (per line, per point)
        int cls = 0;
        if (FAST) {
            bool incut = (tl.jr[31].x <= pts.jw0) && (tl.jr[0].y >= pts.jw1);
            if (incut) {
                float dist = fmaxf(fmaxf((float)tl.bhi[0] - (float)pts.ow1, (float)pts.ow0 - (float)tl.bhi[31]), 0.0f);
                float xm = dist * cmin;
                float z2 = fmaf(xm, xm, amin * amin);
                cls = (z2 >= (float)Tier<R>::z2_far) ? 2 : (z2 >= (float)Tier<R>::z2_fast) ? 1 : 0;
            }
        }
        if (cls == 2) {
            // K = 1: Av H = rho (k0 + rho (k1 + rho F2)), F2 = -2 G B Al, rho = 1/(dnu^2 + gamma^2);
            // the K = 2 terms are below 4e-8 of a line's value here
            fast_k1<R>(tl, pts.ohi, acc);
        } else if (cls == 1) {
            fast_k2<R>(tl, pts.ohi, acc);
        } else if (FAST) {
            mixed_chunk_dispatch<R>(tl, pts, olo, ctab, (float*)dtab, acc);
        } else {
            // FP64: per line (warp-uniform): if every point of the warp is at |z| >= 100
            // use the Lorentz-wing form, masked by the cut only when the line does
            // not cover the whole warp; else choose the Faddeeva tier per point.
            for (int i = 0; i < 32; ++i) {
                const R bh = tl.bhi[i];
                const R4 p2 = tl.r2[i];
                const int2 jr = tl.jr[i];
                const R G = tl.G[i], k0 = tl.k0[i];
                const R4 k = tl.k[i];
                bool line_far = false;
                if (FAST)
                    line_far = all_far((float)bh, (float)bh, (float)pts.ow0, (float)pts.ow1, (float)p2.x, (float)p2.y,
                                       (float)Tier<R>::z2_fast);
                if (line_far) {
                    const bool full = (jr.x <= pts.jw0) && (jr.y >= pts.jw1);
#pragma unroll
                    for (int g = 0; g < LS_G; ++g) {
                        R d = pts.ohi[g] - bh;
                        R rho = rcp_fast(fma(d, d, G));
                        R u = fma(fma(fma(fma(k.w, rho, k.z), rho, k.y), rho, k.x), rho, k0);
                        R v = rho * u;
                        if (full || (pts.jg[g] >= jr.x && pts.jg[g] <= jr.y)) acc[g] += v;
                    }
                } else {
                    const float bl = tl.blo[i];
                    const R cl = tl.clo[i];
                    if (FAST) {
                        // per line, shared by the warp: 1/(n^2 h^2 + a^2) (n = 1..32) for the
                        // small-|z| series, and the 11 coefficients of the K = 5 form in rho
                        const R hn = R(lane + 1) * (R)Tier<R>::h;
                        __syncwarp();
                        dtab[lane] = rcp_fast(fma(hn, hn, p2.y * p2.y));
                        if (lane < 11) ctab[lane] = k5_coeff(lane, (float)k0, (float)rcp_fast(p2.x * p2.x), (float)G);
                        __syncwarp();
                    }
#pragma unroll
                    for (int g = 0; g < LS_G; ++g) {
                        if (pts.jg[g] >= jr.x && pts.jg[g] <= jr.y) {
                            R dh, dl, x, xl;
                            Off<R>::dnu2(pts.ohi[g], olo[g * 32 + lane], bh, bl, &dh, &dl);
                            scaled_pair(dh, dl, p2.x, cl, &x, &xl);
                            const R z2 = fma(x, x, p2.y * p2.y);
                            if (FAST && z2 >= (R)Tier<R>::z2_series) {
                                // |z| >= 8: K = 5 asymptotic form, uniform across the warp
                                R d = dh + dl;
                                R rho = rcp_fast(fma(d, d, G));
                                R u = (R)ctab[10];
#pragma unroll
                                for (int n = 9; n >= 0; --n) u = fma(u, rho, (R)ctab[n]);
                                acc[g] = fma(rho, u, acc[g]);
                            } else if (FAST) {
                                acc[g] = fma(p2.z, (R)voigt_H_series((float)x, (float)xl, (float)p2.y, (float)p2.w,
                                                                     (const float*)dtab),
                                             acc[g]);
                            } else {
                                acc[g] = fma(p2.z, voigt_H<R>(x, xl, p2.y, p2.w, nullptr), acc[g]);
                            }
                        }
                    }
                }
            }
        }
        // fold the 32-line partial into the running compensated sum (TwoSum)
#pragma unroll
        for (int g = 0; g < LS_G; ++g) {
            R sres = shi[g] + acc[g];
            R bb = sres - shi[g];
            slo[g] += (shi[g] - (sres - bb)) + (acc[g] - bb);
            shi[g] = sres;
            acc[g] = R(0);
        }
        __syncwarp();
    }

#pragma unroll
    for (int g = 0; g < LS_G; ++g) {
        if (pts.jg[g] <= jlast) {
            double v = (double)shi[g] + (double)slo[g];
            size_t o = (size_t)layer * N + pts.jg[g];
            if (ksplit == 1) {
                if (sigma_is_float)
                    ((float*)sigma)[o] = (float)(v * unscale);
                else
                    ((double*)sigma)[o] = v * unscale;
            } else {
                partial[((size_t)kc * L_total + nloc) * N + pts.jg[g]] = v; // [ksplit][chunk layers][N]
            }
        }
    }
}

__global__ void combine_kernel(const double* __restrict__ partial, int ksplit, int64_t LN, int64_t off,
                               int64_t cnt, double unscale, void* __restrict__ sigma, int sigma_is_float)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    int64_t o = off + i;
    double s = 0.0, c = 0.0;
    for (int k = 0; k < ksplit; ++k) {
        double v = partial[(size_t)k * LN + i];
        double t = s + v;
        c += (fabs(s) >= fabs(v)) ? (s - t) + v : (v - t) + s;
        s = t;
    }
    s = (s + c) * unscale;
    if (sigma_is_float) ((float*)sigma)[o] = (float)s; else ((double*)sigma)[o] = s;
}

// ------------------------------------------------------------------ K6: adjoint

template <class R>
struct AdjTile {
    R bhi[32];
    float blo[32];
    typename vec4<R>::type r2[32];
    typename vec4<R>::type t[32]; // fast form: f_T = rho (T1 + rho (T2 + rho (T3 + rho T4)))
    typename vec4<R>::type u[32]; // fast form: f_b = rho (U1 + rho (U2 + rho (U3 + rho U4)))
    R G[32], clo[32], aS[32], nn[32];
    int2 jr[32];
    // duplicated constants for the packed fast form (FP32 path only)
    float4 q0[32];           // (-b, -b, G, G)
    float4 qt0[32], qt1[32]; // (T1, T1, T2, T2), (T3, T3, T4, T4)
    float4 qu0[32], qu1[32]; // (U1, U1, U2, U2), (U3, U3, U4, U4)
};

template <class R>
__device__ __forceinline__ void fast_adj(const AdjTile<R>&, const R (&)[LS_G], const R (&)[LS_G], R&, R&)
{
}
// lambda rho P_T(rho) and lambda rho P_U(rho), two points per packed instruction
template <>
__device__ __forceinline__ void fast_adj<float>(const AdjTile<float>& tl, const float (&ohi)[LS_G],
                                                const float (&lam)[LS_G], float& accT, float& accB)
{
    float2 o2[LS_G / 2], l2[LS_G / 2];
#pragma unroll
    for (int p = 0; p < LS_G / 2; ++p) {
        o2[p] = make_float2(ohi[2 * p], ohi[2 * p + 1]);
        l2[p] = make_float2(lam[2 * p], lam[2 * p + 1]);
    }
    float2 aT = make_float2(accT, 0.0f), aB = make_float2(accB, 0.0f);
#pragma unroll 2
    for (int i = 0; i < 32; ++i) {
        const float4 v0 = tl.q0[i], t0 = tl.qt0[i], t1 = tl.qt1[i], u0 = tl.qu0[i], u1 = tl.qu1[i];
        const float2 nb = f2lo(v0), G = f2hi(v0);
#pragma unroll
        for (int p = 0; p < LS_G / 2; ++p) {
            float2 d = __fadd2_rn(o2[p], nb);
            float2 rho = rcp2(__ffma2_rn(d, d, G));
            float2 lr = __fmul2_rn(l2[p], rho);
            float2 pt = __ffma2_rn(__ffma2_rn(__ffma2_rn(f2hi(t1), rho, f2lo(t1)), rho, f2hi(t0)), rho, f2lo(t0));
            float2 pu = __ffma2_rn(__ffma2_rn(__ffma2_rn(f2hi(u1), rho, f2lo(u1)), rho, f2hi(u0)), rho, f2lo(u0));
            aT = __ffma2_rn(lr, pt, aT);
            aB = __ffma2_rn(lr, pu, aB);
        }
    }
    accT = aT.x + aT.y;
    accB = aB.x + aB.y;
}

// Per evaluation the adjoint accumulates
//   f_T = (dlnS/dT) V0 + (1/(2T)) D_beta + (-n/T) D_gamma   and   f_b = D_gamma
// with V0 = Av H, D_beta = beta d sigma/d beta = -Av (H + x H_x + a H_a),
// D_gamma = gamma d sigma/d gamma = Av a H_a, weighted by lambda_j = g_sigma[n][j].
// In the Lorentz-wing form (K = 1 of the asymptotic series, rho = 1/(dnu^2 + gamma^2),
// B = 2 beta^2, G = gamma^2, Al = s gamma/pi):
//   V0 = Al (rho + 1.5 B rho^2 - 2 G B rho^3),  D_beta = Al B (3 rho^2 - 4 G rho^3),
//   D_gamma = Al (rho + (1.5 B - 2 G) rho^2 - 12 G B rho^3 + 12 G^2 B rho^4).
template <class R, bool FAST>
__global__ void __launch_bounds__(LS_THREADS, MinBlocks<R>::v) linesum_adjoint_kernel(
    const double* __restrict__ nu_hat, const int2* __restrict__ jrange,
    const typename vec4<R>::type* __restrict__ rec1, const typename vec4<R>::type* __restrict__ rec2,
    const R* __restrict__ clo, const R* __restrict__ rec3, const float* __restrict__ agg, const double* __restrict__ nu,
    int64_t N, int64_t nl, int layer0, int ksplit, const double* __restrict__ T, const double* __restrict__ g_sigma,
    double lam_scale, double* __restrict__ part, int nstrips)
{
    using R4 = typename vec4<R>::type;
    __shared__ AdjTile<R> tiles[LS_WARPS];
    __shared__ float olo_s[LS_WARPS][32 * LS_G];
    __shared__ R dtab_s[LS_WARPS][32];
    __shared__ double red[2][LS_WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int strip = blockIdx.x, nloc = blockIdx.y, kc = blockIdx.z;
    const int layer = layer0 + nloc;
    const int64_t j0 = (int64_t)strip * LS_STRIP;
    const int64_t jlast = min64(N - 1, j0 + LS_STRIP - 1);
    const R half_invT = (R)(0.5 / T[layer]);
    AdjTile<R>& tl = tiles[w];
    float* olo = olo_s[w];

    double sT = 0.0, sB = 0.0;
    WarpPoints<R> pts;
    if (pts.init(nu, j0 + (int64_t)w * (32 * LS_G), jlast, olo)) {
        int64_t cb, ce;
        strip_window(jrange, nl, j0, jlast, ksplit, kc, &cb, &ce);
        const float cmin = agg[2 * layer], amin = agg[2 * layer + 1];
        const size_t lay = (size_t)nloc * nl;
        const R4* r1g = rec1 + lay;
        const R4* r2g = rec2 + lay;
        const R* clg = clo + lay;
        const R* r3g = rec3 + 2 * lay;
        R lam[LS_G];
#pragma unroll
        for (int g = 0; g < LS_G; ++g)
            lam[g] = (pts.jg[g] <= jlast) ? (R)(g_sigma[(size_t)layer * N + pts.jg[g]] * lam_scale) : R(0);

        LineRec<R> nx;
        R naS = R(0), nnn = R(0);
        if (cb < ce) {
            nx.load(nu_hat, jrange, r1g, r2g, clg, cb + lane, ce);
            if (cb + lane < ce) {
                naS = r3g[2 * (cb + lane)];
                nnn = r3g[2 * (cb + lane) + 1];
            }
        }
        R accT = R(0), accB = R(0);
        for (int64_t t0 = cb; t0 < ce; t0 += 32) {
            {
                R bh;
                float bl;
                Off<R>::make(nx.nu, pts.ref, &bh, &bl);
                tl.bhi[lane] = bh;
                tl.blo[lane] = bl;
                tl.r2[lane] = nx.p2;
                tl.clo[lane] = nx.cl;
                tl.jr[lane] = nx.jr;
                const R G = nx.p1.x, Al = nx.p1.y, F1 = nx.p1.z, F2 = nx.p1.w, aS = naS, nn = nnn;
                R4 tc, uc;
                tc.x = Al * (aS + nn);
                tc.y = aS * F1 + half_invT * R(2) * F1 + nn * (F1 - R(2) * G * Al);
                tc.z = aS * F2 + half_invT * R(2) * F2 + nn * R(6) * F2;
                tc.w = nn * (R(-6) * G * F2);
                uc.x = Al;
                uc.y = F1 - R(2) * G * Al;
                uc.z = R(6) * F2;
                uc.w = R(-6) * G * F2;
                tl.t[lane] = tc;
                tl.u[lane] = uc;
                tl.G[lane] = G;
                tl.aS[lane] = aS;
                tl.nn[lane] = nn;
                if (FAST) {
                    const float nbf = -(float)bh, Gf = (float)G;
                    tl.q0[lane] = make_float4(nbf, nbf, Gf, Gf);
                    tl.qt0[lane] = make_float4((float)tc.x, (float)tc.x, (float)tc.y, (float)tc.y);
                    tl.qt1[lane] = make_float4((float)tc.z, (float)tc.z, (float)tc.w, (float)tc.w);
                    tl.qu0[lane] = make_float4((float)uc.x, (float)uc.x, (float)uc.y, (float)uc.y);
                    tl.qu1[lane] = make_float4((float)uc.z, (float)uc.z, (float)uc.w, (float)uc.w);
                }
            }
            __syncwarp();
            if (t0 + 32 < ce) {
                int64_t l = t0 + 32 + lane;
                nx.load(nu_hat, jrange, r1g, r2g, clg, l, ce);
                naS = (l < ce) ? r3g[2 * l] : R(0);
                nnn = (l < ce) ? r3g[2 * l + 1] : R(0);
            }
            bool fast = false;
            if (FAST) {
                bool incut = (tl.jr[31].x <= pts.jw0) && (tl.jr[0].y >= pts.jw1);
                fast = incut && all_far((float)tl.bhi[0], (float)tl.bhi[31], (float)pts.ow0, (float)pts.ow1, cmin,
                                        amin, (float)Tier<R>::z2_fast_adj);
            }
            if (fast) {
                fast_adj<R>(tl, pts.ohi, lam, accT, accB);
            } else {
                for (int i = 0; i < 32; ++i) {
                    const R bh = tl.bhi[i];
                    const R4 p2 = tl.r2[i];
                    const int2 jr = tl.jr[i];
                    bool line_far = false;
                    if (FAST)
                        line_far = all_far((float)bh, (float)bh, (float)pts.ow0, (float)pts.ow1, (float)p2.x,
                                           (float)p2.y, (float)Tier<R>::z2_fast_adj);
                    if (line_far) {
                        const R G = tl.G[i];
                        const R4 tc = tl.t[i];
                        const R4 uc = tl.u[i];
                        const bool full = (jr.x <= pts.jw0) && (jr.y >= pts.jw1);
#pragma unroll
                        for (int g = 0; g < LS_G; ++g) {
                            R d = pts.ohi[g] - bh;
                            R rho = rcp_fast(fma(d, d, G));
                            R lm = (full || (pts.jg[g] >= jr.x && pts.jg[g] <= jr.y)) ? lam[g] : R(0);
                            R lr = lm * rho;
                            accT = fma(lr, fma(rho, fma(rho, fma(rho, tc.w, tc.z), tc.y), tc.x), accT);
                            accB = fma(lr, fma(rho, fma(rho, fma(rho, uc.w, uc.z), uc.y), uc.x), accB);
                        }
                    } else {
                        const float bl = tl.blo[i];
                        const R cl = tl.clo[i];
                        const R aS = tl.aS[i], nn = tl.nn[i];
                        R* dtab = dtab_s[w];
                        if (FAST) {
                            const R hn = R(lane + 1) * (R)Tier<R>::h;
                            __syncwarp();
                            dtab[lane] = rcp_fast(fma(hn, hn, p2.y * p2.y));
                            __syncwarp();
                        }
#pragma unroll
                        for (int g = 0; g < LS_G; ++g) {
                            if (pts.jg[g] >= jr.x && pts.jg[g] <= jr.y) {
                                R dh, dl, x, xl;
                                Off<R>::dnu2(pts.ohi[g], olo[g * 32 + lane], bh, bl, &dh, &dl);
                                scaled_pair(dh, dl, p2.x, cl, &x, &xl);
                                R a = p2.y;
                                if (FAST && fma(x, x, a * a) >= (R)Tier<R>::z2_fast_adj) {
                                    const R G = tl.G[i];
                                    const R4 tc = tl.t[i];
                                    const R4 uc = tl.u[i];
                                    R d = dh + dl;
                                    R rho = rcp_fast(fma(d, d, G));
                                    R lr = lam[g] * rho;
                                    accT = fma(lr, fma(rho, fma(rho, fma(rho, tc.w, tc.z), tc.y), tc.x), accT);
                                    accB = fma(lr, fma(rho, fma(rho, fma(rho, uc.w, uc.z), uc.y), uc.x), accB);
                                    continue;
                                }
                                R w4[4];
                                voigt_w_dw<R>(x, xl, a, p2.w, w4, FAST ? dtab : nullptr);
                                const R wr = w4[0], dr = w4[2], di = w4[3];
                                // H_x = Re w', H_a = -Im w'
                                R V0 = p2.z * wr;
                                R V1 = p2.z * x * dr;
                                R V2 = -p2.z * a * di;
                                R Db = -(V0 + V1 + V2);
                                R ft = aS * V0 + half_invT * Db + nn * V2;
                                accT = fma(lam[g], ft, accT);
                                accB = fma(lam[g], V2, accB);
                            }
                        }
                    }
                }
            }
            sT += (double)accT;
            sB += (double)accB;
            accT = R(0);
            accB = R(0);
            __syncwarp();
        }
    }
    // fixed-order block reduction
    for (int o = 16; o > 0; o >>= 1) {
        sT += __shfl_xor_sync(0xffffffffu, sT, o);
        sB += __shfl_xor_sync(0xffffffffu, sB, o);
    }
    if (lane == 0) {
        red[0][w] = sT;
        red[1][w] = sB;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < LS_WARPS; ++i) {
            a += red[0][i];
            b += red[1][i];
        }
        size_t o = ((size_t)layer * nstrips + strip) * ksplit + kc;
        part[2 * o] = a;
        part[2 * o + 1] = b;
    }
}

// g_T[n] = sum over (strip, chunk) partials; g_b = sum over layers (fixed order).
__global__ void adjoint_reduce_kernel(const double* __restrict__ part, int L, int per_layer, double unscale,
                                      double inv_sb, double* __restrict__ g_T, double* __restrict__ g_b)
{
    __shared__ double red[256];
    double gb = 0.0;
    for (int n = 0; n < L; ++n) {
        double a = 0.0, b = 0.0;
        for (int i = threadIdx.x; i < per_layer; i += blockDim.x) {
            a += part[2 * ((size_t)n * per_layer + i)];
            b += part[2 * ((size_t)n * per_layer + i) + 1];
        }
        red[threadIdx.x] = a;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) g_T[n] = red[0] * unscale;
        __syncthreads();
        red[threadIdx.x] = b;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) gb += red[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) g_b[0] = gb * unscale * inv_sb;
}

} // namespace xsd

// ====================================================================== host side

using namespace xsd;

namespace {

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

int strips_of(int64_t N) { return (int)((N + LS_STRIP - 1) / LS_STRIP); }

// split the line window of each strip so that the grid holds enough CTAs
int choose_ksplit(int64_t nl, int64_t N, int Lc)
{
    int strips = strips_of(N);
    int64_t ctas = (int64_t)strips * Lc;
    const int64_t target = 152 * 8 * 6; // several waves of 8 resident CTAs per SM
    int k = (int)std::max<int64_t>(1, (target + ctas - 1) / ctas);
    int64_t per_strip = std::max<int64_t>(1, nl); // upper bound of a window
    int kmax = (int)std::max<int64_t>(1, per_strip / 1024);
    return std::min(k, std::min(kmax, 64));
}

struct XsPlan {
    int prec, Lc, ksplit, nchunks;
    size_t off_jr, off_agg, off_rec1, off_rec2, off_rec3, off_clo, off_part, total;
};

XsPlan plan_xs(int64_t nl, int64_t N, int32_t L, int prec, int Lc, bool adjoint)
{
    XsPlan p;
    p.prec = prec;
    p.Lc = Lc;
    size_t rs = (prec == XS_PREC_FP64) ? sizeof(double) : sizeof(float);
    p.ksplit = choose_ksplit(nl, N, Lc);
    size_t off = 0;
    p.off_jr = off;
    off += align256(sizeof(int2) * (size_t)std::max<int64_t>(nl, 1));
    p.off_agg = off;
    off += align256(sizeof(float) * 2 * (size_t)L);
    p.off_rec1 = off;
    off += align256(4 * rs * (size_t)std::max<int64_t>(nl, 1) * Lc);
    p.off_rec2 = off;
    off += align256(4 * rs * (size_t)std::max<int64_t>(nl, 1) * Lc);
    p.off_rec3 = off;
    off += align256(2 * rs * (size_t)std::max<int64_t>(nl, 1) * Lc);
    p.off_clo = off;
    off += align256(rs * (size_t)std::max<int64_t>(nl, 1) * Lc);
    p.off_part = off;
    size_t fwd_part = (p.ksplit > 1) ? sizeof(double) * (size_t)p.ksplit * Lc * N : 0;
    size_t adj_part = sizeof(double) * 2 * (size_t)L * strips_of(N) * p.ksplit;
    off += align256(std::max(fwd_part, adj_part));
    p.total = off;
    p.nchunks = (L + Lc - 1) / Lc;
    (void)adjoint;
    return p;
}

} // namespace

size_t xs_workspace_bytes(int64_t n_lines, int64_t N, int32_t L, int prec)
{
    if (n_lines < 0 || N <= 0 || L <= 0) return 0;
    return plan_xs(n_lines, N, L, prec, L, true).total;
}

size_t xs_workspace_min_bytes(int64_t n_lines, int64_t N, int32_t L, int prec)
{
    if (n_lines < 0 || N <= 0 || L <= 0) return 0;
    return plan_xs(n_lines, N, L, prec, 1, true).total;
}

namespace xsi {

static int pick_plan(int64_t nl, int64_t N, int32_t L, int prec, size_t ws_bytes, XsPlan* out)
{
    int Lc = L;
    while (true) {
        XsPlan p = plan_xs(nl, N, L, prec, Lc, true);
        if (p.total <= ws_bytes) {
            *out = p;
            return XS_OK;
        }
        if (Lc == 1) return XS_EINVAL;
        Lc = (Lc + 1) / 2;
    }
}

template <class R>
static int run_xs(const xs_lines* ln, const double* nu, int64_t N, const double* T, const double* P, int32_t L,
                  double sb, double W, void* sigma, char* ws, const XsPlan& p, bool adjoint,
                  const double* g_sigma, double* g_T, double* g_b, cudaStream_t st, int flags)
{
    // flags: XS_RUN_KEEP_ADJ  (forward) also write the adjoint's per-line records
    //        XS_RUN_REUSE     (adjoint) the records of an immediately preceding forward
    //                         with the same inputs and workspace are still valid
    const bool reuse = adjoint && (flags & XS_RUN_REUSE) && p.nchunks == 1;
    const bool want_rec3 = adjoint || (flags & XS_RUN_KEEP_ADJ);
    using R4 = typename vec4<R>::type;
    const int64_t nl = ln->n;
    const bool mixed = (p.prec == XS_PREC_MIXED);
    const double scale = mixed ? MIXED_SCALE : 1.0;
    const double unscale = mixed ? MIXED_UNSCALE : 1.0;
    int2* jr = (int2*)(ws + p.off_jr);
    float* agg = (float*)(ws + p.off_agg);
    R4* rec1 = (R4*)(ws + p.off_rec1);
    R4* rec2 = (R4*)(ws + p.off_rec2);
    R* rec3 = (R*)(ws + p.off_rec3);
    R* clo = (R*)(ws + p.off_clo);
    double* part = (double*)(ws + p.off_part);
    const int strips = strips_of(N);

    if (nl == 0) {
        if (adjoint) {
            if (cudaMemsetAsync(g_T, 0, sizeof(double) * L, st) != cudaSuccess) return XS_ECUDA;
            if (cudaMemsetAsync(g_b, 0, sizeof(double), st) != cudaSuccess) return XS_ECUDA;
        } else {
            size_t es = mixed ? sizeof(float) : sizeof(double);
            if (cudaMemsetAsync(sigma, 0, es * (size_t)L * N, st) != cudaSuccess) return XS_ECUDA;
        }
        return XS_OK;
    }
    if (!reuse) {
        cut_range_kernel<<<(unsigned)((nl + 255) / 256), 256, 0, st>>>(ln->nu_hat, nl, nu, N, W, jr);
        layer_agg_init_kernel<<<(2 * L + 255) / 256, 256, 0, st>>>(agg, 2 * L);
        count_launch(2);
    }
    for (int c = 0; c < p.nchunks; ++c) {
        int l0 = c * p.Lc;
        int lc = std::min(p.Lc, L - l0);
        if (!reuse) {
            dim3 pg((unsigned)((nl + 255) / 256), (unsigned)lc);
            line_params_kernel<R><<<pg, 256, 0, st>>>(ln->nu_hat, ln->ln_S0, ln->elower, ln->gamma_ref, ln->n_temp,
                                                       nl, ln->mass_amu, ln->q_exponent, T, P, l0, sb, scale, rec1,
                                                       rec2, clo, want_rec3 ? rec3 : nullptr, agg);
            count_launch();
        }
        dim3 grid((unsigned)strips, (unsigned)lc, (unsigned)p.ksplit);
        R4* r1b = rec1;
        R4* r2b = rec2;
        R* r3b = rec3;
        if (!adjoint) {
            prof_begin(0, st);
            linesum_kernel<R, std::is_same<R, float>::value><<<grid, LS_THREADS, 0, st>>>(
                ln->nu_hat, jr, r1b, r2b, clo, agg, nu, N, nl, l0, p.ksplit, unscale, sigma, mixed ? 1 : 0, part, lc);
            prof_end(0, st);
            count_launch();
            if (p.ksplit > 1) {
                count_launch();
                int64_t cnt = (int64_t)lc * N;
                combine_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(part, p.ksplit, cnt, (int64_t)l0 * N,
                                                                              cnt, unscale, sigma, mixed ? 1 : 0);
            }
        } else {
            prof_begin(1, st);
            linesum_adjoint_kernel<R, std::is_same<R, float>::value><<<grid, LS_THREADS, 0, st>>>(
                ln->nu_hat, jr, r1b, r2b, clo, r3b, agg, nu, N, nl, l0, p.ksplit, T, g_sigma, unscale, part, strips);
            prof_end(1, st);
            count_launch();
        }
    }
    if (adjoint) {
        adjoint_reduce_kernel<<<1, 256, 0, st>>>(part, L, strips * p.ksplit, 1.0, 1.0 / sb, g_T, g_b);
        count_launch();
    }
    return (cudaGetLastError() == cudaSuccess) ? XS_OK : XS_ECUDA;
}

int xs_run(const xs_lines* ln, const double* nu, int64_t N, const double* T, const double* P, int32_t L, double sb,
           double W, int prec, void* sigma, void* ws, size_t ws_bytes, bool adjoint, const double* g_sigma,
           double* g_T, double* g_b, cudaStream_t st, int flags)
{
    XsPlan p;
    if (pick_plan(ln->n, N, L, prec, ws_bytes, &p) != XS_OK) return XS_EINVAL;
    if (prec == XS_PREC_FP64)
        return run_xs<double>(ln, nu, N, T, P, L, sb, W, sigma, (char*)ws, p, adjoint, g_sigma, g_T, g_b, st, flags);
    return run_xs<float>(ln, nu, N, T, P, L, sb, W, sigma, (char*)ws, p, adjoint, g_sigma, g_T, g_b, st, flags);
}

int check_sorted(const double* nu_hat, int64_t n, cudaStream_t st, int* flag_dev, bool grid)
{
    if (n < 2) return XS_OK;
    if (cudaMemsetAsync(flag_dev, 0, sizeof(int), st) != cudaSuccess) return XS_ECUDA;
    if (grid)
        grid_check_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nu_hat, n, flag_dev);
    else
        sorted_check_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nu_hat, n, flag_dev);
    count_launch();
    int h = 0;
    if (cudaMemcpyAsync(&h, flag_dev, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return XS_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return XS_ECUDA;
    return h ? XS_EUNSORTED : XS_OK;
}

} // namespace xsi
