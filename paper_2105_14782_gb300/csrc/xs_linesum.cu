// Line-by-line cross-section on sm_103a: per-line/per-layer parameters, the
// direct line-profile sum (Eq. crosssec summed over lines, Sec. 3.1) and its
// reverse-mode adjoint.
//
// Partition.  For every (layer, line) the grid points inside the wing cut are
// split, in FP64, into the line's "near" index range (|z| < NEAR_Z = 16.5, z = x + ia) and
// the rest.  The far part (about 98% of the evaluations) is summed by the main
// kernels with the Lorentz-wing forms of the asymptotic series (Eq. asywofz) in
// packed FP32x2 arithmetic; the near part by the near kernels, one thread per
// grid point (a polynomial in 1/|z|^2 for |z| >= 6, the series below).  Both use
// the same integer ranges, so every (line, point) pair is counted exactly once.
//
// Main kernels.  Lines are sorted by centre.  A CTA owns one strip of 1,024
// consecutive grid points of one layer; each of its 4 warps owns 256 points
// (8 per lane, lane-interleaved) and walks its own line window (all lines with
// an in-cut point among its points, optionally split into K parts across CTAs)
// in 32-line chunks it stages itself in shared memory.  A chunk whose lines all
// cover the warp's points with no near point runs unmasked, with the cheapest
// wing form its |z| bound allows; other chunks mask per (line, point).
//
// Precision (XS_PREC_MIXED): per-line scalars are formed in FP64 and rounded
// once; line-centre offsets to the warp's middle grid point come from per-line
// float pairs (hi + lo where it matters); Voigt values and sums are FP32, with
// each point's running sum an FP32 (hi, lo) pair updated by TwoSum after every
// 32 lines.  XS_PREC_FP64 has no fast forms and no near split: every pair goes
// through the double-precision tiered Faddeeva function.
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
template <class R> struct MinBlocks { static constexpr int v = 4; }; // 128 registers: ILP over occupancy
template <> struct MinBlocks<double> { static constexpr int v = 3; };
// the near/far boundary of the FP32 path: pairs at |z| < NEAR_Z go to the near
// kernels.  At |z| >= 16.5 the K = 2 wing forms truncate the asymptotic series below
// 1e-7 of a term (the first dropped term is 15/(8 |z|^6)); the K = 1 adjoint forms
// are kept for |z| >= 25 (ADJ_K2_Z2) and K = 2 ones used between.
constexpr double NEAR_Z = 16.5;
constexpr float ADJ_K2_Z2 = 625.0f;

// ------------------------------------------------------------------ K0: cut ranges

// For each line: first grid index with nu_j - nu_hat >= -W and last with
// nu_j - nu_hat <= W (double precision, boundary included).  Both are
// non-decreasing along a sorted line list.
__global__ void cut_range_kernel(const double* __restrict__ nu_hat, int64_t nl, const double* __restrict__ nu,
                                 int64_t N, double W, int2* __restrict__ jr, float2* __restrict__ nuf)
{
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nl) return;
    double c = nu_hat[l];
    if (nuf) {
        // centre relative to the first grid point as hi + lo floats, so that the
        // FP32 kernels form line offsets without FP64 arithmetic
        const double o = c - nu[0];
        const float h = (float)o;
        nuf[l] = make_float2(h, (float)(o - (double)h));
    }
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

// agg[4n .. 4n+3] = {min c, min a, max a, unused} of layer n
__global__ void layer_agg_init_kernel(float* agg, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) agg[i] = ((i & 3) < 2) ? __int_as_float(0x7f800000) : 0.0f; // +inf for the minima
}

// Per (layer, line), FP64 math rounded once to R:
//   rec1 = {G = gamma^2, Al = s gamma/pi, F1 = 1.5 B Al, F2 = -2 G B Al}   (B = 2 beta^2)
//   rec2 = {c = 1/(sqrt2 beta), a = gamma c, Av = s c / sqrt(pi), Kc = K(a)}
//   rec3 = {dlnS/dT, -n/T}                                                   (adjoint only)
// s = S(T) * scale.  Per layer: agg[4n .. 4n+2] = min c, min a, max a.
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
// Per layer: agg[4n .. 4n+2] = min c, min a, max a.
template <class R>
__global__ void line_params_kernel(const double* __restrict__ nu_hat, const double* __restrict__ ln_S0,
                                   const double* __restrict__ elower, const double* __restrict__ gamma_ref,
                                   const double* __restrict__ n_temp, int64_t nl, double mass, double qexp,
                                   const double* __restrict__ T, const double* __restrict__ P_bar, int layer0,
                                   double sb, double scale, typename vec4<R>::type* __restrict__ rec1,
                                   typename vec4<R>::type* __restrict__ rec2, R* __restrict__ clo,
                                   R* __restrict__ rec3, float* __restrict__ agg, const double* __restrict__ nu,
                                   int64_t N, const int2* __restrict__ jrange, int2* __restrict__ jnear)
{
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int n = blockIdx.y;
    float cmin = __int_as_float(0x7f800000), amin = cmin, amax = 0.0f;
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
        if (jnear) {
            // near range: in-cut points with |nu_j - nu_hat| < sqrt(NEAR_Z^2 - a^2)/c, i.e. |z| < NEAR_Z
            const double ad = gam * c;
            const double lim = (double)NEAR_Z * NEAR_Z - ad * ad;
            int2 r = make_int2(1, 0); // empty
            if (lim > 0.0) {
                const double del = sqrt(lim) / c;
                int64_t lo = 0, hi = N; // first j with nu[j] - nuh > -del
                while (lo < hi) {
                    int64_t m = (lo + hi) >> 1;
                    if (nu[m] - nuh > -del) hi = m; else lo = m + 1;
                }
                const int64_t jl = lo;
                lo = 0;
                hi = N; // first j with nu[j] - nuh >= del
                while (lo < hi) {
                    int64_t m = (lo + hi) >> 1;
                    if (nu[m] - nuh >= del) hi = m; else lo = m + 1;
                }
                int2 cut = jrange[l];
                if (!XS_CHECK(cut.x >= 0 && cut.y < N)) cut = make_int2(1, 0);
                r.x = (int)max((int64_t)cut.x, jl);
                r.y = (int)min((int64_t)cut.y, lo - 1);
            }
            jnear[idx] = r;
        }
        cmin = (float)cr * (1.0f - 1e-6f);
        amin = (float)a * (1.0f - 1e-6f);
        amax = (float)a * (1.0f + 1e-6f);
    }
    // block min then one atomic per block (positive floats order like their bits)
    for (int o = 16; o > 0; o >>= 1) {
        cmin = fminf(cmin, __shfl_xor_sync(0xffffffffu, cmin, o));
        amin = fminf(amin, __shfl_xor_sync(0xffffffffu, amin, o));
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    }
    if ((threadIdx.x & 31) == 0 && cmin < __int_as_float(0x7f800000)) {
        atomicMin((int*)&agg[4 * (layer0 + n)], __float_as_int(cmin));
        atomicMin((int*)&agg[4 * (layer0 + n) + 1], __float_as_int(amin));
        atomicMax((int*)&agg[4 * (layer0 + n) + 2], __float_as_int(amax));
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
};
template <> struct Off<double> {
    __device__ static void make(double v, double, double* hi, float* lo)
    {
        *hi = v;
        *lo = 0.0f;
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

// Line window of a warp's points (all lines with an in-cut point in [j0, jlast]),
// and part kc of it.  Two ways to split (lb from choose_split):
//   lb == 0: ksplit equal parts of each warp's own window, rounded to whole
//            32-line chunks (balanced work; used when the records of the layers
//            in flight fit in L2 anyway);
//   lb > 0:  the kc-th absolute block [kc lb, (kc + 1) lb) of the sorted line
//            list.  The launch grid has kc as its slowest index, so the strips
//            and layers resident at one time all stream the same block of line
//            records and L2 serves the re-reads of long lists.
// Each warp takes its own window (not the strip's), so no chunk carries lines
// that miss all of the warp's points.  Lane 0 searches, the warp gets the result
// by shuffle.
__device__ __forceinline__ void strip_window(const int2* jrange, int64_t nl, int64_t j0, int64_t jlast, int ksplit,
                                             int64_t lb, int kc, int64_t* cb, int64_t* ce)
{
    long long b = 0, e = 0;
    if ((threadIdx.x & 31) == 0) {
        const int64_t bb = lb_jhi(jrange, nl, (int)j0);
        int64_t ee = lb_jlo(jrange, nl, (int)jlast);
        if (ee < bb) ee = bb;
        if (lb > 0) {
            b = bb > lb * kc ? bb : lb * kc;
            e = ee < lb * (kc + 1) ? ee : lb * (kc + 1);
            if (e < b) e = b;
        } else {
            int64_t per = (ee - bb + ksplit - 1) / ksplit;
            per = (per + 31) & ~(int64_t)31;
            b = min64(ee, bb + per * kc);
            e = min64(ee, b + per);
        }
    }
    *cb = __shfl_sync(0xffffffffu, b, 0);
    *ce = __shfl_sync(0xffffffffu, e, 0);
}

// Grid points of one warp: G per lane, lane-interleaved, offsets to the warp's
// middle point.  init() returns false when the warp has no point in the grid.
template <class R>
struct WarpPoints {
    R ohi[LS_G];
    int jg[LS_G];
    int jw0, jw1; // first and last valid point of the warp
    R ow0, ow1;   // their offsets
    double ref;
    float rh, rl; // ref - nu[0] as hi + lo floats

    __device__ bool init(const double* nu, int64_t jbase, int64_t jlast)
    {
        const int lane = threadIdx.x & 31;
        if (jbase > jlast) return false;
        ref = nu[min64(jlast, jbase + 16 * LS_G)];
        {
            const double o = ref - nu[0];
            rh = (float)o;
            rl = (float)(o - (double)rh);
        }
#pragma unroll
        for (int g = 0; g < LS_G; ++g) {
            int64_t j = jbase + g * 32 + lane;
            jg[g] = (int)j;
            float lo;
            Off<R>::make(nu[min64(j, jlast)], ref, &ohi[g], &lo);
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

__device__ __forceinline__ bool in_range(int j, int2 r) { return j >= r.x && j <= r.y; }

// A point takes a line's far form when it is inside the line's cut and outside
// its near range.
__device__ __forceinline__ bool far_point(int j, int2 cut, int2 nr) { return in_range(j, cut) && !in_range(j, nr); }

// Does the line cover every point of [jw0, jw1] with its far form?
__device__ __forceinline__ bool covers_far(int2 cut, int2 nr, int jw0, int jw1)
{
    const bool full = cut.x <= jw0 && cut.y >= jw1;
    const bool clear = nr.x > nr.y || nr.y < jw0 || nr.x > jw1;
    return full && clear;
}

// Forward tile: the fast-form constants, each duplicated so one broadcast load
// fills a register pair for the packed two-point FP32 instructions (FP32 path),
// plus what the FP64 path needs.
template <class R>
struct LineTile {
    float4 q0[32]; // (-b, -b, G, G)
    float4 q1[32]; // (k0, k0, k1, k1)
    float4 q2[32]; // (k2, k2, k3, k3)
    float4 q3[32]; // (k4, k4, F2, F2)
    int2 jr[32], jn[32];
    R bhi[32];
    typename vec4<R>::type r2[32];
};

// Fast form of a line's term from the asymptotic series with K = 2 (Eq. asywofz),
// written in rho = 1/(dnu^2 + gamma^2):  Av H = rho (k0 + rho (k1 + rho (k2 + rho (k3 + rho k4))))
// with k0 = s gamma/pi = Al, B = 2 beta^2, G = gamma^2 and
//   k1 = 1.5 B Al,  k2 = Al (3.75 B^2 - 2 G B),  k3 = -15 G B^2 Al,  k4 = 12 G^2 B^2 Al;
// the K = 1 form keeps rho (k0 + rho (k1 + rho F2)), F2 = -2 G B Al.
// From rec1 = {G, Al, F1 = 1.5 B Al, F2 = -2 G B Al} and c = 1/sqrt(B):
__device__ __forceinline__ void fast_consts(const float4& p1, float c, float4* k)
{
    const float B = rcp_fast(c * c);
    k->x = p1.z;                        // k1
    k->y = fmaf(2.5f * B, p1.z, p1.w);  // k2
    k->z = 7.5f * B * p1.w;             // k3
    k->w = -6.0f * p1.x * B * p1.w;     // k4
}

__device__ __forceinline__ float2 f2lo(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 f2hi(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 rcp2(float2 v) { return make_float2(rcp_fast(v.x), rcp_fast(v.y)); }
// both reciprocals from one: 1/D1 = D2/(D1 D2), 1/D2 = D1/(D1 D2) (about 1.5 ulp);
// trades a second MUFU op for two FP32 multiplies (0.01 < D < 1e4 in the far forms)
__device__ __forceinline__ float2 rcp2_shared(float2 v)
{
    float r = rcp_fast(v.x * v.y);
    return __fmul2_rn(make_float2(v.y, v.x), make_float2(r, r));
}
// pairs 0 and 1 share one reciprocal, pairs 2 and 3 take one each: this balances
// the MUFU pipe (16 ops/clk/SM) against the FP32 pipe (128 lanes/clk/SM)
__device__ __forceinline__ float2 rcp2_mix(float2 v, int p) { return (p < 2) ? rcp2_shared(v) : rcp2(v); }

// Packed forms over lines [i0, i1) of a tile.  KIND 0: rho (k0 + rho k1), unmasked;
// KIND 1: K = 1, unmasked; KIND 2: K = 2, unmasked; KIND 3: K = 2, masked per
// (line, point) by far_point.
template <int KIND>
__device__ __forceinline__ void far_lines(const LineTile<float>& tl, int i0, int i1, const float2 (&o2)[LS_G / 2],
                                          float2 (&a2)[LS_G / 2], const int (&jg)[LS_G])
{
#pragma unroll 4
    for (int i = i0; i < i1; ++i) {
        const float4 v0 = tl.q0[i], v1 = tl.q1[i], v3 = tl.q3[i];
        const float2 nb = f2lo(v0), G = f2hi(v0), k0 = f2lo(v1), k1 = f2hi(v1);
        float4 v2 = make_float4(0.f, 0.f, 0.f, 0.f);
        int2 cut = make_int2(0, 0), nr = make_int2(1, 0);
        if (KIND != 1) v2 = tl.q2[i];
        if (KIND == 3) {
            cut = tl.jr[i];
            nr = tl.jn[i];
        }
#pragma unroll
        for (int p = 0; p < LS_G / 2; ++p) {
            float2 d = __fadd2_rn(o2[p], nb);
            float2 rho = rcp2_mix(__ffma2_rn(d, d, G), p);
            float2 u;
            if (KIND == 0)
                u = __ffma2_rn(rho, k1, k0);
            else if (KIND == 1)
                u = __ffma2_rn(__ffma2_rn(f2hi(v3), rho, k1), rho, k0);
            else
                u = __ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(f2lo(v3), rho, f2hi(v2)), rho, f2lo(v2)), rho, k1),
                               rho, k0);
            if (KIND == 3) {
                rho.x = far_point(jg[2 * p], cut, nr) ? rho.x : 0.0f;
                rho.y = far_point(jg[2 * p + 1], cut, nr) ? rho.y : 0.0f;
            }
            a2[p] = __ffma2_rn(rho, u, a2[p]);
        }
    }
}

// Lower bound of |z|^2 over a chunk's lines (first and last line offsets -b0,
// -b31 in the tile) and a warp's points: the smallest centre-to-point distance
// times the layer's smallest c, and the layer's smallest a.
__device__ __forceinline__ float chunk_z2min(float nb0, float nb31, const WarpPoints<float>& pts, float cmin,
                                             float amin)
{
    const float dist = fmaxf(fmaxf(-nb0 - pts.ow1, pts.ow0 + nb31), 0.0f);
    const float xm = dist * cmin;
    return fmaf(xm, xm, amin * amin);
}

// One 32-line chunk of the FP32 main kernel.
__device__ __forceinline__ void chunk_far(const LineTile<float>& tl, const WarpPoints<float>& pts, float cmin,
                                          float amin, float amax, float (&acc)[LS_G])
{
    const int lane = threadIdx.x & 31;
    const unsigned ok = __ballot_sync(0xffffffffu, covers_far(tl.jr[lane], tl.jn[lane], pts.jw0, pts.jw1));
    float2 o2[LS_G / 2], a2[LS_G / 2];
#pragma unroll
    for (int p = 0; p < LS_G / 2; ++p) {
        o2[p] = make_float2(pts.ohi[2 * p], pts.ohi[2 * p + 1]);
        a2[p] = make_float2(acc[2 * p], acc[2 * p + 1]);
    }
    if (ok == 0xffffffffu) {
        // every pair at |z| >= NEAR_Z; K = 1 suffices when every pair is at |z| >= 100
        // (the K = 2 terms are below 4e-8 of the leading one), and its F2 term,
        // 2 a^2/|z|^4 of the leading one, is dropped where that is below 2e-8
        const float z2 = chunk_z2min(tl.q0[0].x, tl.q0[31].x, pts, cmin, amin);
        if (z2 >= 1.0e4f) {
            if (2.0f * amax * amax <= 2.0e-8f * z2 * z2)
                far_lines<0>(tl, 0, 32, o2, a2, pts.jg);
            else
                far_lines<1>(tl, 0, 32, o2, a2, pts.jg);
        } else {
            far_lines<2>(tl, 0, 32, o2, a2, pts.jg);
        }
    } else {
        int i = 0;
        while (i < 32) {
            const unsigned rest = ok >> i;
            if (rest & 1u) {
                const unsigned zeros = ~rest;
                const int j = (zeros == 0u) ? 32 : i + __ffs(zeros) - 1;
                far_lines<2>(tl, i, j, o2, a2, pts.jg);
                i = j;
            } else {
                far_lines<3>(tl, i, i + 1, o2, a2, pts.jg);
                ++i;
            }
        }
    }
#pragma unroll
    for (int p = 0; p < LS_G / 2; ++p) {
        acc[2 * p] = a2[p].x;
        acc[2 * p + 1] = a2[p].y;
    }
}

// One 32-line chunk of the FP64 main kernel: every in-cut pair, tiered Faddeeva.
__device__ __forceinline__ void chunk_fp64(const LineTile<double>& tl, const WarpPoints<double>& pts,
                                           double (&acc)[LS_G])
{
    for (int i = 0; i < 32; ++i) {
        const double bh = tl.bhi[i];
        const double4_32a p2 = tl.r2[i];
        const int2 jr = tl.jr[i];
#pragma unroll
        for (int g = 0; g < LS_G; ++g) {
            if (in_range(pts.jg[g], jr)) {
                const double x = fabs(pts.ohi[g] - bh) * p2.x;
                acc[g] = fma(p2.z, voigt_H<double>(x, 0.0, p2.y, p2.w, nullptr), acc[g]);
            }
        }
    }
}

// one lane's line record as loaded from global memory
template <class R>
struct LineRec {
    double nu;  // centre (FP64 path)
    float2 nf;  // centre - nu[0] as hi + lo floats (FP32 path)
    typename vec4<R>::type p1, p2;
    int2 jr, jn;

    __device__ void load(const double* nu_hat, const float2* nuf, const int2* jrange,
                         const typename vec4<R>::type* rec1, const typename vec4<R>::type* rec2, const int2* jnear,
                         int64_t l, int64_t ce)
    {
        constexpr bool FAST = std::is_same<R, float>::value;
        if (l < ce) {
            if (FAST) nf = nuf[l]; else nu = nu_hat[l];
            p1 = rec1[l];
            p2 = rec2[l];
            jr = jrange[l];
            jn = jnear ? jnear[l] : make_int2(1, 0);
        } else {
            // padding: the chunk's last line with zero amplitude keeps every
            // chunk test and offset that of real lines
            if (FAST) nf = nuf[ce - 1]; else nu = nu_hat[ce - 1];
            jr = jrange[ce - 1];
            jn = jnear ? jnear[ce - 1] : make_int2(1, 0);
            p1.x = R(1); p1.y = R(0); p1.z = R(0); p1.w = R(0);
            p2.x = R(1); p2.y = R(1); p2.z = R(0); p2.w = R(0);
        }
    }
};

// Offset of a line's centre to the warp's reference point: FP32 from the float
// pairs (the difference of the hi parts is exact or within half an ulp of the
// result, the lo parts add the rest), FP64 on the FP64 path.
__device__ __forceinline__ void line_offset(const LineRec<float>& r, const WarpPoints<float>& pts, float* bh)
{
    *bh = (r.nf.x - pts.rh) + (r.nf.y - pts.rl);
}
__device__ __forceinline__ void line_offset(const LineRec<double>& r, const WarpPoints<double>& pts, double* bh)
{
    *bh = r.nu;
}

template <class R, bool FAST>
__global__ void __launch_bounds__(LS_THREADS, MinBlocks<R>::v) linesum_kernel(
    const double* __restrict__ nu_hat, const float2* __restrict__ nuf, const int2* __restrict__ jrange,
    const typename vec4<R>::type* __restrict__ rec1, const typename vec4<R>::type* __restrict__ rec2,
    const int2* __restrict__ jnear, const float* __restrict__ agg, const double* __restrict__ nu, int64_t N,
    int64_t nl, int layer0, int ksplit, int64_t lb, double unscale, void* __restrict__ sigma, int sigma_is_float,
    double* __restrict__ partial, int L_total, const double* __restrict__ near_sum)
{
    using R4 = typename vec4<R>::type;
    __shared__ LineTile<R> tiles[LS_WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int strip = blockIdx.x, nloc = blockIdx.y, kc = blockIdx.z;
    const int64_t j0 = (int64_t)strip * LS_STRIP;
    const int64_t jlast = min64(N - 1, j0 + LS_STRIP - 1);
    LineTile<R>& tl = tiles[w];

    WarpPoints<R> pts;
    if (!pts.init(nu, j0 + (int64_t)w * (32 * LS_G), jlast)) return;
    int64_t cb, ce;
    strip_window(jrange, nl, pts.jw0, pts.jw1, ksplit, lb, kc, &cb, &ce);
    if (!XS_CHECK(cb >= 0 && cb <= ce && ce <= nl)) ce = cb;
    const int layer = layer0 + nloc;
    const float cmin = agg[4 * layer], amin = agg[4 * layer + 1], amax = agg[4 * layer + 2];
    const size_t lay = (size_t)nloc * nl; // records hold the current layer chunk
    const R4* r1g = rec1 + lay;
    const R4* r2g = rec2 + lay;
    const int2* jng = FAST ? jnear + lay : nullptr;

    R acc[LS_G], shi[LS_G], slo[LS_G];
#pragma unroll
    for (int g = 0; g < LS_G; ++g) {
        acc[g] = R(0);
        shi[g] = R(0);
        slo[g] = R(0);
    }
    LineRec<R> nx;
    if (cb < ce) nx.load(nu_hat, nuf, jrange, r1g, r2g, jng, cb + lane, ce);

    for (int64_t t0 = cb; t0 < ce; t0 += 32) {
        {
            R bh;
            line_offset(nx, pts, &bh);
            tl.bhi[lane] = bh;
            tl.r2[lane] = nx.p2;
            tl.jr[lane] = nx.jr;
            tl.jn[lane] = nx.jn;
            if (FAST) {
                float4 k;
                fast_consts(make_float4((float)nx.p1.x, (float)nx.p1.y, (float)nx.p1.z, (float)nx.p1.w),
                            (float)nx.p2.x, &k);
                const float nb = -(float)bh, G = (float)nx.p1.x, k0 = (float)nx.p1.y;
                tl.q0[lane] = make_float4(nb, nb, G, G);
                tl.q1[lane] = make_float4(k0, k0, k.x, k.x);
                tl.q2[lane] = make_float4(k.y, k.y, k.z, k.z);
                tl.q3[lane] = make_float4(k.w, k.w, (float)nx.p1.w, (float)nx.p1.w);
            }
        }
        __syncwarp();
        if (t0 + 32 < ce) nx.load(nu_hat, nuf, jrange, r1g, r2g, jng, t0 + 32 + lane, ce); // in flight meanwhile

        if constexpr (FAST)
            chunk_far(tl, pts, cmin, amin, amax, acc);
        else
            chunk_fp64(tl, pts, acc);

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
        if (pts.jg[g] <= jlast && XS_CHECK(pts.jg[g] >= 0 && pts.jg[g] < N)) {
            double v = (double)shi[g] + (double)slo[g];
            if (FAST && kc == 0) v += near_sum[(size_t)nloc * N + pts.jg[g]];
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

// ------------------------------------------------------------------ near kernels (FP32 path)

constexpr int NR_THREADS = 128;

// Lines staged by a near-kernel warp: offsets to the warp's reference point
// (hi + lo), near ranges and per-line scalars.
struct NearTile {
    float bhi[32], blo[32], clo[32];
    float4 r2[32]; // c, a, Av, Kc
    float2 xa[32]; // -c bhi, a^2: x to ~1e-7 for the wing polynomial
    int2 jn[32];
    float4 hc[32][4]; // Av C'_0 .. Av C'_12 of the wing polynomial (6 <= |z| < NEAR_Z)
    float sd[32][SER_TAB]; // series table (|z| < 6, lines with a < 6)
};

struct NearAdjTile {
    float bhi[32], blo[32], clo[32];
    float4 r2[32];
    float2 xa[32];
    int2 jn[32];
    float aS[32], nn[32];
    float4 hf[32][4], hg[32][4]; // f_T and f_b wing polynomials (6 <= |z| < NEAR_Z)
    float sd[32][SER_TAB];
};

// |z|^2 from which the near kernels take the wing polynomial in u = 1/|z|^2;
// below it the series.
constexpr float NEAR_POLY_Z2 = 36.0f;

// u sum_{n<13} C'_n v^n, v = ASY_S u, by Horner from four float4 of coefficients
__device__ __forceinline__ float horner13(const float4* h, float u)
{
    const float v = ASY_S * u;
    const float4 h0 = h[0], h1 = h[1], h2 = h[2], h3 = h[3];
    float p = h3.x;
    p = fmaf(p, v, h2.w);
    p = fmaf(p, v, h2.z);
    p = fmaf(p, v, h2.y);
    p = fmaf(p, v, h2.x);
    p = fmaf(p, v, h1.w);
    p = fmaf(p, v, h1.z);
    p = fmaf(p, v, h1.y);
    p = fmaf(p, v, h1.x);
    p = fmaf(p, v, h0.w);
    p = fmaf(p, v, h0.z);
    p = fmaf(p, v, h0.y);
    p = fmaf(p, v, h0.x);
    return p * u;
}
// u sum_{n<14} F_n v^n
__device__ __forceinline__ float horner14(const float4* h, float u)
{
    const float v = ASY_S * u;
    const float4 h0 = h[0], h1 = h[1], h2 = h[2], h3 = h[3];
    float p = h3.y;
    p = fmaf(p, v, h3.x);
    p = fmaf(p, v, h2.w);
    p = fmaf(p, v, h2.z);
    p = fmaf(p, v, h2.y);
    p = fmaf(p, v, h2.x);
    p = fmaf(p, v, h1.w);
    p = fmaf(p, v, h1.z);
    p = fmaf(p, v, h1.y);
    p = fmaf(p, v, h1.x);
    p = fmaf(p, v, h0.w);
    p = fmaf(p, v, h0.z);
    p = fmaf(p, v, h0.y);
    p = fmaf(p, v, h0.x);
    return p * u;
}

__device__ __forceinline__ void store16(float4* dst, const float* v, int n)
{
#pragma unroll
    for (int q = 0; q < 4; ++q)
        dst[q] = make_float4(4 * q < n ? v[4 * q] : 0.0f, 4 * q + 1 < n ? v[4 * q + 1] : 0.0f,
                             4 * q + 2 < n ? v[4 * q + 2] : 0.0f, 4 * q + 3 < n ? v[4 * q + 3] : 0.0f);
}

// Candidate lines of a warp's 32 points: centres within sqrt(625 - a^2)/c < 25/cmin
// of any of them (binary search on the sorted centres), cut to chunks of 32.
__device__ __forceinline__ void near_window(const double* nu_hat, int64_t nl, double lo_nu, double hi_nu, double del,
                                            int64_t* b, int64_t* e)
{
    long long bb = 0, ee = 0;
    if ((threadIdx.x & 31) == 0) {
        int64_t lo = 0, hi = nl;
        while (lo < hi) {
            int64_t m = (lo + hi) >> 1;
            if (nu_hat[m] < lo_nu - del) lo = m + 1; else hi = m;
        }
        bb = lo;
        lo = bb;
        hi = nl;
        while (lo < hi) {
            int64_t m = (lo + hi) >> 1;
            if (nu_hat[m] <= hi_nu + del) lo = m + 1; else hi = m;
        }
        ee = lo;
    }
    *b = __shfl_sync(0xffffffffu, bb, 0);
    *e = __shfl_sync(0xffffffffu, ee, 0);
}

// near_sum[n][j] = sum over lines with j in their near range of Av H(x, a),
// one thread per grid point, lines in ascending order, Neumaier-compensated.
__global__ void __launch_bounds__(NR_THREADS, 8) near_sum_kernel(const double* __restrict__ nu_hat, int64_t nl,
                                                              const float4* __restrict__ rec2,
                                                              const float* __restrict__ clo,
                                                              const int2* __restrict__ jnear,
                                                              const float* __restrict__ agg,
                                                              const double* __restrict__ nu, int64_t N, int layer0,
                                                              double* __restrict__ near_sum)
{
    __shared__ NearTile tiles[NR_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nloc = blockIdx.y;
    const int64_t jb = (int64_t)blockIdx.x * NR_THREADS + w * 32;
    if (jb >= N) return;
    const int64_t jl = min64(N - 1, jb + 31);
    const int64_t j = jb + lane;
    const int64_t jc = min64(j, N - 1);
    const double ref = nu[jb];
    const double oj = nu[jc] - ref;
    const float ohi = (float)oj, olo = (float)(oj - (double)ohi);
    const float cmin = agg[4 * (layer0 + nloc)];
    const size_t lay = (size_t)nloc * nl;
    NearTile& tl = tiles[w];
    int64_t cb, ce;
    near_window(nu_hat, nl, nu[jb], nu[jl], (double)NEAR_Z / (double)cmin * (1.0 + 1e-6), &cb, &ce);
    if (!XS_CHECK(cb >= 0 && cb <= ce && ce <= nl)) ce = cb;
    const bool live = j <= jl;
    float shi = 0.0f, slo = 0.0f;
    for (int64_t t0 = cb; t0 < ce; t0 += 32) {
        const int64_t l = t0 + lane;
        __syncwarp();
        // stage only lines whose near range meets this warp's points
        bool hit = false;
        if (l < ce) {
            const int2 nr = jnear[lay + l];
            hit = nr.x <= nr.y && nr.x <= (int)jl && nr.y >= (int)jb && XS_CHECK(nr.x >= 0 && nr.y < N);
            if (hit) {
                const double o = nu_hat[l] - ref;
                const float bh = (float)o;
                tl.bhi[lane] = bh;
                tl.blo[lane] = (float)(o - (double)bh);
                const float4 p2 = rec2[lay + l];
                tl.r2[lane] = p2;
                tl.xa[lane] = make_float2(-p2.x * bh, p2.y * p2.y);
                tl.clo[lane] = clo[lay + l];
                tl.jn[lane] = nr;
                float C[ASY_N];
                asy_coeffs(p2.y, p2.z, C);
                store16(tl.hc[lane], C, ASY_N);
                if (p2.y * p2.y < NEAR_POLY_Z2) series_table(p2.y, tl.sd[lane]);
            }
        }
        __syncwarp();
        // the staged lines in ascending order (warp-uniform loop)
        unsigned m = __ballot_sync(0xffffffffu, hit);
        float acc = 0.0f;
        while (m) {
            const int i = __ffs(m) - 1;
            m &= m - 1;
            const bool inr = live && in_range((int)j, tl.jn[i]);
            // x to FP32 accuracy suffices for the polynomial (a rational
            // function of x); the series takes the exact pair
            const float2 xa = tl.xa[i];
            const float xq = fmaf(tl.r2[i].x, ohi, xa.x);
            const float z2 = fmaf(xq, xq, xa.y);
            const bool ser = inr && z2 < NEAR_POLY_Z2;
            if (!__any_sync(0xffffffffu, ser)) {
                // no lane in the series zone: the polynomial, branch-free
                const float hv = horner13(tl.hc[i], rcp_fast(z2));
                acc += inr ? hv : 0.0f;
            } else if (inr) {
                if (!ser) {
                    acc += horner13(tl.hc[i], rcp_fast(z2));
                } else {
                    const float4 p2 = tl.r2[i];
                    float x, xl;
                    scaled_pair(ohi - tl.bhi[i], olo - tl.blo[i], p2.x, tl.clo[i], &x, &xl);
                    float wr, wi;
                    w_series_tab(x, xl, p2.y, p2.w, tl.sd[i], &wr, &wi);
                    acc = fmaf(p2.z, wr, acc);
                }
            }
        }
        // fold the chunk's FP32 partial into the compensated sum (TwoSum)
        const float t = shi + acc;
        const float bb = t - shi;
        slo += (shi - (t - bb)) + (acc - bb);
        shi = t;
    }
    if (live) near_sum[(size_t)nloc * N + j] = (double)shi + (double)slo;
}

// The adjoint's near pairs: per point, sum of lambda_j (f_T, f_b) (see
// linesum_adjoint_kernel), reduced per block into part[layer][block].
__global__ void __launch_bounds__(NR_THREADS, 6) near_adjoint_kernel(
    const double* __restrict__ nu_hat, int64_t nl, const float4* __restrict__ rec2, const float* __restrict__ clo,
    const float* __restrict__ rec3, const int2* __restrict__ jnear, const float* __restrict__ agg,
    const double* __restrict__ nu, int64_t N, int layer0, const double* __restrict__ T,
    const double* __restrict__ g_sigma, double lam_scale, double* __restrict__ part)
{
    __shared__ NearAdjTile tiles[NR_THREADS / 32];
    __shared__ double red[2][NR_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nloc = blockIdx.y;
    const int layer = layer0 + nloc;
    const int64_t jb = (int64_t)blockIdx.x * NR_THREADS + w * 32;
    double sT = 0.0, sB = 0.0;
    if (jb < N) {
        const int64_t jl = min64(N - 1, jb + 31);
        const int64_t j = jb + lane;
        const int64_t jc = min64(j, N - 1);
        const double ref = nu[jb];
        const double oj = nu[jc] - ref;
        const float ohi = (float)oj, olo = (float)(oj - (double)ohi);
        const float cmin = agg[4 * layer];
        const float half_invT = (float)(0.5 / T[layer]);
        const float lam = (j <= jl) ? (float)(g_sigma[(size_t)layer * N + j] * lam_scale) : 0.0f;
        const size_t lay = (size_t)nloc * nl;
        NearAdjTile& tl = tiles[w];
        int64_t cb, ce;
        near_window(nu_hat, nl, nu[jb], nu[jl], (double)NEAR_Z / (double)cmin * (1.0 + 1e-6), &cb, &ce);
        if (!XS_CHECK(cb >= 0 && cb <= ce && ce <= nl)) ce = cb;
        float aT = 0.0f, aB = 0.0f;
        for (int64_t t0 = cb; t0 < ce; t0 += 32) {
            const int64_t l = t0 + lane;
            __syncwarp();
            // stage only lines whose near range meets this warp's points
            bool hit = false;
            if (l < ce) {
                const int2 nr = jnear[lay + l];
                hit = nr.x <= nr.y && nr.x <= (int)jl && nr.y >= (int)jb && XS_CHECK(nr.x >= 0 && nr.y < N);
                if (hit) {
                    const double o = nu_hat[l] - ref;
                    const float bh = (float)o;
                    tl.bhi[lane] = bh;
                    tl.blo[lane] = (float)(o - (double)bh);
                    const float4 p2 = rec2[lay + l];
                    tl.r2[lane] = p2;
                    tl.xa[lane] = make_float2(-p2.x * bh, p2.y * p2.y);
                    tl.clo[lane] = clo[lay + l];
                    tl.jn[lane] = nr;
                    const float aS = rec3[2 * (lay + l)], nn = rec3[2 * (lay + l) + 1];
                    tl.aS[lane] = aS;
                    tl.nn[lane] = nn;
                    float F[ASY_N + 1], G[ASY_N + 1];
                    asy_coeffs_adj(p2.y, p2.z, aS, half_invT, nn, F, G);
                    store16(tl.hf[lane], F, ASY_N + 1);
                    store16(tl.hg[lane], G, ASY_N + 1);
                    if (p2.y * p2.y < NEAR_POLY_Z2) series_table(p2.y, tl.sd[lane]);
                }
            }
            __syncwarp();
            unsigned m = __ballot_sync(0xffffffffu, hit);
            while (m) {
                const int i = __ffs(m) - 1;
                m &= m - 1;
                const bool inr = j <= jl && in_range((int)j, tl.jn[i]);
                const float2 xa = tl.xa[i];
                const float xq = fmaf(tl.r2[i].x, ohi, xa.x);
                const float z2 = fmaf(xq, xq, xa.y);
                const bool ser = inr && z2 < NEAR_POLY_Z2;
                if (!__any_sync(0xffffffffu, ser)) {
                    // no lane in the series zone: the polynomials, branch-free
                    const float u = rcp_fast(z2);
                    const float ft = horner14(tl.hf[i], u), fb = horner14(tl.hg[i], u);
                    aT = fmaf(inr ? lam : 0.0f, inr ? ft : 0.0f, aT);
                    aB = fmaf(inr ? lam : 0.0f, inr ? fb : 0.0f, aB);
                } else if (inr) {
                    float ft, fb;
                    if (!ser) {
                        const float u = rcp_fast(z2);
                        ft = horner14(tl.hf[i], u);
                        fb = horner14(tl.hg[i], u);
                    } else {
                        const float4 p2 = tl.r2[i];
                        float x, xl;
                        scaled_pair(ohi - tl.bhi[i], olo - tl.blo[i], p2.x, tl.clo[i], &x, &xl);
                        const float a = p2.y;
                        float wr, wi;
                        w_series_tab(x, xl, a, p2.w, tl.sd[i], &wr, &wi);
                        // w' = -2 z w + 2i/sqrt(pi);  H_x = Re w', H_a = -Im w'
                        const float dr = -2.0f * (x * wr - a * wi);
                        const float di = -2.0f * (x * wi + a * wr) + (float)(2.0 * INV_SQRTPI);
                        const float V0 = p2.z * wr;
                        const float V1 = p2.z * x * dr;
                        const float V2 = -p2.z * a * di;
                        const float Db = -(V0 + V1 + V2);
                        ft = tl.aS[i] * V0 + half_invT * Db + tl.nn[i] * V2;
                        fb = V2;
                    }
                    aT = fmaf(lam, ft, aT);
                    aB = fmaf(lam, fb, aB);
                }
            }
            sT += (double)aT;
            sB += (double)aB;
            aT = 0.0f;
            aB = 0.0f;
        }
    }
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
        for (int i = 0; i < NR_THREADS / 32; ++i) {
            a += red[0][i];
            b += red[1][i];
        }
        const size_t o = (size_t)layer * gridDim.x + blockIdx.x;
        part[2 * o] = a;
        part[2 * o + 1] = b;
    }
}

// ------------------------------------------------------------------ K6: adjoint

// Per evaluation the adjoint accumulates
//   f_T = (dlnS/dT) V0 + (1/(2T)) D_beta + (-n/T) D_gamma   and   f_b = D_gamma
// with V0 = Av H, D_beta = beta d sigma/d beta = -Av (H + x H_x + a H_a),
// D_gamma = gamma d sigma/d gamma = Av a H_a, weighted by lambda_j = g_sigma[n][j].
// In the Lorentz-wing form (K = 1 of the asymptotic series, rho = 1/(dnu^2 + gamma^2),
// B = 2 beta^2, G = gamma^2, Al = s gamma/pi):
//   V0 = Al (rho + 1.5 B rho^2 - 2 G B rho^3),  D_beta = Al B (3 rho^2 - 4 G rho^3),
//   D_gamma = Al (rho + (1.5 B - 2 G) rho^2 - 12 G B rho^3 + 12 G^2 B rho^4),
// so f_T = rho (T1 + rho (T2 + rho (T3 + rho T4))) and f_b = rho (U1 + ... U4) with
// per-line coefficients.  At |z| >= 25 the K = 2 terms are below 6e-6 of a term.
// With the K = 2 terms (V0 from the forward's degree-5 form, Q = B^2 Al):
//   V0      += Q rho^3 (3.75 - 15 G rho + 12 G^2 rho^2),
//   D_beta  += Q rho^3 (15 - 60 G rho + 48 G^2 rho^2),
//   D_gamma += Q rho^3 (3.75 - 67.5 G rho + 180 G^2 rho^2 - 120 G^3 rho^3),
// degree 6 in rho; used where |z| < 25 (and for the lines of a chunk that has
// masked ones), where they truncate below 7e-7 of a term for |z| >= 16.5.
template <class R>
struct AdjTile {
    float4 q0[32];           // (-b, -b, G, G)
    float4 qt0[32], qt1[32]; // (T1, T1, T2, T2), (T3, T3, T4, T4)
    float4 qu0[32], qu1[32]; // (U1, U1, U2, U2), (U3, U3, U4, U4)
    float4 qt2[32], qu2[32]; // K = 2: (T5, T5, T6, T6), (U5, U5, U6, U6)
    int2 jr[32], jn[32];
    R bhi[32];
    typename vec4<R>::type r2[32];
    R aS[32], nn[32];
};

// Turn lane's line of the tile from the K = 1 adjoint forms into the K = 2 ones.
__device__ __forceinline__ void adj_k2_coeffs(AdjTile<float>& tl, int i, float hT)
{
    const float G = tl.q0[i].z, Al = tl.qu0[i].x, c = tl.r2[i].x;
    const float aS = tl.aS[i], nn = tl.nn[i];
    const float c2 = c * c;
    const float Q = Al * rcp_fast(c2 * c2); // B^2 Al with B = 1/c^2
    const float4 t1 = tl.qt1[i], u1 = tl.qu1[i];
    const float GQ = G * Q, G2Q = G * GQ;
    const float T3 = fmaf(Q, 3.75f * aS + 15.0f * hT + 3.75f * nn, t1.x);
    const float T4 = fmaf(-GQ, 15.0f * aS + 60.0f * hT + 67.5f * nn, t1.z);
    const float T5 = G2Q * (12.0f * aS + 48.0f * hT + 180.0f * nn);
    const float T6 = -120.0f * G * G2Q * nn;
    const float U3 = fmaf(3.75f, Q, u1.x), U4 = fmaf(-67.5f, GQ, u1.z);
    const float U5 = 180.0f * G2Q, U6 = -120.0f * G * G2Q;
    tl.qt1[i] = make_float4(T3, T3, T4, T4);
    tl.qu1[i] = make_float4(U3, U3, U4, U4);
    tl.qt2[i] = make_float4(T5, T5, T6, T6);
    tl.qu2[i] = make_float4(U5, U5, U6, U6);
}

// packed adjoint over lines [i0, i1); MASKED: per (line, point) by far_point;
// DEG2: the K = 1 forms with the rho^3 and rho^4 terms dropped (below 1e-6 of the
// leading one where the caller takes it); K2: the degree-6 K = 2 forms (after
// adj_k2_coeffs); otherwise the K = 1 forms.  Per point sums of f_T and f_b (lambda
// is applied once per chunk by the caller).
template <bool MASKED, bool DEG2 = false, bool K2 = false>
__device__ __forceinline__ void far_adj_lines(const AdjTile<float>& tl, int i0, int i1, const float2 (&o2)[LS_G / 2],
                                              float2 (&aT)[LS_G / 2], float2 (&aB)[LS_G / 2], const int (&jg)[LS_G])
{
    constexpr int UNROLL = K2 ? 2 : 4; // the longer K = 2 forms keep fewer lines in flight
#pragma unroll UNROLL
    for (int i = i0; i < i1; ++i) {
        const float4 v0 = tl.q0[i], t0 = tl.qt0[i], t1 = tl.qt1[i], u0 = tl.qu0[i], u1 = tl.qu1[i];
        float4 t2 = make_float4(0.f, 0.f, 0.f, 0.f), u2 = t2;
        if (K2) {
            t2 = tl.qt2[i];
            u2 = tl.qu2[i];
        }
        const float2 nb = f2lo(v0), G = f2hi(v0);
        int2 cut = make_int2(0, 0), nr = make_int2(1, 0);
        if (MASKED) {
            cut = tl.jr[i];
            nr = tl.jn[i];
        }
#pragma unroll
        for (int p = 0; p < LS_G / 2; ++p) {
            float2 d = __fadd2_rn(o2[p], nb);
            float2 rho = rcp2(__ffma2_rn(d, d, G));
            float2 pt, pu;
            if (DEG2) {
                pt = __ffma2_rn(f2hi(t0), rho, f2lo(t0));
                pu = __ffma2_rn(f2hi(u0), rho, f2lo(u0));
            } else if (K2) {
                pt = __ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(f2hi(t2), rho, f2lo(t2)), rho, f2hi(t1)),
                                                                 rho, f2lo(t1)), rho, f2hi(t0)), rho, f2lo(t0));
                pu = __ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(f2hi(u2), rho, f2lo(u2)), rho, f2hi(u1)),
                                                                 rho, f2lo(u1)), rho, f2hi(u0)), rho, f2lo(u0));
            } else {
                pt = __ffma2_rn(__ffma2_rn(__ffma2_rn(f2hi(t1), rho, f2lo(t1)), rho, f2hi(t0)), rho, f2lo(t0));
                pu = __ffma2_rn(__ffma2_rn(__ffma2_rn(f2hi(u1), rho, f2lo(u1)), rho, f2hi(u0)), rho, f2lo(u0));
            }
            if (MASKED) {
                rho.x = far_point(jg[2 * p], cut, nr) ? rho.x : 0.0f;
                rho.y = far_point(jg[2 * p + 1], cut, nr) ? rho.y : 0.0f;
            }
            aT[p] = __ffma2_rn(rho, pt, aT[p]);
            aB[p] = __ffma2_rn(rho, pu, aB[p]);
        }
    }
}

__device__ __forceinline__ void chunk_far_adj(AdjTile<float>& tl, const WarpPoints<float>& pts,
                                              const float (&lam)[LS_G], float cmin, float amin, float amax, float hT,
                                              float& accT, float& accB)
{
    const int lane = threadIdx.x & 31;
    const unsigned ok = __ballot_sync(0xffffffffu, covers_far(tl.jr[lane], tl.jn[lane], pts.jw0, pts.jw1));
    float2 o2[LS_G / 2], aT[LS_G / 2], aB[LS_G / 2];
#pragma unroll
    for (int p = 0; p < LS_G / 2; ++p) {
        o2[p] = make_float2(pts.ohi[2 * p], pts.ohi[2 * p + 1]);
        aT[p] = make_float2(0.0f, 0.0f);
        aB[p] = make_float2(0.0f, 0.0f);
    }
    if (ok == 0xffffffffu) {
        // the rho^3 and rho^4 terms of f_T and f_b come from the F2 term (relative
        // size up to 12 a^2/|z|^4): dropped where that is below 1e-6; below |z| = 25
        // the K = 2 terms are kept
        const float z2 = chunk_z2min(tl.q0[0].x, tl.q0[31].x, pts, cmin, amin);
        if (z2 < ADJ_K2_Z2) {
            adj_k2_coeffs(tl, lane, hT);
            __syncwarp();
            far_adj_lines<false, false, true>(tl, 0, 32, o2, aT, aB, pts.jg);
        } else if (12.0f * amax * amax <= 1.0e-6f * z2 * z2) {
            far_adj_lines<false, true>(tl, 0, 32, o2, aT, aB, pts.jg);
        } else {
            far_adj_lines<false>(tl, 0, 32, o2, aT, aB, pts.jg);
        }
    } else {
        // a chunk with lines that cover the warp's points only in part: K = 2 forms
        // throughout (its far pairs reach down to the near boundary)
        adj_k2_coeffs(tl, lane, hT);
        __syncwarp();
        int i = 0;
        while (i < 32) {
            const unsigned rest = ok >> i;
            if (rest & 1u) {
                const unsigned zeros = ~rest;
                const int j = (zeros == 0u) ? 32 : i + __ffs(zeros) - 1;
                far_adj_lines<false, false, true>(tl, i, j, o2, aT, aB, pts.jg);
                i = j;
            } else {
                far_adj_lines<true, false, true>(tl, i, i + 1, o2, aT, aB, pts.jg);
                ++i;
            }
        }
    }
#pragma unroll
    for (int p = 0; p < LS_G / 2; ++p) {
        accT = fmaf(lam[2 * p], aT[p].x, fmaf(lam[2 * p + 1], aT[p].y, accT));
        accB = fmaf(lam[2 * p], aB[p].x, fmaf(lam[2 * p + 1], aB[p].y, accB));
    }
}

__device__ __forceinline__ void chunk_fp64_adj(const AdjTile<double>& tl, const WarpPoints<double>& pts,
                                               const double (&lam)[LS_G], double half_invT, double& accT,
                                               double& accB)
{
    for (int i = 0; i < 32; ++i) {
        const double bh = tl.bhi[i];
        const double4_32a p2 = tl.r2[i];
        const int2 jr = tl.jr[i];
        const double aS = tl.aS[i], nn = tl.nn[i];
#pragma unroll
        for (int g = 0; g < LS_G; ++g) {
            if (in_range(pts.jg[g], jr)) {
                const double x = fabs(pts.ohi[g] - bh) * p2.x;
                const double a = p2.y;
                double w4[4];
                voigt_w_dw<double>(x, 0.0, a, p2.w, w4, nullptr);
                // H_x = Re w', H_a = -Im w'
                const double V0 = p2.z * w4[0];
                const double V1 = p2.z * x * w4[2];
                const double V2 = -p2.z * a * w4[3];
                const double Db = -(V0 + V1 + V2);
                const double ft = aS * V0 + half_invT * Db + nn * V2;
                accT = fma(lam[g], ft, accT);
                accB = fma(lam[g], V2, accB);
            }
        }
    }
}

template <class R, bool FAST>
__global__ void __launch_bounds__(LS_THREADS, MinBlocks<R>::v) linesum_adjoint_kernel(
    const double* __restrict__ nu_hat, const float2* __restrict__ nuf, const int2* __restrict__ jrange,
    const typename vec4<R>::type* __restrict__ rec1, const typename vec4<R>::type* __restrict__ rec2,
    const R* __restrict__ rec3, const int2* __restrict__ jnear, const float* __restrict__ agg,
    const double* __restrict__ nu, int64_t N, int64_t nl, int layer0, int ksplit, int64_t lb,
    const double* __restrict__ T, const double* __restrict__ g_sigma, double lam_scale, double* __restrict__ part,
    int nstrips)
{
    using R4 = typename vec4<R>::type;
    __shared__ AdjTile<R> tiles[LS_WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int strip = blockIdx.x, nloc = blockIdx.y, kc = blockIdx.z;
    const int layer = layer0 + nloc;
    const int64_t j0 = (int64_t)strip * LS_STRIP;
    const int64_t jlast = min64(N - 1, j0 + LS_STRIP - 1);
    const R half_invT = (R)(0.5 / T[layer]);
    const float cmin = agg[4 * layer], amin = agg[4 * layer + 1], amax = agg[4 * layer + 2];
    AdjTile<R>& tl = tiles[w];

    double sT = 0.0, sB = 0.0;
    WarpPoints<R> pts;
    if (pts.init(nu, j0 + (int64_t)w * (32 * LS_G), jlast)) {
        int64_t cb, ce;
        strip_window(jrange, nl, pts.jw0, pts.jw1, ksplit, lb, kc, &cb, &ce);
        if (!XS_CHECK(cb >= 0 && cb <= ce && ce <= nl)) ce = cb;
        const size_t lay = (size_t)nloc * nl;
        const R4* r1g = rec1 + lay;
        const R4* r2g = rec2 + lay;
        const R* r3g = rec3 + 2 * lay;
        const int2* jng = FAST ? jnear + lay : nullptr;
        R lam[LS_G];
#pragma unroll
        for (int g = 0; g < LS_G; ++g)
            lam[g] = (pts.jg[g] <= jlast) ? (R)(g_sigma[(size_t)layer * N + pts.jg[g]] * lam_scale) : R(0);

        LineRec<R> nx;
        R naS = R(0), nnn = R(0);
        if (cb < ce) {
            nx.load(nu_hat, nuf, jrange, r1g, r2g, jng, cb + lane, ce);
            if (cb + lane < ce) {
                naS = r3g[2 * (cb + lane)];
                nnn = r3g[2 * (cb + lane) + 1];
            }
        }
        R accT = R(0), accB = R(0);
        for (int64_t t0 = cb; t0 < ce; t0 += 32) {
            {
                R bh;
                line_offset(nx, pts, &bh);
                tl.bhi[lane] = bh;
                tl.r2[lane] = nx.p2;
                tl.jr[lane] = nx.jr;
                tl.jn[lane] = nx.jn;
                tl.aS[lane] = naS;
                tl.nn[lane] = nnn;
                if (FAST) {
                    // fast-form coefficients from G, Al, F1 = 1.5 B Al, F2 = -2 G B Al
                    const float G = (float)nx.p1.x, Al = (float)nx.p1.y, F1 = (float)nx.p1.z, F2 = (float)nx.p1.w;
                    const float aS = (float)naS, nn = (float)nnn, hT = (float)half_invT;
                    const float T1 = Al * (aS + nn);
                    const float T2 = aS * F1 + hT * 2.0f * F1 + nn * (F1 - 2.0f * G * Al);
                    const float T3 = aS * F2 + hT * 2.0f * F2 + nn * 6.0f * F2;
                    const float T4 = nn * (-6.0f * G * F2);
                    const float U1 = Al, U2 = F1 - 2.0f * G * Al, U3 = 6.0f * F2, U4 = -6.0f * G * F2;
                    const float nb = -(float)bh;
                    tl.q0[lane] = make_float4(nb, nb, G, G);
                    tl.qt0[lane] = make_float4(T1, T1, T2, T2);
                    tl.qt1[lane] = make_float4(T3, T3, T4, T4);
                    tl.qu0[lane] = make_float4(U1, U1, U2, U2);
                    tl.qu1[lane] = make_float4(U3, U3, U4, U4);
                }
            }
            __syncwarp();
            if (t0 + 32 < ce) {
                int64_t l = t0 + 32 + lane;
                nx.load(nu_hat, nuf, jrange, r1g, r2g, jng, l, ce);
                naS = (l < ce) ? r3g[2 * l] : R(0);
                nnn = (l < ce) ? r3g[2 * l + 1] : R(0);
            }
            if constexpr (FAST)
                chunk_far_adj(tl, pts, lam, cmin, amin, amax, (float)half_invT, accT, accB);
            else
                chunk_fp64_adj(tl, pts, lam, half_invT, accT, accB);
            sT += (double)accT;
            sB += (double)accB;
            accT = R(0);
            accB = R(0);
            __syncwarp();
        }
    }
    // fixed-order warp reduction; one partial per warp (no block barrier, so a
    // warp that finishes early does not hold the block's slot)
    for (int o = 16; o > 0; o >>= 1) {
        sT += __shfl_xor_sync(0xffffffffu, sT, o);
        sB += __shfl_xor_sync(0xffffffffu, sB, o);
    }
    if (lane == 0) {
        const size_t o = (((size_t)layer * nstrips + strip) * ksplit + kc) * LS_WARPS + w;
        part[2 * o] = sT;
        part[2 * o + 1] = sB;
    }
}

// g_T[n] = sum over the main kernel's (strip, part, warp) partials and the near
// kernel's block partials of layer n (one block per layer, fixed order);
// gbl[n] the same for the broadening term.
__global__ void adjoint_reduce_kernel(const double* __restrict__ part, int per_layer,
                                      const double* __restrict__ part_near, int per_layer_near,
                                      double* __restrict__ g_T, double* __restrict__ gbl)
{
    __shared__ double red[2][256];
    const int n = blockIdx.x;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < per_layer; i += blockDim.x) {
        a += part[2 * ((size_t)n * per_layer + i)];
        b += part[2 * ((size_t)n * per_layer + i) + 1];
    }
    if (part_near)
        for (int i = threadIdx.x; i < per_layer_near; i += blockDim.x) {
            a += part_near[2 * ((size_t)n * per_layer_near + i)];
            b += part_near[2 * ((size_t)n * per_layer_near + i) + 1];
        }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        g_T[n] = red[0][0];
        gbl[n] = red[1][0];
    }
}

// g_b = sum over layers of gbl (in layer order) / s_b
__global__ void broad_sum_kernel(const double* __restrict__ gbl, int L, double inv_sb, double* __restrict__ g_b)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int n = 0; n < L; ++n) s += gbl[n];
        g_b[0] = s * inv_sb;
    }
}

} // namespace xsd

// ====================================================================== host side

using namespace xsd;

namespace {

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

int strips_of(int64_t N) { return (int)((N + LS_STRIP - 1) / LS_STRIP); }
int near_blocks(int64_t N) { return (int)((N + NR_THREADS - 1) / NR_THREADS); }

// Lists whose per-layer records (about 40 bytes a line) for the layers in flight
// (about six at four CTAs per SM) fit in 48 MB of L2 are split into equal parts of
// each warp's window; longer ones into absolute line blocks of at most
// LS_BLOCK_MAX lines, which keeps one block's records for the layers in flight at
// about 16 MB, inside one die's half of the L2.
constexpr int64_t LS_L2_LINES = 200000;
constexpr int64_t LS_BLOCK_MAX = 65536;

// Split of the line windows into ksplit parts: enough CTAs to fill the GPU
// (several waves of 8 resident CTAs per SM); *lb = 0 for equal parts of each
// window, else the absolute block length (a multiple of 32).
void choose_split(int64_t nl, int64_t N, int Lc, int* ksplit, int64_t* lb)
{
    const int strips = strips_of(N);
    const int64_t ctas = (int64_t)strips * Lc;
    const int64_t target = 152 * 8 * 6;
    int64_t k = std::max<int64_t>(1, (target + ctas - 1) / ctas);
    if (nl <= LS_L2_LINES) {
        *ksplit = (int)std::min<int64_t>(k, std::min<int64_t>(std::max<int64_t>(1, nl / 1024), 64));
        *lb = 0;
        return;
    }
    k = std::min<int64_t>(k, nl / 1024);
    k = std::max<int64_t>(k, (nl + LS_BLOCK_MAX - 1) / LS_BLOCK_MAX);
    int64_t b = (nl + k - 1) / k;
    b = (b + 31) & ~(int64_t)31;
    *lb = b;
    *ksplit = (int)((nl + b - 1) / b);
}

struct XsPlan {
    int prec, Lc, ksplit, nchunks;
    int64_t lb; // lines per block of the split
    size_t off_jr, off_nuf, off_agg, off_rec1, off_rec2, off_rec3, off_clo, off_jn, off_near, off_part, off_npart,
        off_gbl, total;
};

XsPlan plan_xs(int64_t nl, int64_t N, int32_t L, int prec, int Lc)
{
    XsPlan p;
    p.prec = prec;
    p.Lc = Lc;
    const bool mixed = (prec == XS_PREC_MIXED);
    const size_t rs = mixed ? sizeof(float) : sizeof(double);
    const size_t n1 = (size_t)std::max<int64_t>(nl, 1);
    choose_split(nl, N, Lc, &p.ksplit, &p.lb);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    p.off_jr = take(sizeof(int2) * n1);
    p.off_nuf = take(mixed ? sizeof(float2) * n1 : 0);
    p.off_agg = take(sizeof(float) * 4 * (size_t)L);
    p.off_rec1 = take(4 * rs * n1 * Lc);
    p.off_rec2 = take(4 * rs * n1 * Lc);
    p.off_rec3 = take(2 * rs * n1 * Lc);
    p.off_clo = take(rs * n1 * Lc);
    p.off_jn = take(mixed ? sizeof(int2) * n1 * Lc : 0);
    p.off_near = take(mixed ? sizeof(double) * (size_t)Lc * N : 0);
    size_t fwd_part = (p.ksplit > 1) ? sizeof(double) * (size_t)p.ksplit * Lc * N : 0;
    size_t adj_part = sizeof(double) * 2 * (size_t)L * strips_of(N) * p.ksplit * LS_WARPS;
    p.off_part = take(std::max(fwd_part, adj_part));
    p.off_gbl = take(sizeof(double) * (size_t)L);
    p.off_npart = take(mixed ? sizeof(double) * 2 * (size_t)L * near_blocks(N) : 0);
    p.total = off;
    p.nchunks = (L + Lc - 1) / Lc;
    return p;
}

} // namespace

size_t xs_workspace_bytes(int64_t n_lines, int64_t N, int32_t L, int prec)
{
    if (n_lines < 0 || N <= 0 || L <= 0) return 0;
    return plan_xs(n_lines, N, L, prec, L).total;
}

size_t xs_workspace_min_bytes(int64_t n_lines, int64_t N, int32_t L, int prec)
{
    if (n_lines < 0 || N <= 0 || L <= 0) return 0;
    return plan_xs(n_lines, N, L, prec, 1).total;
}

namespace xsi {

static int pick_plan(int64_t nl, int64_t N, int32_t L, int prec, size_t ws_bytes, XsPlan* out)
{
    int Lc = L;
    while (true) {
        XsPlan p = plan_xs(nl, N, L, prec, Lc);
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
    constexpr bool FAST = std::is_same<R, float>::value;
    const bool reuse = adjoint && (flags & XS_RUN_REUSE) && p.nchunks == 1;
    const bool want_rec3 = adjoint || (flags & XS_RUN_KEEP_ADJ);
    using R4 = typename vec4<R>::type;
    const int64_t nl = ln->n;
    const double scale = FAST ? MIXED_SCALE : 1.0;
    const double unscale = FAST ? MIXED_UNSCALE : 1.0;
    int2* jr = (int2*)(ws + p.off_jr);
    float2* nuf = FAST ? (float2*)(ws + p.off_nuf) : nullptr;
    float* agg = (float*)(ws + p.off_agg);
    R4* rec1 = (R4*)(ws + p.off_rec1);
    R4* rec2 = (R4*)(ws + p.off_rec2);
    R* rec3 = (R*)(ws + p.off_rec3);
    R* clo = (R*)(ws + p.off_clo);
    int2* jn = FAST ? (int2*)(ws + p.off_jn) : nullptr;
    double* near = FAST ? (double*)(ws + p.off_near) : nullptr;
    double* part = (double*)(ws + p.off_part);
    double* npart = FAST ? (double*)(ws + p.off_npart) : nullptr;
    const int strips = strips_of(N);
    const int nblk = near_blocks(N);

    if (nl == 0) {
        if (adjoint) {
            if (cudaMemsetAsync(g_T, 0, sizeof(double) * L, st) != cudaSuccess) return XS_ECUDA;
            if (cudaMemsetAsync(g_b, 0, sizeof(double), st) != cudaSuccess) return XS_ECUDA;
        } else {
            size_t es = FAST ? sizeof(float) : sizeof(double);
            if (cudaMemsetAsync(sigma, 0, es * (size_t)L * N, st) != cudaSuccess) return XS_ECUDA;
        }
        return XS_OK;
    }
    if (!reuse) {
        cut_range_kernel<<<(unsigned)((nl + 255) / 256), 256, 0, st>>>(ln->nu_hat, nl, nu, N, W, jr, nuf);
        layer_agg_init_kernel<<<(4 * L + 255) / 256, 256, 0, st>>>(agg, 4 * L);
        count_launch(2);
    }
    for (int c = 0; c < p.nchunks; ++c) {
        int l0 = c * p.Lc;
        int lc = std::min(p.Lc, L - l0);
        if (!reuse) {
            dim3 pg((unsigned)((nl + 255) / 256), (unsigned)lc);
            line_params_kernel<R><<<pg, 256, 0, st>>>(ln->nu_hat, ln->ln_S0, ln->elower, ln->gamma_ref, ln->n_temp,
                                                       nl, ln->mass_amu, ln->q_exponent, T, P, l0, sb, scale, rec1,
                                                       rec2, clo, want_rec3 ? rec3 : nullptr, agg, nu, N, jr, jn);
            count_launch();
        }
        dim3 grid((unsigned)strips, (unsigned)lc, (unsigned)p.ksplit);
        dim3 ngrid((unsigned)nblk, (unsigned)lc);
        if (!adjoint) {
            if (FAST) {
                near_sum_kernel<<<ngrid, NR_THREADS, 0, st>>>(ln->nu_hat, nl, (const float4*)rec2, (const float*)clo,
                                                              jn, agg, nu, N, l0, near);
                count_launch();
            }
            prof_begin(0, st);
            linesum_kernel<R, FAST><<<grid, LS_THREADS, 0, st>>>(ln->nu_hat, nuf, jr, rec1, rec2, jn, agg, nu, N, nl, l0,
                                                                 p.ksplit, p.lb, unscale, sigma, FAST ? 1 : 0, part,
                                                                 lc, near);
            prof_end(0, st);
            count_launch();
            if (p.ksplit > 1) {
                count_launch();
                int64_t cnt = (int64_t)lc * N;
                combine_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(part, p.ksplit, cnt, (int64_t)l0 * N,
                                                                              cnt, unscale, sigma, FAST ? 1 : 0);
            }
        } else {
            prof_begin(1, st);
            linesum_adjoint_kernel<R, FAST><<<grid, LS_THREADS, 0, st>>>(ln->nu_hat, nuf, jr, rec1, rec2, rec3, jn, agg,
                                                                         nu, N, nl, l0, p.ksplit, p.lb, T, g_sigma,
                                                                         unscale, part, strips);
            prof_end(1, st);
            count_launch();
            if (FAST) {
                near_adjoint_kernel<<<ngrid, NR_THREADS, 0, st>>>(ln->nu_hat, nl, (const float4*)rec2,
                                                                  (const float*)clo, (const float*)rec3, jn, agg, nu,
                                                                  N, l0, T, g_sigma, unscale, npart);
                count_launch();
            }
        }
    }
    if (adjoint) {
        double* gbl = (double*)(ws + p.off_gbl);
        adjoint_reduce_kernel<<<L, 256, 0, st>>>(part, strips * p.ksplit * LS_WARPS, npart, nblk, g_T, gbl);
        broad_sum_kernel<<<1, 32, 0, st>>>(gbl, L, 1.0 / sb, g_b);
        count_launch(2);
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

XS_CHECK_ACCESSOR(linesum)
