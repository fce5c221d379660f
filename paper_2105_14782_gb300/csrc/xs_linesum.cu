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
constexpr int LS_TILE = LS_THREADS;            // lines per shared-memory tile

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
        double Tn = T[layer0 + n], Pn = P_bar[layer0 + n];
        double nuh = nu_hat[l];
        double qr = pow(Tn / Tref, qexp);
        double boltz = exp(ln_S0[l] - c2 * elower[l] * (1.0 / Tn - 1.0 / Tref));
        double stim = expm1(-c2 * nuh / Tn) / expm1(-c2 * nuh / Tref);
        double S = boltz / qr * stim;
        double beta = sqrt(kB * Tn / (mass * amu)) * nuh / cL;
        double gam = sb * gamma_ref[l] * pow(Tn / Tref, -n_temp[l]) * (Pn / bar_per_atm);
        double s = S * scale;
        double B = 2.0 * beta * beta, G = gam * gam;
        double c = 1.0 / (SQRT2 * beta);
        double a = gam * c;
        double Al = s * gam / PI;
        double Av = s * c * INV_SQRTPI;
        double Kc = 0.0;
        if (a * a < (double)Tier<R>::z2_mid2) {
            const double h = (double)Tier<R>::h;
            double s1 = 0.0;
            for (int k = 1; k <= 40; ++k) {
                double kh = k * h;
                s1 += exp(-kh * kh) / (kh * kh + a * a);
            }
            Kc = erfcx(a) - 2.0 * a * h / PI * s1;
        }
        size_t idx = (size_t)n * nl + l;
        typename vec4<R>::type v1, v2;
        v1.x = (R)G;
        v1.y = (R)Al;
        v1.z = (R)(1.5 * B * Al);
        v1.w = (R)(-2.0 * G * B * Al);
        v2.x = (R)c;
        v2.y = (R)a;
        v2.z = (R)Av;
        v2.w = (R)Kc;
        rec1[idx] = v1;
        rec2[idx] = v2;
        clo[idx] = (R)(c - (double)v2.x); // the part of c the rounded value misses
        if (rec3) {
            double u = c2 * nuh / Tn;
            double dlnS = c2 * elower[l] / (Tn * Tn) - qexp / Tn - (u / Tn) / expm1(u);
            rec3[2 * idx] = (R)dlnS;
            rec3[2 * idx + 1] = (R)(-n_temp[l] / Tn);
        }
        cmin = (float)c * (1.0f - 1e-6f);
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

// Offsets: FP32 path keeps nu relative to the strip reference as hi + lo floats;
// FP64 path keeps absolute doubles.
template <class R> struct Off;
template <> struct Off<float> {
    __device__ static void make(double v, double ref, float* hi, float* lo)
    {
        double o = v - ref;
        *hi = (float)o;
        *lo = (float)(o - (double)*hi);
    }
    __device__ static float dnu(float ohi, float olo, float bhi, float blo) { return (ohi - bhi) + (olo - blo); }
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
    __device__ static double dnu(double ohi, float, double bhi, float) { return ohi - bhi; }
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

template <class R>
struct LsShared {
    R bhi[LS_TILE];
    float blo[LS_TILE];
    typename vec4<R>::type r1[LS_TILE];
    typename vec4<R>::type r2[LS_TILE];
    R clo[LS_TILE];
    int2 jr[LS_TILE];
    float olo[LS_WARPS][32 * LS_G];
    int64_t win[2];
};

template <class R, bool FAST>
__global__ void __launch_bounds__(LS_THREADS) linesum_kernel(
    const double* __restrict__ nu_hat, const int2* __restrict__ jrange,
    const typename vec4<R>::type* __restrict__ rec1, const typename vec4<R>::type* __restrict__ rec2,
    const R* __restrict__ clo, const float* __restrict__ agg, const double* __restrict__ nu, int64_t N, int64_t nl,
    int layer0, int ksplit,
    double unscale, void* __restrict__ sigma, int sigma_is_float, double* __restrict__ partial, int L_total)
{
    using R4 = typename vec4<R>::type;
    __shared__ LsShared<R> sh;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int strip = blockIdx.x, nloc = blockIdx.y, kc = blockIdx.z;
    const int64_t j0 = (int64_t)strip * LS_STRIP;
    const int64_t jlast = min64(N - 1, j0 + LS_STRIP - 1);
    const double ref = nu[min64(jlast, j0 + LS_STRIP / 2)];

    if (tid == 0) {
        int64_t b = lb_jhi(jrange, nl, (int)j0);
        int64_t e = lb_jlo(jrange, nl, (int)jlast);
        if (e < b) e = b;
        int64_t len = e - b;
        int64_t per = (len + ksplit - 1) / ksplit;
        per = (per + 31) & ~(int64_t)31;
        int64_t cb = min64(e, b + per * kc), ce = min64(e, cb + per);
        sh.win[0] = cb;
        sh.win[1] = ce;
    }

    R ohi[LS_G];
    int jg[LS_G];
#pragma unroll
    for (int g = 0; g < LS_G; ++g) {
        int64_t j = j0 + w * (32 * LS_G) + g * 32 + lane;
        int64_t jc = min64(j, jlast);
        jg[g] = (int)j;
        float lo;
        Off<R>::make(nu[jc], ref, &ohi[g], &lo);
        sh.olo[w][g * 32 + lane] = lo;
    }
    // the warp's point span (first and last valid point) for tile classification
    const int jw0 = (int)min64(jlast, j0 + w * (32 * LS_G));
    const int jw1 = (int)min64(jlast, j0 + w * (32 * LS_G) + 32 * LS_G - 1);
    R ow0 = __shfl_sync(0xffffffffu, ohi[0], 0);
    R ow1 = ohi[LS_G - 1];
    {
        // last valid point of the warp may be in a lower (g, lane) slot
        int jl = jw1 - (int)(j0 + w * (32 * LS_G));
        int gl = jl >> 5, ll = jl & 31;
        R v = ohi[0];
#pragma unroll
        for (int g = 0; g < LS_G; ++g)
            if (g == gl) v = ohi[g];
        ow1 = __shfl_sync(0xffffffffu, v, ll);
    }
    const float cmin = agg[2 * (layer0 + nloc)];
    const float amin = agg[2 * (layer0 + nloc) + 1];

    R acc[LS_G], shi[LS_G], slo[LS_G];
#pragma unroll
    for (int g = 0; g < LS_G; ++g) {
        acc[g] = R(0);
        shi[g] = R(0);
        slo[g] = R(0);
    }
    __syncthreads();
    const int64_t cb = sh.win[0], ce = sh.win[1];
    const size_t lay = (size_t)nloc * nl; // records hold the current layer chunk

    for (int64_t t0 = cb; t0 < ce; t0 += LS_TILE) {
        {
            int64_t l = t0 + tid;
            if (l < ce) {
                double v = nu_hat[l];
                R bh;
                float bl;
                Off<R>::make(v, ref, &bh, &bl);
                sh.bhi[tid] = bh;
                sh.blo[tid] = bl;
                sh.r1[tid] = rec1[lay + l];
                sh.r2[tid] = rec2[lay + l];
                sh.clo[tid] = clo[lay + l];
                sh.jr[tid] = jrange[l];
            } else {
                // padding: a copy of the chunk's last line with zero amplitude, so
                // the sub-tile tests and the offsets stay those of real lines
                double v = nu_hat[ce - 1];
                R bh;
                float bl;
                Off<R>::make(v, ref, &bh, &bl);
                sh.bhi[tid] = bh;
                sh.blo[tid] = bl;
                R4 z1, z2;
                z1.x = R(1); z1.y = R(0); z1.z = R(0); z1.w = R(0);
                z2.x = R(1); z2.y = R(1); z2.z = R(0); z2.w = R(0);
                sh.r1[tid] = z1;
                sh.r2[tid] = z2;
                sh.clo[tid] = R(0);
                sh.jr[tid] = jrange[ce - 1];
            }
        }
        __syncthreads();
        const int nt = (int)min64(LS_TILE, ce - t0);
        for (int s0 = 0; s0 < nt; s0 += 32) {
            bool fast = false;
            if (FAST) {
                const int sl = s0 + 31;
                bool incut = (sh.jr[sl].x <= jw0) && (sh.jr[s0].y >= jw1);
                float bf = (float)sh.bhi[s0], bl = (float)sh.bhi[sl];
                float dist = fmaxf(fmaxf(bf - (float)ow1, (float)ow0 - bl), 0.0f);
                float xm = dist * cmin;
                fast = incut && (fmaf(xm, xm, amin * amin) >= (float)Tier<R>::z2_far);
            }
            if (fast) {
#pragma unroll 4
                for (int i = 0; i < 32; ++i) {
                    const R b = sh.bhi[s0 + i];
                    const R4 p = sh.r1[s0 + i];
#pragma unroll
                    for (int g = 0; g < LS_G; ++g) {
                        R d = ohi[g] - b;
                        R rho = rcp_fast(fma(d, d, p.x));
                        R u = fma(p.w, rho, p.z);
                        R q = fma(rho, u, p.y);
                        acc[g] = fma(rho, q, acc[g]);
                    }
                }
            } else {
                const int ns = min(32, nt - s0);
                for (int i = 0; i < ns; ++i) {
                    const int li = s0 + i;
                    const R bh = sh.bhi[li];
                    const float bl = sh.blo[li];
                    const R4 p2 = sh.r2[li];
                    const R cl = sh.clo[li];
                    const int2 jr = sh.jr[li];
#pragma unroll
                    for (int g = 0; g < LS_G; ++g) {
                        if (jg[g] >= jr.x && jg[g] <= jr.y) {
                            R dh, dl, x, xl;
                            Off<R>::dnu2(ohi[g], sh.olo[w][g * 32 + lane], bh, bl, &dh, &dl);
                            scaled_pair(dh, dl, p2.x, cl, &x, &xl);
                            R wr, wi;
                            faddeeva<R>(x, xl, p2.y, p2.w, &wr, &wi);
                            acc[g] = fma(p2.z, wr, acc[g]);
                        }
                    }
                }
            }
            // fold the 32-line partial into the running compensated sum
#pragma unroll
            for (int g = 0; g < LS_G; ++g) {
                R sres = shi[g] + acc[g];
                R bb = sres - shi[g];
                slo[g] += (shi[g] - (sres - bb)) + (acc[g] - bb);
                shi[g] = sres;
                acc[g] = R(0);
            }
        }
        __syncthreads();
    }

    const int layer = layer0 + nloc;
#pragma unroll
    for (int g = 0; g < LS_G; ++g) {
        if (jg[g] <= jlast) {
            double v = (double)shi[g] + (double)slo[g];
            size_t o = (size_t)layer * N + jg[g];
            if (ksplit == 1) {
                if (sigma_is_float)
                    ((float*)sigma)[o] = (float)(v * unscale);
                else
                    ((double*)sigma)[o] = v * unscale;
            } else {
                partial[((size_t)kc * L_total + nloc) * N + jg[g]] = v; // [ksplit][chunk layers][N]
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
struct AdjShared {
    R bhi[LS_TILE];
    float blo[LS_TILE];
    typename vec4<R>::type r2[LS_TILE];
    typename vec4<R>::type t[LS_TILE]; // fast form: f_T = rho (T1 + rho (T2 + rho (T3 + rho T4)))
    typename vec4<R>::type u[LS_TILE]; // fast form: f_b = rho (U1 + rho (U2 + rho (U3 + rho U4)))
    R G[LS_TILE];
    R clo[LS_TILE];
    R aS[LS_TILE], nn[LS_TILE];
    int2 jr[LS_TILE];
    float olo[LS_WARPS][32 * LS_G];
    double red[2][LS_WARPS];
    int64_t win[2];
};

// Per evaluation the adjoint accumulates
//   f_T = (dlnS/dT) V0 + (1/(2T)) D_beta + (-n/T) D_gamma   and   f_b = D_gamma
// with V0 = Av H, D_beta = beta d sigma/d beta = -Av (H + x H_x + a H_a),
// D_gamma = gamma d sigma/d gamma = Av a H_a, weighted by lambda_j = g_sigma[n][j].
template <class R, bool FAST>
__global__ void __launch_bounds__(LS_THREADS) linesum_adjoint_kernel(
    const double* __restrict__ nu_hat, const int2* __restrict__ jrange,
    const typename vec4<R>::type* __restrict__ rec1, const typename vec4<R>::type* __restrict__ rec2,
    const R* __restrict__ clo, const R* __restrict__ rec3, const float* __restrict__ agg, const double* __restrict__ nu,
    int64_t N,
    int64_t nl, int layer0, int ksplit, const double* __restrict__ T, const double* __restrict__ g_sigma,
    double lam_scale, double* __restrict__ part, int nstrips)
{
    using R4 = typename vec4<R>::type;
    __shared__ AdjShared<R> sh;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int strip = blockIdx.x, nloc = blockIdx.y, kc = blockIdx.z;
    const int layer = layer0 + nloc;
    const int64_t j0 = (int64_t)strip * LS_STRIP;
    const int64_t jlast = min64(N - 1, j0 + LS_STRIP - 1);
    const double ref = nu[min64(jlast, j0 + LS_STRIP / 2)];
    const double Tn = T[layer];
    const R half_invT = (R)(0.5 / Tn);

    if (tid == 0) {
        int64_t b = lb_jhi(jrange, nl, (int)j0);
        int64_t e = lb_jlo(jrange, nl, (int)jlast);
        if (e < b) e = b;
        int64_t len = e - b;
        int64_t per = (len + ksplit - 1) / ksplit;
        per = (per + 31) & ~(int64_t)31;
        int64_t cb = min64(e, b + per * kc), ce = min64(e, cb + per);
        sh.win[0] = cb;
        sh.win[1] = ce;
    }
    R ohi[LS_G], lam[LS_G];
    int jg[LS_G];
#pragma unroll
    for (int g = 0; g < LS_G; ++g) {
        int64_t j = j0 + w * (32 * LS_G) + g * 32 + lane;
        int64_t jc = min64(j, jlast);
        jg[g] = (int)j;
        float lo;
        Off<R>::make(nu[jc], ref, &ohi[g], &lo);
        sh.olo[w][g * 32 + lane] = lo;
        lam[g] = (j <= jlast) ? (R)(g_sigma[(size_t)layer * N + j] * lam_scale) : R(0);
    }
    const int jw0 = (int)min64(jlast, j0 + w * (32 * LS_G));
    const int jw1 = (int)min64(jlast, j0 + w * (32 * LS_G) + 32 * LS_G - 1);
    R ow0 = __shfl_sync(0xffffffffu, ohi[0], 0);
    R ow1;
    {
        int jl = jw1 - (int)(j0 + w * (32 * LS_G));
        int gl = jl >> 5, ll = jl & 31;
        R v = ohi[0];
#pragma unroll
        for (int g = 0; g < LS_G; ++g)
            if (g == gl) v = ohi[g];
        ow1 = __shfl_sync(0xffffffffu, v, ll);
    }
    const float cmin = agg[2 * layer];
    const float amin = agg[2 * layer + 1];

    R accT = R(0), accB = R(0);
    double sT = 0.0, sB = 0.0;
    __syncthreads();
    const int64_t cb = sh.win[0], ce = sh.win[1];
    const size_t lay = (size_t)nloc * nl; // records hold the current layer chunk

    for (int64_t t0 = cb; t0 < ce; t0 += LS_TILE) {
        {
            int64_t l = t0 + tid;
            if (l < ce) {
                double v = nu_hat[l];
                R bh;
                float bl;
                Off<R>::make(v, ref, &bh, &bl);
                sh.bhi[tid] = bh;
                sh.blo[tid] = bl;
                R4 p1 = rec1[lay + l];
                R aS = rec3[2 * (lay + l)], nn = rec3[2 * (lay + l) + 1];
                sh.r2[tid] = rec2[lay + l];
                sh.clo[tid] = clo[lay + l];
                sh.jr[tid] = jrange[l];
                sh.G[tid] = p1.x;
                sh.aS[tid] = aS;
                sh.nn[tid] = nn;
                // fast-form coefficients from G, Al, F1 = 1.5 B Al, F2 = -2 G B Al
                R G = p1.x, Al = p1.y, F1 = p1.z, F2 = p1.w;
                R4 tc, uc;
                tc.x = Al * (aS + nn);
                tc.y = aS * F1 + half_invT * R(2) * F1 + nn * (F1 - R(2) * G * Al);
                tc.z = aS * F2 + half_invT * R(2) * F2 + nn * R(6) * F2;
                tc.w = nn * (R(-6) * G * F2);
                uc.x = Al;
                uc.y = F1 - R(2) * G * Al;
                uc.z = R(6) * F2;
                uc.w = R(-6) * G * F2;
                sh.t[tid] = tc;
                sh.u[tid] = uc;
            } else {
                double v = nu_hat[ce - 1];
                R bh;
                float bl;
                Off<R>::make(v, ref, &bh, &bl);
                sh.bhi[tid] = bh;
                sh.blo[tid] = bl;
                R4 z2;
                z2.x = R(1); z2.y = R(1); z2.z = R(0); z2.w = R(0);
                sh.r2[tid] = z2;
                R4 zz;
                zz.x = R(0); zz.y = R(0); zz.z = R(0); zz.w = R(0);
                sh.t[tid] = zz;
                sh.u[tid] = zz;
                sh.G[tid] = R(1);
                sh.clo[tid] = R(0);
                sh.aS[tid] = R(0);
                sh.nn[tid] = R(0);
                sh.jr[tid] = jrange[ce - 1];
            }
        }
        __syncthreads();
        const int nt = (int)min64(LS_TILE, ce - t0);
        for (int s0 = 0; s0 < nt; s0 += 32) {
            bool fast = false;
            if (FAST) {
                const int sl = s0 + 31;
                bool incut = (sh.jr[sl].x <= jw0) && (sh.jr[s0].y >= jw1);
                float bf = (float)sh.bhi[s0], bl = (float)sh.bhi[sl];
                float dist = fmaxf(fmaxf(bf - (float)ow1, (float)ow0 - bl), 0.0f);
                float xm = dist * cmin;
                fast = incut && (fmaf(xm, xm, amin * amin) >= (float)Tier<R>::z2_far);
            }
            if (fast) {
#pragma unroll 2
                for (int i = 0; i < 32; ++i) {
                    const R b = sh.bhi[s0 + i];
                    const R G = sh.G[s0 + i];
                    const R4 tc = sh.t[s0 + i];
                    const R4 uc = sh.u[s0 + i];
#pragma unroll
                    for (int g = 0; g < LS_G; ++g) {
                        R d = ohi[g] - b;
                        R rho = rcp_fast(fma(d, d, G));
                        R ft = rho * fma(rho, fma(rho, fma(rho, tc.w, tc.z), tc.y), tc.x);
                        R fb = rho * fma(rho, fma(rho, fma(rho, uc.w, uc.z), uc.y), uc.x);
                        accT = fma(lam[g], ft, accT);
                        accB = fma(lam[g], fb, accB);
                    }
                }
            } else {
                const int ns = min(32, nt - s0);
                for (int i = 0; i < ns; ++i) {
                    const int li = s0 + i;
                    const R bh = sh.bhi[li];
                    const float bl = sh.blo[li];
                    const R4 p2 = sh.r2[li];
                    const int2 jr = sh.jr[li];
                    const R aS = sh.aS[li], nn = sh.nn[li];
                    const R cl = sh.clo[li];
#pragma unroll
                    for (int g = 0; g < LS_G; ++g) {
                        if (jg[g] >= jr.x && jg[g] <= jr.y) {
                            R dh, dl, x, xl;
                            Off<R>::dnu2(ohi[g], sh.olo[w][g * 32 + lane], bh, bl, &dh, &dl);
                            scaled_pair(dh, dl, p2.x, cl, &x, &xl);
                            R a = p2.y;
                            R wr, wi, dr, di;
                            faddeeva_d<R>(x, xl, a, p2.w, &wr, &wi, &dr, &di);
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
            sT += (double)accT;
            sB += (double)accB;
            accT = R(0);
            accB = R(0);
        }
        __syncthreads();
    }
    // fixed-order block reduction
    for (int o = 16; o > 0; o >>= 1) {
        sT += __shfl_xor_sync(0xffffffffu, sT, o);
        sB += __shfl_xor_sync(0xffffffffu, sB, o);
    }
    if (lane == 0) {
        sh.red[0][w] = sT;
        sh.red[1][w] = sB;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < LS_WARPS; ++i) {
            a += sh.red[0][i];
            b += sh.red[1][i];
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
                  const double* g_sigma, double* g_T, double* g_b, cudaStream_t st)
{
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
    cut_range_kernel<<<(unsigned)((nl + 255) / 256), 256, 0, st>>>(ln->nu_hat, nl, nu, N, W, jr);
    layer_agg_init_kernel<<<(2 * L + 255) / 256, 256, 0, st>>>(agg, 2 * L);
    count_launch(2);
    for (int c = 0; c < p.nchunks; ++c) {
        int l0 = c * p.Lc;
        int lc = std::min(p.Lc, L - l0);
        dim3 pg((unsigned)((nl + 255) / 256), (unsigned)lc);
        line_params_kernel<R><<<pg, 256, 0, st>>>(ln->nu_hat, ln->ln_S0, ln->elower, ln->gamma_ref, ln->n_temp, nl,
                                                   ln->mass_amu, ln->q_exponent, T, P, l0, sb, scale, rec1, rec2, clo,
                                                   adjoint ? rec3 : nullptr, agg);
        count_launch();
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
           double* g_T, double* g_b, cudaStream_t st)
{
    XsPlan p;
    if (pick_plan(ln->n, N, L, prec, ws_bytes, &p) != XS_OK) return XS_EINVAL;
    if (prec == XS_PREC_FP64)
        return run_xs<double>(ln, nu, N, T, P, L, sb, W, sigma, (char*)ws, p, adjoint, g_sigma, g_T, g_b, st);
    return run_xs<float>(ln, nu, N, T, P, L, sb, W, sigma, (char*)ws, p, adjoint, g_sigma, g_T, g_b, st);
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
