// MODIT (Sec. 2.1.2, Eq. MODIT): the cross-section of many lines through a
// lineshape distribution on the log grid and FFT convolution.
//
// Grid: nu_i = nu_min exp(i/R0), i = 0..N-1, R0 = (N-1)/ln(nu_max/nu_min), so the
// variable q = R0 ln(nu/nu_min) steps by 1.  For each layer:
//   1. per layer the min and max of the normalised width gamma' = R0 gamma/nu_hat
//      (modit_range_kernel); per line, once, q_l = R0 ln(nu_hat/nu_min) and the
//      layer-independent parts of S(T) and ln gamma' (modit_prepass_kernel);
//   2. the lineshape distribution S[k][j]: each line adds S(T) (Eq. Slog) to the
//      two q nodes around q_l and the two ln gamma' nodes around its width, with
//      linear weights (modit_lsd_kernel).  One thread per q node takes the lines
//      with floor(q_l) = j (binary search) and hands the upper node's share to its
//      neighbour through shared memory, so the sum has a fixed order (no atomics);
//   3. batched real FFTs of the n_gamma rows (cuFFT);
//   4. Y[f] = sum_k FT(S_k)[f] K_k[f], K_k = exp(-2 pi^2 beta'^2 f^2)
//      (exp(-2 pi gamma'_k |f|) - gamma'_k DFT(A)[f]), beta' = R0 beta/nu_hat (common
//      to all lines of a species at one T), A the sum of a unit Lorentzian's periodic
//      images (its first-order aliasing, removed here);
//   5. inverse FFT per layer, then sigma(nu_i) = sigma(q_i) R0/nu_i.
// The q axis is periodic with the caller's length n_fft (a power of two); node j
// lives at slot j mod n_fft, nodes -(n_fft-N)/2 .. (n_fft+N)/2 - 1 are gathered.
#include <cufft.h>

#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "xs_device.cuh"
#include "xs_internal.h"

namespace xsd {

constexpr int MODIT_MAX_GAMMA = 32;
constexpr int MODIT_THREADS = 128;

template <class R> struct CplxOf;
template <> struct CplxOf<double> { using type = cufftDoubleComplex; };
template <> struct CplxOf<float> { using type = cufftComplex; };

__global__ void modit_range_init_kernel(unsigned long long* range, int L)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < L) {
        range[2 * i] = 0x7ff0000000000000ull; // +inf
        range[2 * i + 1] = 0ull;
    }
}

// per layer min and max of gamma' = R0 gamma/nu_hat (positive doubles order like
// their bit patterns)
__global__ void modit_range_kernel(const double* __restrict__ nu_hat, const double* __restrict__ gamma_ref,
                                   const double* __restrict__ n_temp, int64_t nl, const double* __restrict__ T,
                                   const double* __restrict__ P, double sb, double R0,
                                   unsigned long long* __restrict__ range)
{
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    double gmin = __longlong_as_double(0x7ff0000000000000ll), gmax = 0.0;
    if (l < nl) {
        const double lnTr = log(T[n] / Tref);
        const double g = R0 * sb * gamma_ref[l] * exp(-n_temp[l] * lnTr) * (P[n] / bar_per_atm) / nu_hat[l];
        gmin = g;
        gmax = g;
    }
    for (int o = 16; o > 0; o >>= 1) {
        gmin = fmin(gmin, __shfl_xor_sync(0xffffffffu, gmin, o));
        gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    }
    if ((threadIdx.x & 31) == 0 && gmax > 0.0) {
        atomicMin(&range[2 * n], (unsigned long long)__double_as_longlong(gmin));
        atomicMax(&range[2 * n + 1], (unsigned long long)__double_as_longlong(gmax));
    }
}

// Layer-independent per-line terms: q = R0 ln(nu_hat/nu_min), the stimulated-
// emission denominator expm1(-c2 nu_hat/296) and ln(R0 gamma_ref/nu_hat).
__global__ void modit_prepass_kernel(const double* __restrict__ nu_hat, const double* __restrict__ gamma_ref,
                                     int64_t nl, double nu_min, double R0, double* __restrict__ qv,
                                     double* __restrict__ sden, double* __restrict__ lgref)
{
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nl) return;
    const double nuh = nu_hat[l];
    qv[l] = R0 * log(nuh / nu_min);
    sden[l] = expm1(-c2 * nuh / Tref);
    lgref[l] = log(R0 * gamma_ref[l] / nuh);
}

__device__ __forceinline__ int64_t first_at_least(const double* v, int64_t n, double x) // first i with v[i] >= x
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t m = (lo + hi) >> 1;
        if (v[m] >= x) hi = m; else lo = m + 1;
    }
    return lo;
}

// One thread per (layer, slot); node j = slot, or slot - M for the left padding.
// Each thread takes the lines with floor(q_l) == j (found by binary search on
// the monotone q_l of the prepass), so every line is visited once: weight 1 - w
// goes to node j, w to node j + 1 through shared memory (the slot before the
// block's first comes from an extra halo thread).  Per line and layer: S(T)
// (Eq. Slog) from one exp and one expm1, ln gamma' from the prepass by FMAs.
// Blocks of MODIT_THREADS threads write MODIT_THREADS - 1 slots.
template <class R>
__global__ void __launch_bounds__(MODIT_THREADS) modit_lsd_kernel(
    const double* __restrict__ nu_hat, const double* __restrict__ ln_S0, const double* __restrict__ elower,
    const double* __restrict__ n_temp, const double* __restrict__ qv, const double* __restrict__ sden,
    const double* __restrict__ lgref, int64_t nl, double qexp, const double* __restrict__ T,
    const double* __restrict__ P, double sb, double scale, int64_t N, int64_t M, int ng,
    const unsigned long long* __restrict__ range, R* __restrict__ lsd)
{
    __shared__ double shR[MODIT_THREADS][MODIT_MAX_GAMMA];
    const int t = threadIdx.x;
    const int n = blockIdx.y;
    const int64_t s_raw = (int64_t)blockIdx.x * (MODIT_THREADS - 1) + t - 1;
    const bool valid = s_raw < M;
    const int64_t s = (s_raw + M) % M; // the halo of block 0 is slot M - 1
    const int64_t j = (s < (M + N) / 2) ? s : s - M;
    double accL[MODIT_MAX_GAMMA], accR[MODIT_MAX_GAMMA];
    for (int k = 0; k < ng; ++k) {
        accL[k] = 0.0;
        accR[k] = 0.0;
    }
    if (valid) {
        const double Tn = T[n];
        const double lnTr = log(Tn / Tref);
        const double bT = 1.0 / Tn - 1.0 / Tref;
        const double lgP = log(sb * P[n] / bar_per_atm);
        const double gmin = __longlong_as_double((long long)range[2 * n]);
        const double gmax = __longlong_as_double((long long)range[2 * n + 1]);
        const double lg0 = log(gmin);
        const double dlg = (ng >= 2 && gmax > gmin) ? (log(gmax) - lg0) / (double)(ng - 1) : 0.0;
        const double idlg = dlg > 0.0 ? 1.0 / dlg : 0.0;
        const int64_t b = first_at_least(qv, nl, (double)j);
        const int64_t e = first_at_least(qv, nl, (double)(j + 1));
        for (int64_t l = b; l < e; ++l) {
            const double wq = qv[l] - (double)j;
            const double S = exp(ln_S0[l] - c2 * elower[l] * bT - qexp * lnTr) *
                             (expm1(-c2 * nu_hat[l] / Tn) / sden[l]) * scale;
            int k0 = 0;
            double wk = 0.0;
            if (dlg > 0.0) {
                const double tt = (lgref[l] + lgP - n_temp[l] * lnTr - lg0) * idlg;
                k0 = min(max((int)floor(tt), 0), ng - 2);
                wk = tt - (double)k0;
            }
            const double vl = S * (1.0 - wq), vr = S * wq;
            accL[k0] += vl * (1.0 - wk);
            accR[k0] += vr * (1.0 - wk);
            if (dlg > 0.0) {
                accL[k0 + 1] += vl * wk;
                accR[k0 + 1] += vr * wk;
            }
        }
    }
    for (int k = 0; k < ng; ++k) shR[t][k] = accR[k];
    __syncthreads();
    if (t >= 1 && valid)
        for (int k = 0; k < ng; ++k) lsd[((size_t)n * ng + k) * M + s] = (R)(accL[k] + shR[t - 1][k]);
}

// A(d) = sum over p != 0 of 1/(pi (d + pM)^2) on one period (index d mod M):
// (pi/M)^2/sin^2(pi d/M) - 1/d^2 over pi, near d = 0 from the Laurent series of csc^2.
template <class R>
__global__ void modit_images_kernel(int64_t M, R* __restrict__ A)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const double d = (i < M / 2) ? (double)i : (double)(i - M);
    const double x = PI * d / (double)M;
    double v;
    if (fabs(x) < 0.3) {
        const double x2 = x * x;
        v = (PI / ((double)M * (double)M)) *
            (1.0 / 3 + x2 * (1.0 / 15 + x2 * (2.0 / 189 + x2 * (1.0 / 675 + x2 * (2.0 / 10395)))));
    } else {
        const double sx = sin(x);
        v = ((PI / M) * (PI / M) / (sx * sx) - 1.0 / (d * d)) / PI;
    }
    A[i] = (R)v;
}

// Y[n][m] = sum_k Z[n][k][m] K_k(m) for m = 0..M/2
template <class R>
__global__ void modit_multiply_kernel(const typename CplxOf<R>::type* __restrict__ Z,
                                      const typename CplxOf<R>::type* __restrict__ Ahat, int64_t M, int ng,
                                      const double* __restrict__ T, double mass, double R0,
                                      const unsigned long long* __restrict__ range,
                                      typename CplxOf<R>::type* __restrict__ Y)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    const int64_t H = M / 2 + 1;
    if (m >= H) return;
    const double gmin = __longlong_as_double((long long)range[2 * n]);
    const double gmax = __longlong_as_double((long long)range[2 * n + 1]);
    const double lg0 = log(gmin);
    const double dlg = (ng >= 2 && gmax > gmin) ? (log(gmax) - lg0) / (double)(ng - 1) : 0.0;
    const double bq = sqrt(kB * T[n] / (mass * amu)) * R0 / cL; // beta' (q units)
    const double f = (double)m / (double)M;
    const double gauss = exp(-2.0 * PI * PI * bq * bq * f * f);
    const double ah = (double)Ahat[m].x;
    double yr = 0.0, yi = 0.0;
    for (int k = 0; k < ng; ++k) {
        const double g = exp(lg0 + dlg * (double)k);
        const double K = gauss * (exp(-2.0 * PI * g * f) - g * ah);
        const typename CplxOf<R>::type z = Z[((size_t)n * ng + k) * H + m];
        yr += (double)z.x * K;
        yi += (double)z.y * K;
    }
    Y[(size_t)n * H + m].x = (R)yr;
    Y[(size_t)n * H + m].y = (R)yi;
}

template <class R>
__global__ void modit_finish_kernel(const R* __restrict__ y, int64_t M, int64_t N, int L, double R0, double nu_min,
                                    double unscale, void* __restrict__ sigma)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (i >= N) return;
    const double nu = nu_min * exp((double)i / R0);
    const double v = (double)y[(size_t)n * M + i] / (double)M * R0 / nu * unscale;
    if (std::is_same<R, float>::value) ((float*)sigma)[(size_t)n * N + i] = (float)v;
    else ((double*)sigma)[(size_t)n * N + i] = v;
}


// ------------------------------------------------------------------ adjoint
//
// With lambda = dF/dsigma [L][N] and mu_i = lambda_i R0 unscale/(M nu_i) (so that
// F = sum_i mu_i y_i, y the unnormalised inverse transform), per layer:
//   M^ = FFT(mu); the kernel term sum_m c_m Re(Z_k[m] conj(M^[m])) dK_k[m]/dtheta
//   (c_m = 1 at m = 0 and M/2, else 2); the correlations corr_k = IFFT(K_k M^),
//   so that dF/dLSD_k[j] = corr_k[j]; and per line the distribution term
//   S (dlnS/dT A + B dt/dT), A and B the weight-averaged correlations and their
//   difference across the two gamma' nodes, t the line's fractional gamma' node.
// s_b moves every ln gamma' and both grid ends alike, so it enters through the
// kernels only.

__device__ __forceinline__ double block_sum(double v, double* red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// index of the line attaining the layer's smallest (ext[2n]) and largest
// (ext[2n+1]) gamma' (the same arithmetic as modit_range_kernel)
__global__ void modit_extreme_kernel(const double* __restrict__ nu_hat, const double* __restrict__ gamma_ref,
                                     const double* __restrict__ n_temp, int64_t nl, const double* __restrict__ T,
                                     const double* __restrict__ P, double sb, double R0,
                                     const unsigned long long* __restrict__ range, unsigned long long* __restrict__ ext)
{
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (l >= nl) return;
    const double lnTr = log(T[n] / Tref);
    const double g = R0 * sb * gamma_ref[l] * exp(-n_temp[l] * lnTr) * (P[n] / bar_per_atm) / nu_hat[l];
    const unsigned long long gb = (unsigned long long)__double_as_longlong(g);
    if (gb == range[2 * n]) atomicMin(&ext[2 * n], (unsigned long long)l);
    if (gb == range[2 * n + 1]) atomicMin(&ext[2 * n + 1], (unsigned long long)l);
}

__global__ void modit_ext_init_kernel(unsigned long long* ext, int L)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 2 * L) ext[i] = ~0ull;
}

template <class R>
__global__ void modit_mu_kernel(const double* __restrict__ g_sigma, int64_t N, int64_t M, double R0, double nu_min,
                                double fac, R* __restrict__ mu)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (s >= M) return;
    double v = 0.0;
    if (s < N) v = g_sigma[(size_t)n * N + s] * R0 / (nu_min * exp((double)s / R0)) * fac;
    mu[(size_t)n * M + s] = (R)v;
}

// d ln gamma'_k / dT for node k from the extreme lines' temperature exponents
__device__ __forceinline__ double node_dlng_dT(int k, int ng, double n_lo, double n_hi, double Tn)
{
    const double w = (ng >= 2) ? (double)k / (double)(ng - 1) : 0.0;
    return -((1.0 - w) * n_lo + w * n_hi) / Tn;
}

// kernel term (per layer, block partials) and, in place, X_k = K_k M^ for the
// correlations (overwrites Z after using it)
template <class R>
__global__ void modit_adj_kernel_term(typename CplxOf<R>::type* __restrict__ Z,
                                      const typename CplxOf<R>::type* __restrict__ Mh,
                                      const typename CplxOf<R>::type* __restrict__ Ahat, int64_t M, int ng,
                                      const double* __restrict__ T, double mass, double R0, double sb,
                                      const unsigned long long* __restrict__ range,
                                      const unsigned long long* __restrict__ ext, const double* __restrict__ n_temp,
                                      double* __restrict__ partT, double* __restrict__ partB)
{
    __shared__ double red[256];
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    const int64_t H = M / 2 + 1;
    double gT = 0.0, gB = 0.0;
    if (m < H) {
        const double Tn = T[n];
        const double gmin = __longlong_as_double((long long)range[2 * n]);
        const double gmax = __longlong_as_double((long long)range[2 * n + 1]);
        const double lg0 = log(gmin);
        const double dlg = (ng >= 2 && gmax > gmin) ? (log(gmax) - lg0) / (double)(ng - 1) : 0.0;
        const double n_lo = n_temp[ext[2 * n]], n_hi = n_temp[ext[2 * n + 1]];
        const double bq = sqrt(kB * Tn / (mass * amu)) * R0 / cL;
        const double f = (double)m / (double)M;
        const double G = exp(-2.0 * PI * PI * bq * bq * f * f);
        const double dG_dT = G * (-2.0 * PI * PI * bq * bq * f * f) / Tn;
        const double ah = (double)Ahat[m].x;
        const double cm = (m == 0 || 2 * m == M) ? 1.0 : 2.0;
        const double mr = (double)Mh[(size_t)n * H + m].x, mi = (double)Mh[(size_t)n * H + m].y;
        for (int k = 0; k < ng; ++k) {
            const double g = exp(lg0 + dlg * (double)k);
            const double E = exp(-2.0 * PI * g * f);
            const double K = G * (E - g * ah);
            const double dK_dlng = G * (-2.0 * PI * f * E - ah) * g;
            const size_t zi = ((size_t)n * ng + k) * H + m;
            const typename CplxOf<R>::type z = Z[zi];
            const double Pk = cm * ((double)z.x * mr + (double)z.y * mi); // Re(Z conj(M^))
            gT += Pk * (dG_dT * (E - g * ah) + dK_dlng * node_dlng_dT(k, ng, n_lo, n_hi, Tn));
            gB += Pk * dK_dlng / sb;
            Z[zi].x = (R)(K * mr);
            Z[zi].y = (R)(K * mi);
        }
    }
    gT = block_sum(gT, red);
    gB = block_sum(gB, red);
    if (threadIdx.x == 0) {
        partT[(size_t)n * gridDim.x + blockIdx.x] = gT;
        partB[(size_t)n * gridDim.x + blockIdx.x] = gB;
    }
}

// distribution term per (line, layer), block partials
template <class R>
__global__ void modit_adj_line_term(const double* __restrict__ nu_hat, const double* __restrict__ ln_S0,
                                    const double* __restrict__ elower, const double* __restrict__ n_temp,
                                    const double* __restrict__ qv, const double* __restrict__ sden,
                                    const double* __restrict__ lgref, int64_t nl, double qexp,
                                    const double* __restrict__ T, const double* __restrict__ P, double sb,
                                    double scale, int64_t N, int64_t M, int ng,
                                    const unsigned long long* __restrict__ range,
                                    const unsigned long long* __restrict__ ext, const R* __restrict__ corr,
                                    double* __restrict__ part)
{
    __shared__ double red[256];
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    double gl = 0.0;
    if (l < nl) {
        const double Tn = T[n];
        const double lnTr = log(Tn / Tref);
        const double bT = 1.0 / Tn - 1.0 / Tref;
        const double lgP = log(sb * P[n] / bar_per_atm);
        const double gmin = __longlong_as_double((long long)range[2 * n]);
        const double gmax = __longlong_as_double((long long)range[2 * n + 1]);
        const double lg0 = log(gmin);
        const double dlg = (ng >= 2 && gmax > gmin) ? (log(gmax) - lg0) / (double)(ng - 1) : 0.0;
        const double q = qv[l];
        const double fq = floor(q);
        const int64_t j0 = (int64_t)fq;
        const double wq = q - fq;
        const double u = c2 * nu_hat[l] / Tn;
        const double S = exp(ln_S0[l] - c2 * elower[l] * bT - qexp * lnTr) * (expm1(-u) / sden[l]) * scale;
        const double dlnS = c2 * elower[l] / (Tn * Tn) - qexp / Tn - (u / Tn) / expm1(u);
        int k0 = 0;
        double wk = 0.0, dt = 0.0;
        if (dlg > 0.0) {
            const double t = (lgref[l] + lgP - n_temp[l] * lnTr - lg0) / dlg;
            k0 = min(max((int)floor(t), 0), ng - 2);
            wk = t - (double)k0;
            const double n_lo = n_temp[ext[2 * n]], n_hi = n_temp[ext[2 * n + 1]];
            const double dlg0 = -n_lo / Tn, ddlg = (-n_hi + n_lo) / (Tn * (double)(ng - 1));
            dt = (-n_temp[l] / Tn - dlg0 - t * ddlg) / dlg;
        }
        const int k1 = (dlg > 0.0) ? k0 + 1 : 0;
        // the forward gathers lines whose lower node j0 lies in the window
        // -(M-N)/2 .. (M+N)/2 - 1 and adds to the slots of j0 and j0 + 1 (mod M)
        const int64_t jlo = -(M - N) / 2, jhi = (M + N) / 2;
        double A = 0.0, B = 0.0;
        for (int d = 0; d < 2; ++d) {
            if (j0 < jlo || j0 >= jhi) break;
            const int64_t sl = (((j0 + d) % M) + M) % M;
            const double w = d ? wq : 1.0 - wq;
            const double c0 = (double)corr[((size_t)n * ng + k0) * M + sl];
            const double c1 = (double)corr[((size_t)n * ng + k1) * M + sl];
            A += w * ((1.0 - wk) * c0 + wk * c1);
            B += w * (c1 - c0);
        }
        gl = S * (dlnS * A + B * dt);
    }
    gl = block_sum(gl, red);
    if (threadIdx.x == 0) part[(size_t)n * gridDim.x + blockIdx.x] = gl;
}

// g_T[n] = sum of the line partials + kernel partials; g_b = sum over layers of
// the s_b kernel partials (fixed order)
__global__ void modit_adj_reduce(const double* __restrict__ partL, int nbl, const double* __restrict__ partT,
                                 const double* __restrict__ partB, int nbk, int L, double* __restrict__ g_T,
                                 double* __restrict__ g_b)
{
    __shared__ double red[256];
    double gb = 0.0;
    for (int n = 0; n < L; ++n) {
        double a = 0.0, b = 0.0;
        for (int i = threadIdx.x; i < nbl; i += blockDim.x) a += partL[(size_t)n * nbl + i];
        for (int i = threadIdx.x; i < nbk; i += blockDim.x) {
            a += partT[(size_t)n * nbk + i];
            b += partB[(size_t)n * nbk + i];
        }
        a = block_sum(a, red);
        b = block_sum(b, red);
        if (threadIdx.x == 0) g_T[n] = a;
        gb += b;
    }
    if (threadIdx.x == 0) g_b[0] = gb;
}

} // namespace xsd

namespace {

using namespace xsd;

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

struct ModitPlan {
    size_t range, lines, lsd, Z, A, Ahat, Y, work, total, work_bytes;
    size_t mu, ext, partL, partT, partB; // adjoint only
    int nbl, nbk;
};

ModitPlan modit_plan(int64_t nl, int32_t L, int32_t ng, int64_t M, int prec, bool adjoint = false)
{
    const size_t rs = (prec == XS_PREC_MIXED) ? sizeof(float) : sizeof(double);
    const size_t H = (size_t)M / 2 + 1;
    ModitPlan p{};
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off += al256(b);
        return o;
    };
    p.range = take(2 * sizeof(unsigned long long) * (size_t)L);
    p.lines = take(3 * sizeof(double) * (size_t)std::max<int64_t>(nl, 1)); // q, stim denominator, ln gamma'_ref
    p.lsd = take(rs * (size_t)L * ng * M); // reused for the inverse transforms' output
    p.Z = take(2 * rs * (size_t)L * ng * H);
    p.A = take(rs * (size_t)M);
    p.Ahat = take(2 * rs * H);
    p.Y = take(2 * rs * (size_t)L * H);
    // cuFFT work area: reserved at the size of the largest complex array
    p.work_bytes = std::max<size_t>((size_t)16 << 20, 2 * rs * (size_t)L * ng * H);
    p.work = take(p.work_bytes);
    if (adjoint) {
        p.nbl = (int)((std::max<int64_t>(nl, 1) + 255) / 256);
        p.nbk = (int)((H + 255) / 256);
        p.mu = take(rs * (size_t)L * M);
        p.ext = take(2 * sizeof(unsigned long long) * (size_t)L);
        p.partL = take(sizeof(double) * (size_t)L * p.nbl);
        p.partT = take(sizeof(double) * (size_t)L * p.nbk);
        p.partB = take(sizeof(double) * (size_t)L * p.nbk);
    }
    p.total = off;
    return p;
}

// cuFFT plans, created once per (device, length, batch, type) without their own
// work area (the caller's workspace provides it).
std::mutex g_fft_mu;
std::map<std::tuple<int, int64_t, int64_t, int>, std::pair<cufftHandle, size_t>> g_fft_plans;

int fft_plan(int64_t M, int64_t batch, cufftType type, cufftHandle* out, size_t* work)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return XS_ECUDA;
    auto key = std::make_tuple(dev, M, batch, (int)type);
    auto it = g_fft_plans.find(key);
    if (it != g_fft_plans.end()) {
        *out = it->second.first;
        *work = it->second.second;
        return XS_OK;
    }
    cufftHandle h;
    if (cufftCreate(&h) != CUFFT_SUCCESS) return XS_ECUDA;
    if (cufftSetAutoAllocation(h, 0) != CUFFT_SUCCESS) return XS_ECUDA;
    long long n = M;
    size_t ws = 0;
    const bool fwd = (type == CUFFT_D2Z || type == CUFFT_R2C);
    long long idist = fwd ? M : M / 2 + 1, odist = fwd ? M / 2 + 1 : M;
    if (cufftMakePlanMany64(h, 1, &n, nullptr, 1, idist, nullptr, 1, odist, type, batch, &ws) != CUFFT_SUCCESS) {
        cufftDestroy(h);
        return XS_ECUDA;
    }
    g_fft_plans[key] = {h, ws};
    *out = h;
    *work = ws;
    return XS_OK;
}

template <class R>
int fft_exec(int64_t M, int64_t batch, bool forward, void* in, void* out, void* work, size_t work_bytes,
             cudaStream_t st)
{
    constexpr bool D = std::is_same<R, double>::value;
    const cufftType type = forward ? (D ? CUFFT_D2Z : CUFFT_R2C) : (D ? CUFFT_Z2D : CUFFT_C2R);
    std::lock_guard<std::mutex> lk(g_fft_mu);
    cufftHandle h;
    size_t ws = 0;
    int r = fft_plan(M, batch, type, &h, &ws);
    if (r != XS_OK) return r;
    if (ws > work_bytes) return XS_ETOOBIG;
    if (cufftSetStream(h, st) != CUFFT_SUCCESS || cufftSetWorkArea(h, work) != CUFFT_SUCCESS) return XS_ECUDA;
    cufftResult e;
    if (D) {
        e = forward ? cufftExecD2Z(h, (cufftDoubleReal*)in, (cufftDoubleComplex*)out)
                    : cufftExecZ2D(h, (cufftDoubleComplex*)in, (cufftDoubleReal*)out);
    } else {
        e = forward ? cufftExecR2C(h, (cufftReal*)in, (cufftComplex*)out)
                    : cufftExecC2R(h, (cufftComplex*)in, (cufftReal*)out);
    }
    xsi::count_launch();
    return e == CUFFT_SUCCESS ? XS_OK : XS_ECUDA;
}

template <class R>
int run_modit(const xs_lines* ln, double nu_min, double nu_max, int64_t N, const double* T, const double* P,
              int32_t L, double sb, int32_t ng, int64_t M, void* sigma, char* ws, const ModitPlan& p,
              cudaStream_t st)
{
    using C = typename CplxOf<R>::type;
    constexpr bool FAST = std::is_same<R, float>::value;
    const double R0 = (double)(N - 1) / log(nu_max / nu_min);
    const double scale = FAST ? MIXED_SCALE : 1.0, unscale = FAST ? MIXED_UNSCALE : 1.0;
    const int64_t nl = ln->n;
    const int64_t H = M / 2 + 1;
    auto* range = (unsigned long long*)(ws + p.range);
    R* lsd = (R*)(ws + p.lsd);
    C* Z = (C*)(ws + p.Z);
    R* A = (R*)(ws + p.A);
    C* Ahat = (C*)(ws + p.Ahat);
    C* Y = (C*)(ws + p.Y);
    void* work = ws + p.work;
    if (nl == 0) {
        const size_t es = FAST ? sizeof(float) : sizeof(double);
        return cudaMemsetAsync(sigma, 0, es * (size_t)L * N, st) == cudaSuccess ? XS_OK : XS_ECUDA;
    }
    modit_range_init_kernel<<<(L + 255) / 256, 256, 0, st>>>(range, L);
    modit_range_kernel<<<dim3((unsigned)((nl + 255) / 256), (unsigned)L), 256, 0, st>>>(
        ln->nu_hat, ln->gamma_ref, ln->n_temp, nl, T, P, sb, R0, range);
    double* qv = (double*)(ws + p.lines);
    double* sden = qv + nl;
    double* lgref = sden + nl;
    modit_prepass_kernel<<<(unsigned)((nl + 255) / 256), 256, 0, st>>>(ln->nu_hat, ln->gamma_ref, nl, nu_min, R0, qv,
                                                                        sden, lgref);
    modit_lsd_kernel<R><<<dim3((unsigned)((M + MODIT_THREADS - 2) / (MODIT_THREADS - 1)), (unsigned)L), MODIT_THREADS, 0,
                          st>>>(ln->nu_hat, ln->ln_S0, ln->elower, ln->n_temp, qv, sden, lgref, nl, ln->q_exponent,
                                T, P, sb, scale, N, M, ng, range, lsd);
    modit_images_kernel<R><<<(unsigned)((M + 255) / 256), 256, 0, st>>>(M, A);
    xsi::count_launch(5);
    if (cudaGetLastError() != cudaSuccess) return XS_ECUDA;
    int r = fft_exec<R>(M, (int64_t)L * ng, true, lsd, Z, work, p.work_bytes, st);
    if (r != XS_OK) return r;
    r = fft_exec<R>(M, 1, true, A, Ahat, work, p.work_bytes, st);
    if (r != XS_OK) return r;
    modit_multiply_kernel<R><<<dim3((unsigned)((H + 255) / 256), (unsigned)L), 256, 0, st>>>(
        Z, Ahat, M, ng, T, ln->mass_amu, R0, range, Y);
    xsi::count_launch();
    r = fft_exec<R>(M, L, false, Y, lsd, work, p.work_bytes, st); // y reuses the distribution's memory
    if (r != XS_OK) return r;
    modit_finish_kernel<R><<<dim3((unsigned)((N + 255) / 256), (unsigned)L), 256, 0, st>>>(lsd, M, N, L, R0,
                                                                                         nu_min, unscale, sigma);
    xsi::count_launch();
    return cudaGetLastError() == cudaSuccess ? XS_OK : XS_ECUDA;
}

template <class R>
int run_modit_adjoint(const xs_lines* ln, double nu_min, double nu_max, int64_t N, const double* T, const double* P,
                      int32_t L, double sb, int32_t ng, int64_t M, const double* g_sigma, double* g_T, double* g_b,
                      char* ws, const ModitPlan& p, cudaStream_t st)
{
    using C = typename CplxOf<R>::type;
    constexpr bool FAST = std::is_same<R, float>::value;
    const double R0 = (double)(N - 1) / log(nu_max / nu_min);
    const double scale = FAST ? MIXED_SCALE : 1.0, unscale = FAST ? MIXED_UNSCALE : 1.0;
    const int64_t nl = ln->n;
    const int64_t H = M / 2 + 1;
    auto* range = (unsigned long long*)(ws + p.range);
    auto* ext = (unsigned long long*)(ws + p.ext);
    R* lsd = (R*)(ws + p.lsd);
    C* Z = (C*)(ws + p.Z);
    R* A = (R*)(ws + p.A);
    C* Ahat = (C*)(ws + p.Ahat);
    C* Mh = (C*)(ws + p.Y);
    R* mu = (R*)(ws + p.mu);
    double* partL = (double*)(ws + p.partL);
    double* partT = (double*)(ws + p.partT);
    double* partB = (double*)(ws + p.partB);
    void* work = ws + p.work;
    if (nl == 0) {
        if (cudaMemsetAsync(g_T, 0, sizeof(double) * L, st) != cudaSuccess) return XS_ECUDA;
        return cudaMemsetAsync(g_b, 0, sizeof(double), st) == cudaSuccess ? XS_OK : XS_ECUDA;
    }
    // the forward's distribution and its transform
    modit_range_init_kernel<<<(L + 255) / 256, 256, 0, st>>>(range, L);
    modit_range_kernel<<<dim3((unsigned)((nl + 255) / 256), (unsigned)L), 256, 0, st>>>(
        ln->nu_hat, ln->gamma_ref, ln->n_temp, nl, T, P, sb, R0, range);
    modit_ext_init_kernel<<<(2 * L + 255) / 256, 256, 0, st>>>(ext, L);
    modit_extreme_kernel<<<dim3((unsigned)((nl + 255) / 256), (unsigned)L), 256, 0, st>>>(
        ln->nu_hat, ln->gamma_ref, ln->n_temp, nl, T, P, sb, R0, range, ext);
    double* qv = (double*)(ws + p.lines);
    double* sden = qv + nl;
    double* lgref = sden + nl;
    modit_prepass_kernel<<<(unsigned)((nl + 255) / 256), 256, 0, st>>>(ln->nu_hat, ln->gamma_ref, nl, nu_min, R0, qv,
                                                                        sden, lgref);
    modit_lsd_kernel<R><<<dim3((unsigned)((M + MODIT_THREADS - 2) / (MODIT_THREADS - 1)), (unsigned)L), MODIT_THREADS, 0,
                          st>>>(ln->nu_hat, ln->ln_S0, ln->elower, ln->n_temp, qv, sden, lgref, nl, ln->q_exponent,
                                T, P, sb, scale, N, M, ng, range, lsd);
    modit_images_kernel<R><<<(unsigned)((M + 255) / 256), 256, 0, st>>>(M, A);
    modit_mu_kernel<R><<<dim3((unsigned)((M + 255) / 256), (unsigned)L), 256, 0, st>>>(
        g_sigma, N, M, R0, nu_min, unscale / (double)M, mu);
    xsi::count_launch(8);
    if (cudaGetLastError() != cudaSuccess) return XS_ECUDA;
    int r = fft_exec<R>(M, (int64_t)L * ng, true, lsd, Z, work, p.work_bytes, st);
    if (r != XS_OK) return r;
    r = fft_exec<R>(M, 1, true, A, Ahat, work, p.work_bytes, st);
    if (r != XS_OK) return r;
    r = fft_exec<R>(M, L, true, mu, Mh, work, p.work_bytes, st);
    if (r != XS_OK) return r;
    modit_adj_kernel_term<R><<<dim3((unsigned)p.nbk, (unsigned)L), 256, 0, st>>>(
        Z, Mh, Ahat, M, ng, T, ln->mass_amu, R0, sb, range, ext, ln->n_temp, partT, partB);
    xsi::count_launch();
    r = fft_exec<R>(M, (int64_t)L * ng, false, Z, lsd, work, p.work_bytes, st); // correlations into lsd
    if (r != XS_OK) return r;
    modit_adj_line_term<R><<<dim3((unsigned)p.nbl, (unsigned)L), 256, 0, st>>>(
        ln->nu_hat, ln->ln_S0, ln->elower, ln->n_temp, qv, sden, lgref, nl, ln->q_exponent, T, P, sb, scale, N, M, ng,
        range, ext, lsd, partL);
    modit_adj_reduce<<<1, 256, 0, st>>>(partL, p.nbl, partT, partB, p.nbk, L, g_T, g_b);
    xsi::count_launch(2);
    return cudaGetLastError() == cudaSuccess ? XS_OK : XS_ECUDA;
}

bool pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

} // namespace

extern "C" {

size_t modit_adjoint_workspace_bytes(int64_t n_lines, int32_t L, int32_t n_gamma, int64_t n_fft, int prec)
{
    if (n_lines < 0 || L <= 0 || n_gamma < 1 || n_gamma > MODIT_MAX_GAMMA || !pow2(n_fft)) return 0;
    if (prec != XS_PREC_FP64 && prec != XS_PREC_MIXED) return 0;
    return modit_plan(n_lines, L, n_gamma, n_fft, prec, true).total;
}

int modit_compute_adjoint(const xs_lines* lines, double nu_min, double nu_max, int64_t N, const double* T,
                          const double* P_bar, int32_t L, double broad_scale, int32_t n_gamma, int64_t n_fft,
                          int prec, const double* g_sigma, double* g_T, double* g_broad, void* workspace,
                          size_t workspace_bytes, xs_stream stream)
{
    XS_NVTX("modit_compute_adjoint");
    if (!lines || lines->n < 0 || !T || !P_bar || !g_sigma || !g_T || !g_broad || !workspace || L <= 0 || N < 2)
        return XS_EINVAL;
    if (lines->n > 0 && (!lines->nu_hat || !lines->ln_S0 || !lines->elower || !lines->gamma_ref || !lines->n_temp))
        return XS_EINVAL;
    if (!(nu_min > 0.0) || !(nu_max > nu_min) || !(broad_scale > 0.0) || !(lines->mass_amu > 0.0)) return XS_EINVAL;
    if (n_gamma < 1 || n_gamma > MODIT_MAX_GAMMA || !pow2(n_fft) || n_fft < N + 2) return XS_EINVAL;
    if (prec != XS_PREC_FP64 && prec != XS_PREC_MIXED) return XS_EINVAL;
    const ModitPlan p = modit_plan(lines->n, L, n_gamma, n_fft, prec, true);
    if (workspace_bytes < p.total) return XS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == XS_PREC_FP64)
        return run_modit_adjoint<double>(lines, nu_min, nu_max, N, T, P_bar, L, broad_scale, n_gamma, n_fft, g_sigma,
                                         g_T, g_broad, (char*)workspace, p, st);
    return run_modit_adjoint<float>(lines, nu_min, nu_max, N, T, P_bar, L, broad_scale, n_gamma, n_fft, g_sigma, g_T,
                                    g_broad, (char*)workspace, p, st);
}

size_t modit_workspace_bytes(int64_t n_lines, int32_t L, int32_t n_gamma, int64_t n_fft, int prec)
{
    if (n_lines < 0 || L <= 0 || n_gamma < 1 || n_gamma > MODIT_MAX_GAMMA || !pow2(n_fft)) return 0;
    if (prec != XS_PREC_FP64 && prec != XS_PREC_MIXED) return 0;
    return modit_plan(n_lines, L, n_gamma, n_fft, prec).total;
}

int modit_compute(const xs_lines* lines, double nu_min, double nu_max, int64_t N, const double* T,
                  const double* P_bar, int32_t L, double broad_scale, int32_t n_gamma, int64_t n_fft, int prec,
                  void* sigma, void* workspace, size_t workspace_bytes, xs_stream stream)
{
    XS_NVTX("modit_compute");
    if (!lines || lines->n < 0 || !T || !P_bar || !sigma || !workspace || L <= 0 || N < 2) return XS_EINVAL;
    if (lines->n > 0 && (!lines->nu_hat || !lines->ln_S0 || !lines->elower || !lines->gamma_ref || !lines->n_temp))
        return XS_EINVAL;
    if (!(nu_min > 0.0) || !(nu_max > nu_min) || !(broad_scale > 0.0) || !(lines->mass_amu > 0.0)) return XS_EINVAL;
    if (n_gamma < 1 || n_gamma > MODIT_MAX_GAMMA || !pow2(n_fft) || n_fft < N + 2) return XS_EINVAL;
    if (prec != XS_PREC_FP64 && prec != XS_PREC_MIXED) return XS_EINVAL;
    const ModitPlan p = modit_plan(lines->n, L, n_gamma, n_fft, prec);
    if (workspace_bytes < p.total) return XS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == XS_PREC_FP64)
        return run_modit<double>(lines, nu_min, nu_max, N, T, P_bar, L, broad_scale, n_gamma, n_fft, sigma,
                                 (char*)workspace, p, st);
    return run_modit<float>(lines, nu_min, nu_max, N, T, P_bar, L, broad_scale, n_gamma, n_fft, sigma,
                            (char*)workspace, p, st);
}

} // extern "C"

XS_CHECK_ACCESSOR(modit)
