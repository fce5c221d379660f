// Gaussian-process prior on the layer temperatures (the layer-by-layer retrieval
// of Sec. 6.1): T ~ N(T0 u, K) with
//   K_ij = a_T k_GP(log10 P_i - log10 P_j; tau_P) + eps a_T delta_ij,
// k_GP the RBF kernel k(x; tau) = exp(-x^2 / (2 tau^2)) of Sec. 5.2.3.  One CTA
// builds K in the workspace, factors it K = C C^T (Cholesky, in place, lower
// triangle), solves C y = r and C^T x = y for r = T - T0 u, and writes
//   log p       = -y.y/2 - sum_i log C_ii - (L/2) log(2 pi),
//   dlogp/dT_i  = -x_i,
//   dlogp/dT0   = sum_i x_i.
// FP64 throughout.  L is small (the paper uses 100 layers), so a single block
// does the O(L^3/6) factorisation; every row and column step is a block-wide
// parallel loop with a barrier after it.
#include <cmath>

#include "xs_device.cuh"
#include "xs_internal.h"

namespace xsd {

constexpr int PRIOR_THREADS = 256;

__device__ double block_sum(double v, double* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < PRIOR_THREADS / 32; ++i) s += red[i];  // fixed order
        red[PRIOR_THREADS / 32] = s;
    }
    __syncthreads();
    return red[PRIOR_THREADS / 32];
}

__global__ void __launch_bounds__(PRIOR_THREADS) gp_prior_kernel(const double* __restrict__ T,
                                                                 const double* __restrict__ P, int L, double T0,
                                                                 double aT, double tauP, double eps,
                                                                 double* __restrict__ C, double* __restrict__ y,
                                                                 double* __restrict__ out)
{
    __shared__ double red[PRIOR_THREADS / 32 + 1];
    const int t = threadIdx.x;
    const double inv2t2 = 0.5 / (tauP * tauP);
    // K, lower triangle (row-major L x L)
    for (int k = t; k < L * L; k += PRIOR_THREADS) {
        const int i = k / L, j = k - i * L;
        if (j <= i) {
            const double d = log10(P[i]) - log10(P[j]);
            C[k] = aT * exp(-d * d * inv2t2) + (i == j ? eps * aT : 0.0);
        }
    }
    __syncthreads();
    // right-looking Cholesky: column k scaled by its pivot, then the trailing
    // lower triangle updated by the outer product of column k
    bool ok = true;
    for (int k = 0; k < L; ++k) {
        const double piv = C[(size_t)k * L + k];
        if (!(piv > 0.0)) ok = false;
        const double dk = sqrt(piv);
        __syncthreads();
        if (t == 0) C[(size_t)k * L + k] = dk;
        for (int i = k + 1 + t; i < L; i += PRIOR_THREADS) C[(size_t)i * L + k] /= dk;
        __syncthreads();
        const int m = L - k - 1;  // trailing size
        for (int q = t; q < m * m; q += PRIOR_THREADS) {
            const int i = k + 1 + q / m, j = k + 1 + q % m;
            if (j <= i) C[(size_t)i * L + j] -= C[(size_t)i * L + k] * C[(size_t)j * L + k];
        }
        __syncthreads();
    }
    // forward solve C y = r
    for (int i = 0; i < L; ++i) {
        double s = 0.0;
        for (int j = t; j < i; j += PRIOR_THREADS) s += C[(size_t)i * L + j] * y[j];
        s = block_sum(s, red);
        if (t == 0) y[i] = (T[i] - T0 - s) / C[(size_t)i * L + i];
        __syncthreads();
    }
    // y.y and sum log C_ii
    double q = 0.0, ld = 0.0;
    for (int i = t; i < L; i += PRIOR_THREADS) {
        q += y[i] * y[i];
        ld += log(C[(size_t)i * L + i]);
    }
    q = block_sum(q, red);
    ld = block_sum(ld, red);
    // back solve C^T x = y (x overwrites y from the end)
    for (int i = L - 1; i >= 0; --i) {
        double s = 0.0;
        for (int j = i + 1 + t; j < L; j += PRIOR_THREADS) s += C[(size_t)j * L + i] * y[j];
        s = block_sum(s, red);
        if (t == 0) y[i] = (y[i] - s) / C[(size_t)i * L + i];
        __syncthreads();
    }
    double sx = 0.0;
    for (int i = t; i < L; i += PRIOR_THREADS) {
        out[1 + i] = -y[i];
        sx += y[i];
    }
    sx = block_sum(sx, red);
    if (t == 0) {
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        out[0] = ok ? -0.5 * q - ld - 0.5 * L * log(2.0 * PI) : nan;
        out[1 + L] = ok ? sx : nan;
    }
}

} // namespace xsd

extern "C" {

size_t gp_prior_workspace_bytes(int32_t L)
{
    if (L <= 0 || L > XS_GP_MAX_LAYERS) return 0;
    return sizeof(double) * ((size_t)L * L + (size_t)L);
}

int gp_prior_layers(const double* T, const double* P_bar, int32_t L, double T0, double a_T, double tau_P, double eps,
                    double* out, void* workspace, size_t workspace_bytes, xs_stream stream)
{
    XS_NVTX("gp_prior_layers");
    using namespace xsd;
    if (!T || !P_bar || !out || !workspace || L <= 0 || L > XS_GP_MAX_LAYERS) return XS_EINVAL;
    if (!std::isfinite(T0) || !(a_T > 0.0) || !(tau_P > 0.0) || !(eps >= 0.0)) return XS_EINVAL;
    if (workspace_bytes < gp_prior_workspace_bytes(L)) return XS_EINVAL;
    double* C = (double*)workspace;
    double* y = C + (size_t)L * L;
    gp_prior_kernel<<<1, PRIOR_THREADS, 0, (cudaStream_t)stream>>>(T, P_bar, L, T0, a_T, tau_P, eps, C, y, out);
    xsi::count_launch();
    return cudaGetLastError() == cudaSuccess ? XS_OK : XS_ECUDA;
}

} // extern "C"

XS_CHECK_ACCESSOR(prior)
