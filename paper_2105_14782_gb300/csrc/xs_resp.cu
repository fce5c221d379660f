// Astronomical and instrumental responses (Sec. 4): rigid rotation with
// quadratic limb darkening and a Gaussian instrumental profile with a radial
// velocity, as the normalised kernel sums of Eq. responsenu,
//   F(nu'_i) = sum_j k(c ln(nu'_i/nu_j) + RV) F0_j / sum_j k(c ln(nu'_i/nu_j)),
// and their adjoints (in the input spectrum and in vsini or RV).
//
// One thread per output point; the pairs inside the kernel's support are found
// by binary search on the (increasing) grids.  The rotation kernel vanishes for
// |v| >= vsini; the Gaussian is summed over |v| <= 10 beta (the rest is below
// e^-50 of its peak).  Velocities in km/s.  FP64 throughout (this step is a few
// million kernel evaluations per spectrum).
#include "xs_device.cuh"
#include "xs_internal.h"

namespace xsd {

constexpr double C_KMS = 299792.458;
constexpr int RESP_THREADS = 128;
constexpr double GAUSS_SUPPORT = 10.0;

// zeta(x) of Sec. 4.1 from its disk-integral definition, s = sqrt(1 - x^2):
//   zeta = (2s (1 - u1 - u2) + (pi/2)(u1 + 2u2) s^2 - (4/3) u2 s^3) / (pi (1 - u1/3 - u2/6))
// and d zeta/dx = (2(1 - u1 - u2) + pi (u1 + 2u2) s - 4 u2 s^2)(-x/s) / (pi (1 - u1/3 - u2/6)).
struct RotKernel {
    double inv_v, u1, u2, inv_norm, W;
    __device__ double k(double v) const
    {
        const double x = v * inv_v;
        if (fabs(x) >= 1.0) return 0.0;
        const double s = sqrt(1.0 - x * x);
        return (2.0 * s * (1.0 - u1 - u2) + 0.5 * PI * (u1 + 2.0 * u2) * s * s - (4.0 / 3.0) * u2 * s * s * s) *
               inv_norm;
    }
    // d k / d vsini at fixed v: zeta'(x) (-x/vsini)
    __device__ double dk(double v) const
    {
        const double x = v * inv_v;
        if (fabs(x) >= 1.0) return 0.0;
        const double s = sqrt(1.0 - x * x);
        const double dz = (2.0 * (1.0 - u1 - u2) + PI * (u1 + 2.0 * u2) * s - 4.0 * u2 * s * s) * (-x / s) * inv_norm;
        return dz * (-x * inv_v);
    }
};

// Gaussian IP of Sec. 4.2 (normalisation cancels in Eq. responsenu); dk = d k/d v
struct GaussKernel {
    double inv_b, W;
    __device__ double k(double v) const
    {
        const double t = v * inv_b;
        return exp(-0.5 * t * t);
    }
    __device__ double dk(double v) const
    {
        const double t = v * inv_b;
        return -t * inv_b * exp(-0.5 * t * t);
    }
};

__device__ __forceinline__ int64_t lower_idx(const double* v, int64_t n, double x) // first i with v[i] >= x
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t m = (lo + hi) >> 1;
        if (v[m] >= x) hi = m; else lo = m + 1;
    }
    return lo;
}

// Forward (and, with want_d, the derivative of the output in the kernel's
// parameter: for the rotation d/d vsini of num/den, for the Gaussian d/d RV).
// den[i] is written when den != nullptr.
template <class K, bool ROT>
__global__ void __launch_bounds__(RESP_THREADS) response_kernel(const double* __restrict__ F, const double* __restrict__ nu,
                                                                int64_t N, const double* __restrict__ nu_out,
                                                                int64_t No, K ker, double rv,
                                                                double* __restrict__ out, double* __restrict__ den_out,
                                                                const double* __restrict__ g_out,
                                                                double* __restrict__ part)
{
    __shared__ double red[RESP_THREADS];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double contrib = 0.0;
    if (i < No) {
        const double nui = nu_out[i];
        const double lo = fmin(-ker.W - rv, -ker.W), hi = fmax(ker.W - rv, ker.W);
        // c ln(nu'_i/nu_j) in [lo, hi]  <=>  nu_j in [nu'_i e^{-hi/c}, nu'_i e^{-lo/c}]
        const int64_t b = lower_idx(nu, N, nui * exp(-hi / C_KMS) * (1.0 - 1e-15));
        const int64_t e = lower_idx(nu, N, nui * exp(-lo / C_KMS) * (1.0 + 1e-15));
        double num = 0.0, den = 0.0, dnum = 0.0, dden = 0.0;
        for (int64_t j = b; j < e; ++j) {
            const double a = C_KMS * log(nui / nu[j]); // ratio near 1: log keeps full relative accuracy
            const double Fj = F[j];
            num += ker.k(a + rv) * Fj;
            den += ker.k(a);
            if (g_out) {
                dnum += ker.dk(a + rv) * Fj;
                if (ROT) dden += ker.dk(a);
            }
        }
        const double o = num / den;
        if (out) out[i] = o;
        if (den_out) den_out[i] = den;
        if (g_out) contrib = g_out[i] * (dnum - o * dden) / den;
    }
    if (part) {
        red[threadIdx.x] = contrib;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[blockIdx.x] = red[0];
    }
}

// g_F[j] = sum_i g_out[i] k(c ln(nu'_i/nu_j) + RV) / den[i]  (transpose of Eq. responsenu)
template <class K>
__global__ void __launch_bounds__(RESP_THREADS) response_transpose_kernel(
    const double* __restrict__ g_out, const double* __restrict__ den, const double* __restrict__ nu, int64_t N,
    const double* __restrict__ nu_out, int64_t No, K ker, double rv, double* __restrict__ g_F)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const double nuj = nu[j];
    // c ln(nu'_i/nu_j) + rv in [-W, W]  <=>  nu'_i in [nu_j e^{(-W - rv)/c}, nu_j e^{(W - rv)/c}]
    const int64_t b = lower_idx(nu_out, No, nuj * exp((-ker.W - rv) / C_KMS) * (1.0 - 1e-15));
    const int64_t e = lower_idx(nu_out, No, nuj * exp((ker.W - rv) / C_KMS) * (1.0 + 1e-15));
    double g = 0.0;
    for (int64_t i = b; i < e; ++i) g += g_out[i] * ker.k(C_KMS * log(nu_out[i] / nuj) + rv) / den[i];
    g_F[j] = g;
}

__global__ void sum_parts_kernel(const double* __restrict__ part, int64_t n, double* __restrict__ out)
{
    __shared__ double red[256];
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += part[i];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

} // namespace xsd

namespace {

using namespace xsd;

RotKernel rot_kernel(double vsini, double u1, double u2)
{
    RotKernel k;
    k.inv_v = 1.0 / vsini;
    k.u1 = u1;
    k.u2 = u2;
    k.inv_norm = 1.0 / (PI * (1.0 - u1 / 3.0 - u2 / 6.0));
    k.W = vsini;
    return k;
}

GaussKernel gauss_kernel(double beta)
{
    GaussKernel k;
    k.inv_b = 1.0 / beta;
    k.W = GAUSS_SUPPORT * beta;
    return k;
}

unsigned blocks(int64_t n) { return (unsigned)((n + RESP_THREADS - 1) / RESP_THREADS); }

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

bool grid_ok(const double* nu, int64_t N) { return nu != nullptr && N >= 1; }

int finish(int n_launch)
{
    xsi::count_launch(n_launch);
    return cudaGetLastError() == cudaSuccess ? XS_OK : XS_ECUDA;
}

} // namespace

extern "C" {

int response_rotation(const double* F0, const double* nu, int64_t N, double vsini, double u1, double u2, double* F1,
                      xs_stream stream)
{
    XS_NVTX("response_rotation");
    if (!F0 || !F1 || !grid_ok(nu, N) || !(vsini > 0.0) || !(1.0 - u1 / 3.0 - u2 / 6.0 > 0.0)) return XS_EINVAL;
    response_kernel<RotKernel, true><<<blocks(N), RESP_THREADS, 0, (cudaStream_t)stream>>>(
        F0, nu, N, nu, N, rot_kernel(vsini, u1, u2), 0.0, F1, nullptr, nullptr, nullptr);
    return finish(1);
}

int response_ip_rv(const double* F1, const double* nu, int64_t N, const double* nu_out, int64_t N_out, double beta,
                   double rv, double* F, xs_stream stream)
{
    XS_NVTX("response_ip_rv");
    if (!F1 || !F || !grid_ok(nu, N) || !grid_ok(nu_out, N_out) || !(beta > 0.0) || !(fabs(rv) < C_KMS))
        return XS_EINVAL;
    response_kernel<GaussKernel, false><<<blocks(N_out), RESP_THREADS, 0, (cudaStream_t)stream>>>(
        F1, nu, N, nu_out, N_out, gauss_kernel(beta), rv, F, nullptr, nullptr, nullptr);
    return finish(1);
}

size_t response_workspace_bytes(int64_t N_out)
{
    if (N_out <= 0) return 0;
    return al256(sizeof(double) * (size_t)N_out) + al256(sizeof(double) * (size_t)blocks(N_out));
}

int response_rotation_adjoint(const double* g_F1, const double* F0, const double* nu, int64_t N, double vsini,
                              double u1, double u2, double* g_F0, double* g_vsini, void* workspace,
                              size_t workspace_bytes, xs_stream stream)
{
    XS_NVTX("response_rotation_adjoint");
    if (!g_F1 || !F0 || !g_F0 || !g_vsini || !workspace || !grid_ok(nu, N) || !(vsini > 0.0) ||
        !(1.0 - u1 / 3.0 - u2 / 6.0 > 0.0))
        return XS_EINVAL;
    if (workspace_bytes < response_workspace_bytes(N)) return XS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    double* den = (double*)workspace;
    double* part = (double*)((char*)workspace + al256(sizeof(double) * (size_t)N));
    const RotKernel k = rot_kernel(vsini, u1, u2);
    response_kernel<RotKernel, true><<<blocks(N), RESP_THREADS, 0, st>>>(F0, nu, N, nu, N, k, 0.0, nullptr, den,
                                                                         g_F1, part);
    sum_parts_kernel<<<1, 256, 0, st>>>(part, blocks(N), g_vsini);
    response_transpose_kernel<RotKernel><<<blocks(N), RESP_THREADS, 0, st>>>(g_F1, den, nu, N, nu, N, k, 0.0, g_F0);
    return finish(3);
}

int response_ip_rv_adjoint(const double* g_F, const double* F1, const double* nu, int64_t N, const double* nu_out,
                           int64_t N_out, double beta, double rv, double* g_F1, double* g_rv, void* workspace,
                           size_t workspace_bytes, xs_stream stream)
{
    XS_NVTX("response_ip_rv_adjoint");
    if (!g_F || !F1 || !g_F1 || !g_rv || !workspace || !grid_ok(nu, N) || !grid_ok(nu_out, N_out) ||
        !(beta > 0.0) || !(fabs(rv) < C_KMS))
        return XS_EINVAL;
    if (workspace_bytes < response_workspace_bytes(N_out)) return XS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    double* den = (double*)workspace;
    double* part = (double*)((char*)workspace + al256(sizeof(double) * (size_t)N_out));
    const GaussKernel k = gauss_kernel(beta);
    response_kernel<GaussKernel, false><<<blocks(N_out), RESP_THREADS, 0, st>>>(F1, nu, N, nu_out, N_out, k, rv,
                                                                                nullptr, den, g_F, part);
    sum_parts_kernel<<<1, 256, 0, st>>>(part, blocks(N_out), g_rv);
    response_transpose_kernel<GaussKernel><<<blocks(N), RESP_THREADS, 0, st>>>(g_F, den, nu, N, nu_out, N_out, k,
                                                                               rv, g_F1);
    return finish(3);
}

} // extern "C"

XS_CHECK_ACCESSOR(resp)
