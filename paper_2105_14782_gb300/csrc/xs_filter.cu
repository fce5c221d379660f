// Weak-line pre-filter (App. G): which lines can shape the emission spectrum.
// Per line, in an isothermal atmosphere at the scan temperature where the line's
// strength S(T) (Eq. Slog) is largest: the line-centre layer optical depths
//   dtau_n = dP_n 1e6/(mu m_u g) vmr S/(sqrt(2 pi) beta) erfcx(gamma_n/(sqrt2 beta)),
// the contribution function psi_n = exp(-tau_n) dtau_n P_n/dP_n (tau_n = sum_{k<=n}
// dtau_k) and its argmax n_hat (first on ties).  The grey continuum
// (kappa_coef P cm^2/g) gets its n_hat the same way; a line is kept when
// n_hat <= n_hat_continuum + margin (layer 0 at the top).  One thread per line,
// FP64 (one pass over the layers per line).
#include "xs_device.cuh"
#include "xs_internal.h"

namespace xsd {

constexpr int FILTER_MAX_SCAN = 64;

struct ScanArgs {
    double T[FILTER_MAX_SCAN];
};

__device__ __forceinline__ int contribution_argmax_continuum(const double* P, const double* dP, int L, double fac,
                                                             double kappa)
{
    double tau = 0.0, best = -1.0;
    int arg = 0;
    for (int n = 0; n < L; ++n) {
        const double dt = kappa * P[n] * dP[n] * fac;
        tau += dt;
        const double psi = exp(-tau) * dt * P[n] / dP[n];
        if (psi > best) {
            best = psi;
            arg = n;
        }
    }
    return arg;
}

__global__ void contribution_filter_kernel(const double* __restrict__ nu_hat, const double* __restrict__ ln_S0,
                                           const double* __restrict__ elower, const double* __restrict__ gamma_ref,
                                           const double* __restrict__ n_temp, int64_t nl, double mass, double qexp,
                                           const double* __restrict__ P, const double* __restrict__ dP, int L,
                                           ScanArgs scan, int nT, double vmr, double g, double mu, double kappa,
                                           double sb, int margin, uint8_t* __restrict__ keep,
                                           int32_t* __restrict__ n_hat)
{
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nl) return;
    const double nuh = nu_hat[l];
    // the scan temperature of largest S(T)
    double bestS = -1.0, Ts = scan.T[0];
    const double den = expm1(-c2 * nuh / Tref);
    for (int i = 0; i < nT; ++i) {
        const double T = scan.T[i];
        const double S = exp(ln_S0[l] - c2 * elower[l] * (1.0 / T - 1.0 / Tref) - qexp * log(T / Tref)) *
                         (expm1(-c2 * nuh / T) / den);
        if (S > bestS) {
            bestS = S;
            Ts = T;
        }
    }
    const double beta = sqrt(kB * Ts / (mass * amu)) * nuh / cL;
    const double amp = bestS / (sqrt(2.0 * PI) * beta);
    const double gT = sb * gamma_ref[l] * exp(-n_temp[l] * log(Ts / Tref)) / bar_per_atm;
    const double fac = 1e6 / g;                   // dP [bar] -> dyn/cm^2 over g
    const double col = fac / (mu * amu) * vmr;    // molecules per cm^2 per bar of dP
    double tau = 0.0, best = -1.0;
    int arg = 0;
    for (int n = 0; n < L; ++n) {
        const double a = gT * P[n] / (SQRT2 * beta);
        const double dt = dP[n] * col * amp * erfcx(a);
        tau += dt;
        const double psi = exp(-tau) * dt * P[n] / dP[n];
        if (psi > best) {
            best = psi;
            arg = n;
        }
    }
    const int nc = contribution_argmax_continuum(P, dP, L, fac, kappa);
    keep[l] = (uint8_t)(arg <= nc + margin);
    if (n_hat) n_hat[l] = arg;
}

} // namespace xsd

extern "C" int lines_contribution_filter(const xs_lines* lines, const double* P_bar, const double* dP_bar, int32_t L,
                                         const double* T_scan, int32_t n_scan, double vmr, double gravity, double mu,
                                         double kappa_coef, double broad_scale, int32_t margin, uint8_t* keep,
                                         int32_t* n_hat, xs_stream stream)
{
    XS_NVTX("lines_contribution_filter");
    using namespace xsd;
    if (!lines || lines->n < 0 || !P_bar || !dP_bar || L <= 0 || !T_scan || n_scan < 1 || n_scan > FILTER_MAX_SCAN ||
        !keep)
        return XS_EINVAL;
    if (lines->n > 0 && (!lines->nu_hat || !lines->ln_S0 || !lines->elower || !lines->gamma_ref || !lines->n_temp))
        return XS_EINVAL;
    if (!(vmr > 0.0) || !(gravity > 0.0) || !(mu > 0.0) || !(kappa_coef >= 0.0) || !(broad_scale > 0.0) ||
        !(lines->mass_amu > 0.0))
        return XS_EINVAL;
    ScanArgs sa{};
    for (int i = 0; i < n_scan; ++i) {
        if (!(T_scan[i] > 0.0)) return XS_EINVAL;
        sa.T[i] = T_scan[i];
    }
    if (lines->n == 0) return XS_OK;
    contribution_filter_kernel<<<(unsigned)((lines->n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        lines->nu_hat, lines->ln_S0, lines->elower, lines->gamma_ref, lines->n_temp, lines->n, lines->mass_amu,
        lines->q_exponent, P_bar, dP_bar, L, sa, n_scan, vmr, gravity, mu, kappa_coef, broad_scale, margin, keep,
        n_hat);
    xsi::count_launch();
    return cudaGetLastError() == cudaSuccess ? XS_OK : XS_ECUDA;
}

XS_CHECK_ACCESSOR(filter)
