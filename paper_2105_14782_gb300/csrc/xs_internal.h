// Internal host-side interfaces shared by the translation units of libxs.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/xs.h"

namespace xsi {

// NVTX range named after the library call, around its host-side work and
// launches; costs a few nanoseconds and records nothing unless a profiler
// (nsys, ncu's NVTX filters) is attached
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define XS_NVTX(name) ::xsi::NvtxRange xs_nvtx_range_(name)

// status words of the bounds-checked build, one per translation unit with
// kernels: the largest source line of a failed check (0: none); cleared if asked
int check_status_linesum(int clear);
int check_status_rt(int clear);
int check_status_modit(int clear);
int check_status_resp(int clear);
int check_status_filter(int clear);
int check_status_prior(int clear);

// host-side launch counter (every kernel launch site bumps it)
void count_launch(int n = 1);
// profiling event pairs around line-sum launches (kind 0 forward, 1 adjoint)
void prof_begin(int kind, cudaStream_t st);
void prof_end(int kind, cudaStream_t st);

enum { XS_RUN_KEEP_ADJ = 1, XS_RUN_REUSE = 2 };

// argument checks shared by the entry points (XS_OK or XS_EINVAL, host side only)
int check_lines(const xs_lines* ln);
int check_common(const xs_lines* ln, const double* nu, int64_t N, const double* T, const double* P, int32_t L,
                 double sb, double W, int prec);

// line-sum forward (adjoint == false: writes sigma) or adjoint (writes g_T, g_b);
// flags as above (0 for a self-contained call)
int xs_run(const xs_lines* ln, const double* nu, int64_t N, const double* T, const double* P, int32_t L, double sb,
           double W, int prec, void* sigma, void* ws, size_t ws_bytes, bool adjoint, const double* g_sigma,
           double* g_T, double* g_b, cudaStream_t st, int flags = 0);

// checks ascending (grid == false: non-decreasing centres; grid == true: strictly
// increasing grid) on the device; blocks on `st`; flag_dev is one device int
int check_sorted(const double* v, int64_t n, cudaStream_t st, int* flag_dev, bool grid);

int rt_tau(const void* const* sigma, int32_t S, const double* vmr, const double* P, const double* dP, int32_t L,
           int64_t N, double g, double mu, double kappa, int prec, double* dtau, cudaStream_t st);
int rt_tau_adjoint(const void* const* sigma, int32_t S, const double* vmr, const double* P, const double* dP,
                   int32_t L, int64_t N, double g, double mu, int prec, const double* g_dtau, double* const* g_sigma,
                   double* g_vmr, cudaStream_t st);
int rt_emission(const double* dtau, const double* T, const double* nu, int32_t L, int64_t N, double* F0,
                cudaStream_t st);
size_t rt_emission_ws(int32_t L, int64_t N);
int rt_emission_adjoint(const double* g_F0, const double* dtau, const double* T, const double* nu, int32_t L,
                        int64_t N, double* g_dtau, double* g_T, void* ws, cudaStream_t st);
int rt_loglike(const double* F, const double* d, const double* s, int64_t N, double* logL, double* g_F,
               cudaStream_t st);
int rt_temperatures(double T0, double alpha, const double* P, int32_t L, double* T, cudaStream_t st);
int rt_fill_vmr(const double* theta_dev_unused, int32_t S, int32_t L, const double* log10_vmr_host, double* vmr,
                cudaStream_t st);
int rt_theta_grad(int32_t S, int32_t L, double T0, double alpha, const double* log10_vmr_host, double sb,
                  const double* T, const double* P, const double* g_T, const double* g_vmr, const double* g_b,
                  double* out, cudaStream_t st);
int rt_tau_cia(const double* alpha, const double* Tg, int32_t nT, const double* T, const double* P, const double* dP,
               int32_t L, int64_t N, double vmr1, double vmr2, double g, double mu, int accumulate, double* dtau,
               cudaStream_t st);
int rt_tau_cia_adjoint(const double* g_dtau, const double* alpha, const double* Tg, int32_t nT, const double* T,
                       const double* P, const double* dP, int32_t L, int64_t N, double vmr1, double vmr2, double g,
                       double mu, double* g_T, cudaStream_t st);
int rt_layer_grad(int32_t S, int32_t L, const double* log10_vmr_host, const double* g_T, const double* g_vmr,
                  const double* g_b, double* out, cudaStream_t st);
int rt_accumulate(double* dst, const double* src, int64_t n, int first, cudaStream_t st);

} // namespace xsi
