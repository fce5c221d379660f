// C ABI of libxs: argument checks, workspace plans and the composite model
// calls.  Every entry point returns an xs_status and never throws or prints.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <cstring>
#include <numeric>
#include <vector>

#include "xs_internal.h"

// ------------------------------------------------------------ diagnostics

namespace {
std::atomic<uint64_t> g_launches{0};
std::mutex g_prof_mu;
bool g_prof_on = false;
struct ProfPair {
    cudaEvent_t a, b;
    int kind;
};
std::vector<ProfPair> g_prof;    // pairs recorded since profiling was enabled
std::vector<cudaEvent_t> g_pool; // events kept for reuse
cudaEvent_t take_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
int g_open_kind = -1;
cudaEvent_t g_open_ev = nullptr;
} // namespace

namespace xsi {
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
void prof_begin(int kind, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return;
    g_open_ev = take_event();
    g_open_kind = kind;
    cudaEventRecord(g_open_ev, st);
}
void prof_end(int kind, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on || g_open_ev == nullptr || g_open_kind != kind) return;
    cudaEvent_t e = take_event();
    cudaEventRecord(e, st);
    g_prof.push_back({g_open_ev, e, kind});
    g_open_ev = nullptr;
    g_open_kind = -1;
}
} // namespace xsi

extern "C" {

int xs_profile(int enable)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& p : g_prof) {
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    g_prof.clear();
    g_prof_on = enable != 0;
    return XS_OK;
}

int xs_profile_read(double* fwd_ms, int64_t* fwd_launches, double* adj_ms, int64_t* adj_launches)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    double t[2] = {0.0, 0.0};
    int64_t c[2] = {0, 0};
    for (auto& p : g_prof) {
        if (cudaEventSynchronize(p.b) != cudaSuccess) return XS_ECUDA;
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) return XS_ECUDA;
        t[p.kind] += ms;
        c[p.kind] += 1;
    }
    if (fwd_ms) *fwd_ms = t[0];
    if (fwd_launches) *fwd_launches = c[0];
    if (adj_ms) *adj_ms = t[1];
    if (adj_launches) *adj_launches = c[1];
    return XS_OK;
}

uint64_t xs_launch_count(void) { return g_launches.load(); }

} // extern "C"

namespace {

inline cudaStream_t S(xs_stream s) { return (cudaStream_t)s; }
inline size_t al(size_t v) { return (v + 255) & ~(size_t)255; }
inline bool prec_ok(int p) { return p == XS_PREC_FP64 || p == XS_PREC_MIXED; }
using xsi::check_common;
using xsi::check_lines;

} // namespace

namespace xsi {

int check_lines(const xs_lines* ln)
{
    if (!ln || ln->n < 0) return XS_EINVAL;
    if (ln->n > 0 && (!ln->nu_hat || !ln->ln_S0 || !ln->elower || !ln->gamma_ref || !ln->n_temp)) return XS_EINVAL;
    if (ln->n >= (int64_t)1 << 31) return XS_EINVAL;
    if (!(ln->mass_amu > 0.0) || !std::isfinite(ln->q_exponent)) return XS_EINVAL;
    return XS_OK;
}

int check_common(const xs_lines* ln, const double* nu, int64_t N, const double* T, const double* P, int32_t L,
                 double sb, double W, int prec)
{
    int r = check_lines(ln);
    if (r) return r;
    if (!nu || !T || !P || N <= 0 || L <= 0 || N >= ((int64_t)1 << 31) - 2048) return XS_EINVAL;
    if (!(W > 0.0) || !(sb > 0.0) || !prec_ok(prec)) return XS_EINVAL;
    return XS_OK;
}

} // namespace xsi

extern "C" {

int xs_checked_build(void)
{
#ifdef XS_CHECKED
    return 1;
#else
    return 0;
#endif
}

int xs_check_status(int clear)
{
    XS_NVTX("xs_check_status");
    if (cudaDeviceSynchronize() != cudaSuccess) return XS_ECUDA;
    int (*const f[])(int) = {xsi::check_status_linesum, xsi::check_status_rt, xsi::check_status_modit,
                             xsi::check_status_resp, xsi::check_status_filter, xsi::check_status_prior};
    int worst = 0;
    for (int i = 0; i < 6; ++i) {
        const int v = f[i](clear);
        if (v < 0) return XS_ECUDA;
        if (v > 0 && worst == 0) worst = (i + 1) * 100000 + v;
    }
    return worst;
}

const char* xs_strerror(int status)
{
    switch (status) {
    case XS_OK: return "ok";
    case XS_EINVAL: return "invalid argument";
    case XS_EUNSORTED: return "line centres or grid not in ascending order";
    case XS_ENOMEM: return "out of host memory";
    case XS_ECUDA: return "CUDA error";
    case XS_ETIMEOUT: return "timed out";
    case XS_ETOOBIG: return "problem needs more scratch memory than the fixed or given workspace holds";
    default: return "unknown status";
    }
}

int xs_sort_lines_host(int64_t n, double* nu_hat, double* ln_S0, double* elower, double* gamma_ref, double* n_temp)
{
    if (n < 0) return XS_EINVAL;
    if (n == 0) return XS_OK;
    if (!nu_hat || !ln_S0 || !elower || !gamma_ref || !n_temp) return XS_EINVAL;
    std::vector<int64_t> idx((size_t)n);
    std::iota(idx.begin(), idx.end(), (int64_t)0);
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return nu_hat[a] < nu_hat[b]; });
    std::vector<double> tmp((size_t)n);
    double* f[5] = {nu_hat, ln_S0, elower, gamma_ref, n_temp};
    for (double* a : f) {
        for (int64_t i = 0; i < n; ++i) tmp[(size_t)i] = a[idx[(size_t)i]];
        std::memcpy(a, tmp.data(), sizeof(double) * (size_t)n);
    }
    return XS_OK;
}

int xs_check_sorted(const double* v, int64_t n, int strict, int* flag_dev, xs_stream stream)
{
    XS_NVTX("xs_check_sorted");
    if (n < 0 || (n > 0 && !v) || !flag_dev) return XS_EINVAL;
    return xsi::check_sorted(v, n, S(stream), flag_dev, strict != 0);
}

int xs_compute(const xs_lines* lines, const double* nu, int64_t N, const double* T, const double* P_bar, int32_t L,
               double broad_scale, double wing_cut, int prec, void* sigma, void* workspace, size_t workspace_bytes,
               xs_stream stream)
{
    XS_NVTX("xs_compute");
    int r = check_common(lines, nu, N, T, P_bar, L, broad_scale, wing_cut, prec);
    if (r) return r;
    if (!sigma || !workspace) return XS_EINVAL;
    if (workspace_bytes < xs_workspace_min_bytes(lines->n, N, L, prec)) return XS_EINVAL;
    return xsi::xs_run(lines, nu, N, T, P_bar, L, broad_scale, wing_cut, prec, sigma, workspace, workspace_bytes,
                       false, nullptr, nullptr, nullptr, S(stream));
}

int xs_compute_adjoint(const xs_lines* lines, const double* nu, int64_t N, const double* T, const double* P_bar,
                       int32_t L, double broad_scale, double wing_cut, int prec, const double* g_sigma, double* g_T,
                       double* g_broad, void* workspace, size_t workspace_bytes, xs_stream stream)
{
    XS_NVTX("xs_compute_adjoint");
    int r = check_common(lines, nu, N, T, P_bar, L, broad_scale, wing_cut, prec);
    if (r) return r;
    if (!g_sigma || !g_T || !g_broad || !workspace) return XS_EINVAL;
    if (workspace_bytes < xs_workspace_min_bytes(lines->n, N, L, prec)) return XS_EINVAL;
    return xsi::xs_run(lines, nu, N, T, P_bar, L, broad_scale, wing_cut, prec, nullptr, workspace, workspace_bytes,
                       true, g_sigma, g_T, g_broad, S(stream));
}

int tau_layers(const void* const* sigma, int32_t nsp, const double* vmr, const double* P_bar, const double* dP_bar,
               int32_t L, int64_t N, double gravity, double mu, double kappa_coef, int prec, double* dtau,
               xs_stream stream)
{
    XS_NVTX("tau_layers");
    if (!sigma || nsp < 1 || nsp > XS_MAX_SPECIES || !vmr || !P_bar || !dP_bar || L <= 0 || N <= 0 || !dtau)
        return XS_EINVAL;
    for (int m = 0; m < nsp; ++m)
        if (!sigma[m]) return XS_EINVAL;
    if (!(gravity > 0.0) || !(mu > 0.0) || !prec_ok(prec) || !std::isfinite(kappa_coef)) return XS_EINVAL;
    return xsi::rt_tau(sigma, nsp, vmr, P_bar, dP_bar, L, N, gravity, mu, kappa_coef, prec, dtau, S(stream));
}

int tau_layers_adjoint(const void* const* sigma, int32_t nsp, const double* vmr, const double* P_bar,
                       const double* dP_bar, int32_t L, int64_t N, double gravity, double mu, int prec,
                       const double* g_dtau, double* const* g_sigma, double* g_vmr, xs_stream stream)
{
    XS_NVTX("tau_layers_adjoint");
    if (!sigma || nsp < 1 || nsp > XS_MAX_SPECIES || !vmr || !P_bar || !dP_bar || L <= 0 || N <= 0 || !g_dtau ||
        !g_vmr)
        return XS_EINVAL;
    for (int m = 0; m < nsp; ++m)
        if (!sigma[m]) return XS_EINVAL;
    if (!(gravity > 0.0) || !(mu > 0.0) || !prec_ok(prec)) return XS_EINVAL;
    return xsi::rt_tau_adjoint(sigma, nsp, vmr, P_bar, dP_bar, L, N, gravity, mu, prec, g_dtau, g_sigma, g_vmr,
                               S(stream));
}

int emission_spectrum(const double* dtau, const double* T, const double* nu, int32_t L, int64_t N, double* F0,
                      xs_stream stream)
{
    XS_NVTX("emission_spectrum");
    if (!dtau || !T || !nu || L <= 0 || N <= 0 || !F0) return XS_EINVAL;
    return xsi::rt_emission(dtau, T, nu, L, N, F0, S(stream));
}

int tau_cia(const double* alpha, const double* T_grid, int32_t nT, const double* T, const double* P_bar,
            const double* dP_bar, int32_t L, int64_t N, double vmr1, double vmr2, double gravity, double mu,
            int accumulate, double* dtau, xs_stream stream)
{
    XS_NVTX("tau_cia");
    if (!alpha || !T_grid || nT < 1 || !T || !P_bar || !dP_bar || L <= 0 || N <= 0 || !dtau) return XS_EINVAL;
    if (!(gravity > 0.0) || !(mu > 0.0) || !(vmr1 >= 0.0) || !(vmr2 >= 0.0)) return XS_EINVAL;
    return xsi::rt_tau_cia(alpha, T_grid, nT, T, P_bar, dP_bar, L, N, vmr1, vmr2, gravity, mu, accumulate != 0, dtau,
                           S(stream));
}

int tau_cia_adjoint(const double* g_dtau, const double* alpha, const double* T_grid, int32_t nT, const double* T,
                    const double* P_bar, const double* dP_bar, int32_t L, int64_t N, double vmr1, double vmr2,
                    double gravity, double mu, double* g_T, xs_stream stream)
{
    XS_NVTX("tau_cia_adjoint");
    if (!g_dtau || !alpha || !T_grid || nT < 1 || !T || !P_bar || !dP_bar || L <= 0 || N <= 0 || !g_T)
        return XS_EINVAL;
    if (!(gravity > 0.0) || !(mu > 0.0)) return XS_EINVAL;
    return xsi::rt_tau_cia_adjoint(g_dtau, alpha, T_grid, nT, T, P_bar, dP_bar, L, N, vmr1, vmr2, gravity, mu, g_T,
                                   S(stream));
}

size_t emission_workspace_bytes(int32_t L, int64_t N)
{
    if (L <= 0 || N <= 0) return 0;
    return al(xsi::rt_emission_ws(L, N));
}

int emission_spectrum_adjoint(const double* g_F0, const double* dtau, const double* T, const double* nu, int32_t L,
                              int64_t N, double* g_dtau, double* g_T, void* workspace, size_t workspace_bytes,
                              xs_stream stream)
{
    XS_NVTX("emission_spectrum_adjoint");
    if (!g_F0 || !dtau || !T || !nu || L <= 0 || N <= 0 || !g_dtau || !g_T || !workspace) return XS_EINVAL;
    if (workspace_bytes < emission_workspace_bytes(L, N)) return XS_EINVAL;
    return xsi::rt_emission_adjoint(g_F0, dtau, T, nu, L, N, g_dtau, g_T, workspace, S(stream));
}

int loglike_gauss(const double* F, const double* d, const double* s, int64_t N, double* logL, double* g_F,
                  xs_stream stream)
{
    XS_NVTX("loglike_gauss");
    if (!F || !d || !s || N <= 0 || !logL) return XS_EINVAL;
    return xsi::rt_loglike(F, d, s, N, logL, g_F, S(stream));
}

int layer_temperatures(double T0, double alpha, const double* P_bar, int32_t L, double* T, xs_stream stream)
{
    XS_NVTX("layer_temperatures");
    if (!P_bar || !T || L <= 0 || !(T0 > 0.0) || !std::isfinite(alpha)) return XS_EINVAL;
    return xsi::rt_temperatures(T0, alpha, P_bar, L, T, S(stream));
}

} // extern "C"

// ------------------------------------------------------------ composite model

namespace {

struct ModelPlan {
    size_t T, vmr, sigma, dtau, F0, gF, gdtau, gsig, gvmr, gT, gTtmp, gb, xsws, emws, total;
    size_t xsws_bytes;
    size_t xsws_sp[XS_MAX_SPECIES], xsws_sp_bytes[XS_MAX_SPECIES];
    int64_t max_nl;
};

int check_model(const xs_model* m)
{
    if (!m || m->n_species < 1 || m->n_species > XS_MAX_SPECIES) return XS_EINVAL;
    if (!m->nu || m->N <= 0 || !m->P_bar || !m->dP_bar || m->L <= 0) return XS_EINVAL;
    if (!(m->wing_cut > 0.0) || !(m->gravity > 0.0) || !(m->mu > 0.0) || !prec_ok(m->prec)) return XS_EINVAL;
    for (int s = 0; s < m->n_species; ++s)
        if (check_lines(&m->species[s])) return XS_EINVAL;
    if (m->method != XS_METHOD_LPF && m->method != XS_METHOD_MODIT) return XS_EINVAL;
    if (m->cia_alpha && (!m->cia_T || m->cia_nT < 1 || !(m->cia_vmr1 >= 0.0) || !(m->cia_vmr2 >= 0.0)))
        return XS_EINVAL;
    if (m->method == XS_METHOD_MODIT) {
        if (m->n_gamma < 1 || m->n_gamma > 32 || !(m->nu_min > 0.0) || !(m->nu_max > m->nu_min) || m->N < 2)
            return XS_EINVAL;
        for (int s = 0; s < m->n_species; ++s) {
            const int64_t M = m->n_fft[s];
            if (M < m->N + 2 || (M & (M - 1)) != 0) return XS_EINVAL;
        }
    }
    return XS_OK;
}

ModelPlan plan_model(const xs_model* m)
{
    ModelPlan p{};
    const int Sp = m->n_species;
    const size_t LN = (size_t)m->L * (size_t)m->N;
    const size_t es = (m->prec == XS_PREC_MIXED) ? sizeof(float) : sizeof(double);
    p.max_nl = 0;
    for (int s = 0; s < Sp; ++s) p.max_nl = std::max<int64_t>(p.max_nl, m->species[s].n);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += al(bytes);
        return o;
    };
    p.T = take(sizeof(double) * m->L);
    p.vmr = take(sizeof(double) * Sp * m->L);
    p.sigma = take(es * LN * Sp);
    p.dtau = take(sizeof(double) * LN);
    p.F0 = take(sizeof(double) * m->N);
    p.gF = take(sizeof(double) * m->N);
    p.gdtau = take(sizeof(double) * LN);
    p.gsig = take(sizeof(double) * LN * Sp);
    p.gvmr = take(sizeof(double) * Sp * m->L);
    p.gT = take(sizeof(double) * m->L);
    p.gTtmp = take(sizeof(double) * m->L);
    p.gb = take(sizeof(double) * Sp);
    // one full workspace per species, so the forward's line records stay valid
    // for the adjoint of the same call
    for (int s = 0; s < Sp; ++s) {
        if (m->method == XS_METHOD_MODIT)
            p.xsws_sp_bytes[s] =
                std::max(modit_workspace_bytes(m->species[s].n, m->L, m->n_gamma, m->n_fft[s], m->prec),
                         modit_adjoint_workspace_bytes(m->species[s].n, m->L, m->n_gamma, m->n_fft[s], m->prec));
        else
            p.xsws_sp_bytes[s] = xs_workspace_bytes(m->species[s].n, m->N, m->L, m->prec);
        p.xsws_sp[s] = take(p.xsws_sp_bytes[s]);
    }
    p.xsws_bytes = p.xsws_sp_bytes[0];
    p.xsws = p.xsws_sp[0];
    p.emws = take(emission_workspace_bytes(m->L, m->N));
    p.total = off;
    return p;
}

// theta = (T0, alpha, log10 vmr.., s_b); with T_given (device [L]) the layer
// temperatures are those instead of the power law and theta[0], theta[1] unused.
int model_forward_impl(const xs_model* m, const double* theta, double* F0out, char* ws, const ModelPlan& p,
                       cudaStream_t st, int xs_flags = 0, const double* T_given = nullptr)
{
    const int Sp = m->n_species;
    const size_t LN = (size_t)m->L * (size_t)m->N;
    const size_t es = (m->prec == XS_PREC_MIXED) ? sizeof(float) : sizeof(double);
    double* T = (double*)(ws + p.T);
    double* vmr = (double*)(ws + p.vmr);
    char* sig = ws + p.sigma;
    double* dtau = (double*)(ws + p.dtau);
    int r;
    if (T_given) {
        if (cudaMemcpyAsync(T, T_given, sizeof(double) * m->L, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return XS_ECUDA;
    } else {
        r = xsi::rt_temperatures(theta[0], theta[1], m->P_bar, m->L, T, st);
        if (r) return r;
    }
    r = xsi::rt_fill_vmr(nullptr, Sp, m->L, theta + 2, vmr, st);
    if (r) return r;
    const void* sp[XS_MAX_SPECIES];
    for (int s = 0; s < Sp; ++s) {
        sp[s] = sig + es * LN * s;
        if (m->method == XS_METHOD_MODIT)
            r = modit_compute(&m->species[s], m->nu_min, m->nu_max, m->N, T, m->P_bar, m->L, theta[2 + Sp],
                              m->n_gamma, m->n_fft[s], m->prec, (void*)sp[s], ws + p.xsws_sp[s], p.xsws_sp_bytes[s],
                              st);
        else
            r = xsi::xs_run(&m->species[s], m->nu, m->N, T, m->P_bar, m->L, theta[2 + Sp], m->wing_cut, m->prec,
                            (void*)sp[s], ws + p.xsws_sp[s], p.xsws_sp_bytes[s], false, nullptr, nullptr, nullptr, st,
                            xs_flags);
        if (r) return r;
    }
    r = xsi::rt_tau(sp, Sp, vmr, m->P_bar, m->dP_bar, m->L, m->N, m->gravity, m->mu, m->kappa_coef, m->prec, dtau, st);
    if (r) return r;
    if (m->cia_alpha) {
        r = xsi::rt_tau_cia(m->cia_alpha, m->cia_T, m->cia_nT, T, m->P_bar, m->dP_bar, m->L, m->N, m->cia_vmr1,
                            m->cia_vmr2, m->gravity, m->mu, 1, dtau, st);
        if (r) return r;
    }
    return xsi::rt_emission(dtau, T, m->nu, m->L, m->N, F0out, st);
}

} // namespace

extern "C" {

size_t xs_model_workspace_bytes(const xs_model* model)
{
    if (check_model(model)) return 0;
    return plan_model(model).total;
}

int xs_model_forward(const xs_model* model, const double* theta, double* F0, void* workspace, size_t workspace_bytes,
                     xs_stream stream)
{
    XS_NVTX("xs_model_forward");
    int r = check_model(model);
    if (r) return r;
    if (!theta || !F0 || !workspace) return XS_EINVAL;
    ModelPlan p = plan_model(model);
    if (workspace_bytes < p.total) return XS_EINVAL;
    if (!(theta[0] > 0.0) || !(theta[2 + model->n_species] > 0.0)) return XS_EINVAL;
    return model_forward_impl(model, theta, F0, (char*)workspace, p, S(stream));
}

} // extern "C"

namespace {

// Reverse sweep of the composite model from g_F = dlogL/dF0 (device [N]), after
// a forward with XS_RUN_KEEP_ADJ in the same workspace: out[1 .. 3 + S] = dlogL/dtheta.
int model_adjoint_impl(const xs_model* m, const double* theta, const double* gF, double* out, char* ws,
                       const ModelPlan& p, cudaStream_t st, bool per_layer = false)
{
    const int Sp = m->n_species;
    const size_t LN = (size_t)m->L * (size_t)m->N;
    const size_t es = (m->prec == XS_PREC_MIXED) ? sizeof(float) : sizeof(double);
    double* T = (double*)(ws + p.T);
    double* vmr = (double*)(ws + p.vmr);
    char* sig = ws + p.sigma;
    double* dtau = (double*)(ws + p.dtau);
    double* gdtau = (double*)(ws + p.gdtau);
    double* gsig = (double*)(ws + p.gsig);
    double* gvmr = (double*)(ws + p.gvmr);
    double* gT = (double*)(ws + p.gT);
    double* gTtmp = (double*)(ws + p.gTtmp);
    double* gb = (double*)(ws + p.gb);
    int r;
    if ((r = xsi::rt_emission_adjoint(gF, dtau, T, m->nu, m->L, m->N, gdtau, gT, ws + p.emws, st))) return r;
    if (m->cia_alpha &&
        (r = xsi::rt_tau_cia_adjoint(gdtau, m->cia_alpha, m->cia_T, m->cia_nT, T, m->P_bar, m->dP_bar, m->L, m->N,
                                     m->cia_vmr1, m->cia_vmr2, m->gravity, m->mu, gT, st)))
        return r;
    const void* sp[XS_MAX_SPECIES];
    double* gsp[XS_MAX_SPECIES];
    for (int s = 0; s < Sp; ++s) {
        sp[s] = sig + es * LN * s;
        gsp[s] = gsig + LN * s;
    }
    if ((r = xsi::rt_tau_adjoint(sp, Sp, vmr, m->P_bar, m->dP_bar, m->L, m->N, m->gravity, m->mu, m->prec, gdtau, gsp,
                                 gvmr, st)))
        return r;
    for (int s = 0; s < Sp; ++s) {
        if (m->method == XS_METHOD_MODIT)
            r = modit_compute_adjoint(&m->species[s], m->nu_min, m->nu_max, m->N, T, m->P_bar, m->L, theta[2 + Sp],
                                      m->n_gamma, m->n_fft[s], m->prec, gsp[s], gTtmp, gb + s, ws + p.xsws_sp[s],
                                      p.xsws_sp_bytes[s], st);
        else
            r = xsi::xs_run(&m->species[s], m->nu, m->N, T, m->P_bar, m->L, theta[2 + Sp], m->wing_cut, m->prec,
                            nullptr, ws + p.xsws_sp[s], p.xsws_sp_bytes[s], true, gsp[s], gTtmp, gb + s, st,
                            xsi::XS_RUN_REUSE);
        if (r) return r;
        if ((r = xsi::rt_accumulate(gT, gTtmp, m->L, 0, st))) return r;
    }
    if (per_layer) return xsi::rt_layer_grad(Sp, m->L, theta + 2, gT, gvmr, gb, out, st);
    return xsi::rt_theta_grad(Sp, m->L, theta[0], theta[1], theta + 2, theta[2 + Sp], T, m->P_bar, gT, gvmr, gb, out,
                              st);
}

int model_args(const xs_model* m, const double* theta, void* workspace, size_t workspace_bytes, ModelPlan* p)
{
    int r = check_model(m);
    if (r) return r;
    if (!theta || !workspace) return XS_EINVAL;
    *p = plan_model(m);
    if (workspace_bytes < p->total) return XS_EINVAL;
    if (!(theta[0] > 0.0) || !(theta[2 + m->n_species] > 0.0)) return XS_EINVAL;
    return XS_OK;
}

} // namespace

extern "C" {

int xs_model_logl_grad(const xs_model* m, const double* theta, double* out, double* F0, void* workspace,
                       size_t workspace_bytes, xs_stream stream)
{
    XS_NVTX("xs_model_logl_grad");
    ModelPlan p;
    int r = model_args(m, theta, workspace, workspace_bytes, &p);
    if (r) return r;
    if (!out || !m->d_obs || !m->sig_obs) return XS_EINVAL;
    cudaStream_t st = S(stream);
    char* ws = (char*)workspace;
    double* F = F0 ? F0 : (double*)(ws + p.F0);
    r = model_forward_impl(m, theta, F, ws, p, st, xsi::XS_RUN_KEEP_ADJ);
    if (r) return r;
    double* gF = (double*)(ws + p.gF);
    if ((r = xsi::rt_loglike(F, m->d_obs, m->sig_obs, m->N, out, gF, st))) return r;
    return model_adjoint_impl(m, theta, gF, out, ws, p, st);
}

int xs_model_logl_grad_layers(const xs_model* m, const double* T, const double* log10_vmr, double broad_scale,
                              double* out, double* F0, void* workspace, size_t workspace_bytes, xs_stream stream)
{
    XS_NVTX("xs_model_logl_grad_layers");
    if (!m || !T || !log10_vmr || m->n_species < 1 || m->n_species > XS_MAX_SPECIES) return XS_EINVAL;
    // theta in the composite layout with placeholder T0 = 1, alpha = 0 (unused)
    double theta[3 + XS_MAX_SPECIES];
    theta[0] = 1.0;
    theta[1] = 0.0;
    for (int s = 0; s < m->n_species; ++s) theta[2 + s] = log10_vmr[s];
    theta[2 + m->n_species] = broad_scale;
    ModelPlan p;
    int r = model_args(m, theta, workspace, workspace_bytes, &p);
    if (r) return r;
    if (!out || !m->d_obs || !m->sig_obs) return XS_EINVAL;
    cudaStream_t st = S(stream);
    char* ws = (char*)workspace;
    double* F = F0 ? F0 : (double*)(ws + p.F0);
    r = model_forward_impl(m, theta, F, ws, p, st, xsi::XS_RUN_KEEP_ADJ, T);
    if (r) return r;
    double* gF = (double*)(ws + p.gF);
    if ((r = xsi::rt_loglike(F, m->d_obs, m->sig_obs, m->N, out, gF, st))) return r;
    return model_adjoint_impl(m, theta, gF, out, ws, p, st, true);
}

int xs_model_forward_keep(const xs_model* m, const double* theta, double* F0, void* workspace,
                          size_t workspace_bytes, xs_stream stream)
{
    XS_NVTX("xs_model_forward_keep");
    ModelPlan p;
    int r = model_args(m, theta, workspace, workspace_bytes, &p);
    if (r) return r;
    if (!F0) return XS_EINVAL;
    return model_forward_impl(m, theta, F0, (char*)workspace, p, S(stream), xsi::XS_RUN_KEEP_ADJ);
}

int xs_model_vjp(const xs_model* m, const double* theta, const double* g_F0, double* out, void* workspace,
                 size_t workspace_bytes, xs_stream stream)
{
    XS_NVTX("xs_model_vjp");
    ModelPlan p;
    int r = model_args(m, theta, workspace, workspace_bytes, &p);
    if (r) return r;
    if (!g_F0 || !out) return XS_EINVAL;
    cudaStream_t st = S(stream);
    if (cudaMemsetAsync(out, 0, sizeof(double), st) != cudaSuccess) return XS_ECUDA;
    return model_adjoint_impl(m, theta, g_F0, out, (char*)workspace, p, st);
}

} // extern "C"
