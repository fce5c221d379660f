/*
 * FP64 CPU oracle for the direct line-by-line opacity sum, layer optical depth
 * and Planck-source emission solve of Kawahara et al. (arXiv:2105.14782).
 *
 * TEST INFRASTRUCTURE ONLY.  It exists to check the CUDA library; it is called
 * from tests/, from __graft_entry__.smoke() and from bench.py's CPU-baseline leg,
 * and from nothing else.  It shares no code, header or constant table with the
 * CUDA path.  Plain double precision, no blocking or fusion beyond what the
 * definitions below state; OpenMP only splits independent output elements.
 *
 * What each function follows:
 *   orc_faddeeva      w(z) = exp(-z^2) erfc(-iz), H = Re w, L = Im w (Sec. 2.1.1).
 *                     |z| < 8: the exponentially convergent series behind the
 *                     paper's Eq. algo916 / algo916L (Zaghloul & Ali 2011),
 *                     re-derived here from the erf series of Abramowitz & Stegun
 *                     7.1.29 generalised to step h = 0.5, truncated adaptively.
 *                     |z| >= 8: Laplace continued fraction of w (Gautschi 1970),
 *                     depth 40, bottom-up.
 *   orc_line_params   S(T) of Eq. Slog with Q(T)/Q(296) = (T/296)^q; thermal
 *                     Doppler width of Eq. thermal; pressure width of
 *                     Eq. gammahitran with the self and natural terms dropped,
 *                     P in atm, times a broadening scale s_b.
 *   orc_xs            sigma(nu_j) = sum over lines with |nu_j - nu_hat| <= W of
 *                     S/(sqrt(2 pi) beta) H((nu_j-nu_hat)/(sqrt2 beta),
 *                     gamma/(sqrt2 beta)) (Eq. crosssec, Sec. 3.1), lines in
 *                     ascending centre order, Neumaier-compensated.
 *   orc_tau           Eq. dtau_line plus a continuum kappa_c(P) dP / g.
 *   orc_trans         T = 2 E3(x) = (1 - x) e^{-x} + x^2 E1(x) (Eq. trans).
 *   orc_emission      F0 = sum_n Phi_n (1 - T_n) S_n + Phi_L F_B with
 *                     Phi_n = prod_{k<n} T_k (Eqs. rerr2, rerr_tq, lart) and
 *                     S_n = pi B(T_n) (Eq. sourcepla); F_B = pi B(T_{L-1}).
 *   orc_logl_grad     Gaussian log-likelihood (Eq. likelihood without jitter) and
 *                     its gradient by forward-mode dual numbers (App. D), using
 *                     dw/dz = -2 z w + 2i/sqrt(pi), i.e. the derivative rules of
 *                     H printed in Sec. 2.1.1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define O_PI 3.14159265358979323846
#define O_SQRTPI 1.77245385090551602730
#define O_SQRT2 1.41421356237309504880
#define O_SQRT2PI 2.50662827463100050242

/* CODATA values (cgs) and the paper's c2 (Sec. 2.2, below Eq. Slog). */
static const double o_kB = 1.380649e-16;
static const double o_h = 6.62607015e-27;
static const double o_c = 2.99792458e10;
static const double o_mu = 1.66053906660e-24;
static const double o_c2 = 1.4387773;
static const double o_Tref = 296.0;
static const double o_Patm = 1.01325; /* bar per atm */

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- w(z) --- */

static void w_series(double x, double a, double* re, double* im)
{
    /* x >= 0, a >= 0, x^2 + a^2 < 64.  Step h = 1/2 keeps the series error
     * near exp(-pi^2/h^2) ~ 7e-18. */
    const double h = 0.5;
    int nmax = (int)ceil((x + 6.5) / h);
    double s1 = 0.0, sc = 0.0, ss = 0.0;
    for (int n = 1; n <= nmax; ++n) {
        double nh = n * h;
        double dn = 1.0 / (nh * nh + a * a);
        s1 += exp(-nh * nh) * dn;
        double em = exp(-(nh - x) * (nh - x));
        double ep = exp(-(nh + x) * (nh + x));
        sc += dn * (em + ep);
        ss += nh * dn * (em - ep);
    }
    double erfcx_a = exp(a * a) * erfc(a);
    double K = erfcx_a - 2.0 * a * h / O_PI * s1;
    double th = 2.0 * a * x;
    double sin_ax_over_a = (a > 0.0) ? sin(a * x) / a : x;
    double sin_2ax_over_a = (a > 0.0) ? sin(th) / a : 2.0 * x;
    double ex = exp(-x * x);
    *re = ex * (K * cos(th) + 2.0 * h / O_PI * sin(a * x) * sin_ax_over_a) + a * h / O_PI * sc;
    *im = ex * (-K * sin(th) + h / O_PI * sin_2ax_over_a) + h / O_PI * ss;
}

static void w_contfrac(double x, double a, double* re, double* im)
{
    /* w(z) = (i/sqrt(pi)) / (z - (1/2)/(z - 1/(z - (3/2)/(z - ...)))) */
    double tr = x, ti = a; /* t = z */
    for (int k = 40; k >= 1; --k) {
        double den = tr * tr + ti * ti;
        double qr = 0.5 * k * tr / den, qi = -0.5 * k * ti / den; /* (k/2)/t */
        tr = x - qr;
        ti = a - qi;
    }
    double den = tr * tr + ti * ti; /* i/(sqrt(pi) t) = i conj(t)/(sqrt(pi)|t|^2) */
    *re = ti / (O_SQRTPI * den);
    *im = tr / (O_SQRTPI * den);
}

void orc_faddeeva(double x, double a, double* re, double* im)
{
    double ax = fabs(x);
    if (ax * ax + a * a < 64.0)
        w_series(ax, a, re, im);
    else
        w_contfrac(ax, a, re, im);
    /* On the real axis Re w = exp(-x^2) exactly; the finite continued fraction
     * has no real part there.  (For 0 < a the omitted part is below 1e-27.) */
    if (a == 0.0) *re = exp(-ax * ax);
    if (x < 0.0) *im = -*im;
}

void orc_faddeeva_v(int64_t n, const double* x, const double* a, double* re, double* im)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) orc_faddeeva(x[i], a[i], &re[i], &im[i]);
}

/* ------------------------------------------------------- line physics --- */

static double strength(double lnS0, double elower, double nu_hat, double T, double qexp)
{
    double qr = pow(T / o_Tref, qexp);
    double boltz = exp(lnS0 - o_c2 * elower * (1.0 / T - 1.0 / o_Tref));
    double stim = expm1(-o_c2 * nu_hat / T) / expm1(-o_c2 * nu_hat / o_Tref);
    return boltz / qr * stim;
}

static double doppler_beta(double nu_hat, double T, double mass)
{
    return sqrt(o_kB * T / (mass * o_mu)) * nu_hat / o_c;
}

static double lorentz_gamma(double gamma_ref, double n_temp, double T, double P_bar, double sb)
{
    return sb * gamma_ref * pow(T / o_Tref, -n_temp) * (P_bar / o_Patm);
}

void orc_line_params(int64_t nl, const double* nu_hat, const double* lnS0, const double* elower,
                     const double* gamma_ref, const double* n_temp, double mass, double qexp,
                     double T, double P_bar, double sb, double* S, double* beta, double* gamma)
{
    for (int64_t l = 0; l < nl; ++l) {
        S[l] = strength(lnS0[l], elower[l], nu_hat[l], T, qexp);
        beta[l] = doppler_beta(nu_hat[l], T, mass);
        gamma[l] = lorentz_gamma(gamma_ref[l], n_temp[l], T, P_bar, sb);
    }
}

/* ---------------------------------------------------- sorted line list --- */

typedef struct {
    int64_t n;
    double *nu, *lnS0, *el, *g, *nt;
} sorted_lines;

static const double* g_sort_key;
static int cmp_idx(const void* pa, const void* pb)
{
    int64_t a = *(const int64_t*)pa, b = *(const int64_t*)pb;
    double ka = g_sort_key[a], kb = g_sort_key[b];
    if (ka < kb) return -1;
    if (ka > kb) return 1;
    return (a < b) ? -1 : (a > b); /* stable: ties keep input order */
}

static sorted_lines sort_lines(int64_t nl, const double* nu_hat, const double* lnS0, const double* elower,
                               const double* gamma_ref, const double* n_temp)
{
    sorted_lines s;
    s.n = nl;
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (nl ? nl : 1));
    for (int64_t i = 0; i < nl; ++i) idx[i] = i;
    g_sort_key = nu_hat;
    qsort(idx, (size_t)nl, sizeof(int64_t), cmp_idx);
    double* buf = (double*)malloc(sizeof(double) * 5 * (nl ? nl : 1));
    s.nu = buf;
    s.lnS0 = buf + nl;
    s.el = buf + 2 * nl;
    s.g = buf + 3 * nl;
    s.nt = buf + 4 * nl;
    for (int64_t i = 0; i < nl; ++i) {
        int64_t k = idx[i];
        s.nu[i] = nu_hat[k];
        s.lnS0[i] = lnS0[k];
        s.el[i] = elower[k];
        s.g[i] = gamma_ref[k];
        s.nt[i] = n_temp[k];
    }
    free(idx);
    return s;
}

static void free_lines(sorted_lines* s) { free(s->nu); }

/* first index with nu[i] >= v */
static int64_t lower_bound(const double* nu, int64_t n, double v)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (nu[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* Neumaier-compensated sum over the in-cut lines of one grid point. */
static double xs_point(const sorted_lines* s, const double* S, const double* beta, const double* gam,
                       double nu_j, double W)
{
    int64_t l0 = lower_bound(s->nu, s->n, nu_j - W - 1.0);
    double sum = 0.0, comp = 0.0;
    for (int64_t l = l0; l < s->n; ++l) {
        double d = nu_j - s->nu[l];
        if (d < -W - 1.0) break;
        if (fabs(d) > W) continue;
        double sb2 = O_SQRT2 * beta[l];
        double re, im;
        orc_faddeeva(d / sb2, gam[l] / sb2, &re, &im);
        double term = S[l] / (O_SQRT2PI * beta[l]) * re;
        double t = sum + term;
        if (fabs(sum) >= fabs(term)) comp += (sum - t) + term; else comp += (term - t) + sum;
        sum = t;
    }
    return sum + comp;
}

static void layer_params(const sorted_lines* s, double mass, double qexp, double T, double P, double sb,
                         double* S, double* beta, double* gam)
{
    for (int64_t l = 0; l < s->n; ++l) {
        S[l] = strength(s->lnS0[l], s->el[l], s->nu[l], T, qexp);
        beta[l] = doppler_beta(s->nu[l], T, mass);
        gam[l] = lorentz_gamma(s->g[l], s->nt[l], T, P, sb);
    }
}

/* sigma[L][N] for every layer and grid point. */
void orc_xs(int64_t nl, const double* nu_hat, const double* lnS0, const double* elower,
            const double* gamma_ref, const double* n_temp, double mass, double qexp,
            int64_t N, const double* nu, int32_t L, const double* T, const double* P_bar,
            double sb, double W, double* sigma)
{
    sorted_lines s = sort_lines(nl, nu_hat, lnS0, elower, gamma_ref, n_temp);
    double* par = (double*)malloc(sizeof(double) * 3 * (size_t)(nl ? nl : 1) * (size_t)L);
    for (int32_t n = 0; n < L; ++n)
        layer_params(&s, mass, qexp, T[n], P_bar[n], sb, par + (size_t)3 * nl * n,
                     par + (size_t)3 * nl * n + nl, par + (size_t)3 * nl * n + 2 * nl);
#pragma omp parallel for schedule(dynamic, 16) collapse(2)
    for (int32_t n = 0; n < L; ++n)
        for (int64_t j = 0; j < N; ++j) {
            const double* p = par + (size_t)3 * nl * n;
            sigma[(size_t)n * N + j] = xs_point(&s, p, p + nl, p + 2 * nl, nu[j], W);
        }
    free(par);
    free_lines(&s);
}

/* sigma at selected (layer, grid index) pairs only. */
void orc_xs_points(int64_t nl, const double* nu_hat, const double* lnS0, const double* elower,
                   const double* gamma_ref, const double* n_temp, double mass, double qexp,
                   const double* nu, int32_t L, const double* T, const double* P_bar, double sb, double W,
                   int64_t npts, const int32_t* layer_idx, const int64_t* grid_idx, double* out)
{
    sorted_lines s = sort_lines(nl, nu_hat, lnS0, elower, gamma_ref, n_temp);
    double* par = (double*)malloc(sizeof(double) * 3 * (size_t)(nl ? nl : 1) * (size_t)L);
    for (int32_t n = 0; n < L; ++n)
        layer_params(&s, mass, qexp, T[n], P_bar[n], sb, par + (size_t)3 * nl * n,
                     par + (size_t)3 * nl * n + nl, par + (size_t)3 * nl * n + 2 * nl);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < npts; ++i) {
        const double* p = par + (size_t)3 * nl * layer_idx[i];
        out[i] = xs_point(&s, p, p + nl, p + 2 * nl, nu[grid_idx[i]], W);
    }
    free(par);
    free_lines(&s);
}

/* ---------------------------------------------------- optical depth --- */

/* column factor dP/(mu m_u g) in molecules per cm^2 for a pressure step in bar */
static double column(double dP_bar, double mu, double g) { return dP_bar * 1e6 / (mu * o_mu * g); }

/* Collision-induced absorption (Sec. 2.4, Eq. taucont): for each layer and grid
 * point, dtau = n1 n2 alpha(T, nu) H dP/P with n_i = vmr_i P / (kB T) and the
 * scale height H = kB T / (mu m_u g); alpha interpolated linearly in T between the
 * table's temperatures (clamped at its ends), per grid point.  alpha [nT][N],
 * Tgrid [nT] increasing; dtau [L][N] written. */
void orc_tau_cia(const double* alpha, const double* Tgrid, int32_t nT, const double* T, const double* P_bar,
                 const double* dP_bar, int32_t L, int64_t N, double vmr1, double vmr2, double g, double mu,
                 double* dtau)
{
    for (int32_t n = 0; n < L; ++n) {
        const double Tn = T[n];
        int32_t k = 0;
        double w = 0.0;
        if (Tn <= Tgrid[0]) {
            k = 0;
            w = 0.0;
        } else if (Tn >= Tgrid[nT - 1]) {
            k = nT - 2 < 0 ? 0 : nT - 2;
            w = nT > 1 ? 1.0 : 0.0;
        } else {
            while (k + 1 < nT - 1 && Tgrid[k + 1] <= Tn) ++k;
            w = (Tn - Tgrid[k]) / (Tgrid[k + 1] - Tgrid[k]);
        }
        const double P = P_bar[n] * 1e6, dP = dP_bar[n] * 1e6;
        const double n1 = vmr1 * P / (o_kB * Tn), n2 = vmr2 * P / (o_kB * Tn);
        const double H = o_kB * Tn / (mu * o_mu * g);
        for (int64_t j = 0; j < N; ++j) {
            const double a0 = alpha[(size_t)k * N + j];
            const double a = (nT > 1) ? a0 + w * (alpha[(size_t)(k + 1) * N + j] - a0) : a0;
            dtau[(size_t)n * N + j] = n1 * n2 * a * H * dP / P;
        }
    }
}

/* sigma_all: S species, each [L][N]; vmr [S][L]. */
void orc_tau(int32_t S, const double* const* sigma, const double* vmr, const double* P_bar,
             const double* dP_bar, int32_t L, int64_t N, double g, double mu, double kappa_coef,
             double* dtau)
{
#pragma omp parallel for schedule(static)
    for (int32_t n = 0; n < L; ++n) {
        double col = column(dP_bar[n], mu, g);
        double cont = kappa_coef * P_bar[n] * dP_bar[n] * 1e6 / g;
        for (int64_t j = 0; j < N; ++j) {
            double s = 0.0;
            for (int32_t m = 0; m < S; ++m) s += vmr[(size_t)m * L + n] * sigma[m][(size_t)n * N + j];
            dtau[(size_t)n * N + j] = col * s + cont;
        }
    }
}

/* ------------------------------------------------ exponential integrals --- */

/* E1 by its power series, x in (0, 1]. */
static double e1_series(double x)
{
    const double euler = 0.57721566490153286061;
    double sum = 0.0, term = 1.0;
    for (int k = 1; k < 200; ++k) {
        term *= -x / k;
        double t = term / k;
        sum += t;
        if (fabs(t) < 1e-18 * fabs(sum)) break;
    }
    return -euler - log(x) - sum;
}

/* E_n(x), x > 1, by the continued fraction e^{-x} / (x + n - 1 n /(x + n + 2 - 2(n+1)/(x + n + 4 - ...)))
 * evaluated with the modified Lentz method. */
static double en_contfrac(int n, double x)
{
    const double tiny = 1e-300;
    double b = x + n, c = 1.0 / tiny, d = 1.0 / b, f = d;
    for (int i = 1; i < 1000; ++i) {
        double an = -(double)i * (n - 1 + i);
        b += 2.0;
        d = 1.0 / (an * d + b);
        c = b + an / c;
        double del = c * d;
        f *= del;
        if (fabs(del - 1.0) < 1e-17) break;
    }
    return f * exp(-x);
}

double orc_e1(double x) { return x <= 1.0 ? e1_series(x) : en_contfrac(1, x); }
double orc_e2(double x) { return x <= 1.0 ? exp(-x) - x * e1_series(x) : en_contfrac(2, x); }
double orc_e3(double x) { return x <= 1.0 ? 0.5 * ((1.0 - x) * exp(-x) + x * x * e1_series(x)) : en_contfrac(3, x); }

/* T(x) = 2 E3(x); T(0) = 1 */
double orc_trans(double x)
{
    if (x <= 0.0) return 1.0;
    if (x <= 1.0) return (1.0 - x) * exp(-x) + x * x * e1_series(x);
    return 2.0 * en_contfrac(3, x);
}

void orc_trans_v(int64_t n, const double* x, double* out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_trans(x[i]);
}

/* ---------------------------------------------------- emission solve --- */

/* pi B_nu(T) with nu in cm^-1: erg s^-1 cm^-2 (cm^-1)^-1 */
double orc_planck_pi(double nu, double T)
{
    return O_PI * 2.0 * o_h * o_c * o_c * nu * nu * nu / expm1(o_c2 * nu / T);
}

void orc_emission(const double* dtau, const double* T, const double* nu, int32_t L, int64_t N, double* F0)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < N; ++j) {
        double phi = 1.0, F = 0.0;
        for (int32_t n = 0; n < L; ++n) {
            double tr = orc_trans(dtau[(size_t)n * N + j]);
            F += phi * (1.0 - tr) * orc_planck_pi(nu[j], T[n]);
            phi *= tr;
        }
        F0[j] = F + phi * orc_planck_pi(nu[j], T[L - 1]);
    }
}

/* Same flux by the layer recurrence F_n = T_n F_{n+1} + (1 - T_n) S_n (Eq. rerr). */
void orc_emission_recurrence(const double* dtau, const double* T, const double* nu, int32_t L, int64_t N,
                             double* F0)
{
    for (int64_t j = 0; j < N; ++j) {
        double F = orc_planck_pi(nu[j], T[L - 1]);
        for (int32_t n = L - 1; n >= 0; --n) {
            double tr = orc_trans(dtau[(size_t)n * N + j]);
            F = tr * F + (1.0 - tr) * orc_planck_pi(nu[j], T[n]);
        }
        F0[j] = F;
    }
}

double orc_loglike(const double* F, const double* d, const double* sig, int64_t N)
{
    double s = 0.0;
    for (int64_t j = 0; j < N; ++j) {
        double r = (d[j] - F[j]) / sig[j];
        s += r * r;
    }
    return -0.5 * s;
}

/* ------------------------------------------ forward-mode dual numbers --- */

#define ND 8
typedef struct {
    double v;
    double d[ND];
} dual;

static int g_nd = ND;

static dual dc(double v)
{
    dual r;
    memset(&r, 0, sizeof r);
    r.v = v;
    return r;
}
static dual dadd(dual a, dual b) { for (int i = 0; i < g_nd; ++i) a.d[i] += b.d[i]; a.v += b.v; return a; }
static dual dsub(dual a, dual b) { for (int i = 0; i < g_nd; ++i) a.d[i] -= b.d[i]; a.v -= b.v; return a; }
static dual dmul(dual a, dual b)
{
    dual r;
    r.v = a.v * b.v;
    for (int i = 0; i < g_nd; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
static dual dscale(dual a, double s) { a.v *= s; for (int i = 0; i < g_nd; ++i) a.d[i] *= s; return a; }
static dual ddiv(dual a, dual b)
{
    dual r;
    r.v = a.v / b.v;
    for (int i = 0; i < g_nd; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
    return r;
}
/* apply a scalar function with value f and derivative fp at a.v */
static dual dchain(dual a, double f, double fp)
{
    dual r;
    r.v = f;
    for (int i = 0; i < g_nd; ++i) r.d[i] = fp * a.d[i];
    return r;
}
static dual dexp(dual a) { double e = exp(a.v); return dchain(a, e, e); }
static dual dlog(dual a) { return dchain(a, log(a.v), 1.0 / a.v); }
static dual dsqrt(dual a) { double s = sqrt(a.v); return dchain(a, s, 0.5 / s); }
static dual dexpm1(dual a) { return dchain(a, expm1(a.v), exp(a.v)); }
static dual dpow_c(dual a, double p) { return dchain(a, pow(a.v, p), p * pow(a.v, p - 1.0)); }

/* H(x, a) with dH/dx = 2aL - 2xH and dH/da = 2xL + 2aH - 2/sqrt(pi) (Sec. 2.1.1). */
static dual dvoigt_H(dual x, dual a)
{
    double re, im;
    orc_faddeeva(x.v, a.v, &re, &im);
    double hx = 2.0 * a.v * im - 2.0 * x.v * re;
    double ha = 2.0 * x.v * im + 2.0 * a.v * re - 2.0 / O_SQRTPI;
    dual r;
    r.v = re;
    for (int i = 0; i < g_nd; ++i) r.d[i] = hx * x.d[i] + ha * a.d[i];
    return r;
}

static dual dtrans(dual x)
{
    /* dT/dx = d(2 E3)/dx = -2 E2(x) */
    if (x.v <= 0.0) return dchain(x, 1.0, -2.0);
    return dchain(x, orc_trans(x.v), -2.0 * orc_e2(x.v));
}

static dual dplanck_pi(double nu, dual T)
{
    /* pi 2 h c^2 nu^3 / expm1(c2 nu / T) */
    dual e = dexpm1(ddiv(dc(o_c2 * nu), T));
    return ddiv(dc(O_PI * 2.0 * o_h * o_c * o_c * nu * nu * nu), e);
}

/*
 * Log-likelihood and its gradient with respect to
 *   theta = (T0, alpha, log10 xi_0, ..., log10 xi_{S-1}, s_b)   (3 + S <= 8 entries)
 * for T_n = T0 (P_n / 1 bar)^alpha, xi constant over layers.
 * species s: lines [nl[s]] packed one after another in the five arrays.
 */
double orc_logl_grad(int32_t S, const int64_t* nl, const double* nu_hat, const double* lnS0,
                     const double* elower, const double* gamma_ref, const double* n_temp,
                     const double* mass, const double* qexp, int64_t N, const double* nu, int32_t L,
                     const double* P_bar, const double* dP_bar, double g, double mu, double kappa_coef,
                     double W, const double* theta, const double* dobs, const double* sig_obs,
                     double* grad, double* F0_out)
{
    int np = 3 + S;
    g_nd = np;
    dual T0 = dc(theta[0]), alpha = dc(theta[1]), sb = dc(theta[2 + S]);
    T0.d[0] = 1.0;
    alpha.d[1] = 1.0;
    sb.d[2 + S] = 1.0;
    dual* Tn = (dual*)malloc(sizeof(dual) * L);
    for (int32_t n = 0; n < L; ++n) Tn[n] = dmul(T0, dexp(dscale(alpha, log(P_bar[n]))));

    dual* dtau = (dual*)malloc(sizeof(dual) * (size_t)L * N);
    for (size_t i = 0; i < (size_t)L * N; ++i) {
        dtau[i] = dc(kappa_coef * P_bar[i / N] * dP_bar[i / N] * 1e6 / g);
    }
    int64_t off = 0;
    for (int32_t s = 0; s < S; ++s) {
        sorted_lines sl = sort_lines(nl[s], nu_hat + off, lnS0 + off, elower + off, gamma_ref + off, n_temp + off);
        off += nl[s];
        dual lx = dc(theta[2 + s] * log(10.0));
        lx.d[2 + s] = log(10.0);
        dual xi = dexp(lx);
        dual* par = (dual*)malloc(sizeof(dual) * 3 * (size_t)(sl.n ? sl.n : 1));
        for (int32_t n = 0; n < L; ++n) {
            dual T = Tn[n];
            for (int64_t l = 0; l < sl.n; ++l) {
                /* Eq. Slog */
                dual boltz = dexp(dsub(dc(sl.lnS0[l]), dscale(dsub(ddiv(dc(1.0), T), dc(1.0 / o_Tref)), o_c2 * sl.el[l])));
                dual qr = dpow_c(dscale(T, 1.0 / o_Tref), qexp[s]);
                dual stim = dscale(dexpm1(ddiv(dc(-o_c2 * sl.nu[l]), T)), 1.0 / expm1(-o_c2 * sl.nu[l] / o_Tref));
                par[3 * l] = dmul(ddiv(boltz, qr), stim);
                /* Eq. thermal */
                par[3 * l + 1] = dscale(dsqrt(dscale(T, o_kB / (mass[s] * o_mu))), sl.nu[l] / o_c);
                /* pressure width */
                par[3 * l + 2] = dmul(dscale(sb, sl.g[l] * (P_bar[n] / o_Patm)),
                                      dpow_c(dscale(T, 1.0 / o_Tref), -sl.nt[l]));
            }
            double colv = column(dP_bar[n], mu, g);
#pragma omp parallel for schedule(dynamic, 16)
            for (int64_t j = 0; j < N; ++j) {
                dual sum = dc(0.0);
                double comp = 0.0;
                int64_t l0 = lower_bound(sl.nu, sl.n, nu[j] - W - 1.0);
                for (int64_t l = l0; l < sl.n; ++l) {
                    double dnu = nu[j] - sl.nu[l];
                    if (dnu < -W - 1.0) break;
                    if (fabs(dnu) > W) continue;
                    dual b = par[3 * l + 1];
                    dual sb2 = dscale(b, O_SQRT2);
                    dual x = ddiv(dc(dnu), sb2);
                    dual a = ddiv(par[3 * l + 2], sb2);
                    dual term = dmul(ddiv(par[3 * l], dscale(b, O_SQRT2PI)), dvoigt_H(x, a));
                    double t = sum.v + term.v;
                    if (fabs(sum.v) >= fabs(term.v)) comp += (sum.v - t) + term.v; else comp += (term.v - t) + sum.v;
                    for (int i = 0; i < g_nd; ++i) sum.d[i] += term.d[i];
                    sum.v = t;
                }
                sum.v += comp;
                size_t k = (size_t)n * N + j;
                dtau[k] = dadd(dtau[k], dscale(dmul(xi, sum), colv));
            }
        }
        free(par);
        free_lines(&sl);
    }
    double ll = 0.0;
    double gacc[ND];
    for (int i = 0; i < ND; ++i) gacc[i] = 0.0;
    for (int64_t j = 0; j < N; ++j) {
        dual phi = dc(1.0), F = dc(0.0);
        for (int32_t n = 0; n < L; ++n) {
            dual tr = dtrans(dtau[(size_t)n * N + j]);
            F = dadd(F, dmul(phi, dmul(dsub(dc(1.0), tr), dplanck_pi(nu[j], Tn[n]))));
            phi = dmul(phi, tr);
        }
        F = dadd(F, dmul(phi, dplanck_pi(nu[j], Tn[L - 1])));
        if (F0_out) F0_out[j] = F.v;
        double r = (dobs[j] - F.v) / sig_obs[j];
        ll += -0.5 * r * r;
        for (int i = 0; i < np; ++i) gacc[i] += r / sig_obs[j] * F.d[i];
    }
    for (int i = 0; i < np; ++i) grad[i] = gacc[i];
    free(dtau);
    free(Tn);
    g_nd = ND;
    return ll;
}
