/*
 * libxs — C ABI of the GB300 (sm_103a) line-by-line opacity, optical-depth and
 * emission library for the auto-differentiable spectrum model of Kawahara et al.
 * (arXiv:2105.14782).
 *
 * Conventions shared by every entry point:
 *   - Every array argument is a DEVICE pointer unless it is marked "host".
 *     The caller owns all memory; the library never allocates device memory.
 *     Scratch comes from a caller-provided workspace whose size the matching
 *     *_workspace_bytes() function returns (a 256-byte aligned device buffer).
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *     stream).  Results are valid once the stream reaches that point.
 *   - Layouts are row-major: [L][N] means layer-major, grid index fastest.
 *     Layer 0 is the top of the atmosphere (lowest pressure).
 *   - Units: wavenumber cm^-1, pressure bar, temperature K, cross-section
 *     cm^2/molecule, flux erg s^-1 cm^-2 (cm^-1)^-1 (cgs).
 *   - Return value: XS_OK or a negative xs_status.  Argument errors are detected
 *     on the host before any launch and leave outputs untouched; XS_ECUDA reports
 *     a launch or runtime error (cudaGetLastError).  Nothing is printed and no
 *     entry point aborts the process.
 */
#ifndef XS_H
#define XS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* xs_stream; /* same object as cudaStream_t */

typedef enum {
    XS_OK = 0,
    XS_EINVAL = -1,    /* null pointer, non-positive size, bad precision, too small workspace */
    XS_EUNSORTED = -2, /* line centres not ascending, or grid not strictly increasing */
    XS_ENOMEM = -3,    /* reserved for host-side allocation failure */
    XS_ECUDA = -4,     /* a CUDA launch or runtime call failed */
    XS_ETIMEOUT = -5,  /* a bounded host-side wait ran out */
    XS_ETOOBIG = -6    /* the problem needs more scratch than a fixed or given area holds
                          (xs_compute_noalloc's array; MODIT's reserve for cuFFT's work area) */
} xs_status;

typedef enum {
    XS_PREC_FP64 = 0, /* every step in double precision */
    XS_PREC_MIXED = 1 /* Voigt evaluation and line sum in FP32 (compensated), line-centre
                         offsets and strength exponentials in FP64; sigma stored as float */
} xs_prec;

#define XS_MAX_SPECIES 8

/*
 * One species' line list, structure of arrays, device memory, sorted by nu_hat
 * ascending (xs_sort_lines_host sorts host copies; xs_check_sorted verifies).
 * Fields follow the HITRAN-style parameter table of Sec. 2.2 (Table 1).
 */
typedef struct {
    int64_t n;               /* number of lines (0 allowed) */
    const double* nu_hat;    /* [n] line centre, cm^-1 */
    const double* ln_S0;     /* [n] ln of the line strength at T_ref = 296 K, ln(cm/molecule) */
    const double* elower;    /* [n] lower-state energy E'', cm^-1 */
    const double* gamma_ref; /* [n] Lorentz HWHM at 296 K and 1 atm, cm^-1 atm^-1 */
    const double* n_temp;    /* [n] temperature exponent of the width */
    double mass_amu;         /* molecular mass M in atomic mass units */
    double q_exponent;       /* partition-function ratio Q(T)/Q(296) = (T/296)^q_exponent */
} xs_lines;

/* Human-readable name of a status code (static string). */
const char* xs_strerror(int status);

/*
 * Stable in-place sort of a HOST line list by centre (ties keep input order).
 * All five arrays are permuted together.  Line-list ingest step; Table 1 fields.
 * Returns XS_EINVAL on null arrays with n > 0.
 */
int xs_sort_lines_host(int64_t n, double* nu_hat, double* ln_S0, double* elower, double* gamma_ref,
                       double* n_temp);

/*
 * Synchronously checks the order of a device array v[n]: non-decreasing when
 * strict == 0 (line centres), strictly increasing when strict != 0 (a grid).
 * flag_dev is one caller-owned device int used as scratch.  Returns XS_OK,
 * XS_EUNSORTED or XS_ECUDA; blocks the calling thread until `stream` drains.
 */
int xs_check_sorted(const double* v, int64_t n, int strict, int* flag_dev, xs_stream stream);

/*
 * Bounds-checked build.  Compiled with -DXS_CHECKED (the library file
 * libxs_checked.so), the kernels test the indices they derive from data (line
 * windows, near ranges, cut ranges, grid indices, series table offsets) before
 * each access; a failed test skips the access and records the source line in a
 * device status word of its source file -- no trap, no fault.
 * xs_checked_build: 1 in that build, 0 in the normal one (where the tests are
 * compiled out).
 * xs_check_status: synchronises the device, then returns 0 if no check failed
 * since the last clear, else file * 100000 + line of a failed check (file 1 line
 * sums, 2 radiative transfer, 3 MODIT, 4 responses, 5 pre-filter, 6 prior), or
 * XS_ECUDA; with clear != 0 the words are reset.  Always 0 in the normal build.
 */
int xs_checked_build(void);
int xs_check_status(int clear);

/* Workspace bytes xs_compute / xs_compute_adjoint need for these sizes.  A
 * workspace down to xs_workspace_min_bytes still works (layers are then done in
 * chunks); sizes in between pick the largest chunk that fits. */
size_t xs_workspace_bytes(int64_t n_lines, int64_t N, int32_t L, int prec);
size_t xs_workspace_min_bytes(int64_t n_lines, int64_t N, int32_t L, int prec);

/*
 * Cross-section of one species on a grid for every layer (Eq. crosssec, the
 * direct line-profile sum of Sec. 2.1.1 and Sec. 3.1):
 *   sigma[n][j] = sum over lines l with |nu[j] - nu_hat[l]| <= wing_cut of
 *                 S_l(T_n) / (sqrt(2 pi) beta_l) * H(x, a),
 *   x = (nu[j] - nu_hat[l]) / (sqrt(2) beta_l),  a = gamma_l / (sqrt(2) beta_l),
 * with S(T) of Eq. Slog, beta of Eq. thermal, and
 *   gamma_l = broad_scale * gamma_ref_l * (T_n/296)^(-n_temp_l) * (P_bar[n] / 1.01325)
 * (Eq. gammahitran without the self and natural terms).  The wing-cut test is
 * made in double precision and includes the boundary.
 *   nu      [N] strictly increasing grid (any spacing), cm^-1
 *   T,P_bar [L] layer temperature (K) and pressure (bar), device
 *   sigma   [L][N] output: double for XS_PREC_FP64, float for XS_PREC_MIXED
 * Lines must be sorted by centre.  n == 0 gives sigma = 0.
 */
int xs_compute(const xs_lines* lines, const double* nu, int64_t N, const double* T, const double* P_bar,
               int32_t L, double broad_scale, double wing_cut, int prec, void* sigma, void* workspace,
               size_t workspace_bytes, xs_stream stream);

/*
 * xs_compute without any allocation and without a caller workspace.
 * (No counterpart in the paper: this is a deployment convenience.)
 *
 * For callers that cannot allocate device memory where they need a
 * cross-section -- a host callback or real-time loop that must not block in the
 * driver's allocator, a plugin whose host process owns and caps the memory pool,
 * a tool that may only touch buffers it was handed.  Inputs, outputs and their
 * meaning are exactly those of xs_compute; the scratch comes from a fixed 64 MiB
 * device array inside libxs that every GPU loading the library holds until the
 * process exits.  Problems whose smallest plan (one layer at a time) needs more
 * than 64 MiB, i.e. xs_workspace_min_bytes(n, N, L, prec) > 64 MiB, are
 * rejected with XS_ETOOBIG before any launch.  That plan holds about n * 68
 * bytes (XS_PREC_MIXED) or n * 96 bytes (XS_PREC_FP64) of per-line records, the
 * near-pair sums (N * 8 bytes, mixed) and split-K partials (up to 64 * N * 8
 * bytes); xs_workspace_min_bytes gives the exact figure.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls on a device share the one array and
 * every call overwrites it: calls whose execution overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Nothing in the array has to start at zero: each call writes every region
 * before reading it.  Never calls cudaMalloc, cudaFree or any allocating routine.
 */
int xs_compute_noalloc(const xs_lines* lines, const double* nu, int64_t N, const double* T, const double* P_bar,
                       int32_t L, double broad_scale, double wing_cut, int prec, void* sigma, xs_stream stream);

/*
 * Reverse-mode adjoint of xs_compute.  Given g_sigma[n][j] = dF/dsigma[n][j]
 * (double, [L][N]) it writes
 *   g_T[n]     = sum_j g_sigma[n][j] d sigma[n][j] / d T_n        (through S, beta, gamma)
 *   g_broad[0] = sum_{n,j} g_sigma[n][j] d sigma[n][j] / d broad_scale
 * Voigt values are recomputed, not stored; dH/dx and dH/da follow the
 * relations of Sec. 2.1.1 (dH/dx = 2aL - 2xH, dH/da = 2xL + 2aH - 2/sqrt(pi)).
 * The reduction order is fixed, so repeated calls give identical bits.
 * g_T [L] and g_broad [1] are overwritten (double, device).
 */
int xs_compute_adjoint(const xs_lines* lines, const double* nu, int64_t N, const double* T,
                       const double* P_bar, int32_t L, double broad_scale, double wing_cut, int prec,
                       const double* g_sigma, double* g_T, double* g_broad, void* workspace,
                       size_t workspace_bytes, xs_stream stream);

/*
 * Layer optical depth (Eq. dtau_line) plus a grey continuum:
 *   dtau[n][j] = dP_n 1e6 / (mu m_u g) * sum_m vmr[m][n] sigma_m[n][j]
 *              + kappa_coef * P_n * dP_n * 1e6 / g
 * sigma: HOST array of S device pointers, each [L][N] (double for FP64, float
 * for MIXED).  vmr [S][L] device.  P_bar, dP_bar [L] device (bar).  g in
 * cm s^-2, mu the mean molecular weight.  dtau [L][N] double output.
 */
int tau_layers(const void* const* sigma, int32_t S, const double* vmr, const double* P_bar,
               const double* dP_bar, int32_t L, int64_t N, double gravity, double mu, double kappa_coef,
               int prec, double* dtau, xs_stream stream);

/*
 * Adjoint of tau_layers: from g_dtau [L][N] writes g_sigma[m] = g_dtau * dP 1e6/(mu m_u g) * vmr[m][n]
 * ([L][N] double each; `g_sigma` is a HOST array of S device pointers; a NULL
 * entry skips that species) and g_vmr[m][n] = sum_j g_dtau[n][j] * dtau_m[n][j] / vmr[m][n]
 * ([S][L] double), summed in a fixed order.
 */
int tau_layers_adjoint(const void* const* sigma, int32_t S, const double* vmr, const double* P_bar,
                       const double* dP_bar, int32_t L, int64_t N, double gravity, double mu, int prec,
                       const double* g_dtau, double* const* g_sigma, double* g_vmr, xs_stream stream);

/*
 * Top-of-atmosphere flux of the pure-absorption two-stream solve (Sec. 3):
 *   F0[j] = sum_n Phi_n (1 - T_n) S_n + Phi_L F_B,  Phi_n = prod_{k<n} T_k,
 *   T_n = 2 E3(dtau[n][j]) (Eq. trans), S_n = pi B(nu_j, T_n) (Eq. sourcepla),
 *   F_B = pi B(nu_j, T_{L-1}) (opaque bottom at the deepest layer's temperature).
 * dtau [L][N], T [L], nu [N] double in; F0 [N] double out.
 */
int emission_spectrum(const double* dtau, const double* T, const double* nu, int32_t L, int64_t N, double* F0,
                      xs_stream stream);

/*
 * Collision-induced absorption of one molecule pair (Sec. 2.4, Eq. taucont):
 *   dtau[n][j] (+)= n1 n2 alpha(T_n, nu_j) H dP_n/P_n,  n_i = vmr_i P/(kB T),
 *   H = kB T/(mu m_u g) (Eq. scaleheight),
 * alpha from the table alpha [nT][N] (cm^5, on the model grid) at the temperatures
 * T_grid [nT] (increasing), linear in T and clamped at the ends (the paper
 * interpolates in T only).  T, P_bar, dP_bar [L]; all device.  accumulate = 1 adds
 * to dtau, 0 overwrites.  The adjoint adds to g_T [L] the derivative of
 * sum g_dtau dtau in each T_n (fixed-order sums).
 */
int tau_cia(const double* alpha, const double* T_grid, int32_t nT, const double* T, const double* P_bar,
            const double* dP_bar, int32_t L, int64_t N, double vmr1, double vmr2, double gravity, double mu,
            int accumulate, double* dtau, xs_stream stream);
int tau_cia_adjoint(const double* g_dtau, const double* alpha, const double* T_grid, int32_t nT, const double* T,
                    const double* P_bar, const double* dP_bar, int32_t L, int64_t N, double vmr1, double vmr2,
                    double gravity, double mu, double* g_T, xs_stream stream);

/* Workspace bytes emission_spectrum_adjoint needs. */
size_t emission_workspace_bytes(int32_t L, int64_t N);

/*
 * Adjoint of emission_spectrum.  From g_F0 [N] writes g_dtau [L][N] (overwritten)
 * and g_T [L] (overwritten: the Planck-source part of dF/dT_n only), using the
 * layer recurrence F_n = T_n F_{n+1} + (1 - T_n) S_n (Eq. rerr) swept bottom-up
 * and top-down; dT/d dtau = -2 E2(dtau).  Fixed reduction order.
 */
int emission_spectrum_adjoint(const double* g_F0, const double* dtau, const double* T, const double* nu,
                              int32_t L, int64_t N, double* g_dtau, double* g_T, void* workspace,
                              size_t workspace_bytes, xs_stream stream);

/*
 * Gaussian log-likelihood with fixed per-point errors (Eq. likelihood without
 * the jitter term): logL = -1/2 sum_j ((d_j - F_j)/s_j)^2 written to logL[0];
 * g_F[j] = (d_j - F_j)/s_j^2 if g_F is not NULL.  All device, double.
 */
int loglike_gauss(const double* F, const double* d, const double* s, int64_t N, double* logL, double* g_F,
                  xs_stream stream);

/*
 * Power-law temperature profile of Sec. 5.2: T[n] = T0 * P_bar[n]^alpha (P in bar).
 */
int layer_temperatures(double T0, double alpha, const double* P_bar, int32_t L, double* T, xs_stream stream);

/*
 * A whole emission model: species line lists, grid, layers, observed spectrum.
 * All pointers device.  Used by the composite calls below.
 */
typedef struct {
    int32_t n_species;
    xs_lines species[XS_MAX_SPECIES];
    const double* nu; /* [N] */
    int64_t N;
    const double* P_bar;  /* [L] */
    const double* dP_bar; /* [L] */
    int32_t L;
    double wing_cut;
    double gravity;
    double mu;
    double kappa_coef;
    const double* d_obs;   /* [N] observed spectrum (may be NULL for forward-only use) */
    const double* sig_obs; /* [N] its 1-sigma errors */
    int prec;
    /* Cross-section method.  XS_METHOD_LPF (0, the default of a zeroed struct):
     * the line-by-line sum (xs_compute).  XS_METHOD_MODIT (1): modit_compute, which
     * needs nu to be the log grid from nu_min to nu_max (N points) and per species
     * the padded length n_fft[s]; wing_cut is not used. */
    int method;
    int32_t n_gamma;
    double nu_min, nu_max;
    int64_t n_fft[XS_MAX_SPECIES];
    /* Optional collision-induced absorption (tau_cia) added to the optical depth:
     * table cia_alpha [cia_nT][N] and cia_T [cia_nT] (device), pair mixing ratios;
     * unused when cia_alpha is NULL. */
    const double* cia_alpha;
    const double* cia_T;
    int32_t cia_nT;
    double cia_vmr1, cia_vmr2;
} xs_model;

enum { XS_METHOD_LPF = 0, XS_METHOD_MODIT = 1 };

size_t xs_model_workspace_bytes(const xs_model* model);

/*
 * Forward model for theta = (T0, alpha, log10 vmr_0 .. log10 vmr_{S-1}, broad_scale)
 * (HOST array of 3 + S doubles): layer temperatures (Sec. 5.2 power law), every
 * species' cross-section, optical depth and emission.  F0 [N] device output.
 */
int xs_model_forward(const xs_model* model, const double* theta, double* F0, void* workspace,
                     size_t workspace_bytes, xs_stream stream);

/*
 * Forward model plus the log-likelihood and its gradient by the hand-written
 * adjoints (reverse mode).  out [1 + 3 + S] device doubles: logL, then dlogL/dtheta
 * in theta's order.  F0 [N] is written when not NULL.
 */
int xs_model_logl_grad(const xs_model* model, const double* theta, double* out, double* F0, void* workspace,
                       size_t workspace_bytes, xs_stream stream);

/*
 * MODIT (Sec. 2.1.2, Eqs. FTFT, ftmodit, MODIT): the cross-section of one species
 * on the log grid nu_i = nu_min (nu_max/nu_min)^(i/(N-1)), i = 0..N-1, from a
 * lineshape distribution and FFT convolution instead of a line-by-line sum.
 * With R0 = (N-1)/ln(nu_max/nu_min) and q = R0 ln(nu/nu_min) (unit steps):
 *   - each line adds S(T) (Eq. Slog) to the two q nodes around its centre and the
 *     two of n_gamma log-spaced nodes (per layer, from the smallest to the largest
 *     gamma' = R0 gamma/nu_hat) around its width, with weights linear in q and in
 *     ln gamma';
 *   - sigma(q) = sum_k IFFT[ FFT(S_k) exp(-2 pi^2 beta'^2 f^2) (exp(-2 pi gamma'_k f)
 *     - gamma'_k FFT(A)) ], beta' = R0 beta/nu_hat, and sigma(nu) = sigma(q) R0/nu.
 *     A is the sum of a unit-width Lorentzian's periodic images on the padded q
 *     axis; subtracting it removes the Lorentz aliasing to first order in
 *     gamma'/n_fft (the paper names an aliasing correction without stating it).
 * No wing cut: each profile reaches half the period n_fft on either side.
 * Resolution: the Gaussian factor is applied only up to the Nyquist frequency of
 * the q grid, so the grid must resolve the Doppler width (Sec. 4: R0 >~ 5e5).
 * With beta' below about one q step (cool upper layers on grids coarser than the
 * Doppler width) the cut transform rings and sigma goes negative near lines, by
 * up to a few 1e-2 of the layer maximum; with beta' >= 1.5 in every layer it
 * stays non-negative on the workloads tested.  The call does not check this.
 * n_fft
 * (a power of two, >= N + 2) is the padded period; for profiles that cover the
 * whole grid use n_fft >= 2 (N + m), m the farthest centre outside the grid in q
 * steps.  Lines whose centre lies more than (n_fft - N)/2 q steps outside the grid
 * are left out.  n_gamma 1..32.  Lines sorted by centre (as for xs_compute), device
 * arrays; T, P_bar [L] device; sigma [L][N] device, double (XS_PREC_FP64:
 * FP64 distribution and FFT) or float (XS_PREC_MIXED: FP32 distribution and
 * FFT, strengths scaled by 2^80 inside).  The distribution is summed in a fixed
 * order; the FFTs are cuFFT's (one plan per length and batch, created on first
 * use without a work area of its own).  Errors: XS_EINVAL for bad arguments or a
 * workspace below modit_workspace_bytes; XS_ETOOBIG if cuFFT asks for more work
 * area than the workspace reserves; XS_ECUDA on launch or cuFFT failure.
 */
size_t modit_workspace_bytes(int64_t n_lines, int32_t L, int32_t n_gamma, int64_t n_fft, int prec);
int modit_compute(const xs_lines* lines, double nu_min, double nu_max, int64_t N, const double* T,
                  const double* P_bar, int32_t L, double broad_scale, int32_t n_gamma, int64_t n_fft, int prec,
                  void* sigma, void* workspace, size_t workspace_bytes, xs_stream stream);

/*
 * Reverse-mode adjoint of modit_compute (same grid, lines and arguments).  From
 * g_sigma [L][N] (double, device) it writes g_T [L] = sum_j g_sigma[n][j]
 * dsigma[n][j]/dT_n, through S(T), beta' and every line's and node's gamma', and
 * g_broad [1] = the derivative in broad_scale (which moves all widths and both
 * ends of the gamma' grid alike, so it acts through the kernels only).  The
 * weights are piecewise linear in ln gamma', so the derivative is that of the
 * piece in use.  The forward distribution is recomputed; sums in a fixed order.
 */
size_t modit_adjoint_workspace_bytes(int64_t n_lines, int32_t L, int32_t n_gamma, int64_t n_fft, int prec);
int modit_compute_adjoint(const xs_lines* lines, double nu_min, double nu_max, int64_t N, const double* T,
                          const double* P_bar, int32_t L, double broad_scale, int32_t n_gamma, int64_t n_fft,
                          int prec, const double* g_sigma, double* g_T, double* g_broad, void* workspace,
                          size_t workspace_bytes, xs_stream stream);

/*
 * Astronomical and instrumental responses (Sec. 4, Eq. responsenu):
 *   F(nu'_i) = sum_j k(c ln(nu'_i/nu_j) + RV) F0_j / sum_j k(c ln(nu'_i/nu_j)),
 * velocities in km/s, c = 299792.458 km/s, grids increasing (device arrays).
 * response_rotation: rigid rotation (Sec. 4.1) on the same grid, k(v) = zeta(v/vsini)
 *   with quadratic limb darkening (u1, u2); zeta is taken from its disk-integral
 *   definition, (2s(1-u1-u2) + (pi/2)(u1+2u2)s^2 - (4/3)u2 s^3)/(pi(1-u1/3-u2/6)),
 *   s = sqrt(1-x^2) (the printed closed form does not integrate to one).
 *   F0, F1 [N].
 * response_ip_rv: Gaussian instrumental profile of standard deviation beta (Sec. 4.2;
 *   beta = c/(2 sqrt(2 ln 2) R) for resolving power R) and radial velocity rv, from
 *   the grid nu [N] onto nu_out [N_out]; the Gaussian is summed over |v| <= 10 beta.
 *   nu_out must lie inside nu (every output needs kernel weight).
 * The adjoints write g_F0 [N] (resp. g_F1 [N]) = transpose of the response applied
 * to g_F1 [N] (resp. g_F [N_out]), and g_vsini [1] (resp. g_rv [1]) = the
 * derivative of sum_i g_i F_i in vsini (resp. rv), device doubles, fixed-order
 * sums.  They need response_workspace_bytes(number of outputs) of workspace.
 * XS_EINVAL for bad arguments, XS_ECUDA on launch failure.
 */
int response_rotation(const double* F0, const double* nu, int64_t N, double vsini, double u1, double u2, double* F1,
                      xs_stream stream);
int response_ip_rv(const double* F1, const double* nu, int64_t N, const double* nu_out, int64_t N_out, double beta,
                   double rv, double* F, xs_stream stream);
size_t response_workspace_bytes(int64_t N_out);
int response_rotation_adjoint(const double* g_F1, const double* F0, const double* nu, int64_t N, double vsini,
                              double u1, double u2, double* g_F0, double* g_vsini, void* workspace,
                              size_t workspace_bytes, xs_stream stream);
int response_ip_rv_adjoint(const double* g_F, const double* F1, const double* nu, int64_t N, const double* nu_out,
                           int64_t N_out, double beta, double rv, double* g_F1, double* g_rv, void* workspace,
                           size_t workspace_bytes, xs_stream stream);

/*
 * Layer-by-layer temperatures (the retrieval of Sec. 6 with one temperature per
 * layer): as xs_model_logl_grad with the power law replaced by T [L] (device,
 * Kelvin), log10_vmr [S] (host) and broad_scale; out [1 + L + S + 1] device:
 * logL, dlogL/dT_n for every layer, dlogL/dlog10 vmr_m, dlogL/d broad_scale.
 * The Gaussian-process prior on the T_n is the companion call gp_prior_layers.
 */
int xs_model_logl_grad_layers(const xs_model* model, const double* T, const double* log10_vmr, double broad_scale,
                              double* out, double* F0, void* workspace, size_t workspace_bytes, xs_stream stream);

/*
 * Gaussian-process prior of the layer-by-layer temperatures (Sec. 6.1):
 *   T ~ N(T0 u, K),  K_ij = a_T exp(-(log10 P_i - log10 P_j)^2 / (2 tau_P^2)) + eps a_T delta_ij
 * (the RBF kernel of Sec. 5.2.3; the paper fixes a_T = 1e6, tau_P = 10^0.5, eps = 1e-5).
 *   T, P_bar [L] device (Kelvin, bar), 1 <= L <= XS_GP_MAX_LAYERS
 *   out [L + 2] device doubles: log p(T) (normalised density, with -(L/2) log 2 pi),
 *       d log p / dT_n for every layer, d log p / dT0
 * FP64 Cholesky factorisation of K in the workspace (gp_prior_workspace_bytes(L):
 * L^2 + L doubles, caller-owned), one CTA (O(L^3 / 6) work; milliseconds at the
 * paper's 100 layers), stream-ordered.  A K that is not
 * positive definite in FP64 gives NaN in out[0] and out[L + 1].  XS_EINVAL for
 * null pointers, L out of range, a_T <= 0, tau_P <= 0, eps < 0, a non-finite T0
 * or a short workspace; XS_ECUDA on launch failure.  The posterior of the
 * layer-by-layer retrieval is xs_model_logl_grad_layers' logL plus this log p,
 * and its gradient in T_n the sum of the two.
 */
#define XS_GP_MAX_LAYERS 1024
size_t gp_prior_workspace_bytes(int32_t L);
int gp_prior_layers(const double* T, const double* P_bar, int32_t L, double T0, double a_T, double tau_P, double eps,
                    double* out, void* workspace, size_t workspace_bytes, xs_stream stream);

/*
 * The composite model as a vector-Jacobian product, for likelihoods that are not
 * computed on the model grid (e.g. after the responses of Sec. 4 on an observed
 * grid).  xs_model_forward_keep writes F0 [N] like xs_model_forward and keeps
 * what the reverse sweep needs in the workspace; xs_model_vjp then writes
 * out[1 .. 3 + S] = sum_j g_F0[j] dF0[j]/dtheta (theta's order) and out[0] = 0.
 * xs_model_vjp must follow xs_model_forward_keep with the same model, theta and
 * workspace, with the workspace untouched in between (stream-ordered).  d_obs
 * and sig_obs of the model are not used.  Sizes, errors as xs_model_logl_grad.
 */
int xs_model_forward_keep(const xs_model* model, const double* theta, double* F0, void* workspace,
                          size_t workspace_bytes, xs_stream stream);
int xs_model_vjp(const xs_model* model, const double* theta, const double* g_F0, double* out, void* workspace,
                 size_t workspace_bytes, xs_stream stream);

/*
 * Weak-line pre-filter (App. G).  For every line, at the temperature of T_scan
 * (host [n_scan], n_scan <= 64) where its strength S(T) is largest, in an
 * isothermal atmosphere with mixing ratio vmr: the line-centre layer optical
 * depths dtau_n (the optical-depth formula of tau_layers applied to the
 * line-centre cross-section S erfcx(gamma_n/(sqrt2 beta))/(sqrt(2 pi) beta)),
 * the contribution function psi_n = exp(-tau_n) dtau_n P_n/dP_n with
 * tau_n = sum_{k<=n} dtau_k, and its argmax n_hat (first on ties).  The grey
 * continuum kappa_coef P [cm^2/g] gets its own n_hat; keep[l] = 1 when the
 * line's n_hat <= the continuum's + margin (layer 0 at the top), else 0.
 * keep [n] uint8 and n_hat [n] int32 (may be NULL) device outputs.
 */
int lines_contribution_filter(const xs_lines* lines, const double* P_bar, const double* dP_bar, int32_t L,
                              const double* T_scan, int32_t n_scan, double vmr, double gravity, double mu,
                              double kappa_coef, double broad_scale, int32_t margin, uint8_t* keep, int32_t* n_hat,
                              xs_stream stream);

/*
 * Diagnostics (no paper counterpart).  xs_profile(1) makes the library record a
 * CUDA event pair around every line-sum kernel launch (forward and adjoint,
 * on the launching stream) until xs_profile(0); xs_profile_read synchronises
 * those events and returns the summed kernel times in ms and the launch counts
 * since profiling was enabled.  xs_launch_count returns how many kernels the
 * library has launched since it was loaded (host-side counter, all threads).
 */
int xs_profile(int enable);
int xs_profile_read(double* fwd_ms, int64_t* fwd_launches, double* adj_ms, int64_t* adj_launches);
uint64_t xs_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* XS_H */
