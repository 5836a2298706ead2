/*
 * cyc_oracle.c -- plain FP64 CPU oracle for the cyclic correlation estimator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call this
 * file: only the tests, the package's smoke check and the bench's CPU-baseline leg do.
 * It shares no code, header or table with the CUDA path.
 *
 * What it computes (paper Sec. 2, discrete estimators; Sec. 4, Eq. (impl-corr) with
 * x = y and m >= 0):
 *
 *   R_f[a][m] = (1/N_eff) * sum_{n=0}^{N_eff-1} x[n+m] * c_f(x[n]) * exp(-j 2 pi frac(a*(n0+n)))
 *
 *   c_CONV(z) = conj(z)   (cyclic autocorrelation, Eq. (ACF-def))
 *   c_CONJ(z) = z         (conjugate cyclic correlation, Eq. (CCF-def))
 *   N_eff     = max(0, T - max(lags))  (one common n-range for all lags: no zero padding)
 *   n0        = absolute index of x[0] (phase origin n = 0 at the first sample pushed)
 *
 * frac(a*n) is formed without losing the low bits of a*n: p = a*n rounded, e = fma(a,n,-p)
 * is the exact rounding error (FMA TwoProduct), so a*n = p + e exactly and
 * frac(a*n) = (p - floor(p)) + e with one final rounding.  cos/sin come from libm.
 *
 * Streaming is not modelled: the streaming estimator over any chunking is, by
 * definition, this batch estimator applied to the concatenation of all pushed samples.
 *
 * cyco_estimate_xy is the same equation in full (two inputs, signed lags) and cyco_windows
 * the block's windowed output (window-local phase); both are described where they are
 * defined below.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (contraction is off so that the
 * x86 and Arm builds round identically).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { CYCO_CONV = 1, CYCO_CONJ = 2 };

/* frac(a * n) in [0, 1), exact up to one rounding (see header). */
static double frac_an(double a, int64_t n)
{
    double dn = (double)n;             /* exact for |n| < 2^53 */
    double p = a * dn;
    double e = fma(a, dn, -p);         /* a*dn - p exactly */
    double f = (p - floor(p)) + e;     /* p - floor(p) is exact */
    f -= floor(f);
    if (f >= 1.0) f -= 1.0;
    return f;
}

/* One (form, a, m) entry of the estimator; writes re, im of R. */
static void entry(const double* x, int64_t n_eff, int form, double a, int32_t m,
                  int64_t n0, double* re, double* im)
{
    double sr = 0.0, si = 0.0;
    for (int64_t n = 0; n < n_eff; ++n) {
        double xr = x[2 * (n + m)], xi = x[2 * (n + m) + 1];     /* x[n+m]    */
        double yr = x[2 * n], yi = x[2 * n + 1];                 /* x[n]      */
        if (form == CYCO_CONV) yi = -yi;                         /* conj(x[n]) */
        double pr = xr * yr - xi * yi;                           /* lag product */
        double pi = xr * yi + xi * yr;
        double f = frac_an(a, n0 + n);
        double c = cos(2.0 * M_PI * f), s = -sin(2.0 * M_PI * f);   /* exp(-j 2 pi f) */
        sr += pr * c - pi * s;
        si += pr * s + pi * c;
    }
    *re = sr / (double)n_eff;
    *im = si / (double)n_eff;
}

static int max_lag(const int32_t* lags, int nlags, int32_t* M)
{
    int32_t mx = 0;
    for (int i = 0; i < nlags; ++i) {
        if (lags[i] < 0) return -1;
        if (lags[i] > mx) mx = lags[i];
    }
    *M = mx;
    return 0;
}

/*
 * Full estimate.  x: T interleaved complex FP64 samples.  forms: bitmask CONV=1, CONJ=2.
 * out: [F][nalphas][nlags][2] with F = number of forms set, CONV first.
 * Returns 0, -1 on bad arguments, -2 when N_eff == 0 (out untouched).
 */
int cyco_estimate(const double* x, int64_t T, const int32_t* lags, int nlags,
                  const double* alphas, int nalphas, int forms, int64_t n0,
                  int nthreads, double* out, int64_t* n_eff_out)
{
    int32_t M;
    if (!x || T < 0 || !lags || nlags <= 0 || !alphas || nalphas <= 0 || !out) return -1;
    if ((forms & 3) == 0 || (forms & ~3)) return -1;
    if (max_lag(lags, nlags, &M)) return -1;
    int64_t n_eff = T - M;
    if (n_eff < 0) n_eff = 0;
    if (n_eff_out) *n_eff_out = n_eff;
    if (n_eff == 0) return -2;

    int flist[2], F = 0;
    if (forms & CYCO_CONV) flist[F++] = CYCO_CONV;
    if (forms & CYCO_CONJ) flist[F++] = CYCO_CONJ;
    int64_t total = (int64_t)F * nalphas * nlags;
    if (nthreads <= 0) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int64_t t = 0; t < total; ++t) {
        int f = (int)(t / ((int64_t)nalphas * nlags));
        int ia = (int)((t / nlags) % nalphas);
        int im = (int)(t % nlags);
        entry(x, n_eff, flist[f], alphas[ia], lags[im], n0, &out[2 * t], &out[2 * t + 1]);
    }
    return 0;
}

/*
 * Selected entries only (for parity at sizes where the full grid is too slow on a CPU).
 * form[i] in {1, 2}, alphas[i], lag[i] per entry; M is the max lag of the whole
 * configuration (it fixes N_eff).  out: [nent][2].
 */
int cyco_entries(const double* x, int64_t T, int32_t M, int nent, const int32_t* form,
                 const double* alphas, const int32_t* lag, int64_t n0, int nthreads,
                 double* out, int64_t* n_eff_out)
{
    if (!x || T < 0 || M < 0 || nent < 0 || !form || !alphas || !lag || !out) return -1;
    int64_t n_eff = T - M;
    if (n_eff < 0) n_eff = 0;
    if (n_eff_out) *n_eff_out = n_eff;
    if (n_eff == 0) return -2;
    for (int i = 0; i < nent; ++i)
        if (lag[i] < 0 || lag[i] > M || (form[i] != CYCO_CONV && form[i] != CYCO_CONJ)) return -1;
    if (nthreads <= 0) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int i = 0; i < nent; ++i)
        entry(x, n_eff, form[i], alphas[i], lag[i], n0, &out[2 * i], &out[2 * i + 1]);
    return 0;
}

/* R^0(0) = (1/N_eff) sum_{n<N_eff} |x[n]|^2, the normaliser of the error metric. */
double cyco_r00(const double* x, int64_t T, int32_t M)
{
    int64_t n_eff = T - M;
    if (!x || n_eff <= 0) return 0.0;
    double s = 0.0;
    for (int64_t n = 0; n < n_eff; ++n) s += x[2 * n] * x[2 * n] + x[2 * n + 1] * x[2 * n + 1];
    return s / (double)n_eff;
}

/*
 * The estimator of Eq. (impl-corr) in full: two inputs x, y and signed lags.
 *
 *   R_f[a][m] = (1/N_eff) * sum_{n=Mneg}^{T-Mpos-1} x[n+m] * c_f(y[n]) * exp(-j 2 pi frac(a*(n0+n)))
 *
 *   Mneg  = max(0, -min(lags))   (M^- of Eq. (impl-corr): the window starts Mneg samples in)
 *   Mpos  = max(0,  max(lags))
 *   N_eff = max(0, T - Mneg - Mpos), one common n-range for every lag
 *
 * n is the absolute index of the y sample (phase origin at the first pushed sample); the
 * paper's window-local phase differs by the constant factor exp(+j 2 pi a (n0 + Mneg)).
 * y == NULL means y = x (the cyclic ACF / CCF); with y = x and all lags >= 0 this is
 * exactly cyco_estimate.  Same layout, threads and return codes as cyco_estimate.
 */
static void entry_xy(const double* x, const double* y, int64_t n_lo, int64_t n_eff, int form, double a,
                     int32_t m, int64_t n0, double* re, double* im)
{
    double sr = 0.0, si = 0.0;
    for (int64_t n = n_lo; n < n_lo + n_eff; ++n) {
        double xr = x[2 * (n + m)], xi = x[2 * (n + m) + 1];     /* x[n+m]    */
        double yr = y[2 * n], yi = y[2 * n + 1];                 /* y[n]      */
        if (form == CYCO_CONV) yi = -yi;                         /* conj(y[n]) */
        double pr = xr * yr - xi * yi;
        double pi = xr * yi + xi * yr;
        double f = frac_an(a, n0 + n);
        double c = cos(2.0 * M_PI * f), s = -sin(2.0 * M_PI * f);
        sr += pr * c - pi * s;
        si += pr * s + pi * c;
    }
    *re = sr / (double)n_eff;
    *im = si / (double)n_eff;
}

int cyco_estimate_xy(const double* x, const double* y, int64_t T, const int32_t* lags, int nlags,
                     const double* alphas, int nalphas, int forms, int64_t n0, int nthreads,
                     double* out, int64_t* n_eff_out)
{
    if (!x || T < 0 || !lags || nlags <= 0 || !alphas || nalphas <= 0 || !out) return -1;
    if ((forms & 3) == 0 || (forms & ~3)) return -1;
    if (!y) y = x;
    int32_t lo = 0, hi = 0;
    for (int i = 0; i < nlags; ++i) {
        if (lags[i] < lo) lo = lags[i];
        if (lags[i] > hi) hi = lags[i];
    }
    const int64_t Mneg = -(int64_t)lo, Mpos = hi;
    int64_t n_eff = T - Mneg - Mpos;
    if (n_eff < 0) n_eff = 0;
    if (n_eff_out) *n_eff_out = n_eff;
    if (n_eff == 0) return -2;

    int flist[2], F = 0;
    if (forms & CYCO_CONV) flist[F++] = CYCO_CONV;
    if (forms & CYCO_CONJ) flist[F++] = CYCO_CONJ;
    int64_t total = (int64_t)F * nalphas * nlags;
    if (nthreads <= 0) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int64_t t = 0; t < total; ++t) {
        int f = (int)(t / ((int64_t)nalphas * nlags));
        int ia = (int)((t / nlags) % nalphas);
        int im = (int)(t % nlags);
        entry_xy(x, y, Mneg, n_eff, flist[f], alphas[ia], lags[im], n0, &out[2 * t], &out[2 * t + 1]);
    }
    return 0;
}

/*
 * The block's windowed output (Sec. 4, Eq. (impl-corr) at window start n0 = k * hop):
 *
 *   R_k,f[a][m] = (1/N) sum_{n=0}^{N-1} x[k*hop + Mneg + n + m] * c_f(y[k*hop + Mneg + n])
 *                 * exp(-j 2 pi frac(a * n))
 *
 * with the window-local phase of the equation (n = 0 at the window's first reference
 * sample), N = win_len, for every k with k*hop + Mneg + Mpos + N <= T.  y == NULL: y = x.
 * out: [nwin][F][nalphas][nlags][2]; *nwin_out receives the number of windows (the caller
 * sizes out for max_win windows; more are not written).  Returns 0, -1 on bad arguments.
 */
int cyco_windows(const double* x, const double* y, int64_t T, const int32_t* lags, int nlags,
                 const double* alphas, int nalphas, int forms, int64_t win_len, int64_t hop,
                 int64_t max_win, int nthreads, double* out, int64_t* nwin_out)
{
    if (!x || T < 0 || !lags || nlags <= 0 || !alphas || nalphas <= 0 || !out || win_len <= 0 || hop <= 0)
        return -1;
    if ((forms & 3) == 0 || (forms & ~3)) return -1;
    if (!y) y = x;
    int32_t lo = 0, hi = 0;
    for (int i = 0; i < nlags; ++i) {
        if (lags[i] < lo) lo = lags[i];
        if (lags[i] > hi) hi = lags[i];
    }
    const int64_t Mneg = -(int64_t)lo, Mpos = hi;
    const int64_t span = Mneg + Mpos + win_len;
    int64_t nwin = T >= span ? (T - span) / hop + 1 : 0;
    if (nwin_out) *nwin_out = nwin;
    if (nwin > max_win) nwin = max_win;
    int flist[2], F = 0;
    if (forms & CYCO_CONV) flist[F++] = CYCO_CONV;
    if (forms & CYCO_CONJ) flist[F++] = CYCO_CONJ;
    const int64_t per = (int64_t)F * nalphas * nlags;
    if (nthreads <= 0) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int64_t t = 0; t < nwin * per; ++t) {
        const int64_t k = t / per, r = t % per;
        const int f = (int)(r / ((int64_t)nalphas * nlags));
        const int ia = (int)((r / nlags) % nalphas);
        const int im = (int)(r % nlags);
        /* entry_xy with the reference run starting at k*hop + Mneg and phase index n - that */
        const int64_t s0 = k * hop + Mneg;
        double sr = 0.0, si = 0.0;
        for (int64_t n = 0; n < win_len; ++n) {
            const int64_t i = s0 + n;
            double xr = x[2 * (i + lags[im])], xi = x[2 * (i + lags[im]) + 1];
            double yr = y[2 * i], yi = y[2 * i + 1];
            if (flist[f] == CYCO_CONV) yi = -yi;
            double pr = xr * yr - xi * yi;
            double pi = xr * yi + xi * yr;
            double ph = frac_an(alphas[ia], n);
            double c = cos(2.0 * M_PI * ph), sn = -sin(2.0 * M_PI * ph);
            sr += pr * c - pi * sn;
            si += pr * sn + pi * c;
        }
        out[2 * t] = sr / (double)win_len;
        out[2 * t + 1] = si / (double)win_len;
    }
    return 0;
}

/* Normaliser of the cross error metric: sqrt(mean |x[n]|^2 * mean |y[n]|^2) over the
 * committed n-range [Mneg, T - Mpos) (Cauchy-Schwarz bound of every entry's terms);
 * for y == NULL this is R^0(0) over that range. */
double cyco_r00_xy(const double* x, const double* y, int64_t T, int32_t Mneg, int32_t Mpos)
{
    int64_t n_eff = T - Mneg - Mpos;
    if (!x || n_eff <= 0 || Mneg < 0 || Mpos < 0) return 0.0;
    if (!y) y = x;
    double sx = 0.0, sy = 0.0;
    for (int64_t n = Mneg; n < Mneg + n_eff; ++n) {
        sx += x[2 * n] * x[2 * n] + x[2 * n + 1] * x[2 * n + 1];
        sy += y[2 * n] * y[2 * n] + y[2 * n + 1] * y[2 * n + 1];
    }
    return sqrt(sx / (double)n_eff) * sqrt(sy / (double)n_eff);
}

int cyco_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
