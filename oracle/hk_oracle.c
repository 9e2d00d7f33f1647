/*
 * hk_oracle.c -- plain FP64 CPU oracle for the HELIOS-K 2.0 opacity hot path
 * (Grimm et al. 2021, arXiv:2101.02005).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant with
 * the CUDA path; its constants are typed in here separately and a test checks
 * that the two sets agree.
 *
 * What it computes is the plain definition of the cross section (Sect. 2.2,
 * Eqs. a, u, gammaD, gammaL and S; code parameters of Sect. 2.4.2):
 *
 *     sigma_i = sum_l S_l(T) * Re w(x_il + i y_l) / (alpha_D,l * sqrt(pi))
 *               over every line l with |nu_i - nu0_l| <= cut,
 *     x_il = (nu_i - nu0_l) / alpha_D,l,  y_l = Gamma_L,l / alpha_D,l,
 *     alpha_D = (nu0 / c) sqrt(2 k_B T / m)   (the 1/e Doppler half width),
 *
 * summed in FP64, for every bin in ascending line order, with no tiling,
 * region split or reordering.
 *
 * The Faddeeva function w(z) = exp(-z^2) erfc(-iz) is evaluated with two
 * published methods, chosen by |z|:
 *   |z|^2 <  64 : the trapezoidal rule on w(z) = (i/pi) int exp(-t^2)/(z-t) dt
 *                 with step h = 1/4 plus the exact pole correction
 *                 2 exp(-z^2) / (1 -/+ exp(-2 pi i z / h)), with the node
 *                 lattice shifted by h/2 when x lies near a node (Chiarella &
 *                 Reichel 1968, Math. Comp. 22:137; Matta & Reichel 1971,
 *                 Math. Comp. 25:339).  The quadrature error is of order
 *                 exp(-pi^2/h^2) = 1e-69, so Re w keeps full relative
 *                 accuracy down to the real axis.
 *   |z|^2 >= 64 : the Laplace continued fraction
 *                 w(z) = (i/sqrt(pi)) / (z - (1/2)/(z - 1/(z - (3/2)/(z - ...))))
 *                 (Gautschi 1970, SIAM J. Numer. Anal. 7:187), 40 levels.
 * On the real axis (y == 0) Re w is exp(-x^2) by definition.
 * The derivative w'(z) = -2 z w(z) + 2i/sqrt(pi) (the Faddeeva ODE); for
 * |z|^2 >= 64 its asymptotic series is summed instead to avoid cancellation.
 *
 * Readings of the paper that this file takes (each also listed in the design
 * notes of the repository):
 *   - profile normalisation: area-normalised, phi = Re w / (alpha_D sqrt(pi));
 *   - constants: k_B and c as printed in Sect. 2.2; h from CODATA 2010, which
 *     is consistent with the printed k_B; amu = 1.660538921e-24 g;
 *   - S-mode: S(T) = S_ref (Q(T_ref)/Q(T)) exp(-c2 E'' (1/T - 1/T_ref))
 *                    (1 - exp(-c2 nu0/T)) / (1 - exp(-c2 nu0/T_ref));
 *     A-mode: Eq. S, per molecule, optionally divided by m for cm/g;
 *   - cut: with q = 1/dnu, u = (nu0 - nu_min) * q, i0 = floor(u),
 *     r = u - i0 and W = cut * q (all FP64, one rounding per operation, no
 *     fused multiply-add), bin i is inside iff |(i - i0) - r| <= W; cut <= 0
 *     means no cut (the whole grid).  Mathematically this is
 *     |nu_i - nu0| <= cut; the FP64 form fixes the decision at ties;
 *   - a line with nu0 <= 0 has no Doppler width (Eq. gammaD) and adds nothing;
 *   - plinth (Sect. 2.1): the line's own profile value at exactly its cutting
 *     length, subtracted from every bin inside the cut; no cut, no plinth;
 *   - per-line cuts (Sect. 2.4.3 item 4): factor times the Doppler half width
 *     sqrt(ln 2) alpha_D, evaluated as factor * (nu0 * K_D), or factor times
 *     Gamma_L;
 *   - profiles (Sect. 2.1): Lorentzian (Gamma_L/pi)/(d^2 + Gamma_L^2), Doppler
 *     exp(-(d/alpha_D)^2)/(alpha_D sqrt(pi)), and the binned Gaussian as the
 *     Doppler profile averaged over the bin [d - dnu/2, d + dnu/2];
 *   - HITRAN lists (Sect. 2.2, Eq. gammaL): air/self widths with the self
 *     partial pressure; the pressure shift moves the line to nu0 + delta P/P_ref
 *     while S(T) and alpha_D keep nu0.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- physical constants (oracle copy) ---------------------------------- */
static const double O_C = 2.99792458e10;     /* cm s^-1, Sect. 2.2.2 (Eq. S) */
static const double O_KB = 1.3806489e-16;    /* erg K^-1, Sect. 2.2 (Eq. gammaD) */
static const double O_H = 6.62606957e-27;    /* erg s, CODATA 2010 */
static const double O_AMU = 1.660538921e-24; /* g, CODATA 2010 */
static const double O_PI = 3.14159265358979323846;

void hko_constants(double *out6)
{
    out6[0] = O_C;
    out6[1] = O_KB;
    out6[2] = O_H;
    out6[3] = O_AMU;
    out6[4] = O_H * O_C / O_KB; /* second radiation constant c2 in cm K */
    out6[5] = O_PI;
}

/* ---- Faddeeva function -------------------------------------------------- */

/* Trapezoidal rule with pole correction (Chiarella & Reichel; Matta & Reichel).
 * Requires x >= 0, y >= 0.  Nodes t_n = (n + off) h with |t_n| <= 9.6, where
 * exp(-t^2) < 1e-40 beyond. */
static double complex w_trapezoid(double x, double y)
{
    const double h = 0.25;
    double u = x / h;
    double fr = u - floor(u);
    int shifted = !(fr > 0.25 && fr < 0.75); /* x within h/4 of a node */
    double off = shifted ? 0.5 : 0.0;
    double complex z = x + I * y;
    double complex s = 0.0;
    for (int n = -40; n <= 40; ++n) {
        double t = (n + off) * h;
        if (fabs(t) > 9.6)
            continue;
        s += exp(-t * t) / (z - t);
    }
    double complex w = I * (h / O_PI) * s;
    if (y < O_PI / h) {
        double complex q = cexp(-2.0 * O_PI * I * z / h);
        w += 2.0 * cexp(-z * z) / (shifted ? (1.0 + q) : (1.0 - q));
    }
    return w;
}

/* Laplace continued fraction, 40 levels; accurate to ~1e-14 for |z| >= 8. */
static double complex w_contfrac(double x, double y)
{
    double complex z = x + I * y;
    double complex d = z;
    for (int k = 40; k >= 1; --k)
        d = z - (0.5 * k) / d;
    return (I / sqrt(O_PI)) / d;
}

/* w(x + iy) for y >= 0 and any x. */
static double complex w_eval(double x, double y)
{
    double ax = fabs(x);
    double complex w = (ax * ax + y * y < 64.0) ? w_trapezoid(ax, y) : w_contfrac(ax, y);
    if (y == 0.0)
        w = exp(-ax * ax) + I * cimag(w); /* Re w(x) = exp(-x^2) on the real axis */
    if (x < 0.0)
        w = conj(w); /* w(-x + iy) = conj(w(x + iy)) */
    return w;
}

/* w'(z).  |z|^2 < 64: from the ODE w' = -2 z w + 2i/sqrt(pi).
 * |z|^2 >= 64: asymptotic series w'(z) ~ -(i/sqrt(pi)) sum_k c_k z^-(2k+2),
 * c_0 = 1, c_{k+1} = c_k (2k+3)/2, summed to its smallest term. */
static double complex wprime_eval(double x, double y)
{
    double ax = fabs(x);
    double complex z = ax + I * y;
    double complex d;
    if (ax * ax + y * y < 64.0) {
        d = -2.0 * z * w_eval(ax, y) + 2.0 * I / sqrt(O_PI);
    } else {
        double complex p = 1.0 / (z * z);
        double complex term = p; /* c_0 p^1 */
        double complex sum = 0.0;
        double prev = INFINITY;
        for (int k = 0; k < 200; ++k) {
            double mag = cabs(term);
            if (mag > prev)
                break; /* asymptotic series: stop at the smallest term */
            sum += term;
            if (mag <= 1e-18 * cabs(sum))
                break;
            prev = mag;
            term *= p * (2.0 * k + 3.0) / 2.0;
        }
        d = -(I / sqrt(O_PI)) * sum;
        if (y == 0.0)
            d = -2.0 * ax * exp(-ax * ax) + I * cimag(d);
    }
    if (x < 0.0)
        d = -conj(d); /* w'(-x+iy) = -conj(w'(x+iy)) */
    return d;
}

void hko_faddeeva(int64_t n, const double *x, const double *y, double *re, double *im)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double complex w = w_eval(x[i], y[i]);
        re[i] = creal(w);
        im[i] = cimag(w);
    }
}

void hko_faddeeva_deriv(int64_t n, const double *x, const double *y, double *re, double *im)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double complex d = wprime_eval(x[i], y[i]);
        re[i] = creal(d);
        im[i] = cimag(d);
    }
}

/* ---- per-line quantities (Sect. 2.2, 2.2.2, 2.4.3) ----------------------- */

/* S-mode (HITRAN/ExoMol reference-strength scaling) or A-mode (Eq. S).
 * s_mode 0: S_ref[l] given at T_ref.  s_mode 1: A[l], g_up[l] given.
 * per_gram: divide by m in grams (Eq. S's cm/g convention). */
void hko_line_strength(int64_t n, const double *nu0, const double *S_ref, const double *A,
                       const double *g_up, const double *E_low, int s_mode, double T,
                       double Q_T, double T_ref, double Q_Tref, double mass_amu, int per_gram,
                       double *S_out)
{
    const double c2 = O_H * O_C / O_KB;
    const double m_g = mass_amu * O_AMU;
#pragma omp parallel for schedule(static)
    for (int64_t l = 0; l < n; ++l) {
        double S;
        if (s_mode == 0) {
            double boltz = exp(-c2 * E_low[l] * (1.0 / T - 1.0 / T_ref));
            double stim = -expm1(-c2 * nu0[l] / T) / -expm1(-c2 * nu0[l] / T_ref);
            S = S_ref[l] * (Q_Tref / Q_T) * boltz * stim;
        } else {
            S = A[l] * g_up[l] / (8.0 * O_PI * O_C * nu0[l] * nu0[l] * Q_T) *
                exp(-c2 * E_low[l] / T) * -expm1(-c2 * nu0[l] / T);
        }
        if (per_gram)
            S /= m_g;
        S_out[l] = S;
    }
}

/* alpha_D (Sect. 2.4.2, Eq. alphaD inverted) and Gamma_L (ExoMol form of
 * Sect. 2.2 with the natural term A/(4 pi c)).  A may be NULL (A = 0). */
void hko_widths(int64_t n, const double *nu0, const double *gamma_ref, const double *n_T,
                const double *A, double T, double P, double T_ref, double P_ref,
                double mass_amu, double *alphaD_out, double *gammaL_out)
{
    const double m_g = mass_amu * O_AMU;
#pragma omp parallel for schedule(static)
    for (int64_t l = 0; l < n; ++l) {
        alphaD_out[l] = nu0[l] / O_C * sqrt(2.0 * O_KB * T / m_g);
        double nat = A ? A[l] / (4.0 * O_PI * O_C) : 0.0;
        gammaL_out[l] = nat + gamma_ref[l] * pow(T_ref / T, n_T[l]) * (P / P_ref);
    }
}

/* HITRAN Lorentz half width (Sect. 2.2, Eq. gammaL, air and self broadening):
 * Gamma_L = A/(4 pi c) + (T/T_ref)^-n [gamma_air (P - P_self)/P_ref + gamma_self P_self/P_ref].
 * alpha_D as hko_widths.  A may be NULL (A = 0). */
void hko_widths_hitran(int64_t n, const double *nu0, const double *gamma_air,
                       const double *gamma_self, const double *n_T, const double *A, double T,
                       double P, double P_self, double T_ref, double P_ref, double mass_amu,
                       double *alphaD_out, double *gammaL_out)
{
    const double m_g = mass_amu * O_AMU;
#pragma omp parallel for schedule(static)
    for (int64_t l = 0; l < n; ++l) {
        alphaD_out[l] = nu0[l] / O_C * sqrt(2.0 * O_KB * T / m_g);
        double nat = A ? A[l] / (4.0 * O_PI * O_C) : 0.0;
        gammaL_out[l] = nat + pow(T / T_ref, -n_T[l]) * (gamma_air[l] * (P - P_self) / P_ref +
                                                         gamma_self[l] * P_self / P_ref);
    }
}

/* Pressure-shifted line positions (the shift delta of the HITRAN/HITEMP data,
 * Table binary2, cm^-1 per unit of P_ref): nu0 + delta * (P / P_ref).  The
 * shift moves the line; its strength and Doppler width keep the transition
 * wavenumber nu0. */
void hko_shift(int64_t n, const double *nu0, const double *delta, double P, double P_ref,
               double *out)
{
    const double press = P / P_ref;
#pragma omp parallel for schedule(static)
    for (int64_t l = 0; l < n; ++l)
        out[l] = nu0[l] + delta[l] * press;
}

/* ---- cut predicate ------------------------------------------------------ */

typedef struct {
    int64_t i0;
    double r;
} bin_pos;

static bin_pos line_pos(double nu0, double nu_min, double dnu)
{
    bin_pos p;
    double q = 1.0 / dnu;
    double u = (nu0 - nu_min) * q;
    double f = floor(u);
    p.i0 = (int64_t)f;
    p.r = u - f;
    return p;
}

static int in_cut(int64_t k, double r, double W)
{
    return fabs((double)k - r) <= W;
}

/* Inclusive bin range [*lo, *hi] of a line clipped to [0, nbins); empty if
 * *lo > *hi.  nocut: every bin of the grid; else the bins with
 * |(i - i0) - r| <= W, W = cut / dnu of this line (W >= 0).  The bounds come
 * from the predicate itself: a first guess is walked until in_cut changes, so
 * every bin in the range satisfies in_cut and its neighbours do not. */
static void line_range_w(double nu0, double nu_min, double dnu, int64_t nbins, int nocut,
                         double W, int64_t *lo, int64_t *hi)
{
    if (!(nu0 > 0.0)) { /* no Doppler width (Eq. gammaD is proportional to nu0): ignored */
        *lo = 1;
        *hi = 0;
        return;
    }
    if (nocut) {
        *lo = 0;
        *hi = nbins - 1;
        return;
    }
    bin_pos p = line_pos(nu0, nu_min, dnu);
    /* k offsets relative to i0 */
    int64_t a = (int64_t)floor(p.r - W) - 1;
    int64_t b = (int64_t)ceil(p.r + W) + 1;
    while (in_cut(a, p.r, W))
        --a;
    while (a + 1 <= b && !in_cut(a + 1, p.r, W))
        ++a;
    while (in_cut(b, p.r, W))
        ++b;
    while (b - 1 >= a && !in_cut(b - 1, p.r, W))
        --b;
    int64_t L = p.i0 + a + 1, H = p.i0 + b - 1;
    if (L < 0)
        L = 0;
    if (H > nbins - 1)
        H = nbins - 1;
    *lo = L;
    *hi = H;
}

/* A fixed cutting length: cut <= 0 means no cut (the whole grid). */
static void line_range(double nu0, double nu_min, double dnu, int64_t nbins, double cut,
                       int64_t *lo, int64_t *hi)
{
    line_range_w(nu0, nu_min, dnu, nbins, !(cut > 0.0), cut * (1.0 / dnu), lo, hi);
}

/* Per-line cutting lengths of Sect. 2.4.3 item 4: mode 2 = factor times the
 * Doppler half width Gamma_D = sqrt(ln 2) alpha_D (Eq. gammaD), mode 3 =
 * factor times the Lorentz half width Gamma_L.  The Doppler form is evaluated
 * as factor * (nu0 * K_D) with K_D = sqrt(ln 2) * sqrt(2 k_B T / m) / c (one
 * constant per (T, species)), so that the cut decision is a fixed sequence of
 * correctly rounded operations. */
void hko_line_cuts(int64_t n, const double *nu0, const double *gammaL, int mode, double factor,
                   double T, double mass_amu, double *cut_out)
{
    const double m_g = mass_amu * O_AMU;
    const double K_D = sqrt(0.6931471805599453) * sqrt(2.0 * O_KB * T / m_g) / O_C;
#pragma omp parallel for schedule(static)
    for (int64_t l = 0; l < n; ++l)
        cut_out[l] = mode == 2 ? factor * (nu0[l] * K_D) : factor * gammaL[l];
}

void hko_line_ranges(int64_t n, const double *nu0, double nu_min, double dnu, int64_t nbins,
                     double cut, int64_t *lo, int64_t *hi)
{
#pragma omp parallel for schedule(static)
    for (int64_t l = 0; l < n; ++l)
        line_range(nu0[l], nu_min, dnu, nbins, cut, &lo[l], &hi[l]);
}

/* Pair count with one cutting length per line (cut_l[l] >= 0, in cm^-1). */
int64_t hko_count_pairs_percut(int64_t n, const double *nu0, const double *cut_l, double nu_min,
                               double dnu, int64_t nbins)
{
    int64_t total = 0;
    const double q = 1.0 / dnu;
#pragma omp parallel for schedule(static) reduction(+ : total)
    for (int64_t l = 0; l < n; ++l) {
        int64_t lo, hi;
        line_range_w(nu0[l], nu_min, dnu, nbins, 0, cut_l[l] * q, &lo, &hi);
        if (hi >= lo)
            total += hi - lo + 1;
    }
    return total;
}

int64_t hko_count_pairs(int64_t n, const double *nu0, double nu_min, double dnu, int64_t nbins,
                        double cut)
{
    int64_t total = 0;
#pragma omp parallel for schedule(static) reduction(+ : total)
    for (int64_t l = 0; l < n; ++l) {
        int64_t lo, hi;
        line_range(nu0[l], nu_min, dnu, nbins, cut, &lo, &hi);
        if (hi >= lo)
            total += hi - lo + 1;
    }
    return total;
}

/* ---- cross section (the plain direct sum) ------------------------------- */

/* sigma_out[j] = sigma(bin_lo + j) for j < bin_hi - bin_lo.  Lines need not be
 * sorted; if sorted_nu0 != 0 the candidate lines are narrowed by bisection on
 * nu0 (a superset; the cut predicate still decides).  Parallel over blocks of
 * bins; each bin sums its lines in ascending index order.
 * cut_l: NULL for the fixed cut `cut` (<= 0: no cut), else one cutting
 * length per line (cm^-1, >= 0).  plinth: subtract from every bin inside a
 * line's cut the line's own value at the cutting length,
 * S Re w(cut_l / alpha_D + i y) / (alpha_D sqrt(pi)) (Sect. 2.1, "Removing
 * the Plinth"); a line without a cut has no plinth. */
/* Line profiles (Sect. 2.1): sigma contribution S * phi of one line at
 * offset d = nu - nu0 from its centre.
 *   0 Voigt      phi = Re w(d / alpha_D + i y) / (alpha_D sqrt(pi))
 *   1 Lorentz    phi = (Gamma_L / pi) / (d^2 + Gamma_L^2)
 *   2 Doppler    phi = exp(-(d / alpha_D)^2) / (alpha_D sqrt(pi))
 *   3 binned Gaussian integrated cross section (ExoCross): the Doppler profile
 *                averaged over the bin [d - dnu/2, d + dnu/2],
 *                phi = [erf((d + dnu/2)/alpha_D) - erf((d - dnu/2)/alpha_D)] / (2 dnu),
 *                evaluated with erfc of positive arguments away from the centre
 *                (erf(b) - erf(a) = erfc(a) - erfc(b)) so that no two values near
 *                1 are subtracted. */
static double profile_value(int profile, double S, double d, double aD, double GL, double dnu)
{
    switch (profile) {
    case 1:
        return S * (GL / O_PI) / (d * d + GL * GL);
    case 2: {
        double x = d / aD;
        return S * exp(-x * x) / (aD * sqrt(O_PI));
    }
    case 3: {
        double a = (fabs(d) - 0.5 * dnu) / aD, b = (fabs(d) + 0.5 * dnu) / aD;
        double v = a >= 0.0 ? erfc(a) - erfc(b) : erf(b) + erf(-a);
        return S * v / (2.0 * dnu);
    }
    default:
        return S * creal(w_eval(d / aD, GL / aD)) / (aD * sqrt(O_PI));
    }
}

void hko_sigma_prof(int64_t n, const double *nu0, const double *S, const double *alphaD,
                    const double *gammaL, const double *cut_l, int plinth, int profile,
                    int sorted_nu0, double nu_min, double dnu, int64_t nbins, double cut,
                    int64_t bin_lo, int64_t bin_hi, double *sigma_out, int nthreads);

void hko_sigma_ext(int64_t n, const double *nu0, const double *S, const double *alphaD,
                   const double *gammaL, const double *cut_l, int plinth, int sorted_nu0,
                   double nu_min, double dnu, int64_t nbins, double cut, int64_t bin_lo,
                   int64_t bin_hi, double *sigma_out, int nthreads)
{
    hko_sigma_prof(n, nu0, S, alphaD, gammaL, cut_l, plinth, 0, sorted_nu0, nu_min, dnu, nbins,
                   cut, bin_lo, bin_hi, sigma_out, nthreads);
}

/* As hko_sigma_ext with a choice of line profile (see profile_value); the
 * plinth is the profile's own value at the cutting length. */
void hko_sigma_prof(int64_t n, const double *nu0, const double *S, const double *alphaD,
                    const double *gammaL, const double *cut_l, int plinth, int profile,
                    int sorted_nu0, double nu_min, double dnu, int64_t nbins, double cut,
                    int64_t bin_lo, int64_t bin_hi, double *sigma_out, int nthreads)
{
    const double inv_sqrt_pi = 1.0 / sqrt(O_PI);
    const double q = 1.0 / dnu;
    int64_t nb = bin_hi - bin_lo;
    if (nb <= 0)
        return;
    memset(sigma_out, 0, (size_t)nb * sizeof(double));
    const int nocut = cut_l == NULL && !(cut > 0.0);
    double cmax = cut;
    if (cut_l) {
        cmax = 0.0;
        for (int64_t l = 0; l < n; ++l)
            if (cut_l[l] > cmax)
                cmax = cut_l[l];
    }
    int64_t l_begin = 0, l_end = n;
    if (sorted_nu0 && !nocut && n > 0) {
        double lo_nu = nu_min + (double)bin_lo * dnu - cmax - 2.0 * dnu;
        double hi_nu = nu_min + (double)(bin_hi - 1) * dnu + cmax + 2.0 * dnu;
        int64_t a = 0, b = n;
        while (a < b) {
            int64_t m = (a + b) / 2;
            if (nu0[m] < lo_nu) a = m + 1; else b = m;
        }
        l_begin = a;
        a = l_begin;
        b = n;
        while (a < b) {
            int64_t m = (a + b) / 2;
            if (nu0[m] <= hi_nu) a = m + 1; else b = m;
        }
        l_end = a;
    }
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#endif
    int64_t blk = 64;
    int64_t nblk = (nb + blk - 1) / blk;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t qb = 0; qb < nblk; ++qb) {
        int64_t b0 = bin_lo + qb * blk;
        int64_t b1 = b0 + blk < bin_hi ? b0 + blk : bin_hi;
        for (int64_t l = l_begin; l < l_end; ++l) {
            const double cl = cut_l ? cut_l[l] : cut;
            int64_t lo, hi;
            line_range_w(nu0[l], nu_min, dnu, nbins, nocut, cl * q, &lo, &hi);
            if (lo < b0) lo = b0;
            if (hi > b1 - 1) hi = b1 - 1;
            if (hi < lo)
                continue;
            bin_pos p = line_pos(nu0[l], nu_min, dnu);
            double y = gammaL[l] / alphaD[l];
            double amp = S[l] * inv_sqrt_pi / alphaD[l];
            if (profile == 0) {
                double h = (plinth && !nocut) ? amp * creal(w_eval(cl / alphaD[l], y)) : 0.0;
                for (int64_t i = lo; i <= hi; ++i) {
                    double x = ((double)(i - p.i0) - p.r) * dnu / alphaD[l];
                    sigma_out[i - bin_lo] += amp * creal(w_eval(x, y)) - h;
                }
            } else {
                double h = (plinth && !nocut)
                               ? profile_value(profile, S[l], cl, alphaD[l], gammaL[l], dnu)
                               : 0.0;
                for (int64_t i = lo; i <= hi; ++i) {
                    double d = ((double)(i - p.i0) - p.r) * dnu;
                    sigma_out[i - bin_lo] +=
                        profile_value(profile, S[l], d, alphaD[l], gammaL[l], dnu) - h;
                }
            }
        }
    }
}

void hko_sigma(int64_t n, const double *nu0, const double *S, const double *alphaD,
               const double *gammaL, int sorted_nu0, double nu_min, double dnu, int64_t nbins,
               double cut, int64_t bin_lo, int64_t bin_hi, double *sigma_out, int nthreads)
{
    hko_sigma_ext(n, nu0, S, alphaD, gammaL, NULL, 0, sorted_nu0, nu_min, dnu, nbins, cut,
                  bin_lo, bin_hi, sigma_out, nthreads);
}

/* ---- adjoint (gradient of L = sum_i g_i sigma_i) ------------------------ */

/* For one (T, P) point, S-mode.  Accumulates (+=) into dL_dSref[l] and
 * dL_dgamma[l]; writes *dL_dT and *dL_dP.  Chain rule through
 *   S(T)     : dlnS/dT = -dlnQ/dT + c2 E''/T^2 - (c2 nu0/T^2) / expm1(c2 nu0/T)
 *   alpha_D  : d alpha_D / dT = alpha_D / (2T)
 *   Gamma_L  : dGamma_L/dT = -n (Gamma_L - A/(4 pi c)) / T,  dGamma_L/dP = (Gamma_L - A/(4 pi c)) / P
 *   phi      : phi = Re w(x+iy) / (alpha_D sqrt(pi)),  x = dnu_i/alpha_D, y = Gamma_L/alpha_D,
 *              dRe w/dx = Re w',  dRe w/dy = -Im w'.                                    */
void hko_backward(int64_t n, const double *nu0, const double *S_ref, const double *E_low,
                  const double *gamma_ref, const double *n_T, const double *A, double T,
                  double P, double Q_T, double dlnQ_dT, double T_ref, double P_ref,
                  double Q_Tref, double mass_amu, double nu_min, double dnu, int64_t nbins,
                  double cut, const double *grad_sigma, double *dL_dSref, double *dL_dgamma,
                  double *dL_dT, double *dL_dP, int nthreads)
{
    const double c2 = O_H * O_C / O_KB;
    const double m_g = mass_amu * O_AMU;
    const double inv_sqrt_pi = 1.0 / sqrt(O_PI);
    double gT = 0.0, gP = 0.0;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : gT, gP)
    for (int64_t l = 0; l < n; ++l) {
        double boltz = exp(-c2 * E_low[l] * (1.0 / T - 1.0 / T_ref));
        double stim = -expm1(-c2 * nu0[l] / T) / -expm1(-c2 * nu0[l] / T_ref);
        double ratio = (Q_Tref / Q_T) * boltz * stim; /* S(T) / S_ref */
        double S = S_ref[l] * ratio;
        double dlnS_dT = -dlnQ_dT + c2 * E_low[l] / (T * T) -
                         (c2 * nu0[l] / (T * T)) / expm1(c2 * nu0[l] / T);
        double aD = nu0[l] / O_C * sqrt(2.0 * O_KB * T / m_g);
        double nat = A ? A[l] / (4.0 * O_PI * O_C) : 0.0;
        double press = pow(T_ref / T, n_T[l]) * (P / P_ref);
        double GL = nat + gamma_ref[l] * press;
        double dGL_dT = -n_T[l] * (GL - nat) / T;
        double dGL_dP = gamma_ref[l] * pow(T_ref / T, n_T[l]) / P_ref;
        double y = GL / aD;
        int64_t lo, hi;
        line_range(nu0[l], nu_min, dnu, nbins, cut, &lo, &hi);
        bin_pos p = line_pos(nu0[l], nu_min, dnu);
        double sV = 0.0, sVx = 0.0, sVy = 0.0, sXVx = 0.0;
        for (int64_t i = lo; i <= hi; ++i) {
            double x = ((double)(i - p.i0) - p.r) * dnu / aD;
            double complex w = w_eval(x, y);
            double complex d = wprime_eval(x, y);
            double g = grad_sigma[i];
            sV += g * creal(w);
            sVx += g * creal(d);      /* d Re w / dx */
            sXVx += g * x * creal(d);
            sVy += g * -cimag(d);     /* d Re w / dy */
        }
        /* sigma contribution of line l: S * Re w / (aD sqrt(pi)) */
        double base = inv_sqrt_pi / aD;
        /* d/dS_ref */
        dL_dSref[l] += ratio * base * sV;
        /* d/dgamma_ref: dy/dgamma = press / aD */
        dL_dgamma[l] += S * base * sVy * (press / aD);
        /* d/dT: S(T), 1/aD prefactor, x(aD), y(aD, GL) */
        double daD_dT = aD / (2.0 * T);
        double dy_dT = dGL_dT / aD - y * daD_dT / aD;
        /* dx/dT = -x daD/aD */
        double dT = S * base * (dlnS_dT * sV - (daD_dT / aD) * sV - (daD_dT / aD) * sXVx +
                                dy_dT * sVy);
        gT += dT;
        gP += S * base * sVy * (dGL_dP / aD);
    }
    *dL_dT = gT;
    *dL_dP = gP;
}
