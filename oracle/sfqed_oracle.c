/*
 * Strong-field QED event generator -- plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the
 * benchmark's CPU-baseline leg are the only callers.  The CUDA library never
 * links, loads or calls this file, and this file shares no code, header or
 * table with the CUDA library: everything below is written out a second time,
 * slowly and in the order the method states it, so that each step can be
 * checked against arXiv:2409.17299 and against textbook formulas by eye.
 *
 * Method (arXiv:2409.17299):
 *   Sec. 3, Algorithm 1  per-particle push with an exponential waiting time
 *                        dt_hat = -log(r)/lambda, sub-stepped inside the PIC step
 *   Sec. 3, Algorithm 2  avalanche: every particle born inside the step is
 *                        pushed to the end of the same step
 *   Sec. 3               rates from an approximation of precomputed rates,
 *                        energies by inverse sampling of 2-D (chi, energy) tables
 *   Sec. 3               the accumulated optical-depth scheme of other codes
 *                        (rate once per step, at most one event per step)
 *   Sec. 4.2             per-thread buffers merged after the push; filtering
 *                        and thinning at the merge
 *   Sec. 5.1             "global leveling" resampling keeps the count bounded
 *
 * The paper does not restate the physics; the rate formulas are the standard
 * quasi-classical (LCFA) Baier-Katkov / Ritus probabilities.  Every place where
 * the paper is silent is marked "Reading:".
 *
 * Units: time 1/omega, length c/omega, momentum m c, energy m c^2,
 * fields m c omega / e, for a wavelength of 0.8 um.
 *
 * Parity pins (tests/test_oracle_*.py): Philox against an independent library
 * implementation; Bessel integrals against scipy.special.kv; total rates against
 * direct scipy quadrature and their small/large-chi asymptotes; inverse-CDF
 * tables against the exact CDF (KS, node round trip); Boris against the
 * closed forms for uniform B and uniform E; the event loop against Poisson and
 * waiting-time laws, energy and charge conservation; leveling against its
 * defining equation and weight conservation in expectation; the optical-depth
 * scheme against the per-step event probability 1 - exp(-lambda dt) integrated
 * over its renewal process, against a hand-stepped single particle and
 * against Algorithm 1 in the limit lambda dt -> 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Physical constants (CODATA 2018), lambda = 0.8 um.                  */
/* R = m c^2 / (hbar omega), omega = 2 pi c / lambda.                  */
/* ------------------------------------------------------------------ */
#define OR_ALPHA 7.2973525693e-3
#define OR_R     329718.75885517005
#define OR_PI    3.14159265358979323846

/* Table grids (Reading: the paper gives no layout, only that the inverse CDF
 * is a 2-D function of chi and energy, Sec. 3). */
#define OR_EM_NCHI   121      /* log10 chi in [-3, 3], 20 nodes per decade   */
#define OR_PAIR_NCHI 101      /* log10 chi in [-2, 3], 20 nodes per decade   */
#define OR_EM_NS     257      /* logit u in [-16, 16]                        */
#define OR_PAIR_NS   129      /* logit u in [-16, 0]  (u <= 1/2, symmetric)  */
#define OR_SMAX      16.0
#define OR_CHEB_N    11       /* Chebyshev interpolant of degree 10 per decade */
#define OR_EM_NDEC   6
#define OR_PAIR_NDEC 5
#define OR_PAIR_CHI_MIN 0.01  /* Reading: pair rate is zero below chi = 0.01 */

/* ================================================================== */
/* 1. Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).               */
/*    One round: multiply words 0 and 2 by the two round constants,    */
/*    swap the high halves across and xor in the key; the key is       */
/*    bumped by the two Weyl constants between rounds.                 */
/* ================================================================== */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void or_philox_batch(int64_t n, const uint32_t *ctr, const uint32_t key[2], uint32_t *out)
{
    for (int64_t i = 0; i < n; ++i) or_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* Reading: a uniform double in the open interval (0,1) from two 32-bit words:
 * the top 52 bits of (a,b), plus one half, times 2^-52.  Never 0, never 1. */
double or_u52(uint32_t a, uint32_t b)
{
    uint64_t m = ((uint64_t)a << 20) | (uint64_t)(b >> 12);
    return ((double)m + 0.5) * (1.0 / 4503599627370496.0);
}

/* ================================================================== */
/* 2. Bessel functions K_nu(y) and the integral  int_y^inf K_{1/3}.    */
/*    Large y: trapezoid rule on the integral representations          */
/*      K_nu(y)          = int_0^inf exp(-y cosh t) cosh(nu t) dt      */
/*      int_y^inf K_nu   = int_0^inf exp(-y cosh t) cosh(nu t)/cosh t dt */
/*    (exponentially convergent for these entire integrands, with a     */
/*    step below 0.5/sqrt(y) for large y).                              */
/*    Small y: the ascending series (Abramowitz & Stegun 9.6.2, 9.6.10) */
/*      K_nu = pi/(2 sin nu pi) (I_{-nu} - I_nu),                       */
/*      I_mu(y) = sum_k (y/2)^{2k+mu} / (k! Gamma(k+mu+1)).             */
/* ================================================================== */
#define OR_Y_SERIES 0.5

static double trapezoid_bessel(double nu, double y, int divide_by_cosh)
{
    /* the peak at t = 0 has width ~ 1/sqrt(y): the step shrinks with it so the
     * discretisation error stays near exp(-2 pi^2 / (h^2 y)) < 1e-30 */
    const double h = (y > 16.0) ? 0.5 / sqrt(y) : 0.125;
    if (y > 745.0) return 0.0;            /* exp(-y) underflows in double */
    double sum = 0.5 * exp(-y);           /* t = 0: cosh 0 = 1 */
    for (int j = 1; j < 100000; ++j) {
        double t = j * h;
        double ct = cosh(t);
        double f = exp(-y * ct) * cosh(nu * t);
        if (divide_by_cosh) f /= ct;
        sum += f;
        if (y * ct > 1.0 && f <= 1e-19 * sum) break;
    }
    return h * sum;
}

static double series_I(double mu, double y)
{
    double half = 0.5 * y, s = 0.0;
    for (int k = 0; k < 60; ++k) {
        double term = pow(half, 2.0 * k + mu) / (tgamma(k + 1.0) * tgamma(k + mu + 1.0));
        s += term;
        if (fabs(term) < 1e-19 * fabs(s)) break;
    }
    return s;
}

/* int_0^y I_mu(s) ds, termwise */
static double series_int_I(double mu, double y)
{
    double s = 0.0;
    for (int k = 0; k < 60; ++k) {
        double p = 2.0 * k + mu + 1.0;
        double term = pow(0.5, 2.0 * k + mu) * pow(y, p) / (p * tgamma(k + 1.0) * tgamma(k + mu + 1.0));
        s += term;
        if (fabs(term) < 1e-19 * fabs(s)) break;
    }
    return s;
}

double or_besselK(double nu, double y)
{
    if (y < OR_Y_SERIES && fabs(nu - floor(nu + 0.5)) > 1e-6)
        return OR_PI / (2.0 * sin(nu * OR_PI)) * (series_I(-nu, y) - series_I(nu, y));
    return trapezoid_bessel(nu, y, 0);
}

/* int_y^inf K_{1/3}(s) ds.  int_0^inf K_{1/3} = pi / sqrt(3). */
double or_intK13(double y)
{
    if (y < OR_Y_SERIES) {
        double c = OR_PI / (2.0 * sin(OR_PI / 3.0));
        return OR_PI / sqrt(3.0) - c * (series_int_I(-1.0 / 3.0, y) - series_int_I(1.0 / 3.0, y));
    }
    return trapezoid_bessel(1.0 / 3.0, y, 1);
}

/* ================================================================== */
/* 3. Quasi-classical probabilities (LCFA).                            */
/*    Emission, delta = photon energy / emitter energy,                */
/*      dW/d delta = (alpha R / gamma) / (sqrt3 pi) *                  */
/*        [ ((1-delta) + 1/(1-delta)) K_{2/3}(y) - int_y^inf K_{1/3} ],  */
/*      y = 2 delta / (3 chi (1-delta)).                               */
/*    Pair, delta = electron energy / photon energy,                   */
/*      dW/d delta = (alpha R / k0) / (sqrt3 pi) *                     */
/*        [ (delta/(1-delta) + (1-delta)/delta) K_{2/3}(y) + int_y^inf K_{1/3} ], */
/*      y = 2 / (3 chi delta (1-delta)).                               */
/*    Both are integrated in a variable z on the whole line:           */
/*      emission: y = e^z;  pair: delta = 1/(1+e^-z), z <= 0 (delta <= 1/2). */
/*    g(z) below is the bracket times d delta/dz, so F = c int g dz.    */
/* ================================================================== */
double or_em_bracket(double chi, double delta)
{
    double y = 2.0 * delta / (3.0 * chi * (1.0 - delta));
    return ((1.0 - delta) + 1.0 / (1.0 - delta)) * or_besselK(2.0 / 3.0, y) - or_intK13(y);
}

double or_pair_bracket(double chi, double delta)
{
    double y = 2.0 / (3.0 * chi * delta * (1.0 - delta));
    return (delta / (1.0 - delta) + (1.0 - delta) / delta) * or_besselK(2.0 / 3.0, y) + or_intK13(y);
}

static double g_em(double z, double chi)
{
    double y = exp(z);
    double a = 3.0 * chi * y;
    double one_m = 2.0 / (2.0 + a);            /* 1 - delta */
    double ddelta_dy = 6.0 * chi / ((2.0 + a) * (2.0 + a));
    double bracket = (one_m + 1.0 / one_m) * or_besselK(2.0 / 3.0, y) - or_intK13(y);
    return bracket * ddelta_dy * y;
}

static double g_pair(double z, double chi)
{
    double delta = 1.0 / (1.0 + exp(-z));
    double one_m = 1.0 / (1.0 + exp(z));
    double dd = delta * one_m;                 /* d delta / dz */
    double y = 2.0 / (3.0 * chi * dd);
    double bracket = (delta / one_m + one_m / delta) * or_besselK(2.0 / 3.0, y) + or_intK13(y);
    return bracket * dd;
}

typedef double (*or_gfun)(double, double);

/* Gauss-Legendre nodes on [-1,1] by Newton's method on P_n (textbook). */
#define OR_GL_N 12
static double gl_x[OR_GL_N], gl_w[OR_GL_N];
static int gl_ready = 0;
static void gl_init(void)
{
    if (gl_ready) return;
    int n = OR_GL_N;
    for (int i = 0; i < n; ++i) {
        double x = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        /* recompute derivative at the converged node */
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1; p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    gl_ready = 1;
}

static double gl_integrate(or_gfun g, double chi, double a, double b)
{
    double mid = 0.5 * (a + b), half = 0.5 * (b - a), s = 0.0;
    for (int i = 0; i < OR_GL_N; ++i) s += gl_w[i] * g(mid + half * gl_x[i], chi);
    return s * half;
}

/* Integration ranges in z.  Emission: z in [-120, 8]; below -120 the
 * integrand is C e^{z/3} (K_{2/3} ~ y^{-2/3}), whose tail is 3 g(-120).
 * Above 8 (y > 2980) it is below e^-2980.  Pair: z in [-40, 0]; below -40,
 * y > 1e14 and the integrand is exactly zero in double precision. */
#define OR_EM_ZLO   (-120.0)
#define OR_EM_ZHI   8.0
#define OR_EM_PANEL 0.5
#define OR_EM_NPAN  256
#define OR_PAIR_ZLO (-40.0)
#define OR_PAIR_PANEL 0.125
#define OR_PAIR_NPAN 320

/* F_gamma(chi) = (1/(sqrt3 pi)) int_0^1 [...] d delta */
double or_F_gamma_quad(double chi)
{
    gl_init();
    if (chi <= 0.0) return 0.0;
    double s = 3.0 * g_em(OR_EM_ZLO, chi);
    for (int p = 0; p < OR_EM_NPAN; ++p)
        s += gl_integrate(g_em, chi, OR_EM_ZLO + p * OR_EM_PANEL, OR_EM_ZLO + (p + 1) * OR_EM_PANEL);
    return s / (sqrt(3.0) * OR_PI);
}

/* F_pair(chi) = (1/(sqrt3 pi)) int_0^1 [...] d delta = 2/(sqrt3 pi) int_0^{1/2} */
double or_F_pair_quad(double chi)
{
    gl_init();
    if (chi <= 0.0) return 0.0;
    double s = 0.0;
    for (int p = 0; p < OR_PAIR_NPAN; ++p)
        s += gl_integrate(g_pair, chi, OR_PAIR_ZLO + p * OR_PAIR_PANEL, OR_PAIR_ZLO + (p + 1) * OR_PAIR_PANEL);
    return 2.0 * s / (sqrt(3.0) * OR_PI);
}

/* ================================================================== */
/* 4. Rate approximant (Sec. 3: "polynomial approximations" of the      */
/*    precomputed rates; Sec. 4.3: a fixed number of operations).       */
/*    Reading: on each decade of s = log10 chi a Chebyshev interpolant  */
/*    of degree 10 through the 11 Chebyshev-Gauss points;              */
/*      emission: of F_gamma(chi)/chi on [-3, 3];                       */
/*      pair:     of ln F_pair(chi) + 8/(3 chi) on [-2, 3].             */
/*    Outside: emission F ~ chi * (value at 1e-3) below, chi^{2/3} above; */
/*    pair zero below 0.01, chi^{2/3} above 1e3.                         */
/* ================================================================== */
static void cheb_fit(double (*f)(double), double s_lo, double *coef)
{
    double mid = s_lo + 0.5, half = 0.5, fv[OR_CHEB_N];
    for (int k = 0; k < OR_CHEB_N; ++k) {
        double x = cos(OR_PI * (k + 0.5) / OR_CHEB_N);
        fv[k] = f(mid + half * x);
    }
    for (int j = 0; j < OR_CHEB_N; ++j) {
        double s = 0.0;
        for (int k = 0; k < OR_CHEB_N; ++k) s += fv[k] * cos(OR_PI * j * (k + 0.5) / OR_CHEB_N);
        coef[j] = 2.0 * s / OR_CHEB_N;
    }
}

/* sum_j' c_j T_j(x), first term halved, by the three-term recurrence */
static double cheb_eval(const double *c, double x)
{
    double s = 0.5 * c[0], tm1 = 1.0, t = x;
    for (int j = 1; j < OR_CHEB_N; ++j) {
        s += c[j] * t;
        double tn = 2.0 * x * t - tm1;
        tm1 = t; t = tn;
    }
    return s;
}

static double fit_target_em(double s)   { double chi = pow(10.0, s); return or_F_gamma_quad(chi) / chi; }
static double fit_target_pair(double s) { double chi = pow(10.0, s); return log(or_F_pair_quad(chi)) + 8.0 / (3.0 * chi); }

void or_build_rate_coefs(double *cheb_em /* 6*11 */, double *cheb_pair /* 5*11 */)
{
    gl_init();
    #pragma omp parallel for schedule(dynamic)
    for (int d = 0; d < OR_EM_NDEC + OR_PAIR_NDEC; ++d) {
        if (d < OR_EM_NDEC) cheb_fit(fit_target_em, -3.0 + d, cheb_em + d * OR_CHEB_N);
        else cheb_fit(fit_target_pair, -2.0 + (d - OR_EM_NDEC), cheb_pair + (d - OR_EM_NDEC) * OR_CHEB_N);
    }
}

double or_rate_F(const double *cheb_em, const double *cheb_pair, int is_photon, double chi)
{
    if (!(chi > 0.0)) return 0.0;
    double s = log10(chi);
    if (!is_photon) {
        if (s < -3.0) return chi * cheb_eval(cheb_em, -1.0);
        if (s > 3.0) return 1e3 * cheb_eval(cheb_em + 5 * OR_CHEB_N, 1.0) * pow(chi / 1e3, 2.0 / 3.0);
        int d = (int)floor(s + 3.0);
        if (d > 5) d = 5;
        double x = 2.0 * (s - (-3.0 + d)) - 1.0;
        return chi * cheb_eval(cheb_em + d * OR_CHEB_N, x);
    } else {
        if (chi < OR_PAIR_CHI_MIN) return 0.0;
        if (s > 3.0) return exp(cheb_eval(cheb_pair + 4 * OR_CHEB_N, 1.0) - 8.0 / 3e3) * pow(chi / 1e3, 2.0 / 3.0);
        int d = (int)floor(s + 2.0);
        if (d > 4) d = 4;
        if (d < 0) d = 0;
        double x = 2.0 * (s - (-2.0 + d)) - 1.0;
        return exp(cheb_eval(cheb_pair + d * OR_CHEB_N, x) - 8.0 / (3.0 * chi));
    }
}

/* ================================================================== */
/* 5. Inverse-CDF tables (Sec. 3: inverse sampling through precomputed */
/*    tables of the inverse cumulative probability over chi and energy). */
/*    Reading (layout):                                                 */
/*      node j sits at s_j = logit(u_j) = ln(u_j/(1-u_j)), uniform in s; */
/*      emission stores zeta = ln y(u) with y = 2 delta/(3 chi (1-delta)), */
/*        s_j = -16 + 32 j/256, chi_i = 10^(-3 + i/20);                  */
/*      pair stores ln delta(u) for u <= 1/2 (the spectrum is symmetric */
/*        under delta -> 1-delta), s_j = -16 + 16 j/128,                 */
/*        chi_i = 10^(-2 + i/20).                                        */
/*    Each node is the exact root of CDF = u_j, found by Newton's method */
/*    on the composite Gauss-Legendre cumulative integral.              */
/* ================================================================== */
static double solve_in_panel(or_gfun g, double chi, double za, double zb, double target, int from_top)
{
    /* from_top == 0: find z with int_za^z g = target;
     * from_top == 1: find z with int_z^zb g = target.           */
    double lo = za, hi = zb;
    double whole = gl_integrate(g, chi, za, zb);
    double frac = whole > 0.0 ? target / whole : 0.5;
    if (frac < 0.0) frac = 0.0;
    if (frac > 1.0) frac = 1.0;
    double z = from_top ? zb - frac * (zb - za) : za + frac * (zb - za);
    for (int it = 0; it < 200; ++it) {
        double r, slope;
        if (!from_top) { r = gl_integrate(g, chi, za, z) - target; slope = g(z, chi); }
        else           { r = gl_integrate(g, chi, z, zb) - target; slope = -g(z, chi); }
        /* residual is increasing in z when from_top == 0, decreasing otherwise */
        int above = from_top ? (r < 0.0) : (r > 0.0);
        if (above) hi = z; else lo = z;
        double zn = (slope != 0.0) ? z - r / slope : 0.5 * (lo + hi);
        if (!(zn > lo && zn < hi)) zn = 0.5 * (lo + hi);
        double dz = fabs(zn - z);
        z = zn;
        if (dz < 1e-15 * (1.0 + fabs(z))) break;
        if (hi - lo < 1e-15 * (1.0 + fabs(z))) break;
    }
    return z;
}

/* Invert one CDF on the panels [zlo + p*w, zlo + (p+1)*w], given the mass
 * below zlo ("tail") and, per node, the target lower mass fraction u_j and
 * the upper mass fraction 1-u_j (both exact from s_j).  Writes z_j. */
static void invert_cdf(or_gfun g, double chi, double zlo, double w, int npan, double tail,
                       int ns, const double *s_nodes, double half_total_scale, double *z_out)
{
    double *mass = (double *)malloc(sizeof(double) * npan);
    double *below = (double *)malloc(sizeof(double) * (npan + 1));
    double *above = (double *)malloc(sizeof(double) * (npan + 1));
    for (int p = 0; p < npan; ++p) mass[p] = gl_integrate(g, chi, zlo + p * w, zlo + (p + 1) * w);
    below[0] = tail;
    for (int p = 0; p < npan; ++p) below[p + 1] = below[p] + mass[p];
    above[npan] = 0.0;
    for (int p = npan - 1; p >= 0; --p) above[p] = above[p + 1] + mass[p];
    double total = below[npan] * half_total_scale;   /* pair: the full (0,1) mass is twice the half */
    for (int j = 0; j < ns; ++j) {
        double s = s_nodes[j];
        double u = 1.0 / (1.0 + exp(-s));
        double v = 1.0 / (1.0 + exp(s));            /* 1 - u, without cancellation */
        if (u <= 0.5 || half_total_scale != 1.0) {
            double target = u * total;
            if (target <= tail) {                    /* inside the analytic tail (emission only) */
                /* tail mass is 3 g(z) e^{(z - zlo)/3}-shaped: invert the power law */
                z_out[j] = zlo + 3.0 * log(target / tail);
                continue;
            }
            int p = 0;
            while (p < npan - 1 && below[p + 1] < target) ++p;
            z_out[j] = solve_in_panel(g, chi, zlo + p * w, zlo + (p + 1) * w, target - below[p], 0);
        } else {
            double target = v * total;
            int p = npan - 1;
            while (p > 0 && above[p] < target) --p;
            z_out[j] = solve_in_panel(g, chi, zlo + p * w, zlo + (p + 1) * w, target - above[p + 1], 1);
        }
    }
    free(mass); free(below); free(above);
}

void or_build_icdf_tables(double *icdf_em /* 121*257 */, double *icdf_pair /* 101*129 */)
{
    gl_init();
    double s_em[OR_EM_NS], s_pair[OR_PAIR_NS];
    for (int j = 0; j < OR_EM_NS; ++j) s_em[j] = -OR_SMAX + 2.0 * OR_SMAX * j / (OR_EM_NS - 1);
    for (int j = 0; j < OR_PAIR_NS; ++j) s_pair[j] = -OR_SMAX + OR_SMAX * j / (OR_PAIR_NS - 1);
    #pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < OR_EM_NCHI + OR_PAIR_NCHI; ++r) {
        if (r < OR_EM_NCHI) {
            double chi = pow(10.0, -3.0 + r / 20.0);
            double tail = 3.0 * g_em(OR_EM_ZLO, chi);
            invert_cdf(g_em, chi, OR_EM_ZLO, OR_EM_PANEL, OR_EM_NPAN, tail, OR_EM_NS, s_em, 1.0,
                       icdf_em + (size_t)r * OR_EM_NS);
        } else {
            int i = r - OR_EM_NCHI;
            double chi = pow(10.0, -2.0 + i / 20.0);
            double z[OR_PAIR_NS];
            invert_cdf(g_pair, chi, OR_PAIR_ZLO, OR_PAIR_PANEL, OR_PAIR_NPAN, 0.0, OR_PAIR_NS, s_pair, 2.0, z);
            for (int j = 0; j < OR_PAIR_NS; ++j)
                icdf_pair[(size_t)i * OR_PAIR_NS + j] = -log1p(exp(-z[j]));   /* ln delta */
        }
    }
}

/* Exact CDF values (for tests): fraction of the emission spectrum with
 * photon fraction below delta, and of the pair spectrum with electron
 * fraction below delta. */
double or_em_cdf(double chi, double delta)
{
    gl_init();
    double y = 2.0 * delta / (3.0 * chi * (1.0 - delta));
    double zc = log(y);
    double tail = 3.0 * g_em(OR_EM_ZLO, chi), below = tail, total = tail;
    for (int p = 0; p < OR_EM_NPAN; ++p) {
        double a = OR_EM_ZLO + p * OR_EM_PANEL, b = a + OR_EM_PANEL;
        total += gl_integrate(g_em, chi, a, b);
        if (zc >= b) below += gl_integrate(g_em, chi, a, b);
        else if (zc > a) below += gl_integrate(g_em, chi, a, zc);
    }
    if (zc < OR_EM_ZLO) below = tail * exp((zc - OR_EM_ZLO) / 3.0);
    return below / total;
}

double or_pair_cdf(double chi, double delta)
{
    gl_init();
    int flip = delta > 0.5;
    double d = flip ? 1.0 - delta : delta;
    double zc = log(d) - log1p(-d);
    double below = 0.0, half = 0.0;
    for (int p = 0; p < OR_PAIR_NPAN; ++p) {
        double a = OR_PAIR_ZLO + p * OR_PAIR_PANEL, b = a + OR_PAIR_PANEL;
        double m = gl_integrate(g_pair, chi, a, b);
        half += m;
        if (zc >= b) below += m;
        else if (zc > a) below += gl_integrate(g_pair, chi, a, zc);
    }
    double c = below / (2.0 * half);
    return flip ? 1.0 - c : c;
}

/* Bilinear lookup in (log10 chi, s).  Reading: no extrapolation in chi (the
 * chi coordinate is clamped to the table); linear extrapolation in s beyond
 * +-16 from the end intervals. */
static double table_lookup(const double *tab, int nchi, int ns, double lchi0, double s0, double s_span,
                           double lchi, double s)
{
    double c = (lchi - lchi0) * 20.0;
    if (c < 0.0) c = 0.0;
    if (c > nchi - 1) c = nchi - 1;
    int i0 = (int)floor(c);
    if (i0 > nchi - 2) i0 = nchi - 2;
    double fc = c - i0;
    double t = (s - s0) * (ns - 1) / s_span;
    int j0 = (int)floor(t);
    if (j0 < 0) j0 = 0;
    if (j0 > ns - 2) j0 = ns - 2;
    double ft = t - j0;
    double a = tab[(size_t)i0 * ns + j0], b = tab[(size_t)i0 * ns + j0 + 1];
    double c2 = tab[(size_t)(i0 + 1) * ns + j0], d = tab[(size_t)(i0 + 1) * ns + j0 + 1];
    double lo = a + ft * (b - a), hi = c2 + ft * (d - c2);
    return lo + fc * (hi - lo);
}

/* Photon energy fraction for an emitter at chi with uniform u (Sec. 3).
 * Returns delta and writes 1 - delta without cancellation. */
double or_sample_emission(const double *icdf_em, double chi, double u, double *one_minus)
{
    double s = log(u) - log1p(-u);
    double zeta = table_lookup(icdf_em, OR_EM_NCHI, OR_EM_NS, -3.0, -OR_SMAX, 2.0 * OR_SMAX, log10(chi), s);
    double a = 3.0 * chi * exp(zeta);
    if (one_minus) *one_minus = 2.0 / (2.0 + a);
    return a / (2.0 + a);
}

/* Electron energy fraction for a photon at chi with uniform u (Sec. 3);
 * the spectrum is symmetric, so u > 1/2 maps to 1 - ICDF(1-u). */
double or_sample_pair(const double *icdf_pair, double chi, double u, double *one_minus)
{
    int flip = u > 0.5;
    double uu = flip ? 1.0 - u : u;
    double s = log(uu) - log1p(-uu);
    double ld = table_lookup(icdf_pair, OR_PAIR_NCHI, OR_PAIR_NS, -2.0, -OR_SMAX, OR_SMAX, log10(chi), s);
    double d = exp(ld);
    if (flip) { if (one_minus) *one_minus = d; return 1.0 - d; }
    if (one_minus) *one_minus = 1.0 - d;
    return d;
}

/* ================================================================== */
/* 6. Fields (Sec. 5.1 test problem; analytic field descriptors).       */
/* ================================================================== */
enum { OR_FIELD_UNIFORM = 0, OR_FIELD_ROTATING_E = 1, OR_FIELD_STANDING_CP = 2, OR_FIELD_GRID = 3 };

/* Gridded field (a PIC step's fields, held constant during the step):
 * node values E_x, E_y, E_z, B_x, B_y, B_z on a periodic nx x ny x nz grid
 * over [0, Lx) x [0, Ly) x [0, Lz), node (i, j, k) at (i Lx/nx, j Ly/ny,
 * k Lz/nz); layout [component][k][j][i].  prm = (nx, ny, nz, Lx, Ly, Lz).
 * Trilinear interpolation: linear in x along the four x-edges of the cell,
 * then in y, then in z; each lerp a + f (b - a) as one fused multiply-add. */
static const double *or_grid = NULL;

void or_set_field_grid(const double *g) { or_grid = g; }

static void grid_axis(double x, int n, double inv_h, int *i0, int *i1, double *f)
{
    const double u = x * inv_h;
    const double fl = floor(u);
    long long i = (long long)fl % n;
    if (i < 0) i += n;
    *i0 = (int)i;
    *i1 = (int)((i + 1) % n);
    *f = u - fl;
}

void or_field_grid(const double *prm, const double x[3], double E[3], double B[3])
{
    const int nx = (int)prm[0], ny = (int)prm[1], nz = (int)prm[2];
    int i0, i1, j0, j1, k0, k1;
    double fx, fy, fz;
    grid_axis(x[0], nx, (double)nx / prm[3], &i0, &i1, &fx);
    grid_axis(x[1], ny, (double)ny / prm[4], &j0, &j1, &fy);
    grid_axis(x[2], nz, (double)nz / prm[5], &k0, &k1, &fz);
    const long long plane = (long long)nx * ny, vol = plane * nz;
    for (int c = 0; c < 6; ++c) {
        const double *g = or_grid + c * vol;
        const double a00 = fma(fx, g[k0 * plane + j0 * nx + i1] - g[k0 * plane + j0 * nx + i0], g[k0 * plane + j0 * nx + i0]);
        const double a10 = fma(fx, g[k0 * plane + j1 * nx + i1] - g[k0 * plane + j1 * nx + i0], g[k0 * plane + j1 * nx + i0]);
        const double a01 = fma(fx, g[k1 * plane + j0 * nx + i1] - g[k1 * plane + j0 * nx + i0], g[k1 * plane + j0 * nx + i0]);
        const double a11 = fma(fx, g[k1 * plane + j1 * nx + i1] - g[k1 * plane + j1 * nx + i0], g[k1 * plane + j1 * nx + i0]);
        const double b0 = fma(fy, a10 - a00, a00);
        const double b1 = fma(fy, a11 - a01, a01);
        const double v = fma(fz, b1 - b0, b0);
        if (c < 3) E[c] = v; else B[c - 3] = v;
    }
}

void or_field(int kind, const double *prm, const double x[3], double t, double E[3], double B[3])
{
    if (kind == OR_FIELD_GRID) {
        or_field_grid(prm, x, E, B);
    } else if (kind == OR_FIELD_UNIFORM) {
        E[0] = prm[0]; E[1] = prm[1]; E[2] = prm[2];
        B[0] = prm[3]; B[1] = prm[4]; B[2] = prm[5];
    } else if (kind == OR_FIELD_ROTATING_E) {
        /* E = a0 (cos t, sin t, 0), B = 0 */
        E[0] = prm[0] * cos(t); E[1] = prm[0] * sin(t); E[2] = 0.0;
        B[0] = B[1] = B[2] = 0.0;
    } else {
        /* standing circularly polarised wave, E antinode at x = 0:
         * E = a0 cos x (0, cos t, sin t),  B = a0 sin x (0, cos t, sin t) */
        double ex = prm[0] * cos(x[0]), bx = prm[0] * sin(x[0]);
        E[0] = 0.0; E[1] = ex * cos(t); E[2] = ex * sin(t);
        B[0] = 0.0; B[1] = bx * cos(t); B[2] = bx * sin(t);
    }
}

/* ================================================================== */
/* 7. Quantum parameter chi (Algorithm 1, Calculate chi).               */
/*    lepton: chi = sqrt((gamma E + p x B)^2 - (p.E)^2) / R             */
/*    photon: the same with (k0, k) in place of (gamma, p).             */
/* ================================================================== */
double or_chi(double e0, const double p[3], const double E[3], const double B[3])
{
    double u0 = e0 * E[0] + (p[1] * B[2] - p[2] * B[1]);
    double u1 = e0 * E[1] + (p[2] * B[0] - p[0] * B[2]);
    double u2 = e0 * E[2] + (p[0] * B[1] - p[1] * B[0]);
    double pe = p[0] * E[0] + p[1] * E[1] + p[2] * E[2];
    double q = u0 * u0 + u1 * u1 + u2 * u2 - pe * pe;
    if (q < 0.0) q = 0.0;
    return sqrt(q) / OR_R;
}

/* ================================================================== */
/* 8. Boris push (Boris 1970), charge q = -1 (e-) or +1 (e+).           */
/*    half electric kick, magnetic rotation, half electric kick, then  */
/*    x += p/gamma * h with the new momentum.                           */
/* ================================================================== */
void or_boris(double x[3], double p[3], double q, const double E[3], const double B[3], double h)
{
    double pm[3], t[3], pp[3], s[3];
    for (int i = 0; i < 3; ++i) pm[i] = p[i] + 0.5 * q * h * E[i];
    double gm = sqrt(1.0 + pm[0] * pm[0] + pm[1] * pm[1] + pm[2] * pm[2]);
    for (int i = 0; i < 3; ++i) t[i] = 0.5 * q * h * B[i] / gm;
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int i = 0; i < 3; ++i) s[i] = 2.0 * t[i] / (1.0 + t2);
    double c0 = pm[1] * t[2] - pm[2] * t[1];
    double c1 = pm[2] * t[0] - pm[0] * t[2];
    double c2 = pm[0] * t[1] - pm[1] * t[0];
    pp[0] = pm[0] + c0; pp[1] = pm[1] + c1; pp[2] = pm[2] + c2;
    double d0 = pp[1] * s[2] - pp[2] * s[1];
    double d1 = pp[2] * s[0] - pp[0] * s[2];
    double d2 = pp[0] * s[1] - pp[1] * s[0];
    p[0] = pm[0] + d0 + 0.5 * q * h * E[0];
    p[1] = pm[1] + d1 + 0.5 * q * h * E[1];
    p[2] = pm[2] + d2 + 0.5 * q * h * E[2];
    double g = sqrt(1.0 + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    for (int i = 0; i < 3; ++i) x[i] += p[i] / g * h;
}

/* ================================================================== */
/* 9. Particle ensemble (Sec. 4.1: structure of arrays, one array set  */
/*    per particle type).                                               */
/* ================================================================== */
typedef struct {
    double *x, *y, *z, *px, *py, *pz, *w;
    uint64_t *id;
    uint32_t *nevents;
    double *od;                /* remaining optical depth (optical-depth method); may be NULL */
    int64_t count, capacity;
} or_species;

typedef struct {
    int push_photons;          /* 0: photons recorded, not pushed */
    int soft_photon_filter;    /* 1: drop emitted photons with energy < 2 m c^2 */
    int64_t thin_cap;          /* per species; 0 = off */
    uint64_t seed;
    int field_kind;
    double field_prm[16];
    int event_method;          /* 0: Algorithm 1 sub-stepping; 1: accumulated optical depth */
} or_run_cfg;

typedef struct {
    int64_t particle_steps, emit_events, pair_events;
    int64_t needed_capacity[3];
    int64_t max_subevents;
    int64_t overflow;
} or_stats;

/* one particle while it is being pushed through the step */
typedef struct {
    int sp;                    /* 0 e-, 1 e+, 2 photon */
    double x[3], p[3], w, tau, od;
    uint64_t id;
    uint32_t nevents, k;
    int64_t slot;              /* index in the ensemble, -1 for a newborn */
} or_particle;

typedef struct { or_particle *v; int64_t n, cap; } or_list;

static void list_add(or_list *l, const or_particle *q)
{
    if (l->n == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 16;
        l->v = (or_particle *)realloc(l->v, sizeof(or_particle) * l->cap);
    }
    l->v[l->n++] = *q;
}

typedef struct {
    const double *cheb_em, *cheb_pair, *icdf_em, *icdf_pair;
    const or_run_cfg *cfg;
    double dt, t_n;
    uint32_t step;
    or_stats *st;
} or_step_ctx;

static void philox_event(const or_step_ctx *c, uint64_t id, uint32_t k, uint64_t key64, uint32_t r[4])
{
    uint32_t ctr[4] = { (uint32_t)id, (uint32_t)(id >> 32), c->step, k };
    uint32_t key[2] = { (uint32_t)key64, (uint32_t)(key64 >> 32) };
    or_philox4x32_10(ctr, key, r);
}

/* Reading: children draw their 64-bit id from the same counter under the key
 * seed ^ 0xC0FFEE, so ids do not depend on the order of appends. */
#define OR_CHILD_KEY_XOR 0xC0FFEEull

/* Algorithm 1, ParticlePush, for e- / e+ (Sec. 3). */
static void lepton_push(const or_step_ctx *c, or_particle *P, or_list *photons)
{
    const or_run_cfg *cfg = c->cfg;
    double q = (P->sp == 0) ? -1.0 : 1.0;
    while (P->tau < c->dt) {
        double E[3], B[3];
        or_field(cfg->field_kind, cfg->field_prm, P->x, c->t_n + P->tau, E, B);
        double p2 = P->p[0] * P->p[0] + P->p[1] * P->p[1] + P->p[2] * P->p[2];
        double gamma = sqrt(1.0 + p2);
        double chi = or_chi(gamma, P->p, E, B);
        /* Reading: a lepton exactly at rest has no emission direction; rate 0 */
        double lambda = (p2 > 0.0) ? OR_ALPHA * OR_R / gamma * or_rate_F(c->cheb_em, c->cheb_pair, 0, chi) : 0.0;
        uint32_t r[4];
        double dt_hat;
        if (lambda > 0.0) {
            philox_event(c, P->id, P->k, cfg->seed, r);
            dt_hat = -log(or_u52(r[0], r[1])) / lambda;
        } else {
            dt_hat = INFINITY;
        }
        if (P->tau + dt_hat > c->dt) {
            or_boris(P->x, P->p, q, E, B, c->dt - P->tau);
            P->tau = c->dt;
        } else {
            or_boris(P->x, P->p, q, E, B, dt_hat);
            P->tau += dt_hat;
            /* Reading: chi for the energy draw is taken at the emission point */
            or_field(cfg->field_kind, cfg->field_prm, P->x, c->t_n + P->tau, E, B);
            double pm2 = P->p[0] * P->p[0] + P->p[1] * P->p[1] + P->p[2] * P->p[2];
            double g = sqrt(1.0 + pm2);
            double chi_e = or_chi(g, P->p, E, B);
            double one_m;
            double delta = or_sample_emission(c->icdf_em, chi_e, or_u52(r[2], r[3]), &one_m);
            /* Reading: energy-conserving, collinear recoil */
            double g_after = one_m * g;
            double k0 = delta * g;
            if (g_after < 1.0) { g_after = 1.0; k0 = g - 1.0; }
            double pabs = sqrt(pm2);
            double nx = P->p[0] / pabs, ny = P->p[1] / pabs, nz = P->p[2] / pabs;
            double pa = sqrt((g_after - 1.0) * (g_after + 1.0));
            or_particle ph;
            memset(&ph, 0, sizeof ph);
            ph.sp = 2;
            ph.x[0] = P->x[0]; ph.x[1] = P->x[1]; ph.x[2] = P->x[2];
            ph.p[0] = k0 * nx; ph.p[1] = k0 * ny; ph.p[2] = k0 * nz;
            ph.w = P->w; ph.tau = P->tau; ph.k = 0; ph.nevents = 0; ph.slot = -1;
            uint32_t rid[4];
            philox_event(c, P->id, P->k, cfg->seed ^ OR_CHILD_KEY_XOR, rid);
            ph.id = (uint64_t)rid[0] | ((uint64_t)rid[1] << 32);
            P->p[0] = pa * nx; P->p[1] = pa * ny; P->p[2] = pa * nz;
            P->k += 1;
            P->nevents += 1;
            c->st->emit_events += 1;
            if (!(cfg->soft_photon_filter && k0 < 2.0)) list_add(photons, &ph);
        }
    }
    if ((int64_t)P->k > c->st->max_subevents) c->st->max_subevents = P->k;
}

/* Photon push (Sec. 3: the same scheme; the photon is removed when it
 * creates a pair).  Straight-line motion at the speed of light. */
static void photon_push(const or_step_ctx *c, or_particle *G, or_list *leptons)
{
    const or_run_cfg *cfg = c->cfg;
    while (G->tau < c->dt && G->w > 0.0) {
        double E[3], B[3];
        or_field(cfg->field_kind, cfg->field_prm, G->x, c->t_n + G->tau, E, B);
        double k0 = sqrt(G->p[0] * G->p[0] + G->p[1] * G->p[1] + G->p[2] * G->p[2]);
        if (!(k0 > 0.0)) { G->tau = c->dt; break; }     /* a photon without momentum stays put */
        double chi = or_chi(k0, G->p, E, B);
        double lambda = OR_ALPHA * OR_R / k0 * or_rate_F(c->cheb_em, c->cheb_pair, 1, chi);
        uint32_t r[4];
        double dt_hat;
        if (lambda > 0.0) {
            philox_event(c, G->id, G->k, cfg->seed, r);
            dt_hat = -log(or_u52(r[0], r[1])) / lambda;
        } else {
            dt_hat = INFINITY;
        }
        double nx = G->p[0] / k0, ny = G->p[1] / k0, nz = G->p[2] / k0;
        if (G->tau + dt_hat > c->dt) {
            double h = c->dt - G->tau;
            G->x[0] += nx * h; G->x[1] += ny * h; G->x[2] += nz * h;
            G->tau = c->dt;
        } else {
            G->x[0] += nx * dt_hat; G->x[1] += ny * dt_hat; G->x[2] += nz * dt_hat;
            G->tau += dt_hat;
            or_field(cfg->field_kind, cfg->field_prm, G->x, c->t_n + G->tau, E, B);
            double chi_e = or_chi(k0, G->p, E, B);
            double one_m;
            double delta = or_sample_pair(c->icdf_pair, chi_e, or_u52(r[2], r[3]), &one_m);
            /* Reading: both leptons along k, energies delta k0 and (1-delta) k0,
             * each at least m c^2 */
            double em = delta * k0, ep = one_m * k0;
            if (em < 1.0) em = 1.0;
            if (ep < 1.0) ep = 1.0;
            double pm = sqrt((em - 1.0) * (em + 1.0)), pp = sqrt((ep - 1.0) * (ep + 1.0));
            uint32_t rid[4];
            philox_event(c, G->id, G->k, cfg->seed ^ OR_CHILD_KEY_XOR, rid);
            or_particle a, b;
            memset(&a, 0, sizeof a); memset(&b, 0, sizeof b);
            a.sp = 0; b.sp = 1;
            for (int i = 0; i < 3; ++i) { a.x[i] = G->x[i]; b.x[i] = G->x[i]; }
            a.p[0] = pm * nx; a.p[1] = pm * ny; a.p[2] = pm * nz;
            b.p[0] = pp * nx; b.p[1] = pp * ny; b.p[2] = pp * nz;
            a.w = b.w = G->w; a.tau = b.tau = G->tau; a.slot = b.slot = -1;
            a.id = (uint64_t)rid[0] | ((uint64_t)rid[1] << 32);
            b.id = (uint64_t)rid[2] | ((uint64_t)rid[3] << 32);
            G->k += 1;
            G->nevents += 1;
            G->w = 0.0;                 /* the photon is eliminated */
            c->st->pair_events += 1;
            list_add(leptons, &a);
            list_add(leptons, &b);
        }
    }
    if ((int64_t)G->k > c->st->max_subevents) c->st->max_subevents = G->k;
}

static void load_particle(or_species *S, int sp, int64_t i, or_particle *P)
{
    memset(P, 0, sizeof *P);
    P->sp = sp;
    P->x[0] = S->x[i]; P->x[1] = S->y[i]; P->x[2] = S->z[i];
    P->p[0] = S->px[i]; P->p[1] = S->py[i]; P->p[2] = S->pz[i];
    P->w = S->w[i]; P->id = S->id[i]; P->nevents = S->nevents[i];
    P->od = S->od ? S->od[i] : 0.0;
    P->tau = 0.0; P->k = 0; P->slot = i;
}

static void store_particle(or_species *S, int64_t i, const or_particle *P)
{
    S->x[i] = P->x[0]; S->y[i] = P->x[1]; S->z[i] = P->x[2];
    S->px[i] = P->p[0]; S->py[i] = P->p[1]; S->pz[i] = P->p[2];
    S->w[i] = P->w; S->id[i] = P->id; S->nevents[i] = P->nevents;
    if (S->od) S->od[i] = P->od;
}

/* Returns 0, or 2 when a species ran out of capacity (needed_capacity set). */
static int append_particle(or_species *sp, const or_particle *P, or_stats *st)
{
    or_species *S = &sp[P->sp];
    if (S->count >= S->capacity) {
        st->overflow = 1;
        if (S->count + 1 > st->needed_capacity[P->sp]) st->needed_capacity[P->sp] = S->count + 1;
        S->count += 1;        /* keep counting the demand; nothing is written */
        return 2;
    }
    store_particle(S, S->count, P);
    S->count += 1;
    return 0;
}

/* Algorithm 2, RunAvalanche: push one particle and everything it creates to
 * the end of the step, then save the newborns into the ensemble. */
static int run_avalanche(const or_step_ctx *c, or_species *sp, int species, int64_t i)
{
    or_list leptons = {0}, photons = {0};
    or_particle P;
    load_particle(&sp[species], species, i, &P);
    if (species == 2) list_add(&photons, &P); else list_add(&leptons, &P);
    int64_t cl = 0, cp = 0;
    while (cl != leptons.n || cp != photons.n) {
        for (int64_t k = cl; k < leptons.n; ++k) {
            c->st->particle_steps += 1;
            lepton_push(c, &leptons.v[k], &photons);
        }
        cl = leptons.n;
        for (int64_t k = cp; k < photons.n; ++k) {
            if (c->cfg->push_photons) {
                c->st->particle_steps += 1;
                photon_push(c, &photons.v[k], &leptons);
            }
        }
        cp = photons.n;
    }
    /* SaveGeneratedParticles */
    int rc = 0;
    or_particle *orig = (species == 2) ? &photons.v[0] : &leptons.v[0];
    store_particle(&sp[species], i, orig);
    for (int64_t k = 0; k < leptons.n; ++k)
        if (leptons.v[k].slot < 0 && append_particle(sp, &leptons.v[k], c->st)) rc = 2;
    for (int64_t k = 0; k < photons.n; ++k)
        if (photons.v[k].slot < 0 && append_particle(sp, &photons.v[k], c->st)) rc = 2;
    free(leptons.v); free(photons.v);
    return rc;
}

/* ------------------------------------------------------------------ */
/* The accumulated optical-depth scheme (Sec. 3, the inverse-sampling  */
/* method used by other PIC codes, no sub-cycling).  Reading: the rate */
/* is taken once, at the start of the step; the optical depth d falls  */
/* by lambda * dt (first-order Euler); a particle whose d reaches 0    */
/* has its event at the end of the step (chi at the end point) and     */
/* draws a fresh d.  At most one event per particle and step; the      */
/* children start at the next step with d not drawn yet (0).  A d that  */
/* is not positive on entry is drawn first, from counter word 3 =       */
/* 0xFFFFFFFE; the event uses word 3 = 0 (words 0-1: the new d, 2-3:    */
/* the energy), child ids as in Algorithm 1.                            */
/* ------------------------------------------------------------------ */
#define OR_OD_DRAW 0xFFFFFFFEu

static double od_initial(const or_step_ctx *c, uint64_t id)
{
    uint32_t r[4];
    philox_event(c, id, OR_OD_DRAW, c->cfg->seed, r);
    return -log(or_u52(r[0], r[1]));
}

static void lepton_step_od(const or_step_ctx *c, or_species *sp, int species, int64_t i, int *rc)
{
    const or_run_cfg *cfg = c->cfg;
    or_particle P;
    load_particle(&sp[species], species, i, &P);
    double q = (species == 0) ? -1.0 : 1.0;
    double E[3], B[3];
    or_field(cfg->field_kind, cfg->field_prm, P.x, c->t_n, E, B);
    double p2 = P.p[0] * P.p[0] + P.p[1] * P.p[1] + P.p[2] * P.p[2];
    double gamma = sqrt(1.0 + p2);
    double chi = or_chi(gamma, P.p, E, B);
    double lambda = (p2 > 0.0) ? OR_ALPHA * OR_R / gamma * or_rate_F(c->cheb_em, c->cheb_pair, 0, chi) : 0.0;
    if (!(P.od > 0.0)) P.od = od_initial(c, P.id);
    P.od -= lambda * c->dt;
    or_boris(P.x, P.p, q, E, B, c->dt);
    c->st->particle_steps += 1;
    if (P.od <= 0.0) {
        uint32_t r[4];
        philox_event(c, P.id, 0, cfg->seed, r);
        or_field(cfg->field_kind, cfg->field_prm, P.x, c->t_n + c->dt, E, B);
        double pm2 = P.p[0] * P.p[0] + P.p[1] * P.p[1] + P.p[2] * P.p[2];
        double g = sqrt(1.0 + pm2);
        double one_m;
        double delta = or_sample_emission(c->icdf_em, or_chi(g, P.p, E, B), or_u52(r[2], r[3]), &one_m);
        double g_after = one_m * g, k0 = delta * g;
        if (g_after < 1.0) { g_after = 1.0; k0 = g - 1.0; }
        double pabs = sqrt(pm2);
        double nx = P.p[0] / pabs, ny = P.p[1] / pabs, nz = P.p[2] / pabs;
        double pa = sqrt((g_after - 1.0) * (g_after + 1.0));
        if (!(cfg->soft_photon_filter && k0 < 2.0)) {
            or_particle ph;
            memset(&ph, 0, sizeof ph);         /* od = 0: drawn at its first step */
            ph.sp = 2;
            for (int d = 0; d < 3; ++d) ph.x[d] = P.x[d];
            ph.p[0] = k0 * nx; ph.p[1] = k0 * ny; ph.p[2] = k0 * nz;
            ph.w = P.w; ph.slot = -1;
            uint32_t rid[4];
            philox_event(c, P.id, 0, cfg->seed ^ OR_CHILD_KEY_XOR, rid);
            ph.id = (uint64_t)rid[0] | ((uint64_t)rid[1] << 32);
            if (append_particle(sp, &ph, c->st)) *rc = 2;
        }
        P.p[0] = pa * nx; P.p[1] = pa * ny; P.p[2] = pa * nz;
        P.od = -log(or_u52(r[0], r[1]));
        P.nevents += 1;
        c->st->emit_events += 1;
        if (c->st->max_subevents < 1) c->st->max_subevents = 1;
    }
    store_particle(&sp[species], i, &P);
}

static void photon_step_od(const or_step_ctx *c, or_species *sp, int64_t i, int *rc)
{
    const or_run_cfg *cfg = c->cfg;
    or_particle G;
    load_particle(&sp[2], 2, i, &G);
    c->st->particle_steps += 1;
    double k0 = sqrt(G.p[0] * G.p[0] + G.p[1] * G.p[1] + G.p[2] * G.p[2]);
    if (!(k0 > 0.0)) return;                    /* a photon without momentum stays put */
    double E[3], B[3];
    or_field(cfg->field_kind, cfg->field_prm, G.x, c->t_n, E, B);
    double lambda = OR_ALPHA * OR_R / k0 * or_rate_F(c->cheb_em, c->cheb_pair, 1, or_chi(k0, G.p, E, B));
    if (!(G.od > 0.0)) G.od = od_initial(c, G.id);
    G.od -= lambda * c->dt;
    double nx = G.p[0] / k0, ny = G.p[1] / k0, nz = G.p[2] / k0;
    G.x[0] += nx * c->dt; G.x[1] += ny * c->dt; G.x[2] += nz * c->dt;
    if (G.od <= 0.0) {
        uint32_t r[4], rid[4];
        philox_event(c, G.id, 0, cfg->seed, r);
        or_field(cfg->field_kind, cfg->field_prm, G.x, c->t_n + c->dt, E, B);
        double one_m;
        double delta = or_sample_pair(c->icdf_pair, or_chi(k0, G.p, E, B), or_u52(r[2], r[3]), &one_m);
        double em = delta * k0, ep = one_m * k0;
        if (em < 1.0) em = 1.0;
        if (ep < 1.0) ep = 1.0;
        double pm = sqrt((em - 1.0) * (em + 1.0)), pp = sqrt((ep - 1.0) * (ep + 1.0));
        philox_event(c, G.id, 0, cfg->seed ^ OR_CHILD_KEY_XOR, rid);
        or_particle a, b;
        memset(&a, 0, sizeof a); memset(&b, 0, sizeof b);
        a.sp = 0; b.sp = 1;
        for (int d = 0; d < 3; ++d) { a.x[d] = G.x[d]; b.x[d] = G.x[d]; }
        a.p[0] = pm * nx; a.p[1] = pm * ny; a.p[2] = pm * nz;
        b.p[0] = pp * nx; b.p[1] = pp * ny; b.p[2] = pp * nz;
        a.w = b.w = G.w; a.slot = b.slot = -1;
        a.id = (uint64_t)rid[0] | ((uint64_t)rid[1] << 32);
        b.id = (uint64_t)rid[2] | ((uint64_t)rid[3] << 32);
        if (append_particle(sp, &a, c->st)) *rc = 2;
        if (append_particle(sp, &b, c->st)) *rc = 2;
        G.w = 0.0;                      /* the photon is eliminated */
        G.nevents += 1;
        c->st->pair_events += 1;
        if (c->st->max_subevents < 1) c->st->max_subevents = 1;
    }
    store_particle(&sp[2], i, &G);
}

/* Stable removal of dead entries (weight 0), Sec. 4.2 merge step. */
void or_compact(or_species *S)
{
    int64_t n = 0;
    for (int64_t i = 0; i < S->count; ++i) {
        if (S->w[i] > 0.0) {
            if (n != i) {
                S->x[n] = S->x[i]; S->y[n] = S->y[i]; S->z[n] = S->z[i];
                S->px[n] = S->px[i]; S->py[n] = S->py[i]; S->pz[n] = S->pz[i];
                S->w[n] = S->w[i]; S->id[n] = S->id[i]; S->nevents[n] = S->nevents[i];
                if (S->od) S->od[n] = S->od[i];
            }
            ++n;
        }
    }
    S->count = n;
}

/* ================================================================== */
/* 10. Global leveling (Sec. 1 and Sec. 5.1 name it, after Muraviev et */
/*     al. 2021).  Reading: when the count N exceeds the cap C, find    */
/*     the threshold w* with  sum_i min(1, w_i / w*) = C, keep particle */
/*     i with probability min(1, w_i / w*) (Philox, counter word 3 =    */
/*     0xFFFFFFFF), and raise kept particles below w* to w*.            */
/*     Returns w* (0 when nothing was done).                            */
/* ================================================================== */
double or_level_threshold(const double *w, int64_t n, int64_t cap)
{
    int64_t alive = 0;
    double wmax = 0.0;
    for (int64_t i = 0; i < n; ++i) if (w[i] > 0.0) { ++alive; if (w[i] > wmax) wmax = w[i]; }
    if (cap <= 0 || alive <= cap) return 0.0;
    double lo = 0.0, hi = wmax * (double)alive / (double)cap;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        /* Neumaier compensated sum, so that the computed sum is accurate to
         * working precision and the root is that of the defining equation */
        double s = 0.0, comp = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            if (!(w[i] > 0.0)) continue;
            double term = (w[i] < mid) ? w[i] / mid : 1.0;
            double t = s + term;
            if (fabs(s) >= fabs(term)) comp += (s - t) + term;
            else comp += (term - t) + s;
            s = t;
        }
        s += comp;
        if (s > (double)cap) lo = mid; else hi = mid;
    }
    return hi;
}

double or_level(or_species *S, int64_t cap, uint64_t seed, uint32_t step)
{
    double ws = or_level_threshold(S->w, S->count, cap);
    if (ws <= 0.0) return 0.0;
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (int64_t i = 0; i < S->count; ++i) {
        if (!(S->w[i] > 0.0) || S->w[i] >= ws) continue;
        uint32_t ctr[4] = { (uint32_t)S->id[i], (uint32_t)(S->id[i] >> 32), step, 0xFFFFFFFFu }, r[4];
        or_philox4x32_10(ctr, key, r);
        double u = or_u52(r[0], r[1]);
        if (u < S->w[i] / ws) S->w[i] = ws;
        else S->w[i] = 0.0;
    }
    or_compact(S);
    return ws;
}

/* ================================================================== */
/* 11. nsteps PIC steps of the QED pusher over the whole ensemble.     */
/*     Per step: every particle present at the start of the step runs  */
/*     Algorithm 2; newborns are saved after each avalanche; dead      */
/*     photons are removed; leveling applies per species above the cap. */
/*     Returns 0, or 2 on capacity overflow (the step still completes,  */
/*     children that did not fit are dropped and counted).              */
/* ================================================================== */
int or_push_and_generate(or_species *sp /* [3] */, const double *cheb_em, const double *cheb_pair,
                         const double *icdf_em, const double *icdf_pair, const or_run_cfg *cfg,
                         double dt, int nsteps, int64_t step0, or_stats *st)
{
    int rc = 0;
    for (int s = 0; s < nsteps; ++s) {
        or_step_ctx c;
        c.cheb_em = cheb_em; c.cheb_pair = cheb_pair; c.icdf_em = icdf_em; c.icdf_pair = icdf_pair;
        c.cfg = cfg; c.dt = dt; c.st = st;
        int64_t step = step0 + s;
        c.step = (uint32_t)step;
        c.t_n = (double)step * dt;
        int64_t n0[3] = { sp[0].count, sp[1].count, sp[2].count };
        for (int species = 0; species < 3; ++species) {
            if (species == 2 && !cfg->push_photons) continue;
            for (int64_t i = 0; i < n0[species]; ++i) {
                if (!(sp[species].w[i] > 0.0)) continue;
                if (cfg->event_method == 1) {
                    if (species == 2) photon_step_od(&c, sp, i, &rc);
                    else lepton_step_od(&c, sp, species, i, &rc);
                } else if (run_avalanche(&c, sp, species, i)) {
                    rc = 2;
                }
            }
        }
        if (rc) return rc;
        if (cfg->push_photons) or_compact(&sp[2]);
        if (cfg->thin_cap > 0)
            for (int species = 0; species < 3; ++species) or_level(&sp[species], cfg->thin_cap, cfg->seed, c.step);
    }
    return rc;
}

/* Single-particle helpers exported for the tests. */
double or_rate_lambda(const double *cheb_em, const double *cheb_pair, int is_photon, const double p[3],
                      const double E[3], const double B[3])
{
    double p2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    double e0 = is_photon ? sqrt(p2) : sqrt(1.0 + p2);
    double chi = or_chi(e0, p, E, B);
    if (!(p2 > 0.0)) return 0.0;
    return OR_ALPHA * OR_R / e0 * or_rate_F(cheb_em, cheb_pair, is_photon, chi);
}

/* ================================================================== */
/* 11. Independent cross-check: the subcycled rejection generator.     */
/*     The classic alternative to Algorithm 1 (Sec. 2): the step is     */
/*     split into nsub sub-steps h; in each, a candidate photon energy  */
/*     fraction delta = r^3 (r uniform; the substitution keeps the      */
/*     acceptance bounded although dW/d delta ~ delta^(-2/3) at small   */
/*     delta) is accepted with probability 3 r^2 (dW/d delta) h, the    */
/*     differential LCFA rate evaluated from the Bessel functions       */
/*     directly (no rate approximant, no inverse-CDF table).  Then the  */
/*     lepton is Boris-pushed by h.  Photons are recorded, not pushed.  */
/*     Its own random stream (splitmix64 per particle), so the          */
/*     comparison with Algorithm 1 is statistical.                      */
/* ================================================================== */
static uint64_t splitmix64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double splitmix_u(uint64_t *s) { return ((double)(splitmix64(s) >> 11) + 0.5) * 0x1p-53; }

/* Electrons of E (species 0) only.  Returns the number of emissions; fills
 * delta_out[0..min(n, cap)) with the photon energies (m c^2) and max_accept
 * with the largest acceptance probability met (it must stay well below 1
 * for the method to hold). */
int64_t or_rejection_run(or_species *E, const or_run_cfg *cfg, double dt, int nsteps, int nsub, uint64_t seed,
                         double *delta_out, int64_t delta_cap, double *max_accept)
{
    const double h = dt / nsub;
    const double pref = OR_ALPHA * OR_R / (sqrt(3.0) * M_PI);
    int64_t nev = 0;
    double amax = 0.0;
    for (int64_t i = 0; i < E->count; ++i) {
        uint64_t st = seed ^ (E->id[i] * 0xD1B54A32D192ED03ull);
        double x[3] = { E->x[i], E->y[i], E->z[i] }, p[3] = { E->px[i], E->py[i], E->pz[i] };
        for (int s = 0; s < nsteps; ++s) {
            for (int k = 0; k < nsub; ++k) {
                const double t = (s + (double)k / nsub) * dt;
                double Ef[3], Bf[3];
                or_field(cfg->field_kind, cfg->field_prm, x, t, Ef, Bf);
                const double p2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
                const double gamma = sqrt(1.0 + p2);
                const double chi = or_chi(gamma, p, Ef, Bf);
                const double r = splitmix_u(&st), u = splitmix_u(&st);
                if (p2 > 0.0 && chi > 0.0) {
                    const double delta = r * r * r;
                    const double a = 3.0 * r * r * pref / gamma * or_em_bracket(chi, delta) * h;
                    if (a > amax) amax = a;
                    if (u < a) {
                        /* the same energy-conserving collinear recoil as Algorithm 1 */
                        double g_after = (1.0 - delta) * gamma;
                        if (g_after < 1.0) g_after = 1.0;
                        const double pa = sqrt((g_after - 1.0) * (g_after + 1.0)), inv = 1.0 / sqrt(p2);
                        for (int d = 0; d < 3; ++d) p[d] = pa * p[d] * inv;
                        if (nev < delta_cap) delta_out[nev] = gamma - g_after;   /* photon energy */
                        ++nev;
                    }
                }
                or_boris(x, p, -1.0, Ef, Bf, h);              /* electrons */
            }
        }
        E->x[i] = x[0]; E->y[i] = x[1]; E->z[i] = x[2];
        E->px[i] = p[0]; E->py[i] = p[1]; E->pz[i] = p[2];
    }
    if (max_accept) *max_accept = amax;
    return nev;
}

double or_const(int which)
{
    switch (which) {
    case 0: return OR_ALPHA;
    case 1: return OR_R;
    default: return 0.0;
    }
}

/* ================================================================== */
/* 12. Surrogate of the emission inverse CDF (an extension: the paper  */
/*     samples energies from tables only).  A network                  */
/*     2 -> 64 -> 64 -> 64 -> 1 with SiLU on the hidden layers maps     */
/*     features (log10(chi)/3, logit(u)/16) to zeta/16 + 1/2, where     */
/*     zeta = ln y is the quantity the emission table stores.           */
/*     Parameter layout: W1[64][2], b1[64], W2[64][64], b2[64],         */
/*     W3[64][64], b3[64], W4[64], b4 (8577 numbers, W[out][in]).       */
/*     Plain forward pass and backward pass of the mean squared error.  */
/* ================================================================== */
#define OR_MLP_H 64
#define OR_MLP_NP (OR_MLP_H * 2 + OR_MLP_H + 2 * (OR_MLP_H * OR_MLP_H + OR_MLP_H) + OR_MLP_H + 1)

static double or_silu(double z) { return z / (1.0 + exp(-z)); }
static double or_dsilu(double z) { double s = 1.0 / (1.0 + exp(-z)); return s * (1.0 + z * (1.0 - s)); }

int or_mlp_nparams(void) { return OR_MLP_NP; }

/* The storage rounding of a network that keeps its hidden activations and
   back-propagated deltas as bfloat16: the value rounded to single precision,
   then to bfloat16 (8 significand bits, nearest, ties to even).  qz = 0 is
   the exact network (no rounding). */
static double or_q(double v, int qz)
{
    if (!qz) return v;
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    if ((u & 0x7f800000u) != 0x7f800000u) {
        u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
        memcpy(&f, &u, sizeof f);
    }
    return (double)f;
}

/* one sample: pre-activations z1..z3 and activations h1..h3 (activations
   stored with the rounding qz) */
static double mlp_one_r(const double *P, const double f[2], double z[3][OR_MLP_H], double h[3][OR_MLP_H], int qz)
{
    const double *W1 = P, *b1 = W1 + 2 * OR_MLP_H;
    const double *W2 = b1 + OR_MLP_H, *b2 = W2 + OR_MLP_H * OR_MLP_H;
    const double *W3 = b2 + OR_MLP_H, *b3 = W3 + OR_MLP_H * OR_MLP_H;
    const double *W4 = b3 + OR_MLP_H, *b4 = W4 + OR_MLP_H;
    for (int o = 0; o < OR_MLP_H; ++o) {
        z[0][o] = W1[2 * o] * f[0] + W1[2 * o + 1] * f[1] + b1[o];
        h[0][o] = or_q(or_silu(z[0][o]), qz);
    }
    for (int o = 0; o < OR_MLP_H; ++o) {
        double s = b2[o];
        for (int i = 0; i < OR_MLP_H; ++i) s += W2[o * OR_MLP_H + i] * h[0][i];
        z[1][o] = s;
        h[1][o] = or_q(or_silu(s), qz);
    }
    for (int o = 0; o < OR_MLP_H; ++o) {
        double s = b3[o];
        for (int i = 0; i < OR_MLP_H; ++i) s += W3[o * OR_MLP_H + i] * h[1][i];
        z[2][o] = s;
        h[2][o] = or_q(or_silu(s), qz);
    }
    double y = b4[0];
    for (int i = 0; i < OR_MLP_H; ++i) y += W4[i] * h[2][i];
    return y;
}

static double mlp_one(const double *P, const double f[2], double z[3][OR_MLP_H], double h[3][OR_MLP_H])
{
    return mlp_one_r(P, f, z, h, 0);
}

static void mlp_forward_r(const double *P, int64_t n, const double *feat, double *y, int qz)
{
    double z[3][OR_MLP_H], h[3][OR_MLP_H];
    for (int64_t k = 0; k < n; ++k) y[k] = mlp_one_r(P, feat + 2 * k, z, h, qz);
}

void or_mlp_forward(const double *P, int64_t n, const double *feat /* n x 2 */, double *y)
{
    mlp_forward_r(P, n, feat, y, 0);
}

/* The network with bfloat16 storage of its activations (as a kernel that
   stores them in that format computes it). */
void or_mlp_forward_q(const double *P, int64_t n, const double *feat, double *y)
{
    mlp_forward_r(P, n, feat, y, 1);
}

static double mlp_loss_grad_r(const double *P, int64_t n, const double *feat, const double *t, double *g, int qz);

/* loss = mean_k (y_k - t_k)^2; g = d loss / d P */
double or_mlp_loss_grad(const double *P, int64_t n, const double *feat, const double *t, double *g)
{
    return mlp_loss_grad_r(P, n, feat, t, g, 0);
}

/* The same with bfloat16 storage of the activations h1..h3 and of the
   back-propagated deltas d3, d2, d1 (the products and sums stay exact). */
double or_mlp_loss_grad_q(const double *P, int64_t n, const double *feat, const double *t, double *g)
{
    return mlp_loss_grad_r(P, n, feat, t, g, 1);
}

static double mlp_loss_grad_r(const double *P, int64_t n, const double *feat, const double *t, double *g, int qz)
{
    const double *W1 = P, *b1 = W1 + 2 * OR_MLP_H;
    const double *W2 = b1 + OR_MLP_H, *b2 = W2 + OR_MLP_H * OR_MLP_H;
    const double *W3 = b2 + OR_MLP_H, *b3 = W3 + OR_MLP_H * OR_MLP_H;
    const double *W4 = b3 + OR_MLP_H;
    (void)b2; (void)b3; (void)b1;
    double *gW1 = g, *gb1 = gW1 + 2 * OR_MLP_H;
    double *gW2 = gb1 + OR_MLP_H, *gb2 = gW2 + OR_MLP_H * OR_MLP_H;
    double *gW3 = gb2 + OR_MLP_H, *gb3 = gW3 + OR_MLP_H * OR_MLP_H;
    double *gW4 = gb3 + OR_MLP_H, *gb4 = gW4 + OR_MLP_H;
    memset(g, 0, sizeof(double) * OR_MLP_NP);
    double loss = 0.0;
    double z[3][OR_MLP_H], h[3][OR_MLP_H], d3[OR_MLP_H], d2[OR_MLP_H], d1[OR_MLP_H];
    for (int64_t k = 0; k < n; ++k) {
        const double *f = feat + 2 * k;
        double y = mlp_one_r(P, f, z, h, qz);
        double r = y - t[k];
        loss += r * r;
        double dy = 2.0 * r / (double)n;
        gb4[0] += dy;
        for (int i = 0; i < OR_MLP_H; ++i) {
            gW4[i] += dy * h[2][i];
            d3[i] = or_q(dy * W4[i] * or_dsilu(z[2][i]), qz);
        }
        for (int o = 0; o < OR_MLP_H; ++o) {
            gb3[o] += d3[o];
            for (int i = 0; i < OR_MLP_H; ++i) gW3[o * OR_MLP_H + i] += d3[o] * h[1][i];
        }
        for (int i = 0; i < OR_MLP_H; ++i) {
            double s = 0.0;
            for (int o = 0; o < OR_MLP_H; ++o) s += W3[o * OR_MLP_H + i] * d3[o];
            d2[i] = or_q(s * or_dsilu(z[1][i]), qz);
        }
        for (int o = 0; o < OR_MLP_H; ++o) {
            gb2[o] += d2[o];
            for (int i = 0; i < OR_MLP_H; ++i) gW2[o * OR_MLP_H + i] += d2[o] * h[0][i];
        }
        for (int i = 0; i < OR_MLP_H; ++i) {
            double s = 0.0;
            for (int o = 0; o < OR_MLP_H; ++o) s += W2[o * OR_MLP_H + i] * d2[o];
            d1[i] = or_q(s * or_dsilu(z[0][i]), qz);
        }
        for (int o = 0; o < OR_MLP_H; ++o) {
            gb1[o] += d1[o];
            gW1[2 * o] += d1[o] * f[0];
            gW1[2 * o + 1] += d1[o] * f[1];
        }
    }
    return loss / (double)n;
}

/* Features and target of the surrogate (the reading that defines it). */
void or_mlp_features(double chi, double u, double f[2])
{
    double s = log(u) - log1p(-u);
    if (s > OR_SMAX) s = OR_SMAX;
    if (s < -OR_SMAX) s = -OR_SMAX;
    f[0] = log10(chi) / 3.0;
    f[1] = s / OR_SMAX;
}

/* photon energy fraction from a network output y (zeta = 16 (y - 1/2)) */
double or_mlp_delta(double chi, double y, double *one_minus)
{
    double zeta = 16.0 * (y - 0.5);
    double a = 3.0 * chi * exp(zeta);
    if (one_minus) *one_minus = 2.0 / (2.0 + a);
    return a / (2.0 + a);
}
