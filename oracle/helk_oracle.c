/*
 * helk_oracle.c -- plain, slow FP64 CPU oracle for the HELIOS-K hot path
 * (Grimm & Heng 2015, "HELIOS-K: an ultrafast, open-source opacity
 * calculator for radiative transfer", arXiv:1503.03806).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path (the
 * CUDA library of the paper_1503_03806_gb300 package) shares no code, header,
 * table or constant generator with this file.
 *
 * Built with `gcc -O2 -ffp-contract=off` so that every + - * / is a single
 * correctly rounded IEEE operation in the order written here.
 *
 * What is pinned, and by what, is listed in oracle/__init__.py.  Every
 * function here has at least one pin that does not re-use its own formula
 * (closed forms, mpmath, numpy/scipy library routines, brute force).
 *
 * Readings of the paper taken here (where it is silent or garbled):
 *  - Sec. 2.3 Voigt profile: the integrand is exp(-u'^2) (the printed sign is
 *    lost); Gamma_D uses the shifted line centre.
 *  - Sec. 2.4: region thresholds are inclusive on the cheaper method:
 *    a^2+u^2 >= 100 -> 3-point Gauss-Hermite, >= 1e6 -> 1-point rule.
 *  - "Third-order Gauss-Hermite" = the 3-node rule (nodes 0, +-sqrt(3/2)).
 *  - Algorithm 916 is the series form of Re w(x+iy) derived in
 *    or_K916 below with step h = 1/2 (the cited paper is not available).
 *  - Line-wing cutoff: inclusive |nu_i - nu0'| <= C realised as integer
 *    window bounds; no renormalisation of the truncated profile.
 *  - k-distribution abscissa: g_j = (j + 1/2)/N_b (midpoint of each interval
 *    dy = 1/N_nu of Sec. 2.2); ln is taken of max(kappa, kappa_floor).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ---------------------------------------------------------------------
 * Constants (CGS).  CODATA 2018 exact SI values; T0 = 296 K (Sec. 2.3).
 * ------------------------------------------------------------------- */
#define OR_KB        1.380649e-16                 /* erg / K           */
#define OR_CLIGHT    2.99792458e10                /* cm / s            */
#define OR_AMU       1.66053906660e-24            /* g                 */
#define OR_C2        1.4387768775039338021        /* h c / k_B, cm K   */
#define OR_T0        296.0                        /* K                 */
#define OR_PI        3.1415926535897932384626
#define OR_LN2       0.69314718055994530941723
#define OR_SQRTLN2   0.83255461115769775635316    /* sqrt(ln 2)        */
#define OR_SQRTLN2PI 0.46971863934982566688617    /* sqrt(ln 2 / pi)   */
#define OR_SQRTPI    1.7724538509055160272982     /* sqrt(pi)          */
#define OR_GH3_T     1.2247448713915890490986     /* sqrt(3/2)         */

/* Region thresholds on r^2 = a^2 + u^2 (Sec. 2.4). */
#define OR_R2_GH3    100.0
#define OR_R2_GH1    1.0e6

/* Algorithm 916 series step and number of terms (see or_K916). */
#define OR_A916_H     0.5
#define OR_A916_NTERM 40

/* Cutoff kinds (Sec. 2.4): absolute, multiple of Gamma_L capped, none. */
#define OR_CUT_ABS     0
#define OR_CUT_LORENTZ 1
#define OR_CUT_NONE    2

/* =====================================================================
 * Voigt function H_V(a,u) = Re w(u + i a)   (Sec. 2.3, Eq. for H_V)
 * ===================================================================== */

/* erfcx(y) = exp(y^2) erfc(y), from libm, for 0 <= y < 10 (the only range
 * the core region reaches). */
static double or_erfcx(double y) { return exp(y * y) * erfc(y); }

/*
 * Algorithm 916 (Sec. 2.4): Re w(x + i y) for y >= 0 written with a scaled
 * complementary error function, cosines/sines and three exponentially
 * weighted series that share one loop.
 *
 * Derivation (our own, from w(z) = (i/pi) int e^{-t^2}/(z-t) dt): shift the
 * integration variable by x, subtract the function e^{-x^2} e^{-2ixy}
 * e^{-s^2}/(s - iy) whose integral is e^{-x^2} e^{-2ixy} erfcx(y) and whose
 * pole cancels that of the integrand, and apply the trapezoidal rule with
 * step h to the remaining entire function.  Its aliasing error is of order
 * exp(-pi^2/h^2) ~ 7e-18 for h = 1/2.  The real part is
 *
 *   K(x,y) = e^{-x^2} erfcx(y) cos(2xy)
 *          + (2 h x / pi) e^{-x^2} sin(xy) sinc(xy)
 *          + (2 h / pi) [ -y cos(2xy) e^{-x^2} S1 + (y/2) S2 + (y/2) S3 ]
 *
 *   S1 = sum_{n>=1} e^{-(nh)^2}    / ((nh)^2 + y^2)
 *   S2 = sum_{n>=1} e^{-(nh+x)^2}  / ((nh)^2 + y^2)
 *   S3 = sum_{n>=1} e^{-(nh-x)^2}  / ((nh)^2 + y^2)
 *
 * The oracle sums a fixed 40 terms (nh up to 20); for |x| < 10 every
 * omitted term is below e^{-100} of the largest one.
 */
double or_K916(double x, double y)
{
    const double h = OR_A916_H;
    double ex2, xy, sinc, c2xy, s1 = 0.0, s2 = 0.0, s3 = 0.0, K;
    int n;
    if (x < 0.0) x = -x;                        /* K is even in x */
    ex2  = exp(-(x * x));
    xy   = x * y;
    sinc = (xy == 0.0) ? 1.0 : sin(xy) / xy;
    c2xy = cos(2.0 * xy);
    for (n = 1; n <= OR_A916_NTERM; ++n) {
        double nh = (double)n * h;
        double d  = nh * nh + y * y;
        s1 += exp(-(nh * nh)) / d;
        s2 += exp(-((nh + x) * (nh + x))) / d;
        s3 += exp(-((nh - x) * (nh - x))) / d;
    }
    K  = ex2 * or_erfcx(y) * c2xy;
    K += (2.0 * h * x / OR_PI) * ex2 * sin(xy) * sinc;
    K += (2.0 * h / OR_PI) * (-y * c2xy * ex2 * s1 + 0.5 * y * s2 + 0.5 * y * s3);
    return K;
}

/* Third-order (3-node) Gauss-Hermite quadrature of the Voigt integral
 * (Sec. 2.4): K ~ (y/pi) sum_k w_k / ((x - t_k)^2 + y^2), nodes 0 and
 * +-sqrt(3/2), weights 2 sqrt(pi)/3 and sqrt(pi)/6. */
double or_gh3(double x, double y)
{
    const double w0 = 2.0 * OR_SQRTPI / 3.0, w1 = OR_SQRTPI / 6.0;
    const double t = OR_GH3_T;
    double y2 = y * y;
    double d0 = x * x + y2;
    double d1 = (x - t) * (x - t) + y2;
    double d2 = (x + t) * (x + t) + y2;
    return (y / OR_PI) * (w0 / d0 + w1 / d1 + w1 / d2);
}

/* First-order (1-node) Gauss-Hermite rule (Sec. 2.4): node 0, weight
 * sqrt(pi), i.e. the Lorentz far-wing form y / (sqrt(pi) (x^2 + y^2)). */
double or_gh1(double x, double y)
{
    return (y / OR_PI) * (OR_SQRTPI / (x * x + y * y));
}

/* Region dispatch of Sec. 2.4 on r2 = u*u + a*a (each product and the sum
 * rounded separately).  Returns which method ran in *region if non-NULL:
 * 0 = Algorithm 916, 1 = 3-point GH, 2 = 1-point GH. */
double or_voigt_H(double a, double u, int *region)
{
    double r2 = u * u + a * a;
    if (r2 >= OR_R2_GH1) { if (region) *region = 2; return or_gh1(u, a); }
    if (r2 >= OR_R2_GH3) { if (region) *region = 1; return or_gh3(u, a); }
    if (region) *region = 0;
    return or_K916(u, a);
}

/* =====================================================================
 * Line preparation (Sec. 2.3-2.4): per line and per (T, P) condition.
 * ===================================================================== */

typedef struct {
    /* inputs, SoA; any pointer but nu0/S0/gamma_air may be NULL.
     * mass (amu) and weight (abundance) per line let one list hold several
     * species (Sec. 2.1: mixing ratios applied before the k-distribution). */
    const double *nu0, *S0, *E_lower, *gamma_air, *gamma_self, *n_coll, *delta;
    const double *mass, *weight;
} or_lines;

/* Per-line record.  nu0p = shifted centre, Sp = S sqrt(ln2/pi)/Gamma_D,
 * ku = sqrt(ln2)/Gamma_D, a = sqrt(ln2) Gamma_L / Gamma_D, window [ilo, ihi]
 * (empty when ilo > ihi). */
typedef struct {
    double nu0p, S, Sp, ku, a, gD, gL, cut;
    int64_t ilo, ihi;
} or_rec;

/*
 * One line at (T [K], P [atm], mass [amu]).
 *  - pressure shift  nu0' = nu0 + delta P / P0                (Sec. 2.3)
 *  - line strength   S = S0 (Q0/Q) exp(-c2 E''/T + c2 E''/T0)
 *                        (1 - e^{-c2 nu0/T}) / (1 - e^{-c2 nu0/T0})  (Sec. 2.3)
 *    applied only when E'' is given; q_ratio = Q(T0)/Q(T) is an input.
 *  - Lorentz HWHM    Gamma_L = (T0/T)^n [a_air (P - Pself) + a_self Pself]/P0,
 *                    Pself = P/2, natural width dropped        (Sec. 2.3)
 *  - Doppler HWHM    Gamma_D = nu0' sqrt(2 ln2 k_B T / m) / c  (Sec. 2.3),
 *                    m = the line's own mass when the list carries one
 *  - abundance       S is multiplied by the line's weight when given
 *  - cutoff C and window: inclusive |nu_i - nu0'| <= C        (Sec. 2.4)
 */
static void or_prep_one(const or_lines *L, int64_t l, double T, double P,
                        double mass, double q_ratio, int cut_kind,
                        double cut_value, double cut_cap, double nu_min,
                        double dnu, int64_t ngrid, or_rec *r)
{
    double nu0   = L->nu0[l];
    double delta = L->delta ? L->delta[l] : 0.0;
    double g_air = L->gamma_air[l];
    double g_slf = L->gamma_self ? L->gamma_self[l] : g_air;
    double ncoll = L->n_coll ? L->n_coll[l] : 0.5;
    double S     = L->S0[l];
    double tfac, pself, vth, lo, hi;

    r->nu0p = nu0 + delta * P;

    if (L->E_lower) {
        double E = L->E_lower[l], stim;
        double boltz = exp(-OR_C2 * E / T + OR_C2 * E / OR_T0);
        if (nu0 > 0.0)
            stim = expm1(-OR_C2 * nu0 / T) / expm1(-OR_C2 * nu0 / OR_T0);
        else
            stim = OR_T0 / T;                  /* limit nu0 -> 0 */
        S = S * q_ratio * boltz * stim;
    }
    if (L->weight) S = S * L->weight[l];
    r->S = S;

    tfac  = (ncoll == 0.5) ? sqrt(OR_T0 / T) : pow(OR_T0 / T, ncoll);
    pself = 0.5 * P;
    r->gL = tfac * (g_air * (P - pself) + g_slf * pself);

    if (L->mass) mass = L->mass[l];
    vth   = sqrt(2.0 * OR_LN2 * OR_KB * T / (mass * OR_AMU)) / OR_CLIGHT;
    r->gD = r->nu0p * vth;

    r->a  = OR_SQRTLN2 * r->gL / r->gD;
    r->ku = OR_SQRTLN2 / r->gD;
    r->Sp = S * OR_SQRTLN2PI / r->gD;

    if (cut_kind == OR_CUT_ABS)          r->cut = cut_value;
    else if (cut_kind == OR_CUT_LORENTZ) r->cut = fmin(cut_value * r->gL, cut_cap);
    else                                 r->cut = INFINITY;

    if (cut_kind == OR_CUT_NONE) { r->ilo = 0; r->ihi = ngrid - 1; return; }
    lo = ceil((r->nu0p - r->cut - nu_min) / dnu);
    hi = floor((r->nu0p + r->cut - nu_min) / dnu);
    if (lo < 0.0) lo = 0.0;
    if (hi > (double)(ngrid - 1)) hi = (double)(ngrid - 1);
    if (lo > (double)ngrid) lo = (double)ngrid;
    if (hi < -1.0) hi = -1.0;
    r->ilo = (int64_t)lo;
    r->ihi = (int64_t)hi;
}

/* Exported line preparation: fills the per-line arrays (any may be NULL). */
int or_lineprep(int64_t n, const double *nu0, const double *S0,
                const double *E_lower, const double *gamma_air,
                const double *gamma_self, const double *n_coll,
                const double *delta, const double *mass_l, const double *weight_l,
                double T, double P, double mass,
                double q_ratio, int cut_kind, double cut_value, double cut_cap,
                double nu_min, double dnu, int64_t ngrid,
                double *nu0p, double *S, double *Sp, double *ku, double *a,
                double *gD, double *gL, int64_t *ilo, int64_t *ihi)
{
    or_lines L = { nu0, S0, E_lower, gamma_air, gamma_self, n_coll, delta, mass_l, weight_l };
    int64_t l;
    for (l = 0; l < n; ++l) {
        or_rec r;
        or_prep_one(&L, l, T, P, mass, q_ratio, cut_kind, cut_value, cut_cap,
                    nu_min, dnu, ngrid, &r);
        if (nu0p) nu0p[l] = r.nu0p;
        if (S)    S[l]    = r.S;
        if (Sp)   Sp[l]   = r.Sp;
        if (ku)   ku[l]   = r.ku;
        if (a)    a[l]    = r.a;
        if (gD)   gD[l]   = r.gD;
        if (gL)   gL[l]   = r.gL;
        if (ilo)  ilo[l]  = r.ilo;
        if (ihi)  ihi[l]  = r.ihi;
    }
    return 0;
}

/* =====================================================================
 * Opacity kappa(nu_i) = weight * sum_lines S' H(a, u)   (Sec. 2.3, kappa = S Phi)
 * Grid nu_i = nu_min + i dnu, i in [0, ngrid).  Each point sums its lines
 * in list order.  Threads split the grid into contiguous chunks; the result
 * does not depend on the thread count.
 * ===================================================================== */

typedef struct {
    const or_rec *rec;
    int64_t nlines, g0, g1, evals;
    double nu_min, dnu, weight;
    int accumulate;
    double *kappa;
    int64_t region_count[3];
} or_chunk;

static void *or_opacity_chunk(void *arg)
{
    or_chunk *c = (or_chunk *)arg;
    int64_t l, i;
    double *acc = (double *)calloc((size_t)(c->g1 - c->g0 > 0 ? c->g1 - c->g0 : 1), sizeof(double));
    c->evals = 0;
    c->region_count[0] = c->region_count[1] = c->region_count[2] = 0;
    for (l = 0; l < c->nlines; ++l) {
        const or_rec *r = &c->rec[l];
        int64_t lo = r->ilo > c->g0 ? r->ilo : c->g0;
        int64_t hi = r->ihi < c->g1 - 1 ? r->ihi : c->g1 - 1;
        for (i = lo; i <= hi; ++i) {
            double nu_i = c->nu_min + (double)i * c->dnu;
            double u    = (nu_i - r->nu0p) * r->ku;
            int reg;
            double H    = or_voigt_H(r->a, u, &reg);
            acc[i - c->g0] += r->Sp * H;
            c->region_count[reg]++;
        }
        if (hi >= lo) c->evals += hi - lo + 1;
    }
    for (i = c->g0; i < c->g1; ++i) {
        double v = c->weight * acc[i - c->g0];
        c->kappa[i] = c->accumulate ? c->kappa[i] + v : v;
    }
    free(acc);
    return NULL;
}

/* Full opacity on the grid.  evals_out (optional) receives the number of
 * (line, grid point) pairs evaluated; region_out (optional, 3 entries) the
 * count per method (916, GH3, GH1). */
int or_opacity(int64_t n, const double *nu0, const double *S0,
               const double *E_lower, const double *gamma_air,
               const double *gamma_self, const double *n_coll,
               const double *delta, const double *mass_l, const double *weight_l,
               double T, double P, double mass,
               double q_ratio, int cut_kind, double cut_value, double cut_cap,
               double nu_min, double dnu, int64_t ngrid, double weight,
               int accumulate, double *kappa, int nthreads,
               int64_t *evals_out, int64_t *region_out)
{
    or_lines L = { nu0, S0, E_lower, gamma_air, gamma_self, n_coll, delta, mass_l, weight_l };
    or_rec *rec;
    or_chunk *ch;
    pthread_t *th;
    int64_t l, total = 0, rc[3] = {0, 0, 0};
    int t;
    if (nthreads < 1) nthreads = 1;
    if (ngrid < (int64_t)nthreads) nthreads = (int)(ngrid > 0 ? ngrid : 1);
    rec = (or_rec *)malloc((size_t)(n > 0 ? n : 1) * sizeof(or_rec));
    ch  = (or_chunk *)calloc((size_t)nthreads, sizeof(or_chunk));
    th  = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!rec || !ch || !th) { free(rec); free(ch); free(th); return -2; }
    for (l = 0; l < n; ++l)
        or_prep_one(&L, l, T, P, mass, q_ratio, cut_kind, cut_value, cut_cap,
                    nu_min, dnu, ngrid, &rec[l]);
    for (t = 0; t < nthreads; ++t) {
        ch[t].rec = rec; ch[t].nlines = n;
        ch[t].g0 = ngrid * t / nthreads; ch[t].g1 = ngrid * (t + 1) / nthreads;
        ch[t].nu_min = nu_min; ch[t].dnu = dnu; ch[t].weight = weight;
        ch[t].accumulate = accumulate; ch[t].kappa = kappa;
    }
    if (nthreads == 1) {
        or_opacity_chunk(&ch[0]);
    } else {
        for (t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, or_opacity_chunk, &ch[t]);
        for (t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    }
    for (t = 0; t < nthreads; ++t) {
        total += ch[t].evals;
        rc[0] += ch[t].region_count[0]; rc[1] += ch[t].region_count[1]; rc[2] += ch[t].region_count[2];
    }
    if (evals_out) *evals_out = total;
    if (region_out) { region_out[0] = rc[0]; region_out[1] = rc[1]; region_out[2] = rc[2]; }
    free(rec); free(ch); free(th);
    return 0;
}

/* Opacity at selected grid points only (each computed exactly as or_opacity
 * would, with the same per-point line order).  Used to check large grids on
 * a sample of points. */
int or_opacity_points(int64_t n, const double *nu0, const double *S0,
                      const double *E_lower, const double *gamma_air,
                      const double *gamma_self, const double *n_coll,
                      const double *delta, const double *mass_l,
                      const double *weight_l, double T, double P, double mass,
                      double q_ratio, int cut_kind, double cut_value,
                      double cut_cap, double nu_min, double dnu, int64_t ngrid,
                      int64_t npts, const int64_t *idx, double *kappa_pts,
                      int64_t *evals_out)
{
    or_lines L = { nu0, S0, E_lower, gamma_air, gamma_self, n_coll, delta, mass_l, weight_l };
    int64_t l, p, ev = 0;
    for (p = 0; p < npts; ++p) kappa_pts[p] = 0.0;
    for (l = 0; l < n; ++l) {
        or_rec r;
        or_prep_one(&L, l, T, P, mass, q_ratio, cut_kind, cut_value, cut_cap,
                    nu_min, dnu, ngrid, &r);
        for (p = 0; p < npts; ++p) {
            int64_t i = idx[p];
            if (i < r.ilo || i > r.ihi) continue;
            {
                double nu_i = nu_min + (double)i * dnu;
                double u    = (nu_i - r.nu0p) * r.ku;
                kappa_pts[p] += r.Sp * or_voigt_H(r.a, u, NULL);
                ++ev;
            }
        }
    }
    if (evals_out) *evals_out = ev;
    return 0;
}

/* =====================================================================
 * k-distribution (Sec. 2.2, 2.6): per bin sort, k(g), Chebyshev LS fit.
 * ===================================================================== */

static int or_cmp_double(const void *pa, const void *pb)
{
    double a = *(const double *)pa, b = *(const double *)pb;
    return (a > b) - (a < b);
}

/* Sort each of the nbins contiguous bins of kappa ascending (Sec. 2.6).  The
 * sorted values k_j of one bin are its k-distribution kappa(y) sampled on
 * y_j = (j + 1/2)/N_b. */
int or_sort_bins(const double *kappa, int64_t n, int32_t nbins, double *sorted)
{
    int64_t nb, b;
    if (nbins <= 0 || n % nbins) return -1;
    nb = n / nbins;
    memcpy(sorted, kappa, (size_t)n * sizeof(double));
    for (b = 0; b < nbins; ++b)
        qsort(sorted + b * nb, (size_t)nb, sizeof(double), or_cmp_double);
    return 0;
}

/*
 * Least-squares Chebyshev fit of ln k(g) on one bin (Sec. 2.6):
 * minimise || A c - L ||_2 with A_jk = T_k(t_j), t_j = 2 g_j - 1,
 * g_j = (j + 1/2)/N_b, L_j = ln max(k_j, kappa_floor).  Columns of A come
 * from the recurrence T_0 = 1, T_1 = t, T_{k+1} = 2 t T_k - T_{k-1}.
 * Solved by Householder QR (A = QR, R c = Q^T L), as the paper does.
 */
static int or_chebfit_bin(const double *k, int64_t nb, int ncheb,
                          double kappa_floor, double *A, double *rhs,
                          double *coef)
{
    int64_t j;
    int c, cc;
    for (j = 0; j < nb; ++j) {
        double g = ((double)j + 0.5) / (double)nb;
        double t = 2.0 * g - 1.0;
        double kv = k[j] > kappa_floor ? k[j] : kappa_floor;
        double *row = A + j * ncheb;
        row[0] = 1.0;
        if (ncheb > 1) row[1] = t;
        for (c = 2; c < ncheb; ++c) row[c] = 2.0 * t * row[c - 1] - row[c - 2];
        rhs[j] = log(kv);
    }
    /* Householder QR, column by column, applied to the right-hand side. */
    for (c = 0; c < ncheb; ++c) {
        double norm = 0.0, alpha, vtv, s;
        for (j = c; j < nb; ++j) norm += A[j * ncheb + c] * A[j * ncheb + c];
        norm = sqrt(norm);
        if (norm == 0.0) return -3;
        alpha = A[c * ncheb + c] > 0.0 ? -norm : norm;
        /* v = x - alpha e1 stored in place of column c (rows c..nb-1) */
        A[c * ncheb + c] -= alpha;
        vtv = 0.0;
        for (j = c; j < nb; ++j) vtv += A[j * ncheb + c] * A[j * ncheb + c];
        for (cc = c + 1; cc < ncheb; ++cc) {
            s = 0.0;
            for (j = c; j < nb; ++j) s += A[j * ncheb + c] * A[j * ncheb + cc];
            s = 2.0 * s / vtv;
            for (j = c; j < nb; ++j) A[j * ncheb + cc] -= s * A[j * ncheb + c];
        }
        s = 0.0;
        for (j = c; j < nb; ++j) s += A[j * ncheb + c] * rhs[j];
        s = 2.0 * s / vtv;
        for (j = c; j < nb; ++j) rhs[j] -= s * A[j * ncheb + c];
        /* the diagonal of R is alpha; keep it on the diagonal */
        A[c * ncheb + c] = alpha;
    }
    /* back substitution R c = (Q^T L)[0:ncheb] */
    for (c = ncheb - 1; c >= 0; --c) {
        double s2 = rhs[c];
        for (cc = c + 1; cc < ncheb; ++cc) s2 -= A[c * ncheb + cc] * coef[cc];
        coef[c] = s2 / A[c * ncheb + c];
    }
    return 0;
}

/* Chebyshev coefficients for every bin of an already bin-sorted array, and
 * the bin mean of kappa (= integral of k(g) dg, Sec. 2.1) if mean != NULL. */
int or_chebfit(const double *sorted, int64_t n, int32_t nbins, int32_t ncheb,
               double kappa_floor, double *coeffs, double *mean)
{
    int64_t nb, b, j;
    double *A, *rhs;
    int rc = 0;
    if (nbins <= 0 || n % nbins || ncheb < 1) return -1;
    nb = n / nbins;
    if (ncheb > nb) return -1;
    A   = (double *)malloc((size_t)nb * (size_t)ncheb * sizeof(double));
    rhs = (double *)malloc((size_t)nb * sizeof(double));
    if (!A || !rhs) { free(A); free(rhs); return -2; }
    for (b = 0; b < nbins && rc == 0; ++b) {
        rc = or_chebfit_bin(sorted + b * nb, nb, ncheb, kappa_floor, A, rhs,
                            coeffs + b * ncheb);
        if (mean) {
            double s = 0.0;
            for (j = 0; j < nb; ++j) s += sorted[b * nb + j];
            mean[b] = s / (double)nb;
        }
    }
    free(A); free(rhs);
    return rc;
}

/* Evaluate the fitted k(g) = exp(sum_k c_k T_k(2g - 1)) at ng points g. */
int or_chebeval(const double *coef, int32_t ncheb, int64_t ng, const double *g,
                double *kg)
{
    int64_t j;
    int c;
    for (j = 0; j < ng; ++j) {
        double t = 2.0 * g[j] - 1.0, tkm1 = 1.0, tk = t, s = coef[0];
        if (ncheb > 1) s += coef[1] * t;
        for (c = 2; c < ncheb; ++c) {
            double tkp1 = 2.0 * t * tk - tkm1;
            s += coef[c] * tkp1;
            tkm1 = tk; tk = tkp1;
        }
        kg[j] = exp(s);
    }
    return 0;
}

/*
 * Transmission of each bin for nm column masses m (Sec. 2.1, Eq. for T):
 *   T_b(m) = int_0^1 exp(-k(g) m) dg
 * from the sorted samples (midpoint rule on g_j = (j+1/2)/N_b) into
 * trans_direct[b*nm + i] and, if coeffs != NULL, from the Chebyshev fit on
 * ng midpoints into trans_fit[b*nm + i].
 */
int or_transmission(const double *sorted, int64_t n, int32_t nbins,
                    const double *coeffs, int32_t ncheb, int64_t ng,
                    int32_t nm, const double *m, double *trans_direct,
                    double *trans_fit)
{
    int64_t nb, b, j;
    int i;
    double *g = NULL, *kg = NULL;
    if (nbins <= 0 || n % nbins) return -1;
    nb = n / nbins;
    if (coeffs) {
        g  = (double *)malloc((size_t)ng * sizeof(double));
        kg = (double *)malloc((size_t)ng * sizeof(double));
        if (!g || !kg) { free(g); free(kg); return -2; }
        for (j = 0; j < ng; ++j) g[j] = ((double)j + 0.5) / (double)ng;
    }
    for (b = 0; b < nbins; ++b) {
        const double *k = sorted + b * nb;
        for (i = 0; i < nm; ++i) {
            double s = 0.0;
            for (j = 0; j < nb; ++j) s += exp(-k[j] * m[i]);
            trans_direct[b * nm + i] = s / (double)nb;
        }
        if (coeffs) {
            or_chebeval(coeffs + b * ncheb, ncheb, ng, g, kg);
            for (i = 0; i < nm; ++i) {
                double s = 0.0;
                for (j = 0; j < ng; ++j) s += exp(-kg[j] * m[i]);
                trans_fit[b * nm + i] = s / (double)ng;
            }
        }
    }
    free(g); free(kg);
    return 0;
}
