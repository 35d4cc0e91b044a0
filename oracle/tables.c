/*
 * tables.c -- oracle special functions, cross sections and sampling tables.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Plain FP64, adaptive Gauss-Kronrod
 * (G7/K15) quadrature everywhere; no table or helper is shared with the CUDA
 * library, which uses a different rule.
 *
 * Physics followed here:
 *  - Nonlinear Compton scattering is "the same as EPOCH" (Sec. 2.2), i.e. the
 *    quantum-synchrotron model of Kirk et al. 2009 / Ridgers et al. 2014 with
 *    the Sokolov-Ternov emissivity F(eta, chi).  Its rate prefactor is fixed by
 *    the small-eta Larmor limit (pinned in the tests).
 *  - Bremsstrahlung uses the Tsai screened DCS of Eq. (1) with Tsai's
 *    Thomas-Fermi screening fits (Rev. Mod. Phys. 46, 815, Eqs. 3.38-3.41,
 *    cited at Eq. (1)) and the Davies-Bethe-Maximon Coulomb correction f(Z).
 *  - sigma(E) integrates Eq. (1) from y_cut (hard-photon cut, Sec. 3) to the
 *    kinematic end point; the photon energy is drawn from the partial integral
 *    sigma(y, E) = sigma(E) R2 (Sec. 2.2, text after Eq. 4).
 *  - Bethe-Heitler pair production, which Sec. 2.2 says is implemented like the
 *    bremsstrahlung: Tsai's DCS of the crossed process with the same screening
 *    fits, integrated over the positron fraction x in [1/k, 1 - 1/k], and the
 *    CDF of the partial integral tabulated linearly in x.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Adaptive Gauss-Kronrod 7/15 (QUADPACK node set, Piessens et al. 1983).    */
/* ------------------------------------------------------------------------- */
static const double GK_X[8] = {
    0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
    0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
    0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
    0.207784955007898467600689403773245, 0.0};
static const double GK_WK[8] = {
    0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
    0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
    0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
    0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double GK_WG[4] = {
    0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
    0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

typedef double (*or_fn)(double x, const void* ctx);

static void gk15(or_fn f, const void* ctx, double a, double b, double* k15, double* g7, double* mag) {
    double c = 0.5 * (a + b), h = 0.5 * (b - a);
    double fc = f(c, ctx);
    double sk = GK_WK[7] * fc, sg = GK_WG[3] * fc, sa = GK_WK[7] * fabs(fc);
    for (int i = 0; i < 7; ++i) {
        double dx = h * GK_X[i];
        double f1 = f(c - dx, ctx), f2 = f(c + dx, ctx);
        double s = f1 + f2;
        sk += GK_WK[i] * s;
        sa += GK_WK[i] * (fabs(f1) + fabs(f2));
        if (i & 1) sg += GK_WG[i / 2] * s;
    }
    *k15 = sk * h;
    *g7 = sg * h;
    *mag = sa * fabs(h);
}

/* Recursive bisection.  A panel is accepted when the Kronrod-Gauss
 * difference is below its share of the tolerance, or when that difference is
 * at the level of rounding in the panel sum. */
static double adapt(or_fn f, const void* ctx, double a, double b, double tol_abs, int depth) {
    double k, g, mag;
    gk15(f, ctx, a, b, &k, &g, &mag);
    double err = fabs(k - g);
    if (depth >= 24 || err <= tol_abs || err <= 1e-14 * mag) return k;
    double m = 0.5 * (a + b);
    return adapt(f, ctx, a, m, 0.5 * tol_abs, depth + 1) + adapt(f, ctx, m, b, 0.5 * tol_abs, depth + 1);
}

/* integral of f over [a,b] to relative accuracy rel (with an absolute floor) */
static double integrate(or_fn f, const void* ctx, double a, double b, double rel, double abs_floor) {
    if (b <= a) return 0.0;
    double k, g, mag;
    gk15(f, ctx, a, b, &k, &g, &mag);
    double tol = fmax(rel * fabs(k), abs_floor);
    return adapt(f, ctx, a, b, tol, 0);
}

/* ------------------------------------------------------------------------- */
/* Modified Bessel functions from their integral representations:           */
/*   K_nu(x)          = int_0^inf exp(-x cosh t) cosh(nu t) dt               */
/*   int_x^inf K_53   = int_0^inf exp(-x cosh t) cosh(5t/3) / cosh t dt      */
/* ------------------------------------------------------------------------- */
typedef struct { double x, nu; int kind; } bes_ctx;

static double bes_integrand(double t, const void* vc) {
    const bes_ctx* c = (const bes_ctx*)vc;
    double ch = cosh(t);
    double e = exp(-c->x * ch);
    if (c->kind == 0) return e * cosh(c->nu * t);
    return e * cosh(c->nu * t) / ch;
}

static double bessel_common(double nu, double x, int kind) {
    bes_ctx c = {x, nu, kind};
    /* upper limit: exp(-x cosh T + nu T) is 1e-300 below the value at t = 0 */
    double T = acosh(1.0 + 700.0 / x);
    for (int it = 0; it < 8; ++it) T = acosh(1.0 + (700.0 + nu * T) / x);
    double tpk = asinh(nu / x);          /* maximum of the K_nu integrand       */
    if (tpk > T) tpk = 0.5 * T;
    double r = 0.0;
    /* split into a few panels so the adaptive rule sees the peak and the tail */
    double edges[6] = {0.0, 0.5 * tpk, tpk, tpk + 0.5 * (T - tpk), T, T};
    int ne = 5;
    for (int i = 0; i + 1 < ne; ++i)
        if (edges[i + 1] > edges[i]) r += integrate(bes_integrand, &c, edges[i], edges[i + 1], 1e-14, 1e-300);
    return r;
}

double or_bessel_k(double nu, double x) { return bessel_common(nu, x, 0); }
double or_int_k53(double x) { return bessel_common(5.0 / 3.0, x, 1); }

/* ------------------------------------------------------------------------- */
/* Quantum-synchrotron emissivity.                                           */
/*   F(eta,chi) = (4 chi^2/eta^2) y K_{2/3}(y) + (1 - 2chi/eta) y int_y K53  */
/*   y = 4 chi / (3 eta (eta - 2 chi)),  chi in (0, eta/2).                  */
/* With delta = 2 chi / eta (photon energy fraction) and y = 2 delta/(3 eta  */
/* (1 - delta)):  F = delta^2 y K23(y) + (1 - delta) y IK53(y).              */
/* ------------------------------------------------------------------------- */
static double F_of_y(double eta, double y) {
    double d = 3.0 * eta * y / (2.0 + 3.0 * eta * y);
#ifdef OR_MUTANT_NCS_F_QUANTUM
    return (1.0 - d) * y * or_int_k53(y);
#else
    return d * d * y * or_bessel_k(2.0 / 3.0, y) + (1.0 - d) * y * or_int_k53(y);
#endif
}

double or_ncs_F(double eta, double chi) {
    if (chi <= 0.0 || chi >= 0.5 * eta) return 0.0;
    double y = 4.0 * chi / (3.0 * eta * (eta - 2.0 * chi));
    return F_of_y(eta, y);
}

/* integrand in ln y for int F/chi dchi: dchi/chi = 2/(2 + 3 eta y) d ln y   */
typedef struct { double eta; int classical; } ncs_ctx;
static double ncs_cdf_integrand(double lny, const void* vc) {
    const ncs_ctx* c = (const ncs_ctx*)vc;
    double y = exp(lny);
    if (c->classical) return y * or_int_k53(y);          /* eta -> 0 limit    */
#ifdef OR_MUTANT_NCS_H_JACOBIAN
    return F_of_y(c->eta, y);
#else
    return F_of_y(c->eta, y) * 2.0 / (2.0 + 3.0 * c->eta * y);
#endif
}
/* integrand in ln y for int F dchi: dchi = 3 eta^2 y /(2+3 eta y)^2 d ln y  */
static double ncs_pow_integrand(double lny, const void* vc) {
    const ncs_ctx* c = (const ncs_ctx*)vc;
    double y = exp(lny);
    double q = 2.0 + 3.0 * c->eta * y;
    return F_of_y(c->eta, y) * 3.0 * c->eta * c->eta * y / (q * q);
}

/* integral over y in (0, ymax] of an integrand behaving as y^(p) near 0:
 * numerical on [ylo, ymax] in ln y plus the power-law tail ylo^p/p.         */
static double ln_integral_with_tail(or_fn f, const void* ctx, double ylo, double yhi, double p) {
    double mid = integrate(f, ctx, log(ylo), log(yhi), 1e-14, 1e-300);
    double tail = f(log(ylo), ctx) / p;
    return mid + tail;
}

double or_ncs_power_integral(double eta) {
    ncs_ctx c = {eta, 0};
    /* near y -> 0 the integrand in ln y behaves as y^(4/3) */
    double s = 0.0;
    double lo = 1e-16 / (1.0 + eta);
    double edges[] = {lo, 1e-8, 1e-4, 1e-2, 1.0, 10.0, 200.0};
    for (int i = 0; i < 6; ++i) s += integrate(ncs_pow_integrand, &c, log(edges[i]), log(edges[i + 1]), 1e-14, 1e-300);
    s += ncs_pow_integrand(log(lo), &c) / (4.0 / 3.0);
    return s;
}

double or_ncs_h_direct(double eta) {
    ncs_ctx c = {eta, 0};
    double s = 0.0;
    double lo = 1e-16;
    double edges[] = {lo, 1e-8, 1e-4, 1e-2, 1.0, 10.0, 200.0};
    for (int i = 0; i < 6; ++i) s += integrate(ncs_cdf_integrand, &c, log(edges[i]), log(edges[i + 1]), 1e-14, 1e-300);
    s += ncs_cdf_integrand(log(lo), &c) / (1.0 / 3.0);
    return s;
}

/* ------------------------------------------------------------------------- */
/* Bremsstrahlung, Eq. (1) with Tsai's screening functions.                  */
/* ------------------------------------------------------------------------- */
static const double OR_ALPHA = 7.2973525693e-3;

double or_coulomb_f(double Z) {
    double a2 = (OR_ALPHA * Z) * (OR_ALPHA * Z);
    return a2 * (1.0 / (1.0 + a2) + 0.20206 - 0.0369 * a2 + 0.0083 * a2 * a2 - 0.002 * a2 * a2 * a2);
}

double or_brems_dcs_raw(double Z, double gamma, double y, int complete) {
    /* screening variables: 100 m k / (E E' Z^{1/3}) and 100 m k / (E E' Z^{2/3}) */
    double g = 0.0, e = 0.0;
    if (!complete) {
        g = 100.0 * y / (gamma * (1.0 - y) * cbrt(Z));
        e = 100.0 * y / (gamma * (1.0 - y) * cbrt(Z * Z));
    }
    double phi1 = 20.863 - 2.0 * log(1.0 + (0.55846 * g) * (0.55846 * g))
                  - 4.0 * (1.0 - 0.6 * exp(-0.9 * g) - 0.4 * exp(-1.5 * g));
    double phi2 = phi1 - (2.0 / 3.0) / (1.0 + 6.5 * g + 6.0 * g * g);
    double psi1 = 28.340 - 2.0 * log(1.0 + (3.621 * e) * (3.621 * e))
                  - 4.0 * (1.0 - 0.7 * exp(-8.0 * e) - 0.3 * exp(-29.2 * e));
    double psi2 = psi1 - (2.0 / 3.0) / (1.0 + 40.0 * e + 400.0 * e * e);
    double lnZ = log(Z);
#ifdef OR_MUTANT_BREMS_COULOMB
    double f = 0.0;
#else
    double f = or_coulomb_f(Z);
#endif
    double t1 = (4.0 / 3.0 - 4.0 / 3.0 * y + y * y)
              * (Z * Z * (phi1 - 4.0 / 3.0 * lnZ - 4.0 * f) + Z * (psi1 - 8.0 / 3.0 * lnZ));
    double t2 = (2.0 / 3.0) * (1.0 - y) * (Z * Z * (phi1 - phi2) + Z * (psi1 - psi2));
    return (t1 + t2) / y;
}

typedef struct { double Z, gamma, ycut, L; } br_ctx;
/* integrand in s with y = ycut * exp(s L): y dsigma/dy * L, clamped at 0   */
static double br_integrand(double s, const void* vc) {
    const br_ctx* c = (const br_ctx*)vc;
    double y = c->ycut * exp(s * c->L);
    double d = or_brems_dcs_raw(c->Z, c->gamma, y, 0);
    if (d < 0.0) d = 0.0;
    return y * d * c->L;
}

double or_brems_sigma_direct(double Z, double gamma, double photon_min) {
    double ycut = photon_min / gamma, ymax = 1.0 - 1.0 / gamma;
    if (ycut >= ymax) return 0.0;
    br_ctx c = {Z, gamma, ycut, log(ymax / ycut)};
    return integrate(br_integrand, &c, 0.0, 1.0, 1e-14, 1e-300);
}

/* ------------------------------------------------------------------------- */
/* Bethe-Heitler pair production, which Sec. 2.2 says is implemented like the   */
/* bremsstrahlung: Tsai's screened DCS of the crossed process (Rev. Mod. Phys.  */
/* 46, 815, the reference of Eq. 1) with the same screening fits and Coulomb    */
/* correction.  Photon energy k (m c^2), positron energy fraction x = E+/k,     */
/* E- = (1 - x) k; screening variables 100 m k / (E+ E- Z^{1/3}) and            */
/* 100 m k / (E+ E- Z^{2/3}).                                                   */
/* ------------------------------------------------------------------------- */
double or_bh_dcs_raw(double Z, double k, double x, int complete) {
    double g = 0.0, e = 0.0;
    if (!complete) {
        g = 100.0 / (k * x * (1.0 - x) * cbrt(Z));
        e = 100.0 / (k * x * (1.0 - x) * cbrt(Z * Z));
    }
    double phi1 = 20.863 - 2.0 * log(1.0 + (0.55846 * g) * (0.55846 * g))
                  - 4.0 * (1.0 - 0.6 * exp(-0.9 * g) - 0.4 * exp(-1.5 * g));
    double phi2 = phi1 - (2.0 / 3.0) / (1.0 + 6.5 * g + 6.0 * g * g);
    double psi1 = 28.340 - 2.0 * log(1.0 + (3.621 * e) * (3.621 * e))
                  - 4.0 * (1.0 - 0.7 * exp(-8.0 * e) - 0.3 * exp(-29.2 * e));
    double psi2 = psi1 - (2.0 / 3.0) / (1.0 + 40.0 * e + 400.0 * e * e);
    double lnZ = log(Z);
    double f = or_coulomb_f(Z);
    double xx = x * (1.0 - x);
    double t1 = (1.0 - 4.0 / 3.0 * xx)
              * (Z * Z * (phi1 - 4.0 / 3.0 * lnZ - 4.0 * f) + Z * (psi1 - 8.0 / 3.0 * lnZ));
#ifdef OR_MUTANT_BH_SECOND_TERM
    double t2 = 0.0;
    (void)phi2; (void)psi2;
#else
    double t2 = -(2.0 / 3.0) * xx * (Z * Z * (phi1 - phi2) + Z * (psi1 - psi2));
#endif
    return t1 + t2;
}

typedef struct { double Z, k, xmin, span; } bh_ctx;
/* integrand in s with x = xmin + s span: dsigma/dx * span, clamped at 0 */
static double bh_integrand(double s, const void* vc) {
    const bh_ctx* c = (const bh_ctx*)vc;
    double d = or_bh_dcs_raw(c->Z, c->k, c->xmin + s * c->span, 0);
    if (d < 0.0) d = 0.0;
    return d * c->span;
}

static double bh_raw_s(const bh_ctx* c, double s) { return or_bh_dcs_raw(c->Z, c->k, c->xmin + s * c->span, 0); }

/* integral of the clamped integrand over [a, b] in s.  The clamp puts a kink where the
 * DCS changes sign; each side of it is integrated separately.  The DCS is symmetric about
 * x = 1/2, so the cell is first split there, leaving at most one sign change per part. */
static double bh_cell(const bh_ctx* c, double a, double b) {
    double sm = (0.5 - c->xmin) / c->span;
    if (a < sm && sm < b) return bh_cell(c, a, sm) + bh_cell(c, sm, b);
    double fa = bh_raw_s(c, a), fb = bh_raw_s(c, b);
    if ((fa < 0.0) != (fb < 0.0)) {
        double u = a, v = b;
        for (int it = 0; it < 200 && v - u > 1e-17 * (1.0 + fabs(u)); ++it) {
            double m = 0.5 * (u + v);
            if ((bh_raw_s(c, m) < 0.0) == (fa < 0.0)) u = m; else v = m;
        }
        double r = 0.5 * (u + v);
        return integrate(bh_integrand, c, a, r, 1e-14, 1e-300) + integrate(bh_integrand, c, r, b, 1e-14, 1e-300);
    }
    return integrate(bh_integrand, c, a, b, 1e-14, 1e-300);
}

double or_bh_sigma_direct(double Z, double k) {
    if (!(k > 2.0)) return 0.0;
    bh_ctx c = {Z, k, 1.0 / k, 1.0 - 2.0 / k};
    return bh_cell(&c, 0.0, 1.0);
}

/* ------------------------------------------------------------------------- */
/* Tables                                                                    */
/* ------------------------------------------------------------------------- */
struct or_tables {
    or_table_params p;
    int n_Z;
    double* Z;
    double* h;        /* [n_eta]          */
    double* cdf;      /* [n_eta][n_y]     */
    double* cdf_cl;   /* [n_y]            */
    double cl_total;
    double* sigma;    /* [n_Z][n_E]       */
    double* bcdf;     /* [n_Z][n_E][n_s]  */
    double* bh_sigma; /* [n_Z][n_E]  Bethe-Heitler, k on the log grid [2, gamma_max] */
    double* bh_cdf;   /* [n_Z][n_E][n_s]; both built on first use */
    int bh_built;
};

static double grid_log(double lo, double hi, int i, int n) {
    return exp(log(lo) + (log(hi) - log(lo)) * (double)i / (double)(n - 1));
}

/* one NCS row: cumulative integral of F/chi over y grid, normalised */
static void build_ncs_row(const or_table_params* p, double eta, int classical, double* row, double* total) {
    ncs_ctx c = {eta, classical};
    double ylo = p->y_min * 1e-8;
    /* part below the first grid point: numerical + y^(1/3) power-law tail */
    double cum = ln_integral_with_tail(ncs_cdf_integrand, &c, ylo, p->y_min, 1.0 / 3.0);
    row[0] = cum;
    for (int j = 1; j < p->n_y; ++j) {
        double a = log(grid_log(p->y_min, p->y_max, j - 1, p->n_y));
        double b = log(grid_log(p->y_min, p->y_max, j, p->n_y));
        cum += integrate(ncs_cdf_integrand, &c, a, b, 1e-14, 1e-300);
        row[j] = cum;
    }
    *total = cum;
    for (int j = 0; j < p->n_y; ++j) row[j] /= cum;
    row[p->n_y - 1] = 1.0;
}

static void build_brems_row(const or_table_params* p, double Z, double gamma, double* row, double* sigma) {
    double ycut = p->photon_min / gamma, ymax = 1.0 - 1.0 / gamma;
    int n = p->n_s;
    if (ycut >= ymax) {
        for (int j = 0; j < n; ++j) row[j] = (double)j / (double)(n - 1);
        *sigma = 0.0;
        return;
    }
    br_ctx c = {Z, gamma, ycut, log(ymax / ycut)};
    double cum = 0.0;
    row[0] = 0.0;
    for (int j = 1; j < n; ++j) {
        cum += integrate(br_integrand, &c, (double)(j - 1) / (n - 1), (double)j / (n - 1), 1e-14, 1e-300);
        row[j] = cum;
    }
    *sigma = cum;
    if (cum > 0.0) {
        for (int j = 0; j < n; ++j) row[j] /= cum;
        row[n - 1] = 1.0;
    } else {
        for (int j = 0; j < n; ++j) row[j] = (double)j / (double)(n - 1);
    }
}

static void build_bh_row(const or_table_params* p, double Z, double k, double* row, double* sigma) {
    int n = p->n_s;
    if (!(k > 2.0)) {
        for (int j = 0; j < n; ++j) row[j] = (double)j / (double)(n - 1);
        *sigma = 0.0;
        return;
    }
    bh_ctx c = {Z, k, 1.0 / k, 1.0 - 2.0 / k};
    double cum = 0.0;
    row[0] = 0.0;
    for (int j = 1; j < n; ++j) {
        cum += bh_cell(&c, (double)(j - 1) / (n - 1), (double)j / (n - 1));
        row[j] = cum;
    }
    *sigma = cum;
    if (cum > 0.0) {
        for (int j = 0; j < n; ++j) row[j] /= cum;
        row[n - 1] = 1.0;
    } else {
        for (int j = 0; j < n; ++j) row[j] = (double)j / (double)(n - 1);
    }
}

or_tables* or_tables_build(const or_table_params* p, int n_Z, const double* Z) {
    if (!p || p->n_eta < 2 || p->n_y < 2 || p->n_E < 2 || p->n_s < 2 || n_Z < 0) return NULL;
    or_tables* t = (or_tables*)calloc(1, sizeof(or_tables));
    t->p = *p;
    t->n_Z = n_Z;
    t->Z = (double*)malloc(sizeof(double) * (n_Z > 0 ? n_Z : 1));
    for (int i = 0; i < n_Z; ++i) t->Z[i] = Z[i];
    t->h = (double*)malloc(sizeof(double) * p->n_eta);
    t->cdf = (double*)malloc(sizeof(double) * p->n_eta * p->n_y);
    t->cdf_cl = (double*)malloc(sizeof(double) * p->n_y);
    t->sigma = (double*)malloc(sizeof(double) * (n_Z > 0 ? n_Z : 1) * p->n_E);
    t->bcdf = (double*)malloc(sizeof(double) * (n_Z > 0 ? n_Z : 1) * p->n_E * p->n_s);
    t->bh_sigma = (double*)malloc(sizeof(double) * (n_Z > 0 ? n_Z : 1) * p->n_E);
    t->bh_cdf = (double*)malloc(sizeof(double) * (n_Z > 0 ? n_Z : 1) * p->n_E * p->n_s);

#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < p->n_eta; ++i) {
        double eta = grid_log(p->eta_min, p->eta_max, i, p->n_eta);
        build_ncs_row(p, eta, 0, t->cdf + (int64_t)i * p->n_y, &t->h[i]);
    }
    build_ncs_row(p, 0.0, 1, t->cdf_cl, &t->cl_total);

#pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int iz = 0; iz < n_Z; ++iz)
        for (int i = 0; i < p->n_E; ++i) {
            double g = grid_log(p->gamma_min, p->gamma_max, i, p->n_E);
            build_brems_row(p, Z[iz], g, t->bcdf + ((int64_t)iz * p->n_E + i) * p->n_s,
                            &t->sigma[iz * p->n_E + i]);
        }
    return t;
}

/* the Bethe-Heitler tables, built on the first call that needs them */
static void ensure_bh(const or_tables* tc) {
    or_tables* t = (or_tables*)tc;
    int done;
#pragma omp atomic read
    done = t->bh_built;
    if (done) return;
#pragma omp critical(or_bh_build)
    {
        if (!t->bh_built) {
            const or_table_params* p = &t->p;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
            for (int iz = 0; iz < t->n_Z; ++iz)
                for (int i = 0; i < p->n_E; ++i) {
                    double k = grid_log(2.0, p->gamma_max, i, p->n_E);
                    build_bh_row(p, t->Z[iz], k, t->bh_cdf + ((int64_t)iz * p->n_E + i) * p->n_s,
                                 &t->bh_sigma[iz * p->n_E + i]);
                }
#pragma omp atomic write
            t->bh_built = 1;
        }
    }
}

void or_tables_free(or_tables* t) {
    if (!t) return;
    free(t->Z); free(t->h); free(t->cdf); free(t->cdf_cl); free(t->sigma); free(t->bcdf);
    free(t->bh_sigma); free(t->bh_cdf);
    free(t);
}

double or_tables_classical_total(const or_tables* t) { return t->cl_total; }
double or__photon_min(const or_tables* t) { return t->p.photon_min; }
/* largest tabulated sigma_Z of table iz (the interpolant never exceeds it) */
double or__sigma_max(const or_tables* t, int iz) {
    const double* s = t->sigma + (int64_t)iz * t->p.n_E;
    double m = 0.0;
    for (int i = 0; i < t->p.n_E; ++i) if (s[i] > m) m = s[i];
    return m;
}

int64_t or_tables_export(const or_tables* t, int which, int iz, double* out, int64_t cap) {
    const or_table_params* p = &t->p;
    const double* src = NULL;
    int64_t n = 0;
    switch (which) {
        case 0: src = t->h; n = p->n_eta; break;
        case 1: src = t->cdf; n = (int64_t)p->n_eta * p->n_y; break;
        case 2: src = t->cdf_cl; n = p->n_y; break;
        case 3: if (iz < 0 || iz >= t->n_Z) return -1; src = t->sigma + (int64_t)iz * p->n_E; n = p->n_E; break;
        case 4: if (iz < 0 || iz >= t->n_Z) return -1; src = t->bcdf + (int64_t)iz * p->n_E * p->n_s;
                n = (int64_t)p->n_E * p->n_s; break;
        case 5: if (iz < 0 || iz >= t->n_Z) return -1; ensure_bh(t); src = t->bh_sigma + (int64_t)iz * p->n_E; n = p->n_E; break;
        case 6: if (iz < 0 || iz >= t->n_Z) return -1; ensure_bh(t); src = t->bh_cdf + (int64_t)iz * p->n_E * p->n_s;
                n = (int64_t)p->n_E * p->n_s; break;
        default: return -1;
    }
    if (cap < n) return -1;
    memcpy(out, src, sizeof(double) * n);
    return n;
}

/* ------------------------------------------------------------------------- */
/* Table lookups, as the step uses them.                                     */
/* Rows are interpolated linearly in log eta (log gamma for brems); a sample */
/* is drawn by inverting the row-interpolated CDF, linear in the abscissa    */
/* between grid points.                                                      */
/* ------------------------------------------------------------------------- */
static void row_pos(double v, double lo, double hi, int n, int* i, double* w, int* flag) {
    double tpos = (log(v) - log(lo)) / ((log(hi) - log(lo)) / (double)(n - 1));
    *flag = 0;
    if (tpos >= (double)(n - 1)) { *i = n - 2; *w = 1.0; *flag = 1; return; }
    if (tpos < 0.0) { *i = 0; *w = 0.0; *flag = -1; return; }
    int k = (int)floor(tpos);
    if (k > n - 2) k = n - 2;
    *i = k;
#ifdef OR_MUTANT_ROW_WEIGHT
    *w = 1.0 - (tpos - (double)k);
#else
    *w = tpos - (double)k;
#endif
}

double or_ncs_h_interp(const or_tables* t, double eta, int* range_flag) {
    const or_table_params* p = &t->p;
    if (eta < p->eta_min) { *range_flag = -1; return 5.0 * M_PI / 3.0; }
    int i, fl; double w;
    row_pos(eta, p->eta_min, p->eta_max, p->n_eta, &i, &w, &fl);
    *range_flag = fl;
    return (1.0 - w) * t->h[i] + w * t->h[i + 1];
}

/* largest j with c[j] <= R over the interpolated row (linear scan) */
static double invert_row(const double* ra, const double* rb, double w, int n, double R,
                         double* c0_out, int* j_out, double* frac_out) {
    double c0 = (1.0 - w) * ra[0] + w * rb[0];
    *c0_out = c0;
    if (R < c0) { *j_out = -1; *frac_out = 0.0; return 0.0; }
    int j = 0;
    double cj = c0;
    for (int k = 1; k < n; ++k) {
        double ck = (1.0 - w) * ra[k] + w * rb[k];
        if (ck <= R) { j = k; cj = ck; } else break;
    }
    if (j >= n - 1) { *j_out = n - 1; *frac_out = 0.0; return 0.0; }
    double cn = (1.0 - w) * ra[j + 1] + w * rb[j + 1];
    double fr = (cn > cj) ? (R - cj) / (cn - cj) : 0.0;
    *j_out = j;
    *frac_out = fr;
    return 0.0;
}

double or_sample_ncs_delta(const or_tables* t, double eta, double R, int* below) {
#ifdef OR_MUTANT_NCS_SAMPLE_FLIP
    R = 1.0 - R;
#endif
    const or_table_params* p = &t->p;
    const double *ra, *rb;
    double w;
    *below = 0;
    if (eta < p->eta_min) {
        ra = rb = t->cdf_cl; w = 0.0; *below = 1;
    } else {
        int i, fl;
        row_pos(eta, p->eta_min, p->eta_max, p->n_eta, &i, &w, &fl);
        ra = t->cdf + (int64_t)i * p->n_y;
        rb = t->cdf + (int64_t)(i + 1) * p->n_y;
    }
    double c0, fr; int j;
    invert_row(ra, rb, w, p->n_y, R, &c0, &j, &fr);
    double dly = (log(p->y_max) - log(p->y_min)) / (double)(p->n_y - 1);
    double y;
    if (j < 0) {
        /* below the first grid point the CDF grows as y^(1/3) */
        double q = R / c0;
        y = p->y_min * q * q * q;
    } else if (j >= p->n_y - 1) {
        y = p->y_max;
    } else {
        y = exp(log(p->y_min) + ((double)j + fr) * dly);
    }
#ifdef OR_MUTANT_DELTA_MAP
    return 3.0 * eta * y / (1.0 + 3.0 * eta * y);
#else
    return 3.0 * eta * y / (2.0 + 3.0 * eta * y);
#endif
}

double or_brems_sigma_interp(const or_tables* t, int iz, double gamma, int* above) {
    const or_table_params* p = &t->p;
    int i, fl; double w;
    row_pos(gamma, p->gamma_min, p->gamma_max, p->n_E, &i, &w, &fl);
    *above = (fl == 1);
    const double* s = t->sigma + (int64_t)iz * p->n_E;
    return (1.0 - w) * s[i] + w * s[i + 1];
}

double or_sample_brems_y(const or_tables* t, int iz, double gamma, double R) {
#ifdef OR_MUTANT_BREMS_SAMPLE_FLIP
    R = 1.0 - R;
#endif
    const or_table_params* p = &t->p;
    int i, fl; double w;
    row_pos(gamma, p->gamma_min, p->gamma_max, p->n_E, &i, &w, &fl);
    const double* base = t->bcdf + (int64_t)iz * p->n_E * p->n_s;
    const double* ra = base + (int64_t)i * p->n_s;
    const double* rb = base + (int64_t)(i + 1) * p->n_s;
    double c0, fr; int j;
    invert_row(ra, rb, w, p->n_s, R, &c0, &j, &fr);
    double s;
    if (j < 0) s = 0.0;
    else if (j >= p->n_s - 1) s = 1.0;
    else s = ((double)j + fr) / (double)(p->n_s - 1);
    double ycut = p->photon_min / gamma, ymax = 1.0 - 1.0 / gamma;
    return ycut * exp(s * log(ymax / ycut));
}

/* Bethe-Heitler lookups on the pair grid k in [2, gamma_max] (log spaced) */
double or_bh_sigma_interp(const or_tables* t, int iz, double k, int* above) {
    const or_table_params* p = &t->p;
    ensure_bh(t);
    *above = 0;
    if (!(k > 2.0)) return 0.0;
    int i, fl; double w;
    row_pos(k, 2.0, p->gamma_max, p->n_E, &i, &w, &fl);
    *above = (fl == 1);
    const double* s = t->bh_sigma + (int64_t)iz * p->n_E;
    return (1.0 - w) * s[i] + w * s[i + 1];
}

double or_sample_bh_x(const or_tables* t, int iz, double k, double R) {
    const or_table_params* p = &t->p;
    ensure_bh(t);
    int i, fl; double w;
    row_pos(k, 2.0, p->gamma_max, p->n_E, &i, &w, &fl);
    const double* base = t->bh_cdf + (int64_t)iz * p->n_E * p->n_s;
    const double* ra = base + (int64_t)i * p->n_s;
    const double* rb = base + (int64_t)(i + 1) * p->n_s;
    double c0, fr; int j;
    invert_row(ra, rb, w, p->n_s, R, &c0, &j, &fr);
    double s;
    if (j < 0) s = 0.0;
    else if (j >= p->n_s - 1) s = 1.0;
    else s = ((double)j + fr) / (double)(p->n_s - 1);
    return 1.0 / k + s * (1.0 - 2.0 / k);
}

/* ------------------------------------------------------------------------- */
/* Breit-Wheeler pair production of a photon in a locally constant crossed    */
/* field (Sec. 1 names the process; the rate is the one of the same LCFA      */
/* model as the NCS module).  Per unit positron energy fraction x, with       */
/* xi = 2 / (3 chi x (1 - x)):                                                */
/*   G(chi, x) = (x/(1-x) + (1-x)/x) K_{2/3}(xi) + int_xi^inf K_{1/3}(t) dt   */
/* and the rate W = alpha (m c^2/hbar) (m c^2 / (hbar omega)) T(chi),         */
/*   T(chi) = (1 / (sqrt 3 pi)) int_0^1 G(chi, x) dx.                         */
/* ------------------------------------------------------------------------- */
double or_int_k13(double x) { return bessel_common(1.0 / 3.0, x, 1); }

double or_bw_G(double chi, double x) {
    if (!(chi > 0.0) || !(x > 0.0) || !(x < 1.0)) return 0.0;
    double xi = 2.0 / (3.0 * chi * x * (1.0 - x));
    if (xi > 700.0) return 0.0;                  /* below 1e-300 of the peak */
    return (x / (1.0 - x) + (1.0 - x) / x) * or_bessel_k(2.0 / 3.0, xi) + or_int_k13(xi);
}

/* the x grid of the tables: x_j = (1 - cos(pi s_j)) / 2, s_j = j / (n - 1), which
 * clusters the nodes at both ends where the spectrum of large chi peaks */
#ifdef OR_MUTANT_BW_X_NODES
static double bw_x_of_s(double s) { return s; }
#else
static double bw_x_of_s(double s) { return 0.5 * (1.0 - cos(M_PI * s)); }
#endif

typedef struct { double chi; } bw_ctx;
static double bw_integrand_s(double s, const void* vc) {
    const bw_ctx* c = (const bw_ctx*)vc;
    return or_bw_G(c->chi, bw_x_of_s(s)) * 0.5 * M_PI * sin(M_PI * s);      /* dx = (pi/2) sin(pi s) ds */
}

/* int_0^1 G dx over the cells of an n-node s grid, each cell by a fixed 15-point
 * Gauss-Kronrod rule on two halves (G is smooth in s within a cell; a fixed rule keeps
 * the cost bounded where the nested Bessel quadratures carry rounding noise), cumulative
 * values into row if given (row[0] = 0) */
static double bw_cumulate(double chi, int n, double* row) {
    bw_ctx c = {chi};
    double cum = 0.0;
    if (row) row[0] = 0.0;
    for (int j = 1; j < n; ++j) {
        double a = (double)(j - 1) / (double)(n - 1), b = (double)j / (double)(n - 1), m = 0.5 * (a + b);
        double k1, g1, m1, k2, g2, m2;
        gk15(bw_integrand_s, &c, a, m, &k1, &g1, &m1);
        gk15(bw_integrand_s, &c, m, b, &k2, &g2, &m2);
        cum += k1 + k2;
        if (row) row[j] = cum;
    }
    return cum;
}

/* T = int G dx / (sqrt3 pi) */
#ifdef OR_MUTANT_BW_NORM
#define BW_NORM (sqrt(3.0) * 2.0 * M_PI)
#else
#define BW_NORM (sqrt(3.0) * M_PI)
#endif
/* by the same rule on 256 cells (no table) */
double or_bw_T_direct(double chi) {
    if (!(chi > 0.0)) return 0.0;
    return bw_cumulate(chi, 257, NULL) / BW_NORM;
}

struct or_bw_tables {
    int n_chi, n_x;
    double chi_min, chi_max;
    double* T;        /* [n_chi] T(chi_i), chi_i log spaced on [chi_min, chi_max] */
    double* cdf;      /* [n_chi][n_x] normalised cumulative G over x_j            */
};

or_bw_tables* or_bw_tables_build(int n_chi, double chi_min, double chi_max, int n_x) {
    if (n_chi < 2 || n_x < 2 || !(chi_min > 0.0) || !(chi_max > chi_min)) return NULL;
    or_bw_tables* t = (or_bw_tables*)calloc(1, sizeof(or_bw_tables));
    t->n_chi = n_chi; t->n_x = n_x; t->chi_min = chi_min; t->chi_max = chi_max;
    t->T = (double*)calloc((size_t)n_chi, sizeof(double));
    t->cdf = (double*)calloc((size_t)n_chi * n_x, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n_chi; ++i) {
        double chi = grid_log(chi_min, chi_max, i, n_chi);
        double* row = t->cdf + (int64_t)i * n_x;
        double tot = bw_cumulate(chi, n_x, row);
        t->T[i] = tot / BW_NORM;
        for (int j = 0; j < n_x; ++j) row[j] = tot > 0.0 ? row[j] / tot : (double)j / (double)(n_x - 1);
    }
    return t;
}

void or_bw_tables_free(or_bw_tables* t) {
    if (!t) return;
    free(t->T); free(t->cdf); free(t);
}

int64_t or_bw_tables_export(const or_bw_tables* t, int which, double* out, int64_t cap) {
    int64_t n = which == 0 ? t->n_chi : which == 1 ? (int64_t)t->n_chi * t->n_x : -1;
    if (n < 0 || n > cap) return -1;
    memcpy(out, which == 0 ? t->T : t->cdf, (size_t)n * sizeof(double));
    return n;
}

/* T(chi) between nodes: ln(T e^{8/(3 chi)}) linear in ln chi (the factor takes out the
 * exponential of the small-chi limit, which no polynomial in ln chi follows); 0 below the
 * table (flag -1), the last node above it (flag 1) */
double or_bw_T_interp(const or_bw_tables* t, double chi, int* flag) {
    if (!(chi >= t->chi_min)) { *flag = -1; return 0.0; }
    int i; double w;
    row_pos(chi, t->chi_min, t->chi_max, t->n_chi, &i, &w, flag);
    if (*flag == 1) return t->T[t->n_chi - 1];
    double ca = grid_log(t->chi_min, t->chi_max, i, t->n_chi), cb = grid_log(t->chi_min, t->chi_max, i + 1, t->n_chi);
    double la = log(t->T[i]) + 8.0 / (3.0 * ca), lb = log(t->T[i + 1]) + 8.0 / (3.0 * cb);
    return exp((1.0 - w) * la + w * lb - 8.0 / (3.0 * chi));
}

/* positron energy fraction x from the CDF rows interpolated at chi (weights linear
 * in ln chi, clamped to the table), inverted linearly in s between nodes */
double or_bw_sample_x(const or_bw_tables* t, double chi, double R) {
    int i, fl; double w;
    if (!(chi >= t->chi_min)) chi = t->chi_min;
    row_pos(chi, t->chi_min, t->chi_max, t->n_chi, &i, &w, &fl);
    const double* ra = t->cdf + (int64_t)i * t->n_x;
    const double* rb = ra + t->n_x;
    double c0, fr; int j;
    invert_row(ra, rb, w, t->n_x, R, &c0, &j, &fr);
    double s;
    if (j < 0) s = 0.0;
    else if (j >= t->n_x - 1) s = 1.0;
    else s = ((double)j + fr) / (double)(t->n_x - 1);
    return bw_x_of_s(s);
}
