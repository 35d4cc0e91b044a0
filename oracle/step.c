/*
 * step.c -- oracle particle step.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * One particle at a time, FP64, in the order of the method:
 *   E, B at (x^n, t^n)                         prescribed laser (Sec. 3 setup)
 *   Boris push u^{n-1/2} -> u^{n+1/2}           "particle pusher" (Sec. 2.2)
 *   eta from u^{n+1/2} and E, B                 Sec. 2.1 (quantum parameter)
 *   NCS optical depth tau -= dN/dt dt; emit at tau <= 0     Sec. 2.2 (EPOCH)
 *   brems: P = 1 - exp(-n sigma v dt), event iff R1 < P      Eq. (4)
 *          photon energy from sigma(y,E) = sigma(E) R2, k along v  Sec. 2.2
 *   photons below m c^2 are created but not stored           Sec. 3
 *   x^{n+1} = x^n + dt u^{n+1/2} / gamma
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 */
#define C_ALPHA 7.2973525693e-3
#define C_RE 2.8179403262e-15          /* classical electron radius, m  */
#define C_MEC2_MEV 0.51099895000       /* m_e c^2, MeV                  */
#define C_HBARC_MEVM 197.3269804e-15   /* hbar c, MeV m                 */
#define C_LIGHT 299792458.0
#define HIST_EMAX_MEV 10000.0          /* top of the energy histogram   */

/* OR_MUTANT_* (never defined in a normal build, here and in tables.c): each plants one
 * plausible mistake (a dropped term, a wrong sign, a missing factor, a lag, a wrong
 * constant) so that the tests can show that a pin fails for it (tests/test_oracle_mutants.py). */

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, from its published definition (Salmon et al., SC'11):      */
/* 10 rounds of two 32x32->64 multiplies (M0 = 0xD2511F53, M1 = 0xCD9E8D57), */
/* key bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85) between rounds. */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
#ifdef OR_MUTANT_PHILOX_MULT
        uint64_t p0 = (uint64_t)0xD2511F55u * (uint64_t)c0;
#else
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
#endif
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
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

/* purposes of the per-particle Philox streams */
enum { PUR_BREMS = 0, PUR_NCS = 1, PUR_TAU0 = 2, PUR_POS = 3, PUR_MJ = 4, PUR_WAIT = 256 };
/* photon streams: counter word 0 = the photon's id_mech, word 3 = PUR_BH + emission step */
#define PUR_BH 0x40000000u
/* free-path draws: word 3 = PUR_BH_FREE + emission step (emission steps below 2^28) */
#define PUR_BH_FREE 0x50000000u

static void draw(const or_run_params* r, int64_t id, uint32_t step, uint32_t purpose, uint32_t w[4]) {
    uint32_t ctr[4] = {(uint32_t)id, r->run_id, step, purpose};
    uint32_t key[2] = {(uint32_t)(r->seed & 0xffffffffu), (uint32_t)(r->seed >> 32)};
    or_philox4x32_10(ctr, key, w);
}
static uint64_t word64(uint32_t lo, uint32_t hi) { return ((uint64_t)hi << 32) | (uint64_t)lo; }
/* uniform in (0,1) with 53 random bits */
static double u53(uint64_t v) { return ((double)(v >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
/* uniform in (0,1) with 32 random bits */
static double u32(uint32_t v) { return ((double)v + 0.5) * (1.0 / 4294967296.0); }

/* ------------------------------------------------------------------------- */
/* Units                                                                     */
/* ------------------------------------------------------------------------- */
double or_schwinger_field(double lambda_m) {
    /* E_S = m^2 c^3 / (e hbar) in units of m c omega / e  =  m c^2 / (hbar omega) */
    double hbar_omega_mev = 2.0 * M_PI * C_HBARC_MEVM / lambda_m;
    return C_MEC2_MEV / hbar_omega_mev;
}
double or_critical_density(double lambda_m) {
    /* n_c = eps0 m omega^2 / e^2 = pi / (r_e lambda^2) */
    return M_PI / (C_RE * lambda_m * lambda_m);
}

/* ------------------------------------------------------------------------- */
/* Prescribed laser fields.  The pulse is defined through its vector         */
/* potential A(phi) with phi = t - x, so E and B carry no DC part:           */
/*   g(phi): sin^2 ramp over ramp_periods, flat top flat_s, cos^2 ramp;      */
/*   LP:  A = a0 g sin(phi) y^;   CP: A = a0 g (sin(phi) y^ - cos(phi) z^);  */
/*   E = -dA/dt, B = curl A = x^ cross E for the plane wave.                 */
/* The 2D focus multiplies the transverse profile sqrt(w0/w) exp(-y^2/w^2)   */
/* and adds the paraxial curvature and Gouy phase plus the first-order       */
/* longitudinal components required by div E = 0 and div B = 0.              */
/* ------------------------------------------------------------------------- */
static void envelope(const or_run_params* r, double phi, double* g, double* dg) {
    double pr = 2.0 * M_PI * r->ramp_periods;
    double pf = 2.0 * M_PI * r->flat_s * C_LIGHT / r->lambda_m;
    if (phi <= 0.0 || phi >= 2.0 * pr + pf) { *g = 0.0; *dg = 0.0; return; }
    if (phi < pr) {
        double s = sin(0.5 * M_PI * phi / pr);
        *g = s * s;
        *dg = (0.5 * M_PI / pr) * sin(M_PI * phi / pr);
        return;
    }
    if (phi <= pr + pf) { *g = 1.0; *dg = 0.0; return; }
    double q = phi - pr - pf;
    double c = cos(0.5 * M_PI * q / pr);
    *g = c * c;
#ifdef OR_MUTANT_ENVELOPE_FALL
    *dg = (0.5 * M_PI / pr) * sin(M_PI * q / pr);
#else
    *dg = -(0.5 * M_PI / pr) * sin(M_PI * q / pr);
#endif
}

static void incident_fields(const or_run_params* r, double x, double y, double t, double E[3], double B[3]) {
    E[0] = E[1] = E[2] = 0.0;
    B[0] = B[1] = B[2] = 0.0;
    if (r->geometry == OR_CONST) {
        for (int k = 0; k < 3; ++k) { E[k] = r->E_const[k]; B[k] = r->B_const[k]; }
        return;
    }
    double phi = t - x;
    double g, dg;
    envelope(r, phi, &g, &dg);
    if (g == 0.0 && dg == 0.0) return;
    double a0 = r->a0;
    double S = 1.0, theta = phi, inv_R = 0.0, inv_w2 = 0.0;
    if (r->geometry == OR_GAUSS_2D) {
        double kl = 2.0 * M_PI / r->lambda_m;         /* lengths -> c/omega     */
        double w0 = r->w0_m * kl;
        double zr = 0.5 * w0 * w0;
        double xi = x - r->focus_x_m * kl;
        double w2 = w0 * w0 * (1.0 + xi * xi / (zr * zr));
        inv_w2 = 1.0 / w2;
        inv_R = xi / (xi * xi + zr * zr);
#ifdef OR_MUTANT_AMPLITUDE
        S = (w0 / sqrt(w2)) * exp(-y * y * inv_w2);
#else
        S = sqrt(w0 / sqrt(w2)) * exp(-y * y * inv_w2);
#endif
#if defined(OR_MUTANT_GOUY_SIGN)
        theta = phi - 0.5 * y * y * inv_R - 0.5 * atan(xi / zr);
#elif defined(OR_MUTANT_CURVATURE_SIGN)
        theta = phi + 0.5 * y * y * inv_R + 0.5 * atan(xi / zr);
#else
        theta = phi - 0.5 * y * y * inv_R + 0.5 * atan(xi / zr);
#endif
    }
    double st = sin(theta), ct = cos(theta);
    /* y-polarised component: E_y = B_z = -a0 S (g' sin + g cos) */
#ifdef OR_MUTANT_INCIDENT_SIGN
    double ey = a0 * S * (dg * st + g * ct);
#else
    double ey = -a0 * S * (dg * st + g * ct);
#endif
    E[1] = ey;
    B[2] = ey;
    if (r->geometry == OR_GAUSS_2D)
        E[0] = a0 * g * S * (y * inv_R * ct + 2.0 * y * inv_w2 * st);
    if (r->polarisation == OR_CP) {
        /* z-polarised component, a quarter period behind: E_z = -B_y */
        double ez = a0 * S * (dg * ct - g * st);
        E[2] = ez;
        B[1] = -ez;
        if (r->geometry == OR_GAUSS_2D)
            B[0] = a0 * g * S * (2.0 * y * inv_w2 * ct - y * inv_R * st);
    }
}

static void add_reflected(const or_run_params* r, double x, double t, double E[3], double B[3]);
void or_fields(const or_run_params* r, double x, double y, double t, double E[3], double B[3]) {
    incident_fields(r, x, y, t, E, B);
    if (r->geometry == OR_PLANE_1D && r->reflect_r != 0.0) add_reflected(r, x, t, E, B);
}

/* Transverse E of the 1D plane pulse at phase p (the y and z components above). */
static void plane_e(const or_run_params* r, double p, double* ey, double* ez) {
    double g, dg;
    envelope(r, p, &g, &dg);
    double st = sin(p), ct = cos(p);
#ifdef OR_MUTANT_MIRROR_SIGN
    *ey = r->a0 * (dg * st + g * ct);
#else
    *ey = -r->a0 * (dg * st + g * ct);
#endif
    *ez = (r->polarisation == OR_CP) ? r->a0 * (dg * ct - g * st) : 0.0;
}

/* Reflected wave: the mirror image of the incident vector potential in the
 * plane x = x_m, A_r(t, x) = -r A(t + x - 2 x_m).  It travels along -x, so
 * E_r = -r e(psi) with psi = t + x - 2 x_m and B_r = -x^ cross E_r; for r = 1
 * the transverse E vanishes on the mirror plane at all times.                */
static void add_reflected(const or_run_params* r, double x, double t, double E[3], double B[3]) {
    double kl = 2.0 * M_PI / r->lambda_m;
    double psi = t + x - 2.0 * r->mirror_x_m * kl;
    double ey, ez;
    plane_e(r, psi, &ey, &ez);
#ifdef OR_MUTANT_REFL_SQUARED
    double ery = -r->reflect_r * r->reflect_r * ey, erz = -r->reflect_r * r->reflect_r * ez;
#else
    double ery = -r->reflect_r * ey, erz = -r->reflect_r * ez;
#endif
    E[1] += ery;
    E[2] += erz;
    B[1] += erz;
    B[2] -= ery;
}

/* ------------------------------------------------------------------------- */
/* Boris push for charge -e, mass m (normalised: du/dt = -(E + u x B/gamma)) */
/* ------------------------------------------------------------------------- */
void or_boris(double u[3], const double E[3], const double B[3], double dt) {
    double h = 0.5 * dt;
    double um[3] = {u[0] - h * E[0], u[1] - h * E[1], u[2] - h * E[2]};
    double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
#ifdef OR_MUTANT_BORIS_SIGN
    double tv[3] = {h * B[0] / gm, h * B[1] / gm, h * B[2] / gm};
#else
    double tv[3] = {-h * B[0] / gm, -h * B[1] / gm, -h * B[2] / gm};
#endif
    double t2 = tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2];
    double sv[3] = {2.0 * tv[0] / (1.0 + t2), 2.0 * tv[1] / (1.0 + t2), 2.0 * tv[2] / (1.0 + t2)};
    double up[3] = {um[0] + (um[1] * tv[2] - um[2] * tv[1]),
                    um[1] + (um[2] * tv[0] - um[0] * tv[2]),
                    um[2] + (um[0] * tv[1] - um[1] * tv[0])};
    double uq[3] = {um[0] + (up[1] * sv[2] - up[2] * sv[1]),
                    um[1] + (up[2] * sv[0] - up[0] * sv[2]),
                    um[2] + (up[0] * sv[1] - up[1] * sv[0])};
    u[0] = uq[0] - h * E[0];
    u[1] = uq[1] - h * E[1];
    u[2] = uq[2] - h * E[2];
}

/* ------------------------------------------------------------------------- */
/* Quantum parameter (Sec. 2.1; garbled there, read as the standard          */
/* invariant):  eta E_S = sqrt( (gamma E + u x B)^2 - (u.E)^2 ).             */
/* Evaluated through an exact rewriting that avoids cancellation for         */
/* electrons riding a wave along x:  with dB = B - x^ x E and                */
/* V = (gamma - u_x) E + u x dB, one has gamma E + u x B = V + x^ (u.E), so   */
/* the invariant equals |V|^2 + 2 V_x (u.E).  gamma - u_x is formed as       */
/* (1 + u_y^2 + u_z^2)/(gamma + u_x) when u_x > 0.                           */
/* ------------------------------------------------------------------------- */
double or_eta(const double u[3], const double E[3], const double B[3], double E_S) {
    double gamma = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#ifdef OR_MUTANT_ETA_GM
    double gm = (u[0] > 0.0) ? (u[1] * u[1] + u[2] * u[2]) / (gamma + u[0]) : gamma - u[0];
#else
    double gm = (u[0] > 0.0) ? (1.0 + u[1] * u[1] + u[2] * u[2]) / (gamma + u[0]) : gamma - u[0];
#endif
    double dB[3] = {B[0], B[1] + E[2], B[2] - E[1]};
    double V[3] = {gm * E[0] + (u[1] * dB[2] - u[2] * dB[1]),
                   gm * E[1] + (u[2] * dB[0] - u[0] * dB[2]),
                   gm * E[2] + (u[0] * dB[1] - u[1] * dB[0])};
    double uE = u[0] * E[0] + u[1] * E[1] + u[2] * E[2];
#ifdef OR_MUTANT_ETA_UE
    double q = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    (void)uE;
#else
    double q = V[0] * V[0] + V[1] * V[1] + V[2] * V[2] + 2.0 * V[0] * uE;
#endif
    return q > 0.0 ? sqrt(q) / E_S : 0.0;
}

/* ------------------------------------------------------------------------- */
/* 128-bit fixed-point energy tally: value = hi + lo * 2^-64                 */
/* ------------------------------------------------------------------------- */
static void fx_add(uint64_t* w, double v) {
    if (!(v > 0.0)) return;
    double ip = floor(v);
    double fr = v - ip;
    uint64_t lo = (uint64_t)(fr * 18446744073709551616.0);
    uint64_t old = w[0];
    w[0] = old + lo;
    if (w[0] < old) w[1] += 1;
    w[1] += (uint64_t)ip;
}

/* ------------------------------------------------------------------------- */
/* Null-collision bremsstrahlung (the speed-up the paper names for the MC    */
/* collision, Sec. 4; method of Skullerud 1968).  Candidate collisions come  */
/* from a majorant process that ignores position and energy: per step a      */
/* candidate with probability P_hat = 1 - exp(-x_hat), x_hat = n_i c dt times */
/* the largest tabulated sigma_Z (beta <= 1 and the slab indicator <= 1).    */
/* The steps between candidates are geometric, drawn as floor(-ln U/x_hat).  */
/* A candidate becomes a collision with probability P/P_hat, P the Eq. 4     */
/* probability of the step, so a collision happens in a step with            */
/* probability P exactly, as in the direct method.                           */
/* ------------------------------------------------------------------------- */
extern double or__sigma_max(const or_tables* t, int iz);
double or_null_x_hat(const or_tables* t, const or_run_params* r) {
    double kl = 2.0 * M_PI / r->lambda_m;
    double dt = r->dt_over_T * 2.0 * M_PI;
    double n_i = r->ne_over_nc * or_critical_density(r->lambda_m) / r->charge_state;
    double smax = or__sigma_max(t, r->iz);
    return n_i * C_ALPHA * C_RE * C_RE * (dt / kl) * smax;
}
/* steps to the next candidate: floor(-ln U / x_hat), OR_WAIT_NEVER when that
 * does not fit in 32 bits (or x_hat = 0)                                    */
static uint32_t wait_draw(double x_hat, uint64_t v) {
#ifdef OR_MUTANT_WAIT_SCALE
    double q = -log(u53(v)) / (2.0 * x_hat);
#else
    double q = -log(u53(v)) / x_hat;
#endif
    if (!(q < 4294967295.0)) return OR_WAIT_NEVER;
    return (uint32_t)floor(q);
}

/* ------------------------------------------------------------------------- */
/* Run context                                                               */
/* ------------------------------------------------------------------------- */
typedef struct {
    double dt, E_S, C_ncs, K_br, x0, x1, yh, box0, box1, log_emax;
    double photon_min;
    double x_hat, P_hat;          /* null-collision majorant (brems_method NULL) */
} run_ctx;

static void make_ctx(const or_tables* t, const or_run_params* r, run_ctx* c, double photon_min) {
    double kl = 2.0 * M_PI / r->lambda_m;              /* 1/m -> c/omega units */
    c->dt = r->dt_over_T * 2.0 * M_PI;
    c->E_S = or_schwinger_field(r->lambda_m);
    /* dN/dt = sqrt(3) alpha /(2 pi) * (m c^2/hbar) * (eta/gamma) h(eta); in 1/omega units */
    c->C_ncs = sqrt(3.0) * C_ALPHA / (2.0 * M_PI) * c->E_S;
    /* x_b = n_i sigma beta c dt; sigma in alpha r_e^2, c dt in metres */
    double n_i = r->ne_over_nc * or_critical_density(r->lambda_m) / r->charge_state;
    c->K_br = n_i * C_ALPHA * C_RE * C_RE * (c->dt / kl);
    c->x0 = r->slab_x0_m * kl;
    c->x1 = (r->slab_x0_m + r->slab_thick_m) * kl;
    c->yh = r->y_half_m * kl;
    c->box0 = r->box_x_m[0] * kl;
    c->box1 = r->box_x_m[1] * kl;
    c->log_emax = log(HIST_EMAX_MEV / C_MEC2_MEV);
    c->photon_min = photon_min;
    c->x_hat = or_null_x_hat(t, r);
    c->P_hat = -expm1(-c->x_hat);
}

/* table params are needed for photon_min; fetch through the export API */
extern double or__photon_min(const or_tables* t);

int or_init(const or_tables* t, const or_run_params* r, const int64_t* ids, int64_t n_ids, double* st,
            uint32_t* wait) {
    if (r->brems_method == OR_BREMS_NULL && !wait && n_ids > 0) return -1;
    run_ctx c;
    make_ctx(t, r, &c, or__photon_min(t));
#ifdef OR_MUTANT_MJ_TEMPERATURE
    double theta = 0.5 * r->T_mev / C_MEC2_MEV;
#else
    double theta = r->T_mev / C_MEC2_MEV;
#endif
    for (int64_t k = 0; k < n_ids; ++k) {
        int64_t id = ids[k];
        uint32_t w[4];
        double* s = st + 6 * k;
        draw(r, id, 0, PUR_POS, w);
        /* a beam enters at the front face of the slab (Sec. 2.2 bunch benchmark) */
#ifdef OR_MUTANT_INIT_SPREAD
        s[0] = (r->init_dist == OR_BEAM) ? c.x0 : c.x0 + 2.0 * (c.x1 - c.x0) * u32(w[0]);
#else
        s[0] = (r->init_dist == OR_BEAM) ? c.x0 : c.x0 + (c.x1 - c.x0) * u32(w[0]);
#endif
        s[1] = (r->geometry == OR_GAUSS_2D) ? -c.yh + 2.0 * c.yh * u32(w[1]) : 0.0;
        s[2] = s[3] = s[4] = 0.0;
        if (r->init_dist == OR_MAXWELL_JUTTNER) {
            /* Sobol (1976) rejection for the Maxwell-Juttner momentum magnitude */
            double um = 0.0;
            for (uint32_t round = 0; round < 64; ++round) {
                uint32_t m[4];
                draw(r, id, 0, PUR_MJ + round, m);
                double X1 = u32(m[0]), X2 = u32(m[1]), X3 = u32(m[2]), X4 = u32(m[3]);
                double uu = -theta * log(X1 * X2 * X3);
                double ee = -theta * log(X1 * X2 * X3 * X4);
                if (ee * ee - uu * uu > 1.0) { um = uu; break; }
            }
            /* isotropic direction from the position draw's last two words */
            double X5 = u32(w[2]), X6 = u32(w[3]);
            double sn = 2.0 * sqrt(X5 * (1.0 - X5));
            s[2] = um * (2.0 * X5 - 1.0);
            s[3] = um * sn * cos(2.0 * M_PI * X6);
            s[4] = um * sn * sin(2.0 * M_PI * X6);
        } else if (r->init_dist == OR_BEAM) {
            s[2] = sqrt(r->beam_gamma * r->beam_gamma - 1.0);
        }
        draw(r, id, 0, PUR_TAU0, w);
        s[5] = -log(u53(word64(w[0], w[1])));
        if (r->brems_method == OR_BREMS_NULL) {
            draw(r, id, 0, PUR_WAIT, w);
            wait[k] = wait_draw(c.x_hat, word64(w[0], w[1]));
        }
    }
    return 0;
}

typedef struct { or_photon* v; int64_t n, cap; } plist;
static void plist_push(plist* l, const or_photon* p) {
    if (l->n == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 8;
        l->v = (or_photon*)realloc(l->v, sizeof(or_photon) * l->cap);
    }
    l->v[l->n++] = *p;
}

static void record(const run_ctx* c, double x, double y, double ew, const double k[3], uint32_t step,
                   int64_t id, int mech, plist* pl, uint64_t* hist, uint64_t* tally) {
    or_photon p;
    p.x = (float)x; p.y = (float)y; p.energy = (float)ew;
    p.kx = (float)k[0]; p.ky = (float)k[1]; p.kz = (float)k[2];
    p.step = step;
    p.id_mech = (uint32_t)id | ((uint32_t)mech << 31);
    plist_push(pl, &p);
#ifdef OR_MUTANT_HIST_SHIFT
    int eb = (int)floor((double)OR_HIST_E_BINS * log(ew) / c->log_emax) + 1;
#else
    int eb = (int)floor((double)OR_HIST_E_BINS * log(ew) / c->log_emax);
#endif
    if (eb >= OR_HIST_E_BINS) { eb = OR_HIST_E_BINS - 1; tally[ORT_N_HIST_OVER]++; }
    if (eb < 0) eb = 0;
    double th = atan2(k[1], k[0]);
    int tb = (int)floor((th + M_PI) / (2.0 * M_PI) * (double)OR_HIST_T_BINS);
    if (tb < 0) tb = 0;
    if (tb >= OR_HIST_T_BINS) tb = OR_HIST_T_BINS - 1;
    hist[mech * OR_HIST_E_BINS + eb]++;
    hist[2 * OR_HIST_E_BINS + mech * OR_HIST_T_BINS + tb]++;
}

/* energy-conserving recoil along u: gamma' = gamma - w, u' = u^ sqrt(gamma'^2 - 1) */
static void recoil(double u[3], double gamma, double w, double khat[3]) {
    double um = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#ifdef OR_MUTANT_PHOTON_BACKWARD
    if (um > 0.0) { khat[0] = -u[0] / um; khat[1] = -u[1] / um; khat[2] = -u[2] / um; }
#else
    if (um > 0.0) { khat[0] = u[0] / um; khat[1] = u[1] / um; khat[2] = u[2] / um; }
#endif
    else { khat[0] = 1.0; khat[1] = 0.0; khat[2] = 0.0; }
    double g2 = gamma - w;
    double un = (g2 > 1.0) ? sqrt(g2 * g2 - 1.0) : 0.0;
    u[0] = khat[0] * un; u[1] = khat[1] * un; u[2] = khat[2] * un;
}

static void note_event(uint64_t* ev, int64_t n, int mech) {
    if (!ev) return;
    uint32_t cnt = (uint32_t)(*ev & 0xffffffffu), hs = (uint32_t)(*ev >> 32);
    cnt += mech ? 0x10000u : 1u;
    hs += (uint32_t)(n + 1) * (mech ? 0x9E3779B1u : 1u);
    *ev = ((uint64_t)hs << 32) | cnt;
}

/* One step n of one particle in the fields E, B at (x^n, t^n) (Sec. 2.2 order):
 * push, NCS optical depth and emission, brems test (Eq. 4, direct or null
 * collisions), position update, absorbing box.                               */
static void particle_step(const or_tables* t, const or_run_params* r, const run_ctx* c, int64_t id, int64_t n,
                          double* px, double* py, double u[3], double* ptau, uint32_t* wait, const double E[3],
                          const double B[3], plist* pl, uint64_t* hist, uint64_t* tally, uint64_t* ev) {
    double x = *px, y = *py, tau = *ptau;
    or_boris(u, E, B, c->dt);
    double gamma = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (r->enable_ncs) {
        double eta = or_eta(u, E, B, c->E_S);
        int fl;
        double h = or_ncs_h_interp(t, eta, &fl);
        if (fl == 1) tally[ORT_N_ETA_ABOVE]++;
#if defined(OR_MUTANT_NCS_NO_GAMMA)
        tau -= c->C_ncs * eta * h * c->dt;
        if (tau <= 0.0) {
#elif defined(OR_MUTANT_NCS_LAG)
        const double tau_before = tau;
        tau -= c->C_ncs * (eta / gamma) * h * c->dt;
        if (tau_before <= 0.0) {
#else
        tau -= c->C_ncs * (eta / gamma) * h * c->dt;
        if (tau <= 0.0) {
#endif
            uint32_t w[4];
            draw(r, id, (uint32_t)n, PUR_NCS, w);
            int below;
            double delta = or_sample_ncs_delta(t, eta, u53(word64(w[0], w[1])), &below);
            if (below) tally[ORT_N_ETA_BELOW]++;
            double ew = delta * gamma;
#ifdef OR_MUTANT_CLAMP_GAMMA
            if (ew > gamma) { ew = gamma; tally[ORT_N_CLAMP]++; }
#else
            if (ew > gamma - 1.0) { ew = gamma - 1.0; tally[ORT_N_CLAMP]++; }
#endif
            double k[3];
            recoil(u, gamma, ew, k);
            note_event(ev, n, 0);
            double gn = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#ifdef OR_MUTANT_RECOIL_TALLY
            fx_add(tally + ORT_E_RECOIL_NCS, gn - gamma);
#else
            fx_add(tally + ORT_E_RECOIL_NCS, gamma - gn);
#endif
            if (ew >= c->photon_min) {
                tally[ORT_N_NCS_STORED]++;
                tally[ORT_N_PHOTONS]++;
                fx_add(tally + ORT_E_NCS_STORED, ew);
                record(c, x, y, ew, k, (uint32_t)n, id, 0, pl, hist, tally);
            } else {
                tally[ORT_N_NCS_BELOW]++;
                fx_add(tally + ORT_E_NCS_BELOW, ew);
            }
            gamma = gn;
#ifndef OR_MUTANT_TAU_NO_RESET
            tau = -log(u53(word64(w[2], w[3])));
#endif
        }
    }
    if (r->enable_brems) {
        int in_slab = (x >= c->x0 && x <= c->x1);
#ifndef OR_MUTANT_TARGET_Y
        if (r->geometry == OR_GAUSS_2D && fabs(y) > c->yh) in_slab = 0;
#endif
        int nullc = (r->brems_method == OR_BREMS_NULL);
        /* direct method: every step in the slab is a test (Eq. 4); null
         * collisions: only the candidate steps of the majorant process  */
        int test = nullc ? (*wait == 0) : (in_slab && gamma > 1.0 + c->photon_min);
        if (nullc && !test && *wait != OR_WAIT_NEVER) --*wait;
        if (test) {
            double P = 0.0;                  /* Eq. 4 probability of this step */
            if (in_slab && gamma > 1.0 + c->photon_min) {
                int above;
                double sig = or_brems_sigma_interp(t, r->iz, gamma, &above);
                if (above) tally[ORT_N_GAMMA_ABOVE]++;
                double um = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#ifdef OR_MUTANT_BREMS_NO_BETA
                double xb = c->K_br * sig;
                (void)um;
#else
                double xb = c->K_br * sig * (um / gamma);
#endif
                P = -expm1(-xb);
            }
#ifdef OR_MUTANT_NULL_THINNING
            double p_acc = P;
#else
            double p_acc = nullc ? P / c->P_hat : P;
#endif
            /* direct: one draw of purpose 0 at step n (test word, photon-energy word);
             * null: one draw of purpose 256 at step n + 1 (next-wait word, test word),
             * and purpose 0 at step n only for a collision (photon-energy word)  */
            uint32_t w[4], v[4];
            uint64_t U;
            if (nullc) {
                draw(r, id, (uint32_t)n + 1u, PUR_WAIT, v);
                U = word64(v[2], v[3]);
            } else {
                draw(r, id, (uint32_t)n, PUR_BREMS, w);
                U = word64(w[0], w[1]);
            }
            uint64_t thr = (uint64_t)floor(p_acc * 18446744073709551616.0);
            if (p_acc >= 1.0) thr = UINT64_MAX;
            if (U < thr) {
                if (nullc) draw(r, id, (uint32_t)n, PUR_BREMS, w);
                double yy = or_sample_brems_y(t, r->iz, gamma, u53(word64(w[2], w[3])));
                double ew = yy * gamma;
                double k[3];
                recoil(u, gamma, ew, k);
                note_event(ev, n, 1);
                double gn = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                fx_add(tally + ORT_E_RECOIL_BR, gamma - gn);
                if (ew >= c->photon_min) {
                    tally[ORT_N_BR_STORED]++;
                    tally[ORT_N_PHOTONS]++;
                    fx_add(tally + ORT_E_BR_STORED, ew);
                    record(c, x, y, ew, k, (uint32_t)n, id, 1, pl, hist, tally);
                } else {
                    tally[ORT_N_BR_BELOW]++;
                    fx_add(tally + ORT_E_BR_BELOW, ew);
                }
                gamma = gn;
            }
            if (nullc) *wait = wait_draw(c->x_hat, word64(v[0], v[1]));
        }
    }
#ifdef OR_MUTANT_POSITION_NO_GAMMA
    x += c->dt * u[0];
#else
    x += c->dt * u[0] / gamma;
#endif
#ifdef OR_MUTANT_Y_UPDATE
    if (r->geometry == OR_GAUSS_2D) y += c->dt * u[2] / gamma;
#else
    if (r->geometry == OR_GAUSS_2D) y += c->dt * u[1] / gamma;
#endif
#ifdef OR_MUTANT_BOX_ONE_SIDED
    if (r->box_enable && x > c->box1) {
#else
    if (r->box_enable && (x < c->box0 || x > c->box1)) {
#endif
        x = NAN;
        tally[ORT_N_KILLED]++;
        tally[ORT_KILLED_STEPS] += (uint64_t)(n + 1);
    }
    *px = x; *py = y; *ptau = tau;
}

static void run_one(const or_tables* t, const or_run_params* r, const run_ctx* c, int64_t id,
                    int64_t step0, int64_t n_steps, double* s, uint32_t* wait, plist* pl, uint64_t* hist,
                    uint64_t* tally, uint64_t* ev) {
    double x = s[0], y = s[1];
    double u[3] = {s[2], s[3], s[4]};
    double tau = s[5];
    for (int64_t n = step0; n < step0 + n_steps; ++n) {
        if (isnan(x)) break;
        double tn = (double)n * c->dt;
        double E[3], B[3];
        or_fields(r, x, y, tn, E, B);
        particle_step(t, r, c, id, n, &x, &y, u, &tau, wait, E, B, pl, hist, tally, ev);
    }
    s[0] = x; s[1] = y; s[2] = u[0]; s[3] = u[1]; s[4] = u[2]; s[5] = tau;
}

int or_run(const or_tables* t, const or_run_params* r, const int64_t* ids, int64_t n_ids,
           int64_t step0, int64_t n_steps, double* state, uint32_t* wait,
           or_photon* photons, int64_t cap, int64_t* n_photons,
           uint64_t* hist, uint64_t* tally, uint64_t* events, int n_threads) {
    if (!t || !r || n_ids < 0 || n_steps < 0) return -1;
    if (r->brems_method == OR_BREMS_NULL && !wait && n_ids > 0) return -1;
    run_ctx c;
    make_ctx(t, r, &c, or__photon_min(t));
    plist* lists = (plist*)calloc(n_ids > 0 ? n_ids : 1, sizeof(plist));
    int nt = n_threads > 0 ? n_threads : 1;
    uint64_t* th_hist = (uint64_t*)calloc((size_t)nt * OR_HIST_WORDS, sizeof(uint64_t));
    uint64_t* th_tally = (uint64_t*)calloc((size_t)nt * ORT_WORDS, sizeof(uint64_t));
#pragma omp parallel for num_threads(nt) schedule(dynamic, 16)
    for (int64_t k = 0; k < n_ids; ++k) {
        int me = 0;
#ifdef _OPENMP
        me = omp_get_thread_num();
#endif
        run_one(t, r, &c, ids[k], step0, n_steps, state + 6 * k, wait ? wait + k : NULL, &lists[k],
                th_hist + (size_t)me * OR_HIST_WORDS, th_tally + (size_t)me * ORT_WORDS,
                events ? events + k : NULL);
    }
    for (int k = 0; k < nt; ++k) {
        const uint64_t* th = th_tally + (size_t)k * ORT_WORDS;
        for (int i = 0; i < OR_HIST_WORDS; ++i) hist[i] += th_hist[(size_t)k * OR_HIST_WORDS + i];
        for (int i = 0; i < ORT_E_NCS_STORED; ++i) tally[i] += th[i];
        /* 128-bit fixed-point pairs (lo, hi) */
        for (int i = ORT_E_NCS_STORED; i <= ORT_E_RECOIL_BR; i += 2) {
            uint64_t old = tally[i];
            tally[i] = old + th[i];
            if (tally[i] < old) tally[i + 1] += 1;
            tally[i + 1] += th[i + 1];
        }
    }
    int64_t total = 0;
    for (int64_t k = 0; k < n_ids; ++k) {
        for (int64_t j = 0; j < lists[k].n; ++j) {
            if (total < cap) photons[total] = lists[k].v[j];
            ++total;
        }
        free(lists[k].v);
    }
    *n_photons = total;
    free(lists); free(th_hist); free(th_tally);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* 1D electromagnetic PIC around the step.                                   */
/* Normalised Maxwell equations (c = 1, E and B in m c omega / e, J in        */
/* e n_c c, so that dE/dt = curl B - J).  In 1D the transverse fields split   */
/* into waves along +x and -x: F+- = E_y +- B_z and G+- = E_z -+ B_y obey     */
/* dF+-/dt +- dF+-/dx = -J_y and dG+-/dt +- dG+-/dx = -J_z.  With dx = dt      */
/* each is carried one cell per step along its characteristic, the current   */
/* taken at the midpoint of the path (half node, half step):                  */
/*   F+_i^{n+1} = F+_{i-1}^n - dt J_y,i-1/2^{n+1/2},                          */
/*   F-_i^{n+1} = F-_{i+1}^n - dt J_y,i+1/2^{n+1/2}  (same for G with J_z),   */
/* which propagates vacuum waves exactly and, unlike the Yee scheme at        */
/* dx = dt, stays stable with a plasma; E_x^{n+1} = E_x^n - dt J_x^{n+1/2} at */
/* half nodes (Gauss's law is kept by the charge-conserving current).  The    */
/* laser enters at x = 0 (F+_0 = 2 g_y, G+_0 = 2 g_z, g the incident field);   */
/* nothing enters at x = L (F-_N = G-_N = 0); outgoing waves leave freely.    */
/* One step: particles in E^n, B^n (gathered by linear weights) -> x^{n+1};   */
/* an electron that leaves [0, L] deposits its last move, so Gauss's law      */
/* holds on the grid with its charge gone through the boundary, and is then  */
/* removed;                                                                  */
/* currents J^{n+1/2} by linear weighting; fields to n + 1.  Currents are     */
/* summed in 2^-36 fixed point per contribution (exact and order-free, the    */
/* same rule the device code uses).                                          */
/* ------------------------------------------------------------------------- */
#define PIC_FX 68719476736.0                  /* 2^36 */

/* weight of grid point k (node, or half node with off = 0.5) for a particle at s = x/dx */
static double lin_w(double s, int64_t k, double off) {
    double d = fabs(s - ((double)k + off));
    return d < 1.0 ? 1.0 - d : 0.0;
}

void or_pic_gather(int n_cells, double dx, const double* grid, double x, double E[3], double B[3]) {
    const int64_t n = n_cells;
    const double* ex = grid;
    const double* fp = ex + n;
    const double* fm = fp + n + 1;
    const double* gp = fm + n + 1;
    const double* gm = gp + n + 1;
    double s = x / dx;
    int64_t i = (int64_t)floor(s);
    double f = s - (double)i;
    double v[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int k = 0; k < 2; ++k) {
        int64_t m = i + k;
        if (m >= 0 && m <= n) { v[0][k] = fp[m]; v[1][k] = fm[m]; v[2][k] = gp[m]; v[3][k] = gm[m]; }
    }
    double Fp = (1.0 - f) * v[0][0] + f * v[0][1], Fm = (1.0 - f) * v[1][0] + f * v[1][1];
    double Gp = (1.0 - f) * v[2][0] + f * v[2][1], Gm = (1.0 - f) * v[3][0] + f * v[3][1];
    E[1] = 0.5 * (Fp + Fm);
    B[2] = 0.5 * (Fp - Fm);
    E[2] = 0.5 * (Gp + Gm);
#ifdef OR_MUTANT_PIC_BY_SIGN
    B[1] = 0.5 * (Gp - Gm);
#else
    B[1] = 0.5 * (Gm - Gp);
#endif
    B[0] = 0.0;
    /* E_x at half nodes j + 1/2 */
#ifdef OR_MUTANT_PIC_GATHER_NODE
    double sh = s;
#else
    double sh = s - 0.5;
#endif
    int64_t j = (int64_t)floor(sh);
    double fh = sh - (double)j;
    double h0 = (j >= 0 && j < n) ? ex[j] : 0.0, h1 = (j + 1 >= 0 && j + 1 < n) ? ex[j + 1] : 0.0;
    E[0] = (1.0 - fh) * h0 + fh * h1;
}

int or_pic_init(const or_run_params* r, int n_cells, double weight, const double* state, int64_t n, double* grid) {
    if (n_cells < 4 || !grid) return -1;
    memset(grid, 0, sizeof(double) * (size_t)OR_PIC_GRID_WORDS(n_cells));
    double* rho = grid + n_cells + 4 * ((int64_t)n_cells + 1);
    double dx = r->dt_over_T * 2.0 * M_PI;
    for (int64_t p = 0; p < n; ++p) {
        double x = state[6 * p];
        if (isnan(x)) continue;
        double s = x / dx;
        int64_t i0 = (int64_t)floor(s);
        for (int64_t k = i0; k <= i0 + 1; ++k)
            if (k >= 0 && k <= n_cells) rho[k] += weight * lin_w(s, k, 0.0) / dx;   /* ions +, electrons - */
    }
    return 0;
}

/* Current of one electron moving from x_old to x_new (|x_new - x_old| < dx) with
 * velocity (u/gamma): J_x at half nodes from the change of its node weights
 * (cumulative, charge conserving), J_y, J_z at half nodes with the mean of its
 * half-node weights at the two positions.  Accumulated as dimensionless
 * fixed-point sums; the caller applies the weight and the charge sign.       */
static void pic_deposit(double dx, int n_cells, double x_old, double x_new, const double u[3], double gamma,
                        int64_t* ax, int64_t* ay, int64_t* az) {
    double so = x_old / dx, sn = x_new / dx;
    int64_t ia = (int64_t)floor(fmin(so, sn));
    double cum = 0.0;
    for (int64_t k = ia; k <= ia + 1; ++k) {          /* half nodes ia, ia+1 (node ia+2 closes the sum) */
        cum += lin_w(sn, k, 0.0) - lin_w(so, k, 0.0);
#ifdef OR_MUTANT_PIC_CURRENT_SIGN
        if (k >= 0 && k < n_cells) ax[k] -= (int64_t)nearbyint(cum * PIC_FX);
#else
        if (k >= 0 && k < n_cells) ax[k] += (int64_t)nearbyint(cum * PIC_FX);
#endif
    }
    double vy = u[1] / gamma, vz = u[2] / gamma;
    for (int64_t k = ia - 1; k <= ia + 1; ++k) {      /* half nodes touched by either position */
#ifdef OR_MUTANT_PIC_JY_WEIGHT
        double sbar = lin_w(sn, k, 0.5);
#else
        double sbar = 0.5 * (lin_w(so, k, 0.5) + lin_w(sn, k, 0.5));
#endif
        if (sbar > 0.0 && k >= 0 && k < n_cells) {
            ay[k] += (int64_t)nearbyint(vy * sbar * PIC_FX);
            az[k] += (int64_t)nearbyint(vz * sbar * PIC_FX);
        }
    }
}

int or_pic_run(const or_tables* t, const or_run_params* r0, int n_cells, double weight, const int64_t* ids,
               int64_t n_ids, int64_t step0, int64_t n_steps, double* state, uint32_t* wait, double* grid,
               or_photon* photons, int64_t cap, int64_t* n_photons, uint64_t* hist, uint64_t* tally,
               uint64_t* events, int n_threads) {
    if (!t || !r0 || n_ids < 0 || n_steps < 0 || n_cells < 4 || !grid) return -1;
    if (r0->brems_method == OR_BREMS_NULL && !wait && n_ids > 0) return -1;
    or_run_params rr = *r0;
    const double kl = 2.0 * M_PI / rr.lambda_m;
    const double dt = rr.dt_over_T * 2.0 * M_PI, dx = dt;
    const int64_t n = n_cells;
    rr.box_enable = 0;              /* electrons leaving the grid are removed below, after their current */
    const double L = (double)n * dx;
    const or_run_params* r = &rr;
    run_ctx c;
    make_ctx(t, r, &c, or__photon_min(t));
    int nt = n_threads > 0 ? n_threads : 1;
    plist* lists = (plist*)calloc(n_ids > 0 ? n_ids : 1, sizeof(plist));
    uint64_t* th_hist = (uint64_t*)calloc((size_t)nt * OR_HIST_WORDS, sizeof(uint64_t));
    uint64_t* th_tally = (uint64_t*)calloc((size_t)nt * ORT_WORDS, sizeof(uint64_t));
    int64_t* acc = (int64_t*)calloc((size_t)nt * 3 * n, sizeof(int64_t));
    int64_t* jsum = (int64_t*)calloc((size_t)3 * n, sizeof(int64_t));
    double* tmp = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    double* ex = grid;
    double* fp = ex + n;
    double* fm = fp + n + 1;
    double* gp = fm + n + 1;
    double* gm = gp + n + 1;
    for (int64_t s_ = step0; s_ < step0 + n_steps; ++s_) {
        memset(acc, 0, sizeof(int64_t) * (size_t)nt * 3 * n);
        /* particles in E^n, B^n; currents J^{n+1/2} */
#pragma omp parallel for num_threads(nt) schedule(static)
        for (int64_t k = 0; k < n_ids; ++k) {
            int me = 0;
#ifdef _OPENMP
            me = omp_get_thread_num();
#endif
            double* s = state + 6 * k;
            if (isnan(s[0])) continue;
            double x = s[0], y = s[1], u[3] = {s[2], s[3], s[4]}, tau = s[5];
            double E[3], B[3];
            or_pic_gather(n_cells, dx, grid, x, E, B);
            double x_old = x;
            particle_step(t, r, &c, ids[k], s_, &x, &y, u, &tau, wait ? wait + k : NULL, E, B, &lists[k],
                          th_hist + (size_t)me * OR_HIST_WORDS, th_tally + (size_t)me * ORT_WORDS,
                          events ? events + k : NULL);
            double gamma = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            int64_t* a = acc + (size_t)me * 3 * n;
            pic_deposit(dx, n_cells, x_old, x, u, gamma, a, a + n, a + 2 * n);
            if (x < 0.0 || x > L) {     /* it left through a boundary face, carrying its charge out */
                x = NAN;
                uint64_t* tl = th_tally + (size_t)me * ORT_WORDS;
                tl[ORT_N_KILLED]++;
                tl[ORT_KILLED_STEPS] += (uint64_t)(s_ + 1);
            }
            s[0] = x; s[1] = y; s[2] = u[0]; s[3] = u[1]; s[4] = u[2]; s[5] = tau;
        }
        memset(jsum, 0, sizeof(int64_t) * 3 * (size_t)n);
        for (int th = 0; th < nt; ++th)
            for (int64_t k = 0; k < 3 * n; ++k) jsum[k] += acc[(size_t)th * 3 * n + k];
        /* J_x = (w/dt) sum dS (the electron charge -1 included), J_y,z = -(w/dx) sum v S */
        const double kx = weight / dt / PIC_FX, kyz = -weight / dx / PIC_FX;
        const int64_t* jx = jsum;
        const int64_t* jy = jsum + n;
        const int64_t* jz = jsum + 2 * n;
#ifdef OR_MUTANT_PIC_EX_SIGN
        for (int64_t j = 0; j < n; ++j) ex[j] += dt * kx * (double)jx[j];
#else
        for (int64_t j = 0; j < n; ++j) ex[j] -= dt * kx * (double)jx[j];
#endif
        /* waves along +x: node i from node i - 1 through half node i - 1 */
        double gy, gz;
        plane_e(r, (double)(s_ + 1) * dt, &gy, &gz);      /* incident field at x = 0, t^{n+1} */
        memcpy(tmp, fp, sizeof(double) * (size_t)(n + 1));
        for (int64_t i = 1; i <= n; ++i) fp[i] = tmp[i - 1] - dt * kyz * (double)jy[i - 1];
#ifdef OR_MUTANT_PIC_INJECT_HALF
        fp[0] = gy;
#else
        fp[0] = 2.0 * gy;
#endif
        memcpy(tmp, gp, sizeof(double) * (size_t)(n + 1));
        for (int64_t i = 1; i <= n; ++i) gp[i] = tmp[i - 1] - dt * kyz * (double)jz[i - 1];
        gp[0] = 2.0 * gz;
        /* waves along -x: node i from node i + 1 through half node i */
        memcpy(tmp, fm, sizeof(double) * (size_t)(n + 1));
        for (int64_t i = 0; i < n; ++i) fm[i] = tmp[i + 1] - dt * kyz * (double)jy[i];
        fm[n] = 0.0;
        memcpy(tmp, gm, sizeof(double) * (size_t)(n + 1));
        for (int64_t i = 0; i < n; ++i) gm[i] = tmp[i + 1] - dt * kyz * (double)jz[i];
        gm[n] = 0.0;
    }
    for (int k = 0; k < nt; ++k) {
        const uint64_t* th = th_tally + (size_t)k * ORT_WORDS;
        for (int i = 0; i < OR_HIST_WORDS; ++i) hist[i] += th_hist[(size_t)k * OR_HIST_WORDS + i];
        for (int i = 0; i < ORT_E_NCS_STORED; ++i) tally[i] += th[i];
        for (int i = ORT_E_NCS_STORED; i <= ORT_E_RECOIL_BR; i += 2) {
            uint64_t old = tally[i];
            tally[i] = old + th[i];
            if (tally[i] < old) tally[i + 1] += 1;
            tally[i + 1] += th[i + 1];
        }
    }
    int64_t total = 0;
    for (int64_t k = 0; k < n_ids; ++k) {
        for (int64_t j = 0; j < lists[k].n; ++j) {
            if (total < cap) photons[total] = lists[k].v[j];
            ++total;
        }
        free(lists[k].v);
    }
    *n_photons = total;
    free(lists); free(th_hist); free(th_tally); free(acc); free(jsum); free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Bethe-Heitler conversion of the photons in the target (Sec. 2.2: "similar */
/* to the bremsstrahlung"): the direct MC collision of Eq. (4) per step with */
/* sigma_BH, photons moving at c along their direction.                      */
/* ------------------------------------------------------------------------- */
/* conversion of photon j at step m with the fraction word (w2, w3): record and tallies */
static void pair_record(const or_tables* t, const or_run_params* r, const run_ctx* c, const or_photon* ph,
                        int64_t j, int64_t m, double k, double px, double py, int two_d, uint32_t w2, uint32_t w3,
                        or_pair* pairs, int64_t cap, uint64_t* tally) {
    double x = or_sample_bh_x(t, r->iz, k, u53(word64(w2, w3)));
    double ep = x * k;
    int64_t q = (int64_t)tally[ORP_N_PAIRS]++;
    fx_add(tally + ORP_E_PAIRS, k);
    fx_add(tally + ORP_E_POSITRONS, ep);
    (void)c;
    if (q < cap) {
        or_pair* o = pairs + q;
        o->x = (float)px; o->y = (float)(two_d ? py : 0.0);
        o->e_minus = (float)(k - ep); o->e_plus = (float)ep;
        o->kx = ph->kx; o->ky = ph->ky; o->kz = ph->kz;
        o->step = (uint32_t)m; o->photon = (uint32_t)j; o->id_mech = ph->id_mech;
    }
}

int or_pair_transport(const or_tables* t, const or_run_params* r, const or_photon* photons, int64_t n_photons,
                      int64_t step_end, or_pair* pairs, int64_t cap, uint64_t* tally, int method) {
    if (method != OR_PAIR_DIRECT && method != OR_PAIR_FREE_PATH) return -1;
    run_ctx c;
    make_ctx(t, r, &c, or__photon_min(t));
    for (int k = 0; k < ORP_WORDS; ++k) tally[k] = 0;
    const int two_d = (r->geometry == OR_GAUSS_2D);
    for (int64_t j = 0; j < n_photons; ++j) {
        const or_photon* ph = photons + j;
        double k = (double)ph->energy;
        if (!(k > 2.0)) continue;
        double kx = (double)ph->kx, ky = (double)ph->ky, kz = (double)ph->kz;
        double xe = (double)ph->x, ye = (double)ph->y;
        int64_t ne = (int64_t)ph->step;
        int above;
        double sig = or_bh_sigma_interp(t, r->iz, k, &above);
        double P = -expm1(-c.K_br * sig);                  /* beta = 1 */
        uint64_t thr = (uint64_t)floor(P * 18446744073709551616.0);
        if (P >= 1.0) thr = UINT64_MAX;
        uint32_t key[2] = {(uint32_t)(r->seed & 0xffffffffu), (uint32_t)(r->seed >> 32)};
        int was_in = 0;
        int64_t first = -1, last = -1;                     /* the run of steps inside the target */
        for (int64_t m = ne + 1; m < step_end; ++m) {
            double tt = (double)(m - ne) * c.dt;
            double px = fma(kx, tt, xe), py = fma(ky, tt, ye);
            int in = (px >= c.x0 && px <= c.x1);
            if (two_d && fabs(py) > c.yh) in = 0;
            if (!in) {
                if (was_in) break;                         /* left the target */
                if ((px < c.x0 && kx <= 0.0) || (px > c.x1 && kx >= 0.0)) break;
                if (two_d && fabs(py) > c.yh && py * ky >= 0.0) break;
                continue;
            }
            if (!was_in) {
                was_in = 1;
                first = m;
                tally[ORP_N_ENTERED]++;
                if (above) tally[ORP_N_K_ABOVE]++;
            }
            last = m;
            if (method == OR_PAIR_FREE_PATH) continue;     /* the run only; one draw below */
            uint32_t ctr[4] = {ph->id_mech, r->run_id, (uint32_t)m, PUR_BH + (uint32_t)ne};
            uint32_t w[4];
            or_philox4x32_10(ctr, key, w);
            tally[ORP_N_TESTS]++;
            if (word64(w[0], w[1]) < thr) {
                pair_record(t, r, &c, ph, j, m, k, px, py, two_d, w[2], w[3], pairs, cap, tally);
                break;
            }
        }
        if (method == OR_PAIR_FREE_PATH && first >= 0 && c.K_br * sig > 0.0) {
            /* the per-step trials of one crossing, all with probability P = 1 - exp(-lam) (Eq. 4,
             * lam = n_i sigma c dt), fail a geometric number of times before the first success:
             * j = floor(ln U / ln(1 - P)) = floor(-ln U / lam) */
            uint32_t ctr[4] = {ph->id_mech, r->run_id, (uint32_t)first, PUR_BH_FREE + (uint32_t)ne};
            uint32_t w[4];
            or_philox4x32_10(ctr, key, w);
            tally[ORP_N_TESTS]++;
#ifdef OR_MUTANT_BH_FREE_PATH
            double q = floor(-log(u53(word64(w[0], w[1]))) / (2.0 * c.K_br * sig));
#else
            double q = floor(-log(u53(word64(w[0], w[1]))) / (c.K_br * sig));
#endif
            if (q <= (double)(last - first)) {
                int64_t m = first + (int64_t)q;
                double tt = (double)(m - ne) * c.dt;
                pair_record(t, r, &c, ph, j, m, k, fma(kx, tt, xe), fma(ky, tt, ye), two_d, w[2], w[3], pairs, cap,
                            tally);
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Photon quantum parameter: the electron's eta with u -> kvec, gamma -> |k|, */
/* in the same cancellation-safe arrangement (k - k_x = k_perp^2/(k + k_x)).  */
/* ------------------------------------------------------------------------- */
double or_chi_photon(const double kv[3], const double E[3], const double B[3], double E_S) {
    double k = sqrt(kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2]);
    double gm = (kv[0] > 0.0) ? (kv[1] * kv[1] + kv[2] * kv[2]) / (k + kv[0]) : k - kv[0];
    double dB[3] = {B[0], B[1] + E[2], B[2] - E[1]};
    double V[3] = {gm * E[0] + (kv[1] * dB[2] - kv[2] * dB[1]),
                   gm * E[1] + (kv[2] * dB[0] - kv[0] * dB[2]),
                   gm * E[2] + (kv[0] * dB[1] - kv[1] * dB[0])};
    double kE = kv[0] * E[0] + kv[1] * E[1] + kv[2] * E[2];
#ifdef OR_MUTANT_CHI_KE
    double q = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    (void)kE;
#else
    double q = V[0] * V[0] + V[1] * V[1] + V[2] * V[2] + 2.0 * V[0] * kE;
#endif
    return q > 0.0 ? sqrt(q) / E_S : 0.0;
}

/* ------------------------------------------------------------------------- */
/* Breit-Wheeler pair production of the photons in the laser field.  Each     */
/* photon moves at c along its direction from its emission point; at step m   */
/* (n_e < m < step_end) it is at p_m = x_e + k^ (m - n_e) c dt, where the     */
/* fields at (p_m, t_m = m dt) give its chi.  An optical depth tau_0 = -ln U  */
/* falls by W(chi, k) dt per step and the photon converts at the first step   */
/* where it is <= 0: the per-step optical-depth method of the NCS module.     */
/* Photons do not feel the fields, so following each one after the run       */
/* equals stepping it with the electrons (prescribed fields).                 */
/* ------------------------------------------------------------------------- */
#define PUR_BW_TAU 0x60000000u   /* tau_0: counter (id_mech, run id, n_e, PUR_BW_TAU + n_e) */
#define PUR_BW_X 0x70000000u     /* x at the conversion step m: (id_mech, run id, m, PUR_BW_X + n_e) */

int or_bw_transport(const or_bw_tables* bt, const or_tables* t, const or_run_params* r, const or_photon* photons,
                    int64_t n_photons, int64_t step_end, or_pair* pairs, int64_t cap, uint64_t* tally) {
    if (r->geometry == OR_PIC_1D) return -1;     /* self-consistent fields are not stored */
    run_ctx c;
    make_ctx(t, r, &c, or__photon_min(t));
    for (int k = 0; k < ORP_WORDS; ++k) tally[k] = 0;
    const int two_d = (r->geometry == OR_GAUSS_2D);
    const double coef = C_ALPHA * c.E_S * c.dt;          /* W dt = coef T(chi) / k */
    uint32_t key[2] = {(uint32_t)(r->seed & 0xffffffffu), (uint32_t)(r->seed >> 32)};
    for (int64_t j = 0; j < n_photons; ++j) {
        const or_photon* ph = photons + j;
        double k = (double)ph->energy;
        if (!(k > 2.0)) continue;
        double kx = (double)ph->kx, ky = (double)ph->ky, kz = (double)ph->kz;
        double kvec[3] = {k * kx, k * ky, k * kz};
        double xe = (double)ph->x, ye = (double)ph->y;
        int64_t ne = (int64_t)ph->step;
        uint32_t ctr[4] = {ph->id_mech, r->run_id, (uint32_t)ne, PUR_BW_TAU + (uint32_t)ne};
        uint32_t w[4];
        or_philox4x32_10(ctr, key, w);
        double tau = -log(u53(word64(w[0], w[1])));
        tally[ORP_N_ENTERED]++;
        for (int64_t m = ne + 1; m < step_end; ++m) {
            double tt = (double)(m - ne) * c.dt;
#ifdef OR_MUTANT_BW_PHOTON_STILL
            double px = xe, py = ye;
            (void)tt;
#else
            double px = fma(kx, tt, xe), py = fma(ky, tt, ye);
#endif
            double E[3], B[3];
            or_fields(r, px, py, (double)m * c.dt, E, B);
            double chi = or_chi_photon(kvec, E, B, c.E_S);
            int fl;
            double T = or_bw_T_interp(bt, chi, &fl);
            tally[ORP_N_TESTS]++;
            if (fl == 1) tally[ORP_N_K_ABOVE]++;
            tau -= coef * T / k;
            if (tau <= 0.0) {
                uint32_t cx[4] = {ph->id_mech, r->run_id, (uint32_t)m, PUR_BW_X + (uint32_t)ne};
                or_philox4x32_10(cx, key, w);
                double x = or_bw_sample_x(bt, chi, u53(word64(w[0], w[1])));
                double ep = x * k;
                int64_t q = (int64_t)tally[ORP_N_PAIRS]++;
                fx_add(tally + ORP_E_PAIRS, k);
                fx_add(tally + ORP_E_POSITRONS, ep);
                if (q < cap) {
                    or_pair* o = pairs + q;
                    o->x = (float)px; o->y = (float)(two_d ? py : 0.0);
                    o->e_minus = (float)(k - ep); o->e_plus = (float)ep;
                    o->kx = ph->kx; o->ky = ph->ky; o->kz = ph->kz;
                    o->step = (uint32_t)m; o->photon = (uint32_t)j; o->id_mech = ph->id_mech;
                }
                break;
            }
        }
    }
    return 0;
}
