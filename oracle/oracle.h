/*
 * oracle.h -- FP64 CPU oracle for the per-macroparticle photon-emission step of
 * Wan, Lv, Jia, Sang & Xie, "Photon emission by bremsstrahlung and nonlinear
 * Compton scattering in the interaction of ultraintense laser and plasmas"
 * (arXiv:1612.07592).
 *
 * TEST INFRASTRUCTURE ONLY.  This directory is the independent reference the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library.
 *
 * Everything is plain scalar C99 in double precision, one particle at a time,
 * in the order the method states its steps:
 *   fields at (x^n, t^n) -> Boris push -> quantum parameter eta (Sec. 2.1)
 *   -> nonlinear-Compton optical depth (Sec. 2.2, "same as EPOCH")
 *   -> bremsstrahlung direct MC collision (Sec. 2.2, Eq. 4, Eq. 1)
 *   -> position update.
 *
 * Units: time in 1/omega_L, length in c/omega_L, momentum u = p/(m c),
 * fields in m c omega_L / e, energies in m c^2.
 */
#ifndef PE_ORACLE_H
#define PE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) -------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* ---- special functions (integral representations, own quadrature) -------- */
double or_bessel_k(double nu, double x);          /* K_nu(x)                    */
double or_int_k53(double x);                      /* int_x^inf K_{5/3}(t) dt    */
/* Quantum-synchrotron emissivity F(eta, chi) (Sokolov-Ternov form used by
 * Kirk 2009 / Ridgers 2014, which the paper's NCS module follows).            */
double or_ncs_F(double eta, double chi);
/* integral of F over chi in (0, eta/2): the radiated power shape (Larmor pin) */
double or_ncs_power_integral(double eta);
/* h(eta) = int_0^{eta/2} F/chi dchi, by direct quadrature (no table)          */
double or_ncs_h_direct(double eta);

/* ---- bremsstrahlung: Tsai screened DCS, Eq. (1) ---------------------------- */
double or_coulomb_f(double Z);
/* d sigma / d y per atom in units of alpha r_e^2; y = k/E, E = gamma m c^2.
 * complete != 0 forces the screening variables to zero (complete screening).
 * Not clamped: returns the raw bracket value.                                 */
double or_brems_dcs_raw(double Z, double gamma, double y, int complete);
/* sigma_Z(gamma) = int_{ycut}^{ymax} dsigma/dy dy (clamped integrand >= 0),
 * ycut = photon_min/gamma, ymax = 1 - 1/gamma; units alpha r_e^2.            */
double or_brems_sigma_direct(double Z, double gamma, double photon_min);

/* ---- Bethe-Heitler pair production (Sec. 2.2: implemented like the brems) --
 * d sigma / d x per atom in units of alpha r_e^2 for a photon of energy k (m c^2)
 * giving a positron of energy x k and an electron of energy (1 - x) k; Tsai's
 * DCS of the crossed process with the screening fits of Eq. (1).  Not clamped. */
double or_bh_dcs_raw(double Z, double k, double x, int complete);
/* sigma_BH(k) = int_{1/k}^{1-1/k} max(dsigma/dx, 0) dx (0 for k <= 2), alpha r_e^2 */
double or_bh_sigma_direct(double Z, double k);

/* ---- tables ---------------------------------------------------------------- */
typedef struct {
    int n_eta, n_y;           /* NCS rows (log eta) x columns (log y)          */
    double eta_min, eta_max;
    double y_min, y_max;      /* CDF abscissa y = 2 delta / (3 eta (1-delta))  */
    int n_E, n_s;             /* brems rows (log gamma) x columns (s in [0,1]) */
    double gamma_min, gamma_max;
    double photon_min;        /* hard-photon cut in m c^2 (Sec. 3: 0.511 MeV)  */
} or_table_params;

typedef struct or_tables or_tables;
or_tables* or_tables_build(const or_table_params* p, int n_Z, const double* Z);
void or_tables_free(or_tables* t);
/* which: 0 = h(eta_i) [n_eta], 1 = NCS CDF [n_eta*n_y], 2 = classical CDF [n_y],
 *        3 = sigma_Z(gamma_i) [n_E] for Z index iz, 4 = brems CDF [n_E*n_s],
 *        5 = sigma_BH(k_i) [n_E] with k_i log spaced on [2, gamma_max],
 *        6 = Bethe-Heitler CDF over s [n_E*n_s], x = 1/k + s (1 - 2/k).
 * Returns the number of doubles written, or -1.                               */
int64_t or_tables_export(const or_tables* t, int which, int iz, double* out, int64_t cap);
/* classical-limit total int_0^inf (int_y^inf K53) dy as integrated (5 pi/3)  */
double or_tables_classical_total(const or_tables* t);

/* inverse-CDF samplers exactly as the step uses them (exposed for tests)      */
double or_sample_ncs_delta(const or_tables* t, double eta, double R, int* below);
double or_sample_brems_y(const or_tables* t, int iz, double gamma, double R);
double or_ncs_h_interp(const or_tables* t, double eta, int* range_flag);
double or_brems_sigma_interp(const or_tables* t, int iz, double gamma, int* above);
double or_bh_sigma_interp(const or_tables* t, int iz, double k, int* above);
double or_sample_bh_x(const or_tables* t, int iz, double k, double R);

/* ---- Breit-Wheeler pair production in the laser field ----------------------
 * Sec. 1 names the process; as for the NCS module the rate is that of a locally
 * constant crossed field.  For a photon of energy k (m c^2) with quantum
 * parameter chi (or_chi_photon) the pair rate per unit time (1/omega_L) is
 *   W = alpha E_S T(chi) / k,   T(chi) = (1/(sqrt 3 pi)) int_0^1 G(chi, x) dx,
 *   G(chi, x) = (x/(1-x) + (1-x)/x) K_{2/3}(xi) + int_xi^inf K_{1/3}(t) dt,
 *   xi = 2 / (3 chi x (1 - x)),
 * x the positron's share of k (E_S = m c^2 / (hbar omega_L) in these units).   */
double or_int_k13(double x);                      /* int_x^inf K_{1/3}(t) dt     */
double or_bw_G(double chi, double x);
double or_bw_T_direct(double chi);                /* by quadrature (no table)    */
/* chi = sqrt((k E + kvec x B)^2 - (kvec . E)^2) / E_S for the photon momentum kvec
 * (|kvec| = k): the electron's eta with u -> kvec and gamma -> k                */
double or_chi_photon(const double kvec[3], const double E[3], const double B[3], double E_S);
/* tables: T(chi_i) on n_chi log-spaced chi in [chi_min, chi_max] and the CDF of G
 * over x at n_x nodes x_j = (1 - cos(pi j/(n_x - 1)))/2 (clustered at both ends).
 * which: 0 = T [n_chi], 1 = CDF [n_chi * n_x].                                  */
typedef struct or_bw_tables or_bw_tables;
or_bw_tables* or_bw_tables_build(int n_chi, double chi_min, double chi_max, int n_x);
void or_bw_tables_free(or_bw_tables* t);
int64_t or_bw_tables_export(const or_bw_tables* t, int which, double* out, int64_t cap);
/* ln T linear in ln chi; 0 below the table (flag -1), the last node above (flag 1) */
double or_bw_T_interp(const or_bw_tables* t, double chi, int* flag);
/* x from the CDF rows interpolated at chi, inverted linearly in s = acos(1-2x)/pi */
double or_bw_sample_x(const or_bw_tables* t, double chi, double R);

/* ---- run description ------------------------------------------------------- */
enum { OR_LP_Y = 0, OR_CP = 1 };
enum { OR_PLANE_1D = 0, OR_GAUSS_2D = 1, OR_CONST = 2, OR_PIC_1D = 3 };
enum { OR_REST = 0, OR_MAXWELL_JUTTNER = 1, OR_BEAM = 2 };

typedef struct {
    double a0, lambda_m;
    int polarisation, geometry;
    double w0_m, focus_x_m;
    double flat_s, ramp_periods;
    double E_const[3], B_const[3];       /* OR_CONST only (normalised units)    */
    double Z, charge_state, ne_over_nc;
    double slab_x0_m, slab_thick_m, y_half_m;
    double dt_over_T;
    int init_dist;
    double T_mev;                        /* Maxwell-Juttner temperature         */
    double beam_gamma;                   /* OR_BEAM: u = (sqrt(g^2-1), 0, 0) at x = slab front */
    uint64_t seed;
    uint32_t run_id;
    int enable_ncs, enable_brems;
    int box_enable; double box_x_m[2];   /* absorbing box in x                  */
    int iz;                              /* index of Z in the table set         */
    /* reflected wave (OR_PLANE_1D): the incident pulse plus its mirror image in
     * the plane x = mirror_x_m with amplitude coefficient reflect_r (0 = none) */
    double reflect_r, mirror_x_m;
    int brems_method;                    /* OR_BREMS_DIRECT | OR_BREMS_NULL     */
} or_run_params;
enum { OR_BREMS_DIRECT = 0, OR_BREMS_NULL = 1 };
/* wait value meaning "no further candidate collision in this run"            */
#define OR_WAIT_NEVER 0xFFFFFFFFu

/* photon record, 32 bytes */
typedef struct {
    float x, y, energy, kx, ky, kz;
    uint32_t step;
    uint32_t id_mech;                    /* particle id | (mechanism << 31)      */
} or_photon;

/* tally words (uint64) */
enum {
    ORT_N_NCS_STORED = 0, ORT_N_NCS_BELOW = 1, ORT_N_BR_STORED = 2, ORT_N_BR_BELOW = 3,
    ORT_N_PHOTONS = 4, ORT_N_ETA_ABOVE = 5, ORT_N_ETA_BELOW = 6, ORT_N_GAMMA_ABOVE = 7,
    ORT_N_KILLED = 8, ORT_KILLED_STEPS = 9, ORT_N_CLAMP = 10, ORT_N_HIST_OVER = 11,
    ORT_E_NCS_STORED = 16, ORT_E_NCS_BELOW = 18, ORT_E_BR_STORED = 20, ORT_E_BR_BELOW = 22,
    ORT_E_RECOIL_NCS = 24, ORT_E_RECOIL_BR = 26,
    ORT_WORDS = 32
};
#define OR_HIST_E_BINS 512
#define OR_HIST_T_BINS 180
#define OR_HIST_WORDS (2 * OR_HIST_E_BINS + 2 * OR_HIST_T_BINS)

/* Initial state of the listed particles (x, y, ux, uy, uz, tau per particle).
 * wait (one per particle) receives the steps to the first candidate collision
 * of the null-collision brems method; it may be NULL for OR_BREMS_DIRECT.    */
int or_init(const or_tables* t, const or_run_params* r, const int64_t* ids, int64_t n_ids,
            double* state, uint32_t* wait);
/* Advance the listed particles from step0 for n_steps.  state is in/out (6
 * doubles per particle).  Photons of these particles are written in particle
 * order to photons[0..cap); *n_photons receives the true count.  hist and
 * tally are accumulated (not cleared).  Returns 0 on success.                 */
int or_run(const or_tables* t, const or_run_params* r, const int64_t* ids, int64_t n_ids,
           int64_t step0, int64_t n_steps, double* state, uint32_t* wait,
           or_photon* photons, int64_t cap, int64_t* n_photons,
           uint64_t* hist, uint64_t* tally, uint64_t* events, int n_threads);
/* events (nullable): per particle, low 32 bits = NCS count | brems count << 16,
 * high 32 bits = sum over emissions of (step + 1) * (1 or 0x9E3779B1 for brems)
 * mod 2^32 -- a fingerprint of the particle's event list.                     */

/* ---- 1D electromagnetic PIC around the step ------------------------------
 * Geometry OR_PIC_1D: the fields at the particles come from a grid that the
 * electrons' own currents and the injected laser drive (the paper's PIC host with
 * the field solver and weighting on).  n_cells cells over [0, L], dx = c dt;
 * grid layout (doubles, n = n_cells):
 *   ex[n]     E_x at half nodes (i + 1/2) dx
 *   fp[n+1]   E_y + B_z at nodes i dx (moves along +x)
 *   fm[n+1]   E_y - B_z (moves along -x)
 *   gp[n+1]   E_z - B_y (moves along +x)
 *   gm[n+1]   E_z + B_y (moves along -x)
 *   rho[n+1]  immobile ion charge density at the nodes (the electrons' initial
 *             charge with the opposite sign)
 * weight: areal density of one macro-electron (n_c c/omega units).           */
#define OR_PIC_GRID_WORDS(n) (6 * (int64_t)(n) + 5)
/* grid after or_init: zero fields, rho from the initial electrons (state) */
int or_pic_init(const or_run_params* r, int n_cells, double weight, const double* state, int64_t n, double* grid);
/* Advance particles and grid together (step-major); arguments as or_run.  The
 * particle list must be the whole run (the currents of all electrons drive the
 * fields).  Electrons leaving [0, L] are removed after depositing their last
 * move (their charge leaves through the boundary).                           */
int or_pic_run(const or_tables* t, const or_run_params* r, int n_cells, double weight, const int64_t* ids,
               int64_t n_ids, int64_t step0, int64_t n_steps, double* state, uint32_t* wait, double* grid,
               or_photon* photons, int64_t cap, int64_t* n_photons, uint64_t* hist, uint64_t* tally,
               uint64_t* events, int n_threads);
/* fields at x from the grid (linear weights; zero beyond the grid) */
void or_pic_gather(int n_cells, double dx, const double* grid, double x, double E[3], double B[3]);

/* ---- Bethe-Heitler conversion of the emitted photons in the target ----------
 * Each photon record (k = energy > 2 m c^2) moves at c along its direction from
 * its emission point: at step m (emission step n_e < m < step_end) its position
 * is p = x_e + k^ (m - n_e) c dt.  At every step with p inside the target (the
 * slab, and |y| <= y_half in 2D) it takes the test of Eq. (4) with sigma_BH:
 * P = 1 - exp(-n_i sigma_BH(k) c dt), one draw of counter (id_mech, run id, m,
 * 0x40000000 + n_e): test word = words 0-1 against floor(P 2^64), fraction word
 * = words 2-3.  On conversion x is drawn from the CDF (u53 of the fraction word),
 * E+ = x k, E- = k - E+, both along k^; the photon is gone.  A photon that leaves
 * the target, or is outside and moving away from it, is not followed further. */
typedef struct {
    float x, y;               /* conversion point (position at the start of `step`) */
    float e_minus, e_plus;    /* total energies of the electron and the positron, m c^2 */
    float kx, ky, kz;         /* direction of the converted photon                */
    uint32_t step;            /* step of the conversion                           */
    uint32_t photon;          /* index of the photon record                       */
    uint32_t id_mech;         /* the photon's id_mech                             */
} or_pair;
enum { ORP_N_PAIRS = 0, ORP_N_ENTERED = 1, ORP_N_K_ABOVE = 2, ORP_N_TESTS = 3, ORP_E_PAIRS = 4, ORP_E_POSITRONS = 6,
       ORP_WORDS = 8 };
/* pairs in photon order to pairs[0..cap); tally (ORP_WORDS, cleared here):
 * pair count (true count), photons that entered the target, of them above the
 * table's k range, tests taken (draws), and 128-bit fixed-point sums of k and E+
 * of the conversions.                                                         */
enum { OR_PAIR_DIRECT = 0, OR_PAIR_FREE_PATH = 1 };
/* method OR_PAIR_FREE_PATH: the same law by one draw per photon (the random free path):
 * the trials of a crossing all have probability P, so the number of failures before the
 * first success is geometric, j = floor(ln U / ln(1 - P)) = floor(-ln U / lam) (Eq. 4:
 * 1 - P = exp(-lam), lam = n_i sigma c dt, taken as computed) with U the u53 of words 0-1 of
 * the draw (id_mech, run id, first step inside, 0x50000000 + n_e); the photon converts at
 * the first step inside + j if that is still inside, with the fraction word 2-3.  The
 * tests tally then counts draws.  Returns -1 for an unknown method.                      */
int or_pair_transport(const or_tables* t, const or_run_params* r, const or_photon* photons, int64_t n_photons,
                      int64_t step_end, or_pair* pairs, int64_t cap, uint64_t* tally, int method);

/* ---- Breit-Wheeler conversion of the emitted photons in the laser field ----
 * Each photon record (k > 2 m c^2) moves at c along its direction from its
 * emission point; at step m (n_e < m < step_end) it is at x_e + k^ (m - n_e) c dt
 * and the fields there at t = m dt give its chi (or_chi_photon, kvec = k k^).
 * tau_0 = -ln U, U the u53 of words 0-1 of the draw (id_mech, run id, n_e,
 * 0x60000000 + n_e), falls by alpha E_S T(chi) dt / k per step (T from the table,
 * or_bw_T_interp); at the first step with tau <= 0 the photon converts: x from
 * words 0-1 of the draw (id_mech, run id, m, 0x70000000 + n_e) by or_bw_sample_x,
 * E+ = x k, E- = k - E+, both along k^, at the photon's position.  The tally
 * words are those of the Bethe-Heitler transport with: [1] photons followed,
 * [2] photon-steps with chi above the table, [3] photon-steps taken.  Not for
 * OR_PIC_1D runs (returns -1).                                                */
int or_bw_transport(const or_bw_tables* bt, const or_tables* t, const or_run_params* r, const or_photon* photons,
                    int64_t n_photons, int64_t step_end, or_pair* pairs, int64_t cap, uint64_t* tally);

/* normalised helpers (exposed for unit pins) */
double or_schwinger_field(double lambda_m);   /* E_S in m c omega / e          */
double or_critical_density(double lambda_m);  /* n_c in m^-3                   */
void or_fields(const or_run_params* r, double x, double y, double t, double E[3], double B[3]);
/* majorant of the null-collision method: x_hat = n_i max_gamma(sigma_Z) c dt  */
double or_null_x_hat(const or_tables* t, const or_run_params* r);
double or_eta(const double u[3], const double E[3], const double B[3], double E_S);
void or_boris(double u[3], const double E[3], const double B[3], double dt);

#ifdef __cplusplus
}
#endif
#endif
