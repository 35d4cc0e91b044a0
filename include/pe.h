/*
 * pe.h -- C ABI of the GB300 photon-emission step library (libpe.so).
 *
 * The library advances laser-driven electrons through the per-macroparticle
 * emission step of Wan, Lv, Jia, Sang & Xie, arXiv:1612.07592 ("Photon
 * emission by bremsstrahlung and nonlinear Compton scattering in the
 * interaction of ultraintense laser and plasmas"), in the paper's own test
 * mode (Sec. 2.2: field solver and weighting off, "only particle pusher and
 * bremsstrahlung MC module", here with the NCS module as well) under
 * prescribed laser fields with the paper's setup (Sec. 3).
 *
 * Per particle and step:
 *   E, B at (x^n, t^n)                       prescribed pulse (Sec. 3)
 *   Boris push u^{n-1/2} -> u^{n+1/2}         particle pusher (Sec. 2.2)
 *   eta = sqrt((gamma E + u x B)^2 - (u.E)^2) / E_S       (Sec. 2.1)
 *   NCS: tau -= dN/dt dt against the tabulated quantum-synchrotron rate;
 *        tau <= 0 -> photon energy by inverse CDF, recoil, new tau (Sec. 2.2)
 *   brems: P = 1 - exp(-n_i sigma(E) v dt) (Eq. 4, sign as intended), event
 *        iff a 64-bit uniform is below P 2^64; photon energy from
 *        sigma(y, E) = sigma(E) R2 (text after Eq. 4) with the screened Tsai
 *        cross section of Eq. (1); photon along v
 *   photons below m c^2 are created but only tallied (Sec. 3)
 *   x^{n+1} = x^n + dt u^{n+1/2} / gamma
 *
 * Units inside the library: time 1/omega_L, length c/omega_L, u = p/(m c),
 * fields m c omega_L / e, energies m c^2.  Parameters are SI unless stated.
 *
 * Conventions.  Every call returns pe_status; no exception crosses the ABI.
 * On an error pe_last_error() (thread-local) describes it.  The library owns
 * the opaque handles and the device copies of the tables; the caller owns
 * every particle, photon, histogram and tally buffer (device memory, e.g.
 * torch tensors) and keeps them alive until pe_destroy().  Streams are passed
 * as void* (cudaStream_t).  All work is asynchronous on the run's stream
 * except pe_create_tables, pe_tally and the export calls, which synchronise.
 */
#ifndef PE_H
#define PE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PE_OK = 0,
    PE_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, bad enum)     */
    PE_ERR_CUDA = 2,         /* a CUDA runtime call failed                              */
    PE_ERR_NOMEM = 3,        /* the library could not allocate its own device memory    */
    PE_ERR_BUFFER_FULL = 4,  /* photon buffer overflowed; counts stay exact             */
    PE_ERR_TABLE_RANGE = 5,  /* reserved: out-of-table values are counted, not fatal    */
    PE_ERR_TIMEOUT = 6,      /* tally word 12 is set (no kernel of this build waits)     */
    PE_ERR_STATE = 7         /* call out of order (e.g. mixed precisions in one batch)  */
} pe_status;

enum { PE_LP_Y = 0, PE_CP = 1 };                          /* polarisation                */
enum { PE_PLANE_1D = 0, PE_GAUSS_2D = 1, PE_CONST = 2, PE_PIC_1D = 3 };  /* field geometry */
enum { PE_F64 = 0, PE_F32 = 1 };                          /* arithmetic of the step      */
enum { PE_REST = 0, PE_MAXWELL_JUTTNER = 1, PE_BEAM = 2, PE_CALLER = 3 };  /* initial state */
enum { PE_BREMS_DIRECT = 0, PE_BREMS_NULL = 1 };          /* bremsstrahlung MC method    */
#define PE_WAIT_NEVER 0xFFFFFFFFu   /* brems_wait value: no further candidate in this run */
#define PE_PIC_GRID_WORDS(n) (6 * (int64_t)(n) + 5)   /* grid words of a PE_PIC_1D run */
#define PE_PIC_MAX_CELLS 4096

#define PE_HIST_E_BINS 512    /* log bins of photon energy over [0.511 MeV, 10 GeV]      */
#define PE_HIST_T_BINS 180    /* bins of theta = atan2(k_y, k_x) over [-pi, pi)          */
#define PE_HIST_WORDS (2 * PE_HIST_E_BINS + 2 * PE_HIST_T_BINS)
#define PE_TALLY_WORDS 32
#define PE_MAX_BATCH 64       /* runs in one batched launch                              */

/* tally word indices (uint64).  Energies are 128-bit fixed point in m c^2:
 * value = word[i+1] + word[i] * 2^-64, summed exactly (order independent).   */
enum {
    PE_T_N_NCS_STORED = 0, PE_T_N_NCS_BELOW = 1, PE_T_N_BR_STORED = 2, PE_T_N_BR_BELOW = 3,
    PE_T_N_PHOTONS = 4,      /* photons appended (true count, also beyond capacity)       */
    PE_T_N_ETA_ABOVE = 5,    /* particle-steps with eta above the table (row clamped)      */
    PE_T_N_ETA_BELOW = 6,    /* NCS emissions sampled from the classical (eta->0) row      */
    PE_T_N_GAMMA_ABOVE = 7,  /* brems tests with gamma above the table (row clamped)       */
    PE_T_N_KILLED = 8, PE_T_KILLED_STEPS = 9, PE_T_N_CLAMP = 10, PE_T_N_HIST_OVER = 11,
    PE_T_N_WAIT_TIMEOUT = 12, /* reserved for device waits that run out; pe_tally returns
                                 PE_ERR_TIMEOUT when it is set.  No kernel of this library waits
                                 on another thread, CTA or copy, so it stays 0              */
    PE_T_N_NONFINITE = 13,   /* particles removed because a momentum was NaN or infinite (also in N_KILLED) */
    PE_T_E_NCS_STORED = 16, PE_T_E_NCS_BELOW = 18, PE_T_E_BR_STORED = 20, PE_T_E_BR_BELOW = 22,
    PE_T_E_RECOIL_NCS = 24, PE_T_E_RECOIL_BR = 26
};

/* Sampling-table description (Sec. 2.2).
 * NCS: h(eta) and the photon-energy CDF on n_eta log-spaced eta in
 *   [eta_min, eta_max] x n_y log-spaced y in [y_min, y_max], where
 *   y = 2 delta / (3 eta (1 - delta)) and delta = photon energy / electron energy.
 * Brems: sigma_Z(gamma) and the CDF of sigma(y, E) = sigma(E) R2 on n_E
 *   log-spaced gamma in [gamma_min, gamma_max] x n_s points s in [0, 1] with
 *   y = y_cut (y_max / y_cut)^s, y_cut = photon_min_mc2 / gamma, y_max = 1 - 1/gamma.
 * One brems table per entry of Z[0..n_Z).                                     */
typedef struct {
    int n_eta, n_y;
    double eta_min, eta_max, y_min, y_max;
    int n_E, n_s;
    double gamma_min, gamma_max;
    double photon_min_mc2;           /* hard-photon cut, m c^2 (Sec. 3: 1.0)        */
    int n_Z;
    const double* Z;                 /* host array, copied                          */
} pe_table_params;

/* One run (one laser-target configuration, Sec. 3). */
typedef struct {
    double a0, lambda_m;             /* peak normalised vector potential per component, wavelength */
    int polarisation, geometry;      /* PE_LP_Y | PE_CP ; PE_PLANE_1D | PE_GAUSS_2D | PE_CONST     */
    double w0_m, focus_x_m;          /* PE_GAUSS_2D waist and focal plane                           */
    double flat_s, ramp_periods;     /* flat top (Sec. 3: 30 fs) and sin^2 ramps in periods          */
    double E_const[3], B_const[3];   /* PE_CONST fields, normalised units                           */
    double Z, charge_state, ne_over_nc;          /* target: atomic number, ion charge, n_e / n_c   */
    double slab_x0_m, slab_thick_m, y_half_m;    /* slab [x0, x0+thick] (and |y| <= y_half in 2D)  */
    double dt_over_T;                /* time step in laser periods                                  */
    int precision;                   /* PE_F64 | PE_F32                                             */
    int init_dist;                   /* PE_REST | PE_MAXWELL_JUTTNER | PE_BEAM | PE_CALLER          */
    double T_mev, beam_gamma;        /* Maxwell-Juttner temperature; PE_BEAM Lorentz factor         */
    uint64_t seed;                   /* Philox key                                                  */
    uint32_t run_id;                 /* Philox counter word 1                                       */
    int enable_ncs, enable_brems;
    int box_enable;                  /* absorbing boundary in x (Sec. 3), default off               */
    double box_x_m[2];
    /* Reflected wave (PE_PLANE_1D only): the incident pulse plus its mirror
     * image in the plane x = mirror_x_m, A_r(t, x) = -reflect_r A(t + x - 2 x_m),
     * a fixed stand-in for the reflecting plasma surface of Sec. 3.  The image
     * travels along -x; for reflect_r = 1 the transverse E vanishes on the plane.
     * The fields are not cut at the plane.  reflect_r in [0, 1], 0 = no
     * reflected wave.                                                           */
    double reflect_r, mirror_x_m;
    /* PE_BREMS_DIRECT: the test of Eq. 4 in every step in the slab.
     * PE_BREMS_NULL: null collisions (the speed-up Sec. 4 names for the MC
     * collision): candidates from a majorant process with
     * x_hat = n_i c dt max_gamma sigma_Z per step, independent of position and
     * energy; the steps between candidates are geometric, floor(-ln U / x_hat),
     * kept per particle in pe_buffers.brems_wait; a candidate is a collision
     * with probability P / (1 - exp(-x_hat)), P the Eq. 4 probability of the
     * step, so collisions have the law of the direct method.  Philox purposes:
     * 256 at step 0 (first wait) and at candidate step + 1 (next wait, test
     * word), 0 at the candidate step only for a collision (photon energy).      */
    int brems_method;
    /* PE_PIC_1D: the 1D electromagnetic PIC around the step (the paper's host
     * with the field solver and current weighting on, Sec. 2.2, Sec. 3): the
     * fields at the electrons come from a grid of n_cells cells over [0, L],
     * dx = c dt, driven by the electrons' currents and by the laser (a0,
     * polarisation, envelope as for PE_PLANE_1D) entering at x = 0.  Ions are
     * immobile at the electrons' initial positions (neutral start).  Each
     * macro-electron carries the areal density ne_over_nc x slab thickness / n.
     * Electrons leaving [0, L] are removed.  In 1D the transverse fields move as
     * F+- = E_y +- B_z and G+- = E_z -+ B_y along +-x: one cell per step along
     * the characteristics with the current at the midpoint (exact in vacuum);
     * E_x follows -J_x of the charge-conserving linear weighting.             */
    int n_cells;
    /* Global id of the run's particle 0.  Particle i of the buffers draws its
     * random numbers with Philox counter word 0 = id0 + i, and its photons carry
     * that id.  Electrons are independent under prescribed fields, so one run of
     * N electrons can be split into runs over contiguous id ranges [id0, id0 + n)
     * (one per GPU or process, same seed and run_id): each range gives exactly
     * the particles, photons and events the unsplit run gives for those ids, and
     * the tallies and histograms of the parts add up exactly (integers and
     * 128-bit fixed point) to the unsplit run's.  0 for an unsplit run;
     * id0 + n must not exceed 2^32.                                              */
    uint32_t id0;
} pe_run_params;

/* Caller-owned device buffers of one run.
 *   x, y             : n positions, 8 bytes each: a double for PE_F64; for
 *                      PE_F32 a pair of floats (hi, lo) whose sum is the
 *                      position, advanced by compensated adds so the laser
 *                      phase t - x keeps ~1e-12 accuracy; y is only read and
 *                      written for PE_GAUSS_2D but must be valid.
 *   ux, uy, uz       : n momenta, float (PE_F32) or double (PE_F64).
 *   tau              : n optical depths, 8 bytes each: a double for PE_F64; for
 *                      PE_F32 a pair of floats (hi, lo) whose sum is the value,
 *                      kept exact to ~2^-48 by compensated subtraction.
 *   photons          : photon_capacity records of 32 bytes
 *                      {float x, y, energy, kx, ky, kz; uint32 step; uint32 id | mech << 31}
 *   hist             : PE_HIST_WORDS uint64 (zeroed by pe_init_particles)
 *   tally            : PE_TALLY_WORDS uint64 (zeroed by pe_init_particles)
 *   events           : optional (may be NULL), n uint64 per-particle event
 *                      fingerprints, zeroed by pe_init_particles: low 32 bits =
 *                      NCS emissions | brems emissions << 16, high 32 bits =
 *                      sum over emissions of (step + 1) * (1, or 0x9E3779B1 for
 *                      brems) mod 2^32.  Used to compare event lists.
 *   grid             : PE_PIC_1D only (NULL otherwise): PE_PIC_GRID_WORDS(n_cells)
 *                      words, double (PE_F64) or float (PE_F32): E_x at the n half
 *                      nodes, then F+, F-, G+, G- and the ion charge density at
 *                      the n + 1 nodes (n = n_cells); set by pe_init_particles
 *                      (zero fields, ion charge from the initial electrons) and
 *                      advanced by pe_step.
 *   brems_wait       : n uint32, steps to each particle's next candidate
 *                      collision (PE_WAIT_NEVER: none); written by
 *                      pe_init_particles, required for PE_BREMS_NULL, ignored
 *                      (may be NULL) for PE_BREMS_DIRECT.
 * Pointers must be 16-byte aligned.                                            */
typedef struct {
    void *x, *y, *ux, *uy, *uz, *tau;
    void* photons;
    int64_t photon_capacity;
    void* hist;
    void* tally;
    void* events;
    void* brems_wait;
    void* grid;
} pe_buffers;

/* Launch shape of the persistent kernels (the autotuner's knobs).
 * block: electrons per tile (64, 128, 192 or 256); the FP32 kernel covers a
 * tile with block/2 threads, two electrons each, the FP64 kernel with block
 * threads; ctas_per_sm: CTAs per SM in the grid; steps_per_launch: steps done
 * per launch with the state held in registers (1 = state round-trips memory
 * every step).  Zeros pick defaults: 256 electrons per tile; three times the
 * CTAs that fit on an SM for the FP32 kernel (once for the one-step form of a
 * single plane-wave run, launches of at most 4 steps), twice for the FP64
 * kernel; min(steps, 4096) steps per launch.                                   */
typedef struct {
    int block, ctas_per_sm, steps_per_launch;
} pe_launch_config;

/* Host copy of a run's results. */
typedef struct {
    uint64_t tally[PE_TALLY_WORDS];
    uint64_t hist[PE_HIST_WORDS];
    int64_t n_particles, steps_done;
    int64_t photons_stored;          /* min(true count, capacity)                   */
    double live_particle_steps;      /* sum over particles of steps advanced alive  */
    double e_ncs_stored, e_ncs_below, e_br_stored, e_br_below, e_recoil_ncs, e_recoil_br;  /* m c^2 */
} pe_tally_out;

typedef struct pe_tables pe_tables;
typedef struct pe_run pe_run;

/* Build the NCS and brems tables on the host in FP64 (Sec. 2.2; Eq. 1 with
 * Tsai's screening functions) and upload FP64 and FP32 copies to the current
 * device.  Synchronous.  Errors: PE_ERR_ARG, PE_ERR_NOMEM, PE_ERR_CUDA.     */
pe_status pe_create_tables(const pe_table_params* params, pe_tables** out);
pe_status pe_destroy_tables(pe_tables* tables);

/* Copy one table to host memory: which = 0 h(eta) [n_eta], 1 NCS CDF
 * [n_eta*n_y], 2 classical CDF [n_y], 3 sigma_Z [n_E] (iz), 4 brems CDF
 * [n_E*n_s] (iz), 5 Bethe-Heitler sigma_BH [n_E] (iz; k log spaced on
 * [2, gamma_max] m c^2, alpha r_e^2), 6 Bethe-Heitler CDF [n_E*n_s] (iz; over
 * s with positron fraction x = 1/k + s (1 - 2/k)).  Kinds 5 and 6 build the
 * pair tables on first use.  *n_out receives the element count; cap too small
 * -> ARG.                                                                     */
pe_status pe_tables_export(const pe_tables* tables, int which, int iz, double* host_out,
                           int64_t cap, int64_t* n_out);

/* Bind buffers to a new run and, unless init_dist == PE_CALLER, draw the
 * initial positions (uniform in the slab; a beam starts at the slab's front
 * face) and momenta (rest, Maxwell-Juttner by Sobol's rejection, or a beam
 * along +x) from the particle's Philox
 * stream; always draws the initial optical depth tau = -ln U and, for
 * PE_BREMS_NULL, the first candidate wait.  Zeroes hist,
 * tally and the photon count.  Asynchronous on cuda_stream.  The run refers
 * to tables, which must outlive it.  Z must be one of the table set's Z.
 * Errors: PE_ERR_ARG (null, n < 0, n >= 2^31, Z not in tables, misaligned,
 * reflect_r outside [0, 1] or set for a geometry other than PE_PLANE_1D,
 * unknown brems_method, PE_BREMS_NULL without brems_wait).                   */
pe_status pe_init_particles(const pe_tables* tables, const pe_run_params* params, int64_t n,
                            const pe_buffers* buffers, void* cuda_stream, pe_run** out);

/* Resume a run from a checkpoint: the caller's buffers (the same layout as for
 * pe_init_particles) already hold the state a run reached after step0 steps --
 * positions, momenta, optical depths, null-collision waits, event words,
 * photons, histograms, tallies and, for PE_PIC_1D, the grid -- for instance
 * copied to the host and back.  Nothing is drawn or cleared; the run's step
 * index is step0, so the next pe_step continues exactly where the checkpointed
 * run stopped (the draws are keyed on the step) and the results equal those of
 * the uninterrupted run bit for bit.  params and n must be those of the run that
 * was checkpointed.  A library extension for long jobs (the paper has no
 * counterpart).  Errors: as pe_init_particles, and step0 outside [0, 2^32).    */
pe_status pe_resume_particles(const pe_tables* tables, const pe_run_params* params, int64_t n,
                              const pe_buffers* buffers, int64_t step0, void* cuda_stream, pe_run** out);

/* Advance runs by n_steps.  n_runs == 1: PE_F64 runs use the plain kernel
 * (one launch per step); PE_F32 runs use the persistent kernel.  n_runs > 1
 * (<= PE_MAX_BATCH): all runs must be PE_F32 and share the first run's
 * stream; they advance together, one persistent launch per field kind present
 * per steps_per_launch steps.  Asynchronous.  cfg may be NULL.
 * Precision: the FP32 kernels form the laser phase t^n - x with t^n = n dt_hi +
 * n dt_lo, dt_hi holding 11 significant bits, so n dt_hi is exact up to step
 * 8192 (the paper's runs take 4000); later steps add one rounding of about
 * 2^-24 t^n to the phase (1e-4 rad at step 50000).  FP64 runs are unaffected. */
pe_status pe_step(pe_run* const* runs, int n_runs, int64_t n_steps);
pe_status pe_step_ex(pe_run* const* runs, int n_runs, int64_t n_steps, const pe_launch_config* cfg);

/* A CUDA graph of the batched persistent launches that advance runs by
 * steps_per_replay steps (one kernel node per launch: per field kind present
 * and per steps_per_launch chunk).  pe_graph_launch replays it on the first
 * run's stream, first setting each node's step index to where the runs are,
 * so every replay continues the runs; results are identical to pe_step_ex
 * with the same configuration.  All runs must share tables and precision
 * (PE_F32 or PE_F64); the runs must not be stepped by other calls while the
 * graph exists.  The graph refers to the runs, which must outlive it. */
typedef struct pe_graph pe_graph;
pe_status pe_graph_create(pe_run* const* runs, int n_runs, int64_t steps_per_replay, const pe_launch_config* cfg,
                          pe_graph** out);
pe_status pe_graph_launch(pe_graph* graph);
pe_status pe_graph_destroy(pe_graph* graph);

/* Synchronise the run's stream and copy tally, histograms and counters to
 * *out.  Returns PE_ERR_BUFFER_FULL (after filling *out) if more photons
 * were produced than the buffer holds; the counts stay exact.               */
pe_status pe_tally(pe_run* run, pe_tally_out* out);

pe_status pe_destroy(pe_run* run);

/* Kinetic-energy spectrum of the run's live electrons (the electron spectra of
 * the paper's Fig. 5): counts (uint64, device memory of the caller, n_bins
 * words, 16-byte aligned, cleared by the call) in n_bins log bins of (gamma - 1)
 * m c^2 over [e_min_mev, e_max_mev); energies outside are not counted.
 * Asynchronous on the run's stream.  Errors: PE_ERR_ARG (null, n_bins outside
 * [1, 4096], bad range, misaligned), PE_ERR_CUDA.                             */
pe_status pe_electron_spectrum(pe_run* run, int n_bins, double e_min_mev, double e_max_mev, void* counts);

/* Map of the stored photons over emission position x and energy (the photon
 * density maps of the paper's Fig. 4, reduced to 1D): counts (uint64, device
 * memory of the caller, nx * ne words, x-major, cleared by the call) in nx
 * linear bins of x over [x_min_m, x_max_m) and ne log bins of the photon
 * energy over [e_min_mev, e_max_mev).  Reads the stored count on the device
 * (min(appended, capacity)).  Asynchronous on the run's stream.  Errors:
 * PE_ERR_ARG (null, nx * ne outside [1, 2^24], bad ranges, misaligned),
 * PE_ERR_CUDA.                                                                */
pe_status pe_photon_map(pe_run* run, int nx, double x_min_m, double x_max_m, int ne, double e_min_mev,
                        double e_max_mev, void* counts);

/* Bethe-Heitler pair production of emitted photons in the target.  Sec. 2.2
 * says pair production by photons in the field of the nuclei is implemented
 * like the bremsstrahlung: a direct MC collision of Eq. (4) with the pair
 * cross section, here Tsai's DCS of the crossed process with the screening
 * fits of Eq. (1), clamped at zero, over the positron energy fraction x in
 * [1/k, 1 - 1/k] (k the photon energy in m c^2; no pairs for k <= 2).
 *
 * Each photon record (the 32-byte layout of the photon buffer) moves at c
 * along its direction from its emission point: at step m (emission step n_e
 * < m < step_end) it is at p = x_e + k^ (m - n_e) c dt.  At every step with p
 * in the run's target (the slab; and |y| <= y_half in 2D) it takes the test
 * P = 1 - exp(-n_i sigma_BH(k) c dt) with one Philox draw of counter
 * (id_mech, run id, m, 0x40000000 + n_e) under the run's seed: words 0-1
 * against floor(P 2^64), words 2-3 (53 bits) for x by the inverse CDF.  A
 * conversion writes one pe_pair (E+ = x k, E- = k - E+, both along k^) and
 * ends the photon; a photon that has left the target, or is outside it and
 * moving away, is not followed further.  Photons do not feel the fields, so
 * following each one after the fact equals stepping it with the electrons.
 *
 * method PE_PAIR_FREE_PATH samples the same law with one draw per photon:
 * the tests of one crossing all have the same P (sigma_BH(k) and n_i are
 * constant along it), so the number of failures before the first success is
 * geometric, j = floor(ln U / ln(1 - P)) = floor(-ln U / lam), with lam =
 * n_i sigma_BH(k) c dt the exponent of Eq. (4).  One Philox draw of counter
 * (id_mech, run id, a, 0x50000000 + n_e), a the first step in the target:
 * words 0-1 give U (53 bits), words 2-3 x; the photon converts at step a + j
 * if that is within its run of steps in the target.  The conversions differ
 * draw by draw from PE_PAIR_DIRECT's but follow the same distribution; the
 * tests tally counts one per photon that had a draw.
 *   run       : the run whose target, step, seed, run id and Z apply
 *   photons   : device array of n_photons records (for instance the run's own
 *               photon buffer); 4-byte aligned; read only
 *   step_end  : first step not taken (-1: the run's steps done so far)
 *   pairs     : device array of capacity pe_pair records (may be null if
 *               capacity is 0); written in no particular order
 *   tally     : device array of PE_PAIR_TALLY_WORDS uint64, cleared by the
 *               call: the true pair count (it may exceed capacity; the
 *               excess is not written), photons that entered the target,
 *               of them above the table's k range (last row used), tests
 *               taken (one draw each), and 128-bit fixed-point (lo, hi;
 *               2^-64 m c^2) sums of k and E+ of the conversions
 *   method    : PE_PAIR_DIRECT (per-step tests) or PE_PAIR_FREE_PATH
 * Asynchronous on the run's stream.  The first call on a table set builds
 * its pair tables on the host and uploads them (synchronous).
 * Errors: PE_ERR_ARG (null, n_photons < 0 or >= 2^31, capacity < 0,
 * misaligned, step_end beyond the run, unknown method), PE_ERR_NOMEM,
 * PE_ERR_CUDA.                                                               */
typedef struct {
    float x, y;               /* conversion point: the photon's position at `step` (y = 0 in 1D) */
    float e_minus, e_plus;    /* total energies of the electron and the positron, m c^2 */
    float kx, ky, kz;         /* direction of the converted photon */
    uint32_t step;            /* step of the conversion */
    uint32_t photon;          /* index of the photon record */
    uint32_t id_mech;         /* the photon's id_mech */
} pe_pair;
#define PE_PAIR_TALLY_WORDS 8
enum {
    PE_PT_N_PAIRS = 0, PE_PT_N_ENTERED = 1, PE_PT_N_K_ABOVE = 2, PE_PT_N_TESTS = 3, PE_PT_E_PAIRS = 4,
    PE_PT_E_POSITRONS = 6
};
enum { PE_PAIR_DIRECT = 0, PE_PAIR_FREE_PATH = 1 };
pe_status pe_pair_transport(pe_run* run, const void* photons, int64_t n_photons, int64_t step_end, void* pairs,
                            int64_t capacity, void* tally, int method);

/* Breit-Wheeler pair production of a photon in the laser field (Sec. 1 names the
 * process; its rate is the one of a locally constant crossed field, the model of
 * the NCS module): a photon of energy k (m c^2) with quantum parameter
 * chi = sqrt((k E + kvec x B)^2 - (kvec . E)^2) / E_S makes pairs at the rate
 *   W = alpha (m c^2/hbar) T(chi) / k,   T(chi) = (1/(sqrt 3 pi)) int_0^1 G dx,
 *   G(chi, x) = (x/(1-x) + (1-x)/x) K_{2/3}(xi) + int_xi^inf K_{1/3}(t) dt,
 *   xi = 2 / (3 chi x (1 - x)), x the positron's share of k.
 * Computed on the host (no device needed):
 *   T   : n_chi doubles, T(chi_i) for chi_i log spaced on [chi_min, chi_max]
 *   cdf : n_chi * n_x doubles (row i = chi_i), the normalised cumulative integral
 *         of G over x at the nodes x_j = (1 - cos(pi j / (n_x - 1))) / 2
 * Both arrays belong to the caller.  Errors: PE_ERR_ARG (null, n_chi or n_x
 * outside [2, 4096], not 0 < chi_min < chi_max).                                */
pe_status pe_bw_tables_host(int n_chi, double chi_min, double chi_max, int n_x, double* T, double* cdf);

/* The same Breit-Wheeler tables on the current device (library-owned): T as
 * L_i = ln T(chi_i) + 8 / (3 chi_i), linear in ln chi between nodes (the factor
 * takes out the small-chi exponential), and the CDF rows.  Synchronous.
 * Errors: as pe_bw_tables_host; PE_ERR_ARG also if T underflows at chi_min;
 * PE_ERR_NOMEM, PE_ERR_CUDA.                                                 */
typedef struct pe_bw_tables pe_bw_tables;
pe_status pe_bw_tables_create(int n_chi, double chi_min, double chi_max, int n_x, pe_bw_tables** out);
pe_status pe_bw_tables_destroy(pe_bw_tables* tables);

/* Breit-Wheeler conversion of photon records in the run's prescribed laser
 * fields (Sec. 1).  Each record (the 32-byte photon layout; photons with
 * k <= 2 m c^2 are skipped) moves at c along its direction from its emission
 * point: at step m (n_e < m < step_end) it is at x_e + k^ (m - n_e) c dt and
 * the run's fields at (that point, t = m dt) give chi = sqrt((k E + kvec x B)^2
 * - (kvec . E)^2) / E_S, kvec = k k^.  An optical depth tau_0 = -ln U, U from
 * words 0-1 (53 bits) of the Philox draw (id_mech, run id, n_e, 0x60000000 + n_e),
 * falls by W dt = alpha E_S dt T(chi) / k per step; at the first step with
 * tau <= 0 the photon converts: x from words 0-1 of the draw (id_mech, run id,
 * m, 0x70000000 + n_e) by the CDF (rows interpolated in ln chi, chi clamped to
 * the table, inverted linearly in s, x = (1 - cos(pi s)) / 2), one pe_pair with
 * E+ = x k, E- = k - E+, both along k^, at the photon's position.  Tally words
 * (PE_PAIR_TALLY_WORDS uint64, cleared by the call): [0] the true pair count,
 * [1] photons followed, [2] photon-steps with chi above the table (last node
 * used), [3] photon-steps taken, [4-5] and [6-7] 128-bit fixed-point sums of k
 * and E+ of the conversions.  A photon behind a pulse for good (the fields
 * vanish there) stops early with its remaining steps counted as taken.  FP64
 * runs step in double; FP32 runs in float (optical depth as a compensated float
 * pair) and at most 8192 steps.  Asynchronous on the run's stream.
 *   run, bw   : the run whose fields, step, seed and run id apply; the tables
 *   photons   : device array of n_photons records, 4-byte aligned, read only
 *   step_end  : first step not taken (-1: the run's steps done so far)
 *   pairs     : device array of capacity pe_pair records (excess not written)
 * Errors: PE_ERR_ARG (null, n_photons < 0 or >= 2^31, capacity < 0, misaligned,
 * step_end beyond the run or above 8192 for FP32), PE_ERR_STATE (a PE_PIC_1D run:
 * its fields are not stored), PE_ERR_CUDA.                                   */
pe_status pe_bw_transport(pe_run* run, const pe_bw_tables* bw, const void* photons, int64_t n_photons,
                          int64_t step_end, void* pairs, int64_t capacity, void* tally);

/* a0 of a pulse of intensity I (W/cm^2) at wavelength lambda (Sec. 3: a0 = 0.86 sqrt(I_18)
 * at 1 um; here 0.855 lambda_um sqrt(I_18) for LP, divided by sqrt(2) per component for CP). */
double pe_a0_from_intensity(double I_wcm2, double lambda_m, int polarisation);

/* PIC steps that allocate nothing.  The paper has no counterpart: this is an
 * interface choice of this library.  pe_init_particles allocates, for a
 * PE_PIC_1D run, the device memory in which each step sums the electrons'
 * currents.  Some callers cannot call cudaMalloc at all: programs whose device
 * memory is handed out by a host framework or a fixed pool they must not
 * bypass, or that run under a memory budget that forbids new allocations
 * once the simulation is set up.  This entry point advances such a caller's
 * PIC state by n_steps steps from step index step0 with the same kernels and
 * results as pe_step on a run made by pe_init_particles with the same
 * parameters and buffers, but it sums the currents in a fixed array compiled
 * into the library ((3 x PE_PIC_MAX_CELLS + 1) x 8 bytes = 96 KiB + 8 bytes: the
 * sums and the count of CTAs done with a step, held on every GPU that loads
 * the library until the process exits).  It calls no cudaMalloc or
 * cudaFree and no routine that allocates.
 *   tables, params, n and buffers describe the run as for pe_init_particles
 *   (params->geometry = PE_PIC_1D); the caller owns every buffer, which must
 *   hold a PIC state (for instance one set up by pe_init_particles, or a grid
 *   cleared to zero with the caller's own electrons).  hist and tally
 *   accumulate as in pe_step.  Asynchronous on cuda_stream.
 *   The first call on a device looks up the array's device address with that
 *   device current (cudaGetSymbolAddress) and keeps it for the life of the
 *   process; make that first call before any stream capture, and do not reset
 *   the device (cudaDeviceReset) or tear down its primary context after it: the
 *   module may then load at another address and the kept one is stale.  Every
 *   call shares the one array and clears it before use, so calls whose work
 *   overlaps on the GPU (other streams, other host threads) race and give wrong
 *   currents: serialise them.  The checks and the run description are those of
 *   pe_init_particles (the same code).
 * Errors: PE_ERR_ARG (null, wrong geometry, n_cells outside [4,
 * PE_PIC_MAX_CELLS] -- the array's limit --, bad sizes or alignment, Z not in
 * the tables), PE_ERR_CUDA.                                                    */
pe_status pe_pic_step_noalloc(const pe_tables* tables, const pe_run_params* params, int64_t n,
                              const pe_buffers* buffers, int64_t step0, int64_t n_steps, void* cuda_stream);

/* Diagnostics (the paper has no counterpart): the library's own single-precision
 * device forms, evaluated on given inputs so that tests can bound their error.
 *   fn = PE_MATH_RCP      1/d for d >= 1 as the FP32 step forms it (the hardware
 *                         reciprocal estimate of -d refined by one Newton-Raphson
 *                         step; the probe returns minus that result, an exact negation)
 *        PE_MATH_SIN/_COS the carrier-phase sine and cosine of the paired FP32 step
 *                         (Cody-Waite reduction by 2 pi with a two-part constant,
 *                         then the hardware sine and cosine); _SIN1/_COS1 the same
 *                         in the one-electron FP32 step (the 1D PIC)
 *        PE_MATH_BREMS_P  1 - e^-x as the paired step forms the probability of Eq. 4
 *                         (a four-term Taylor series below 2^-5, expm1f above);
 *                         _BREMS_P1 the same in the one-electron step (the 1D PIC)
 *        PE_MATH_CUDA_RCP, _SIN, _COS, _EXPM1: CUDA's __frcp_rn, sinf, cosf and
 *                         -expm1f(-x), for comparison
 *        PE_MATH_GOUY_C/_S  at a = (x - x_f) / z_R, the factors (1 + a^2)^(-1/4) cos(atan(a)/2)
 *                         and (1 + a^2)^(-1/4) sin(atan(a)/2) of the paired 2D focus
 *                         (amplitude sqrt(w0/w) and Gouy phase, formed without an arctangent)
 *        PE_MATH_EXP_NEG  e^(-x) for x >= 0 as the paired 2D focus forms its transverse
 *                         profile (the hardware base-2 exponential)
 *        PE_MATH_TAU      the optical depth -ln U every FP32 kernel draws after an
 *                         emission (Sec. 2.2), U the 53-bit uniform of a 64-bit random
 *                         word: `in` then holds 2n floats, read as the bit patterns of n
 *                         word pairs (w_lo at in[2i], w_hi at in[2i + 1])
 *   in, out : n floats of device memory (2n for PE_MATH_TAU; 4-byte aligned);
 *             asynchronous on stream.
 * Errors: PE_ERR_ARG (null, n < 0, unknown fn), PE_ERR_CUDA.                  */
enum { PE_MATH_RCP = 0, PE_MATH_SIN = 1, PE_MATH_COS = 2, PE_MATH_SIN1 = 3, PE_MATH_COS1 = 4,
       PE_MATH_BREMS_P = 5, PE_MATH_BREMS_P1 = 6, PE_MATH_CUDA_RCP = 7, PE_MATH_CUDA_SIN = 8,
       PE_MATH_CUDA_COS = 9, PE_MATH_CUDA_EXPM1 = 10, PE_MATH_GOUY_C = 11, PE_MATH_GOUY_S = 12,
       PE_MATH_EXP_NEG = 13, PE_MATH_TAU = 14 };
pe_status pe_math_probe(int fn, const float* in, float* out, int64_t n, void* cuda_stream);

/* Peak of an arithmetic pipe, for the roofline of the ALU-bound step kernel (the
 * paper has no counterpart): one launch of blocks x threads threads, each running
 * `iters` rounds of *chains_out independent fused multiply-add chains -- kind
 * PE_FMA_F32 (FFMA), PE_FMA_F32X2 (the paired FFMA2: two FMAs per instruction) or
 * PE_FMA_F64 (DFMA).  out (device memory, blocks x threads floats, or doubles for
 * PE_FMA_F64) receives each thread's sums so the work is kept.  The caller times the
 * launch on cuda_stream (CUDA events); it performs 2 x chains x iters x blocks x
 * threads flops (twice that for PE_FMA_F32X2).  Asynchronous.  Errors: PE_ERR_ARG
 * (unknown kind, blocks or iters < 1, threads not a multiple of 32 in [32, 256]). */
enum { PE_FMA_F32 = 0, PE_FMA_F32X2 = 1, PE_FMA_F64 = 2 };
pe_status pe_fma_peak(int kind, int blocks, int threads, int iters, void* out, void* cuda_stream,
                      int* chains_out);

/* Debug builds.  A library compiled with PE_DEBUG checks every table row and
 * column, guide entry and histogram bin a kernel indexes against its array; an
 * index out of range is counted in a word of the table set and clamped into
 * range, so the access stays in bounds and nothing traps (the substitute for a
 * memory checker).  pe_debug_build returns 1 for such a library, 0 otherwise.
 * pe_debug_count synchronises the device and returns the sum of the counts of
 * the given table sets (either may be NULL; 0 in a release build).
 * Errors: PE_ERR_ARG (both NULL, out NULL), PE_ERR_CUDA.                      */
int pe_debug_build(void);
pe_status pe_debug_count(const pe_tables* tables, const pe_bw_tables* bw, uint64_t* out);

/* Number of kernel launches the library has issued (all runs, this process). */
int64_t pe_launch_count(void);

const char* pe_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
