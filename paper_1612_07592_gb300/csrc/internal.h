// internal.h -- descriptors shared by the host API and the kernels of libpe.
// Everything here is passed to kernels by value (kernel parameters up to
// 32 KB), so a launch needs no device-side descriptor copies and can be
// captured in a CUDA graph as is.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pe.h"

namespace pe {

// physical constants (CODATA 2018)
constexpr double kAlpha = 7.2973525693e-3;
constexpr double kRe = 2.8179403262e-15;        // classical electron radius [m]
constexpr double kMec2MeV = 0.51099895000;      // m_e c^2 [MeV]
constexpr double kHbarcMeVm = 197.3269804e-15;  // hbar c [MeV m]
constexpr double kC = 299792458.0;              // [m/s]
constexpr double kPi = 3.14159265358979323846;
constexpr double kHistEmaxMeV = 10000.0;        // top edge of the energy histogram

// Table constants in the arithmetic of the step (float copies for the FP32 path,
// so no double->float conversion runs per step).
template <typename R>
struct TabC {
    R eta_min, ln_eta_min, inv_dln_eta;   // row position = (ln eta - ln eta_min) * inv
    R ln_y_min, dln_y, y_min, y_max;
    R ln_g_min, inv_dln_g;
    R photon_min;
    R h_classical;                        // 5 pi / 3
    R eta_last, g_last;                   // n_eta - 1 and n_E - 1 (last row position)
    R s_step;                             // 1 / (n_s - 1)
    R ln_k_min, inv_dln_k;                // Bethe-Heitler rows: k log spaced on [2, gamma_max]
};

// Device view of one table set.  f32 and f64 copies of every table.
struct TablesDev {
    const float* h32;   const double* h64;      // [n_eta]
    const float* cdf32; const double* cdf64;    // [(n_eta + 1) * n_y]; row n_eta = classical limit
    const float* sig32; const double* sig64;    // [n_Z * n_E]
    const float* bcdf32; const double* bcdf64;  // [n_Z * n_E * n_s]
    const float* cdf32lo;                       // float-pair remainders: value = cdf32 + cdf32lo
    const float* bcdf32lo;
    // FP32 emission tables by pairs of adjacent rows: entry (i, j) holds column j of
    // rows i and i+1 as float pairs (hi_i, lo_i, hi_i+1, lo_i+1), so one 16-byte load
    // gives both values the row interpolation needs.  NCS: pair-rows 0..n_eta-2 and
    // pair-row n_eta-1 = (classical, classical); brems: n_E - 1 pair-rows per Z.
    const float4* cdfq;                         // [n_eta * n_y]
    const float4* bcdfq;                        // [n_Z * (n_E - 1) * n_s]
    // Guide tables (Chen & Asau 1974) of the pair-rows: for m in [0, M), entry m holds
    // (J_i(m/M), J_i+1(m/M), J_i((m+1)/M), J_i+1((m+1)/M)) with J_r(u) the largest
    // column j with CDF_r[j] <= u (-1 if none).  The inverse of the interpolated row
    // at u in [m/M, (m+1)/M) lies between the smallest and the largest of them.
    const short4* gq;                           // [n_eta * M_y]
    const short4* bgq;                          // [n_Z * (n_E - 1) * M_s]
    // Bethe-Heitler pair production (FP64 only; built on the first pair call): sigma_BH [n_Z * n_E]
    // and the CDF over s [n_Z * n_E * n_s], x = 1/k + s (1 - 2/k), rows k log spaced on [2, gamma_max]
    const double* bhsig64;
    const double* bhcdf64;
    unsigned long long* dbg;                    // debug builds: count of table indices found out of range
    int M_y, M_s;                               // guide sizes (powers of two >= n_y, n_s)
    float fM_y, fM_s;
    int n_eta, n_y, n_E, n_s, n_Z;
    TabC<float> cf;
    TabC<double> cd;
};

// Per-step constants of one run, in the arithmetic of the step.
template <typename R>
struct StepC {
    R dt, dt_hi, dt_lo;       // dt split so that n * dt_hi is exact in float for n < 2^13
    R inv_ES, ncs_coef;       // ncs_coef = sqrt(3) alpha / (2 pi) * E_S * dt
    R K_br;                   // n_i alpha r_e^2 (c dt): x_b = K_br * sigma[alpha r_e^2] * beta
    R x0, x1, yh;             // slab (normalised)
    R box0, box1;
    R inv_log_emax;           // 1 / ln(E_hist_max / m c^2)
    R a0, w0, zr, xf, phi_r, phi_f, k_env;   // fields; k_env = pi / (2 phi_r)
    R inv_zr, inv_w0sq;       // 1 / z_R, 1 / w0^2 (2D focus)
    R E_const[3], B_const[3];
    R refl_r;                 // reflected wave amplitude coefficient
    R xm2_hi, xm2_lo;         // 2 x_m (mirror plane) as hi + lo: in float an exact pair
    R P_hat;                  // null collisions: candidate probability 1 - exp(-x_hat) per step
    R pic_kx, pic_kyz;        // 1D PIC: J_x = pic_kx * sum, J_y,z = pic_kyz * sum (fixed-point sums)
    R bw_coef;                // Breit-Wheeler: alpha E_S dt (W dt = bw_coef T(chi) / k)
};

// Device view of one run.  Optical depth: double for PE_F64, a float pair
// (hi, lo) with value hi + lo for PE_F32; 8 bytes per particle either way.
template <typename R>
struct RunDevT {
    void *x, *y, *ux, *uy, *uz;
    void* tau;
    uint8_t* photons;
    unsigned long long* hist;
    unsigned long long* tally;
    unsigned long long* events;   // optional per-particle event fingerprints
    int64_t n;
    int64_t capacity;
    int64_t step0;                // step index of the first step of this launch
    StepC<R> c;
    int geometry, polarisation;
    int enable_ncs, enable_brems, box_enable;
    int iz;                       // brems table index
    uint32_t run_id;
    uint32_t id0;                 // global id of particle 0 (Philox counter word 0 = id0 + index)
    uint32_t seed_lo, seed_hi;
    int fk;                       // field kind (physics.cuh)
    int brems_method;             // PE_BREMS_DIRECT | PE_BREMS_NULL
    uint32_t* wait;               // null collisions: steps to the next candidate
    double x_hat;                 // null collisions: majorant optical depth per step (both precisions)
    void* grid;                   // 1D PIC: field grid (the run's precision, layout in pe.h)
    unsigned long long* jacc;     // 1D PIC: current sums of one step (3 n_cells, 2^-36 fixed point)
    int n_cells;                  // 1D PIC: cells of the grid (0 otherwise)
};
using RunDev = RunDevT<double>;

// Batched launch: runs and their tile prefix.
template <typename R>
struct BatchDevT {
    int n_runs;
    int tile;                           // particles per tile
    int64_t tile_start[PE_MAX_BATCH + 1];
    RunDevT<R> runs[PE_MAX_BATCH];
};

inline RunDevT<float> to_float(const RunDevT<double>& d) {
    RunDevT<float> f;
    f.x = d.x; f.y = d.y; f.ux = d.ux; f.uy = d.uy; f.uz = d.uz; f.tau = d.tau;
    f.photons = d.photons; f.hist = d.hist; f.tally = d.tally; f.events = d.events;
    f.n = d.n; f.capacity = d.capacity; f.step0 = d.step0;
    const double* src = &d.c.dt;
    float* dst = &f.c.dt;
    for (size_t k = 0; k < sizeof(StepC<double>) / sizeof(double); ++k) dst[k] = (float)src[k];
    f.geometry = d.geometry; f.polarisation = d.polarisation;
    f.enable_ncs = d.enable_ncs; f.enable_brems = d.enable_brems; f.box_enable = d.box_enable;
    f.iz = d.iz; f.run_id = d.run_id; f.id0 = d.id0; f.seed_lo = d.seed_lo; f.seed_hi = d.seed_hi;
    f.fk = d.fk; f.brems_method = d.brems_method; f.wait = d.wait; f.x_hat = d.x_hat;
    f.grid = d.grid; f.jacc = d.jacc; f.n_cells = d.n_cells;
    return f;
}

// diagnostics (kernels.cu)
void launch_electron_spectrum(const RunDev& r, int precision, double e_lo, double e_hi, int n_bins,
                              unsigned long long* out, cudaStream_t s);
void launch_photon_map(const RunDev& r, double x_lo, double x_hi, int nx, double e_lo, double e_hi, int ne,
                       unsigned long long* out, cudaStream_t s);

// 1D PIC (kernels_pic.cu)
void launch_pic_rho(const RunDev& r, int precision, cudaStream_t s);
void launch_pic_step(const TablesDev& t, const RunDev& r, int precision, int sms, cudaStream_t s);

// host-side table build (tables.cpp)
struct HostTables {
    pe_table_params p;
    std::vector<double> Z;
    std::vector<double> h;       // n_eta
    std::vector<double> cdf;     // (n_eta + 1) * n_y, last row classical
    std::vector<double> sigma;   // n_Z * n_E
    std::vector<double> bcdf;    // n_Z * n_E * n_s
    double classical_total = 0;
};
bool build_host_tables(const pe_table_params& p, HostTables& out, std::string* err);
// Bethe-Heitler tables of the same parameters: sigma_BH [n_Z * n_E], CDF [n_Z * n_E * n_s]
void build_host_bh_tables(const HostTables& h, std::vector<double>& sigma, std::vector<double>& cdf);
// Breit-Wheeler tables on the host: T(chi_i) [n_chi] and the CDF over x_j [n_chi * n_x]
void build_host_bw_tables(int n_chi, double chi_min, double chi_max, int n_x, double* T, double* cdf);

// Breit-Wheeler tables on the device: T by L_i = ln T(chi_i) + 8 / (3 chi_i), linear in
// ln chi between nodes (T = exp(L - 8 / (3 chi))), and the CDF over x at the nodes
// x_j = (1 - cos(pi j / (n_x - 1))) / 2
struct BwDev {
    const double* L64;            // [n_chi]
    const float* L32;             // [n_chi], float copy for the FP32 transport
    const double* cdf64;          // [n_chi * n_x]
    unsigned long long* dbg;      // debug builds: count of table indices found out of range
    double T_last, chi_min, ln_chi_min, inv_dln_chi;
    float fT_last, fchi_min, fln_chi_min, finv_dln_chi, f_last;   // f_last = n_chi - 1
    int n_chi, n_x;
};
// kernels_bw.cu: Breit-Wheeler conversion of photon records in the run's prescribed fields
void launch_bw_transport(const BwDev& b, const RunDev& r, int precision, const void* photons, int64_t n_photons,
                         int64_t step_end, void* pairs, int64_t capacity, unsigned long long* tally, cudaStream_t s);

// kernels_pair.cu: Bethe-Heitler conversion of photon records in the run's target
void launch_pair_transport(const TablesDev& t, const RunDev& r, const void* photons, int64_t n_photons,
                           int64_t step_end, void* pairs, int64_t capacity, unsigned long long* tally, int method,
                           cudaStream_t s);

// kernels_diag.cu
void launch_math_probe(int fn, const float* in, float* out, int64_t n, cudaStream_t s);
void launch_fma_peak(int kind, int blocks, int threads, int iters, void* out, cudaStream_t s);
int fma_chains();

// kernels.cu
void launch_init(const RunDev& r, int precision, int init_dist, double theta, double beam_u, cudaStream_t s);
void launch_step_plain_f64(const TablesDev& t, const RunDev& r, cudaStream_t s);
void launch_step_persistent_f32(const TablesDev& t, const BatchDevT<float>& b, int steps, int grid, int block,
                                cudaStream_t s);
void launch_step_persistent_f64(const TablesDev& t, const BatchDevT<double>& b, int steps, int grid, int block,
                                cudaStream_t s);
int persistent_smem_bytes(const TablesDev& t, int precision);
int default_ctas_per_sm_f32(int fk, int block, int smem, int steps_per_launch);
// every run of the launch has the paper's setup: NCS on, direct brems, no absorbing box (the FP32
// kernels then take these flags as compile-time constants)
inline bool common_flags_f32(const BatchDevT<float>& b) {
    for (int k = 0; k < b.n_runs; ++k) {
        const RunDevT<float>& r = b.runs[k];
        if (!r.enable_ncs || !r.enable_brems || r.brems_method != PE_BREMS_DIRECT || r.box_enable) return false;
    }
    return true;
}
const void* persistent_kernel_f32(const BatchDevT<float>& b, int steps, int smem, int block, int* threads,
                                  int* smem_out);
const void* persistent_kernel_f64(const BatchDevT<double>& b, int smem, int block, int* threads);
int persistent_occupancy_f64(int block, int smem);

}  // namespace pe
