// kernels.cuh -- the emission-step kernels for sm_103a (device code).
//
//  k_init            one thread per particle: initial position, momentum and
//                    optical depth from the particle's Philox stream.
//  k_step_plain      FP64, one thread per particle, one step per launch,
//                    tables read from global memory, histograms and tallies
//                    by global atomics (the plain per-run path).
//  k_step_persistent grid-stride over tiles of one or many runs, K steps per
//                    launch with the particle state in registers, the rate
//                    tables (h(eta), sigma_Z(gamma)) staged in shared memory,
//                    photons appended inside the emission branch (one atomic per
//                    group of lanes there together), histograms and tallies
//                    accumulated in shared memory and flushed once per run per
//                    CTA.  Instantiated for double; the FP32 step runs on the
//                    paired kernels (pair_f32.cuh), and the FP32 PIC kernel
//                    uses step_one below.
//
// Step order per particle (Sec. 2.2): fields at (x^n, t^n) -> Boris push ->
// eta -> NCS optical depth (emission at tau <= 0) -> brems test (Eq. 4) ->
// position update.  Both emissions may fire in one step; brems sees the
// momentum after the NCS recoil.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "physics.cuh"
#include "rare_f32.cuh"

namespace pe {

// ---------------------------------------------------------------------------
// accumulation helpers
// ---------------------------------------------------------------------------
// 128-bit fixed-point add of v >= 0 (m c^2) into (lo, hi): exact, order-free
__device__ __forceinline__ void fx_add(unsigned long long* w, double v) {
    if (!(v > 0.0)) return;
    double ip = floor(v);
    unsigned long long lo = __double2ull_rz((v - ip) * 0x1.0p64);
    unsigned long long old = atomicAdd(w, lo);
    unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
    unsigned long long hi = (unsigned long long)ip + carry;
    if (hi) atomicAdd(w + 1, hi);
}

struct Photon {
    float x, y, e, kx, ky, kz;
    uint32_t step, id_mech;
};

// pair record of the pair-production transports (the pe_pair layout)
struct PairRec {
    float x, y, e_minus, e_plus, kx, ky, kz;
    uint32_t step, photon, id_mech;
};
static_assert(sizeof(PairRec) == 40, "pe_pair layout");
static_assert(sizeof(Photon) == 32, "photon record layout");

// a photon's coordinate (direction component d, emission coordinate e) at step m, as the
// definition computes it: e + d ((m - n_e) c dt), one rounding for the step product and one
// for the fused multiply-add
__device__ __forceinline__ double photon_pos(const StepC<double>& c, double d, double e, int64_t ne, int64_t m) {
    return __fma_rn(d, __dmul_rn((double)(m - ne), c.dt), e);
}

// Appends a photon from inside an emission branch: the lanes that are in the branch together
// (__activemask) take consecutive slots with one atomic of their leader, so no photon is held
// across the rest of the step (and the step loop has no per-step vote for appends).
template <typename R>
__device__ __forceinline__ void append_now(const RunDevT<R>& r, const Photon& p) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(r.tally + PE_T_N_PHOTONS, (unsigned long long)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    const unsigned long long slot = base + __popc(mask & ((1u << lane) - 1u));
    if (slot < (unsigned long long)r.capacity) {
        float4* dst = reinterpret_cast<float4*>(r.photons + slot * 32);
        dst[0] = make_float4(p.x, p.y, p.e, p.kx);
        dst[1] = make_float4(p.ky, p.kz, __uint_as_float(p.step), __uint_as_float(p.id_mech));
    }
}

// ---------------------------------------------------------------------------
// one step of one particle
// ---------------------------------------------------------------------------
template <typename R>
struct Particle {
    R x, y, u[3];
    R x_lo, y_lo;               // compensation of the float position update (0 in double)
    R tau, tau_lo;              // optical depth; float path keeps it as the pair tau + tau_lo
    uint32_t ev_cnt, ev_hash;   // event fingerprint (only kept when r.events != nullptr)
    uint32_t wait;              // null collisions: steps to the next candidate
};
template <typename R>
__device__ __forceinline__ void note_event(Particle<R>& P, uint32_t n, int mech) {
    P.ev_cnt += mech ? 0x10000u : 1u;
    P.ev_hash += (n + 1u) * (mech ? 0x9E3779B1u : 1u);
}
// optical depth arithmetic: tau -= d (compensated in float), emission test, reset
__device__ __forceinline__ void tau_sub(Particle<double>& P, double d) { P.tau -= d; }
__device__ __forceinline__ void tau_sub(Particle<float>& P, float d) {
    float s = P.tau - d;
    float bb = s - P.tau;
    float e = (P.tau - (s - bb)) + (-d - bb);
    P.tau = s;
    P.tau_lo += e;
}
template <typename R>
__device__ __forceinline__ bool tau_crossed(const Particle<R>& P) { return P.tau + P.tau_lo <= (R)0; }
// rare-branch arithmetic by precision: the FP64 path in double, the FP32 path in
// float pairs and integers (no FP64 or conversion instructions, see rare_f32.cuh)
__device__ __forceinline__ void tau_draw(Particle<double>& P, uint4 w) {
    P.tau = -log(uni53(w64(w.z, w.w)));
    P.tau_lo = 0;
}
__device__ __forceinline__ void tau_draw(Particle<float>& P, uint4 w) {
    P.tau = tau_draw_f32(w.z, w.w);
    P.tau_lo = 0;
}
__device__ __forceinline__ double sample_delta(const TablesDev& t, double eta, uint4 w, bool& below) {
    return sample_ncs_delta<double>(t, t.cdf64, eta, uni53(w64(w.x, w.y)), below);
}
__device__ __forceinline__ float sample_delta(const TablesDev& t, float eta, uint4 w, bool& below) {
    return sample_ncs_delta_f32(t, eta, w.x, w.y, below);
}
__device__ __forceinline__ double sample_y(const TablesDev& t, int iz, double gamma, uint4 w) {
    return sample_brems_y<double>(t, t.bcdf64 + (size_t)iz * t.n_E * t.n_s, gamma, uni53(w64(w.z, w.w)));
}
__device__ __forceinline__ float sample_y(const TablesDev& t, int iz, float gamma, uint4 w) {
    return sample_brems_y_f32(t, iz, gamma, w.z, w.w);
}
__device__ __forceinline__ void fx_add_r(unsigned long long* p, double v) { fx_add(p, v); }
__device__ __forceinline__ void fx_add_r(unsigned long long* p, float v) { fx_add_f32(p, v); }
__device__ __forceinline__ bool brems_event(double P, uint4 w) { return below_threshold(P, w.x, w.y); }
__device__ __forceinline__ bool brems_event(float P, uint4 w) { return below_threshold_f32(P, w.x, w.y); }
__device__ __forceinline__ void hist_bins(double e, double kx, double ky, double inv_log_emax, int& eb, int& tb,
                                          bool& over) {
    eb = (int)floor((double)PE_HIST_E_BINS * log(e) * inv_log_emax);
    over = eb >= PE_HIST_E_BINS;
    if (over) eb = PE_HIST_E_BINS - 1;
    if (eb < 0) eb = 0;
    tb = (int)floor((atan2(ky, kx) + kPi) / (2.0 * kPi) * (double)PE_HIST_T_BINS);
    if (tb < 0) tb = 0;
    if (tb >= PE_HIST_T_BINS) tb = PE_HIST_T_BINS - 1;
}
__device__ __forceinline__ void hist_bins(float e, float kx, float ky, float inv_log_emax, int& eb, int& tb,
                                          bool& over) {
    hist_bins_f32(e, kx, ky, inv_log_emax, eb, tb, over);
}

template <typename R>
__device__ __forceinline__ void hist_add(unsigned long long* hist, unsigned long long* tally, int mech, R e,
                                         R kx, R ky, R inv_log_emax, unsigned long long* dbg) {
    int eb, tb;
    bool over;
    hist_bins(e, kx, ky, inv_log_emax, eb, tb, over);
    eb = dbg_idx(dbg, eb, PE_HIST_E_BINS);
    tb = dbg_idx(dbg, tb, PE_HIST_T_BINS);
    if (over) atomicAdd(tally + PE_T_N_HIST_OVER, 1ull);
    atomicAdd(hist + mech * PE_HIST_E_BINS + eb, 1ull);
    atomicAdd(hist + 2 * PE_HIST_E_BINS + mech * PE_HIST_T_BINS + tb, 1ull);
}


// The emission branches are real calls (__noinline__): compiled once per
// precision, so every kernel that steps a particle (single run or batch, any
// launch shape) performs bit-identical emission arithmetic, and the rarely taken
// code stays out of the step loop's instruction stream.  They take the particle
// by value and return it (no address of the loop-carried state escapes, so it
// stays in registers).  The paired FP32 kernels inline both branches instead
// (ncs_emit_body, brems_emit_body): with 72 registers a thread, a call's register
// convention cost spills on the common path (measured 9 % of the headline job).  Their
// translation unit rounds every operation as written, so all of their instances
// (single run or batch, resident or streaming: compared bit for bit in the tests)
// round the inlined branches alike.
template <typename R>
struct Emission {
    Particle<R> P;     // particle after the branch
    R gamma;           // its Lorentz factor
    bool stored;       // a photon above the cut was produced
    Photon ph;
};

// NCS emission at a crossing of the optical depth (Sec. 2.2): photon energy by
// inverse CDF, recoil along u, tallies, new optical depth.
template <typename R>
__device__ __forceinline__ Emission<R> ncs_emit_body(const TablesDev& t, const RunDevT<R>& r, uint32_t id, uint32_t n,
                                                     Particle<R> P, R gamma, R eta, R xn, R yn,
                                                     unsigned long long* hist, unsigned long long* tally) {
    Emission<R> out;
    out.stored = false;
    const StepC<R>& c = r.c;
    const R photon_min = tabc<R>(t).photon_min;
    uint4 w = draw(r, id, n, PUR_NCS);
    bool below;
    R delta = sample_delta(t, eta, w, below);
    if (below) atomicAdd(tally + PE_T_N_ETA_BELOW, 1ull);
    R ew = delta * gamma;
    if (ew > gamma - (R)1) { ew = gamma - (R)1; atomicAdd(tally + PE_T_N_CLAMP, 1ull); }
    R k[3];
    recoil<R>(P.u, gamma, ew, k);
    note_event<R>(P, n, 0);
    R gn = m_sqrt((R)1 + P.u[0] * P.u[0] + P.u[1] * P.u[1] + P.u[2] * P.u[2]);
    fx_add_r(tally + PE_T_E_RECOIL_NCS, gamma - gn);
    if (ew >= photon_min) {
        atomicAdd(tally + PE_T_N_NCS_STORED, 1ull);
        fx_add_r(tally + PE_T_E_NCS_STORED, ew);
        hist_add<R>(hist, tally, 0, ew, k[0], k[1], c.inv_log_emax, t.dbg);
        out.stored = true;
        out.ph = Photon{(float)xn, (float)yn, (float)ew, (float)k[0], (float)k[1], (float)k[2], n, id};
    } else {
        atomicAdd(tally + PE_T_N_NCS_BELOW, 1ull);
        fx_add_r(tally + PE_T_E_NCS_BELOW, ew);
    }
    tau_draw(P, w);
    out.P = P;
    out.gamma = gn;
    return out;
}
template <typename R>
__device__ __noinline__ Emission<R> ncs_emit(const TablesDev& t, const RunDevT<R>& r, uint32_t id, uint32_t n,
                                             Particle<R> P, R gamma, R eta, R xn, R yn, unsigned long long* hist,
                                             unsigned long long* tally) {
    return ncs_emit_body<R>(t, r, id, n, P, gamma, eta, xn, yn, hist, tally);
}

// 1 - e^{-x} in FP32 (the probability of Eq. 4): below 2^-5 by the Taylor series
// x (1 - x/2 + x^2/6 - x^3/24), whose truncation is below x^4/120 < 2^-26 relative (the per-step
// x_b of solid targets is 1e-6 to 1e-3); above it by expm1f
__device__ __forceinline__ float one_minus_exp_neg_f32(float x) {
    if (x < 0x1.0p-5f) return x * fmaf(x, fmaf(x, fmaf(x, -1.0f / 24.0f, 1.0f / 6.0f), -0.5f), 1.0f);
    return -expm1f(-x);
}

// Probability of a brems collision in this step, Eq. (4): P = 1 - exp(-x_b) with
// x_b = n_i sigma_Z(gamma) beta c dt, for an electron in the slab.
template <typename R>
__device__ __forceinline__ R brems_prob(const TablesDev& t, const RunDevT<R>& r, const R* sig_tab,
                                        const Particle<R>& P, R gamma, unsigned long long* tally) {
    bool above;
    R sig = sigma_of<R>(t, sig_tab, gamma, above);
    if (above) atomicAdd(tally + PE_T_N_GAMMA_ABOVE, 1ull);
    R um = m_sqrt(P.u[0] * P.u[0] + P.u[1] * P.u[1] + P.u[2] * P.u[2]);
    R xb = r.c.K_br * sig * (um / gamma);
    if constexpr (sizeof(R) == 4) return one_minus_exp_neg_f32(xb);
    else return -m_expm1(-xb);
}

// Brems photon (text after Eq. 4): y from sigma(y, E) = sigma(E) R2, k^ = v^,
// recoil, tallies.
template <typename R>
__device__ __forceinline__ Emission<R> brems_emit_body(const TablesDev& t, const RunDevT<R>& r, uint32_t id,
                                                       uint32_t n, Particle<R> P, R gamma, R xn, R yn, uint4 w,
                                                       unsigned long long* hist, unsigned long long* tally) {
    Emission<R> out;
    out.stored = false;
    const R photon_min = tabc<R>(t).photon_min;
    R yy = sample_y(t, r.iz, gamma, w);
    R ew = yy * gamma;
    R k[3];
    recoil<R>(P.u, gamma, ew, k);
    note_event<R>(P, n, 1);
    R gn = m_sqrt((R)1 + P.u[0] * P.u[0] + P.u[1] * P.u[1] + P.u[2] * P.u[2]);
    fx_add_r(tally + PE_T_E_RECOIL_BR, gamma - gn);
    if (ew >= photon_min) {
        atomicAdd(tally + PE_T_N_BR_STORED, 1ull);
        fx_add_r(tally + PE_T_E_BR_STORED, ew);
        hist_add<R>(hist, tally, 1, ew, k[0], k[1], r.c.inv_log_emax, t.dbg);
        out.stored = true;
        out.ph = Photon{(float)xn, (float)yn, (float)ew, (float)k[0], (float)k[1], (float)k[2], n, id | 0x80000000u};
    } else {
        atomicAdd(tally + PE_T_N_BR_BELOW, 1ull);
        fx_add_r(tally + PE_T_E_BR_BELOW, ew);
    }
    out.P = P;
    out.gamma = gn;
    return out;
}
template <typename R>
__device__ __noinline__ Emission<R> brems_emit(const TablesDev& t, const RunDevT<R>& r, uint32_t id, uint32_t n,
                                               Particle<R> P, R gamma, R xn, R yn, uint4 w, unsigned long long* hist,
                                               unsigned long long* tally) {
    return brems_emit_body<R>(t, r, id, n, P, gamma, xn, yn, w, hist, tally);
}

// copy an emission branch's result back into the caller's state
template <typename R>
__device__ __forceinline__ void take(const Emission<R>& e, Particle<R>& P, R& gamma, bool& stored, Photon& ph) {
    P = e.P;
    gamma = e.gamma;
    stored = e.stored;
    ph = e.ph;
}

// Bremsstrahlung direct MC collision (Eq. 4 and the text after it) for an
// electron in the slab: event test, photon energy, recoil.  gamma is updated.
template <typename R>
__device__ __forceinline__ void brems_collide(const TablesDev& t, const RunDevT<R>& r, const R* sig_tab,
                                              uint32_t id, uint32_t n, Particle<R>& P, R& gamma, R xn, R yn,
                                              bool& stored, Photon& ph, unsigned long long* hist,
                                              unsigned long long* tally) {
    R Pbr = brems_prob<R>(t, r, sig_tab, P, gamma, tally);
    uint4 w = draw(r, id, n, PUR_BREMS);
    if (brems_event(Pbr, w)) take(brems_emit<R>(t, r, id, n, P, gamma, xn, yn, w, hist, tally), P, gamma, stored, ph);
}

// steps to the next candidate of the majorant process, floor(-ln U / x_hat), in
// double in both precisions (once per candidate; the 32-bit count must not move
// by a step against the FP64 reference)
__device__ __forceinline__ uint32_t wait_draw(double x_hat, uint32_t lo, uint32_t hi) {
    double q = -log(uni53(w64(lo, hi))) / x_hat;
    if (!(q < 4294967295.0)) return PE_WAIT_NEVER;
    return (uint32_t)floor(q);
}

// Null-collision candidate (majorant process, see pe.h): a collision with
// probability P / P_hat (P of Eq. 4, 0 outside the slab), then the next wait.
template <typename R>
__device__ __noinline__ Emission<R> brems_candidate(const TablesDev& t, const RunDevT<R>& r, const R* sig_tab,
                                                    uint32_t id, uint32_t n, Particle<R> P, R gamma, bool in_slab,
                                                    R xn, R yn, unsigned long long* hist, unsigned long long* tally) {
    Emission<R> out;
    out.stored = false;
    out.gamma = gamma;
    R p_acc = 0;
    if (in_slab && gamma > (R)1 + tabc<R>(t).photon_min)
        p_acc = brems_prob<R>(t, r, sig_tab, P, gamma, tally) / r.c.P_hat;
    // one draw of purpose 256 at step n + 1: the next wait (x, y) and the test word (z, w);
    // purpose 0 at step n only for a collision (the photon-energy word, as in the direct method)
    uint4 v = draw(r, id, n + 1u, PUR_WAIT);
    if (brems_event(p_acc, make_uint4(v.z, v.w, 0u, 0u)))
        out = brems_emit<R>(t, r, id, n, P, gamma, xn, yn, draw(r, id, n, PUR_BREMS), hist, tally);
    else
        out.P = P;
    out.P.wait = wait_draw(r.x_hat, v.x, v.y);
    return out;
}

// absorbing boundary in x (Sec. 3): the electron is removed (x = NaN)
template <typename R>
__device__ __forceinline__ void box_check(const RunDevT<R>& r, Particle<R>& P, uint32_t n, unsigned long long* tally) {
    if (r.box_enable && (P.x < r.c.box0 || P.x > r.c.box1)) {
        P.x = (R)NAN;
        atomicAdd(tally + PE_T_N_KILLED, 1ull);
        atomicAdd(tally + PE_T_KILLED_STEPS, (unsigned long long)n + 1ull);
    }
}

// kCommon: the run has NCS on, direct brems and no absorbing box (the paper's setup), known at
// compile time, so the step carries no test of the run's flags; otherwise they are read from the run.
template <typename R, int G, bool kCommon = false>
__device__ __forceinline__ void step_one(const TablesDev& t, const RunDevT<R>& r, const R* h_tab, const R* sig_tab,
                                         uint32_t id, uint32_t n, R nf, Particle<R>& P,
                                         unsigned long long* hist, unsigned long long* tally) {
    bool st;           // an emission branch stored a photon, appended at once (append_now)
    Photon ph;
    const StepC<R>& c = r.c;
    const R photon_min = tabc<R>(t).photon_min;
    const R dt = c.dt;
    R E[3], B[3];
    fields<R, G>(r, P.x, P.x_lo, P.y, nf, E, B);
    boris<R>(P.u, E, B, dt);
    // gamma; in FP32 also 1/gamma from one reciprocal square root (v / gamma below becomes
    // v * (1/gamma); an emission refreshes it)
    R gamma, inv_g = 0;
    if constexpr (sizeof(R) == 4) {
        const float g2 = 1.0f + P.u[0] * P.u[0] + P.u[1] * P.u[1] + P.u[2] * P.u[2];
        inv_g = rsqrtf(g2);
        gamma = g2 * inv_g;
    } else {
        gamma = m_sqrt((R)1 + P.u[0] * P.u[0] + P.u[1] * P.u[1] + P.u[2] * P.u[2]);
    }
    auto over_gamma = [&](R v) -> R {
        if constexpr (sizeof(R) == 4) return v * inv_g;
        else return v / gamma;
    };
    auto refresh = [&]() {
        if constexpr (sizeof(R) == 4) inv_g = 1.0f / gamma;
    };
    const R xn = P.x, yn = P.y;

    if (kCommon || r.enable_ncs) {
        R eta = eta_of<R, G>(P.u, gamma, E, B, c.inv_ES);
        int fl;
        R h = h_of_eta<R>(t, h_tab, eta, fl);
        if (fl == 1) atomicAdd(tally + PE_T_N_ETA_ABOVE, 1ull);
        // dN/dt dt = sqrt(3) alpha/(2 pi) (m c^2/hbar) (eta/gamma) h(eta) dt
        tau_sub(P, c.ncs_coef * over_gamma(eta) * h);
        if (tau_crossed(P)) {
            take(ncs_emit<R>(t, r, id, n, P, gamma, eta, xn, yn, hist, tally), P, gamma, st, ph);
            if (st) append_now(r, ph);
            refresh();
        }
    }

    if (kCommon || r.enable_brems) {
        bool in_slab = (xn >= c.x0 && xn <= c.x1);
        if ((G == FK_GAUSS_LP || G == FK_GAUSS_CP) && fabs(yn) > c.yh) in_slab = false;
        if (!kCommon && r.brems_method == PE_BREMS_NULL) {
            if (P.wait == 0u) {
                const R g_before = gamma;
                take(brems_candidate<R>(t, r, sig_tab, id, n, P, gamma, in_slab, xn, yn, hist, tally), P, gamma, st, ph);
                if (st) append_now(r, ph);
                if (gamma != g_before) refresh();
            } else if (P.wait != PE_WAIT_NEVER) {
                --P.wait;
            }
        } else if (in_slab && gamma > (R)1 + photon_min) {
            const R g_before = gamma;
            st = false;
            brems_collide<R>(t, r, sig_tab, id, n, P, gamma, xn, yn, st, ph, hist, tally);
            if (st) append_now(r, ph);
            if (gamma != g_before) refresh();
        }
    }

    advance(P.x, P.x_lo, over_gamma(dt * P.u[0]));
    if (G == FK_GAUSS_LP || G == FK_GAUSS_CP) advance(P.y, P.y_lo, over_gamma(dt * P.u[1]));
    if (!kCommon) box_check<R>(r, P, n, tally);
}

__device__ __forceinline__ void load_tau(const RunDevT<double>& r, int64_t i, Particle<double>& P) {
    P.tau = ((const double*)r.tau)[i];
    P.tau_lo = 0;
}
__device__ __forceinline__ void load_tau(const RunDevT<float>& r, int64_t i, Particle<float>& P) {
    float2 v = ((const float2*)r.tau)[i];
    P.tau = v.x;
    P.tau_lo = v.y;
}
__device__ __forceinline__ void store_tau(const RunDevT<double>& r, int64_t i, const Particle<double>& P) {
    ((double*)r.tau)[i] = P.tau;
}
__device__ __forceinline__ void store_tau(const RunDevT<float>& r, int64_t i, const Particle<float>& P) {
    ((float2*)r.tau)[i] = make_float2(P.tau, P.tau_lo);
}

__device__ __forceinline__ void load_pos(const RunDevT<double>& r, int64_t i, Particle<double>& P) {
    P.x = ((const double*)r.x)[i];
    P.y = (r.geometry == PE_GAUSS_2D) ? ((const double*)r.y)[i] : 0.0;
    P.x_lo = 0;
    P.y_lo = 0;
}
__device__ __forceinline__ void load_pos(const RunDevT<float>& r, int64_t i, Particle<float>& P) {
    float2 v = ((const float2*)r.x)[i];
    P.x = v.x;
    P.x_lo = v.y;
    if (r.geometry == PE_GAUSS_2D) {
        float2 q = ((const float2*)r.y)[i];
        P.y = q.x;
        P.y_lo = q.y;
    } else {
        P.y = 0;
        P.y_lo = 0;
    }
}
__device__ __forceinline__ void store_pos(const RunDevT<double>& r, int64_t i, const Particle<double>& P) {
    ((double*)r.x)[i] = P.x;
    if (r.geometry == PE_GAUSS_2D) ((double*)r.y)[i] = P.y;
}
// pairs are stored exactly as held in registers, so a launch boundary changes nothing
__device__ __forceinline__ void store_pos(const RunDevT<float>& r, int64_t i, const Particle<float>& P) {
    ((float2*)r.x)[i] = make_float2(P.x, P.x_lo);
    if (r.geometry == PE_GAUSS_2D) ((float2*)r.y)[i] = make_float2(P.y, P.y_lo);
}

template <typename R>
__device__ __forceinline__ void load_particle(const RunDevT<R>& r, int64_t i, Particle<R>& P) {
    load_pos(r, i, P);
    P.u[0] = ((const R*)r.ux)[i];
    P.u[1] = ((const R*)r.uy)[i];
    P.u[2] = ((const R*)r.uz)[i];
    load_tau(r, i, P);
    P.wait = r.wait ? r.wait[i] : PE_WAIT_NEVER;
    if (r.events) {
        unsigned long long e = r.events[i];
        P.ev_cnt = (uint32_t)e;
        P.ev_hash = (uint32_t)(e >> 32);
    } else {
        P.ev_cnt = P.ev_hash = 0;
    }
}
template <typename R>
__device__ __forceinline__ void store_particle(const RunDevT<R>& r, int64_t i, const Particle<R>& P) {
    store_pos(r, i, P);
    ((R*)r.ux)[i] = P.u[0];
    ((R*)r.uy)[i] = P.u[1];
    ((R*)r.uz)[i] = P.u[2];
    store_tau(r, i, P);
    if (r.wait) r.wait[i] = P.wait;
    if (r.events) r.events[i] = ((unsigned long long)P.ev_hash << 32) | P.ev_cnt;
}

// At a launch boundary (the state just loaded for step n): false for a removed particle
// (x = NaN with finite momenta: left the box or the PIC grid, or removed here before).  A
// particle whose momentum is NaN or infinite (from the caller's buffers, or arithmetic that
// overflowed) is removed here: x = NaN, momenta zeroed so it is counted once, stored back,
// and counted in N_NONFINITE and N_KILLED with its n steps alive.
template <typename R>
__device__ __forceinline__ bool live_or_kill(const RunDevT<R>& r, int64_t i, Particle<R>& P, uint32_t n,
                                             unsigned long long* tally) {
    if (isfinite(P.u[0]) && isfinite(P.u[1]) && isfinite(P.u[2])) return !isnan(P.x);
    P.x = (R)NAN;
    P.u[0] = P.u[1] = P.u[2] = (R)0;
    store_particle<R>(r, i, P);
    atomicAdd(tally + PE_T_N_NONFINITE, 1ull);
    atomicAdd(tally + PE_T_N_KILLED, 1ull);
    atomicAdd(tally + PE_T_KILLED_STEPS, (unsigned long long)n);
    return false;
}

// ---------------------------------------------------------------------------
// persistent kernel: grid-stride over tiles of all runs, K steps per launch
// ---------------------------------------------------------------------------
template <typename R>
__device__ void flush_shared(unsigned long long* s_hist, unsigned long long* s_tally, const RunDevT<R>& r) {
    __syncthreads();
    for (int k = threadIdx.x; k < PE_HIST_WORDS; k += blockDim.x) {
        unsigned long long v = s_hist[k];
        if (v) { atomicAdd(r.hist + k, v); s_hist[k] = 0; }
    }
    if (threadIdx.x < PE_T_E_NCS_STORED) {
        unsigned long long v = s_tally[threadIdx.x];
        if (v) { atomicAdd(r.tally + threadIdx.x, v); s_tally[threadIdx.x] = 0; }
    } else if (threadIdx.x < PE_TALLY_WORDS && ((threadIdx.x - PE_T_E_NCS_STORED) & 1) == 0 &&
               threadIdx.x <= PE_T_E_RECOIL_BR) {
        int k = threadIdx.x;
        unsigned long long lo = s_tally[k], hi = s_tally[k + 1];
        if (lo || hi) {
            unsigned long long old = atomicAdd(r.tally + k, lo);
            if (old + lo < old) hi += 1;
            if (hi) atomicAdd(r.tally + k + 1, hi);
            s_tally[k] = 0;
            s_tally[k + 1] = 0;
        }
    }
    __syncthreads();
}

// K steps of one particle with its state in registers
template <typename R, int G, bool kCommon>
__device__ __forceinline__ void tile_steps(const TablesDev& t, const RunDevT<R>& r, const R* s_h, const R* sig_z,
                                           int64_t i, bool active, Particle<R>& P, int steps,
                                           unsigned long long* s_hist, unsigned long long* s_tally) {
    const uint32_t n0 = (uint32_t)r.step0;
    R nf = (R)n0;                      // step index as a float, advanced by exact +1
    for (int s = 0; s < steps; ++s, nf += (R)1) {
        if (active) {
            step_one<R, G, kCommon>(t, r, s_h, sig_z, r.id0 + (uint32_t)i, n0 + (uint32_t)s, nf, P, s_hist, s_tally);
            if (!kCommon && r.box_enable && isnan(P.x)) { active = false; store_particle<R>(r, i, P); }
        }
    }
    if (active) store_particle<R>(r, i, P);
}

// Every run of a launch has field kind G.  kSingle: one run, its descriptor read
// straight from the kernel parameters (constant-bank operands); otherwise the
// current run's descriptor is copied to shared memory once per tile, so no step
// reads an indexed kernel parameter.
// Resident CTAs of 256 threads per SM the register budget is sized for (64 registers; the FP64
// persistent kernels)
#ifndef PE_MIN_CTAS
#define PE_MIN_CTAS 4
#endif
template <typename R, bool kSingle, int G, bool kCommon = false>
__global__ void __launch_bounds__(256, PE_MIN_CTAS) k_step_persistent(TablesDev t, BatchDevT<R> b, int steps) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ RunDevT<R> s_run;
    unsigned long long* s_hist = reinterpret_cast<unsigned long long*>(smem);
    unsigned long long* s_tally = s_hist + PE_HIST_WORDS;
    R* s_h = reinterpret_cast<R*>(s_tally + PE_TALLY_WORDS);
    R* s_sig = s_h + t.n_eta;
    const R* g_h = (sizeof(R) == 4) ? (const R*)t.h32 : (const R*)t.h64;
    const R* g_sig = (sizeof(R) == 4) ? (const R*)t.sig32 : (const R*)t.sig64;

    for (int k = threadIdx.x; k < PE_HIST_WORDS + PE_TALLY_WORDS; k += blockDim.x) s_hist[k] = 0;
    for (int k = threadIdx.x; k < t.n_eta; k += blockDim.x) s_h[k] = g_h[k];
    for (int k = threadIdx.x; k < t.n_Z * t.n_E; k += blockDim.x) s_sig[k] = g_sig[k];
    __syncthreads();

    const int64_t n_tiles = b.tile_start[b.n_runs];
    int cur = -1;
    int run_idx = 0;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        if (!kSingle) {
            while (run_idx + 1 < b.n_runs && b.tile_start[run_idx + 1] <= tile) ++run_idx;
            if (run_idx != cur) {
                if (cur >= 0) flush_shared<R>(s_hist, s_tally, s_run);
                constexpr int kWords = sizeof(RunDevT<R>) / 4;
                static_assert(kWords <= 256, "run descriptor larger than one word per thread");
                if (threadIdx.x < kWords)
                    reinterpret_cast<uint32_t*>(&s_run)[threadIdx.x] =
                        reinterpret_cast<const uint32_t*>(&b.runs[run_idx])[threadIdx.x];
                __syncthreads();
                cur = run_idx;
            }
        }
        const RunDevT<R>& r = kSingle ? b.runs[0] : s_run;
        int64_t i = (tile - b.tile_start[run_idx]) * b.tile + threadIdx.x;
        bool active = i < r.n;
        Particle<R> P;
        if (active) {
            load_particle<R>(r, i, P);
            active = live_or_kill<R>(r, i, P, (uint32_t)r.step0, s_tally);
        }
        const R* sig_z = s_sig + (size_t)r.iz * t.n_E;
        tile_steps<R, G, kCommon>(t, r, s_h, sig_z, i, active, P, steps, s_hist, s_tally);
        cur = kSingle ? 0 : cur;
    }
    if (kSingle) {
        if (gridDim.x > 0 && n_tiles > 0) flush_shared<R>(s_hist, s_tally, b.runs[0]);
    } else if (cur >= 0) {
        flush_shared<R>(s_hist, s_tally, s_run);
    }
}


}  // namespace pe
