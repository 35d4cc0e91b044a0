// pair_f32.cuh -- the FP32 step for the 1D plane-wave field kinds with two
// electrons per thread.  Blackwell issues paired single-precision arithmetic
// (FFMA2/FADD2/FMUL2: two FP32 results per instruction), so the common path of
// the step -- fields, Boris push, eta, rate lookup, optical depth, the
// bremsstrahlung probability of Eq. 4, position -- runs on float2 values holding
// the two electrons, with the operations of the one-electron float step in the
// same order (where a form differs -- a Newton-refined reciprocal for a
// division, a series for 1 - e^{-x} at small x, Fast2Sum for the optical depth
// -- the comment at the spot says why it holds).  The draws of the
// bremsstrahlung test, emissions and the absorbing boundary leave the packed
// path and run per electron.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace pe {

// ---- paired arithmetic -----------------------------------------------------------
__device__ __forceinline__ float2 P2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b with one paired instruction: (-1) b + a
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, P2(-1.0f), a); }
__device__ __forceinline__ float2 neg2(float2 a) { return __fmul2_rn(a, P2(-1.0f)); }
// per-electron operations (no paired form)
__device__ __forceinline__ float2 sqrt2(float2 a) { return make_float2(sqrtf(a.x), sqrtf(a.y)); }
__device__ __forceinline__ float2 rsqrt2(float2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }
// 1/d for d >= 1 (both uses below): the hardware reciprocal estimate refined by one Newton-Raphson
// step, r' = r + r (1 - d r), which squares its relative error (about 1 ulp after it); it replaces
// an IEEE division, whose special-case check and branch cost more than the estimate and two FMAs
__device__ __forceinline__ float2 rcp2(float2 d) {
    float2 r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(d.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(d.y));
    const float2 e = fma2(neg2(d), r, P2(1.0f));
    return fma2(r, e, r);
}
__device__ __forceinline__ float2 log2v(float2 a) { return make_float2(__log2f(a.x), __log2f(a.y)); }
__device__ __forceinline__ float2 sel2(bool cx, bool cy, float2 a, float2 b) {
    return make_float2(cx ? a.x : b.x, cy ? a.y : b.y);
}
__device__ __forceinline__ float2 clamp2(float2 a, float lo, float hi) {
    return make_float2(fminf(fmaxf(a.x, lo), hi), fminf(fmaxf(a.y, lo), hi));
}
__device__ __forceinline__ float comp(float2 a, int k) { return k ? a.y : a.x; }
__device__ __forceinline__ void set_comp(float2& a, int k, float v) { if (k) a.y = v; else a.x = v; }

// TwoSum on pairs: (s, e) with s + e = a + b exactly
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
    s = add2(a, b);
    float2 bb = sub2(s, a);
    e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}

// ramp sine/cosine of the envelope (0 <= v <= pi/2), paired: the hardware units
__device__ __forceinline__ void ramp_sincos2(float2 v, float2& s_out, float2& c_out) {
    s_out = make_float2(__sinf(v.x), __sinf(v.y));
    c_out = make_float2(__cosf(v.x), __cosf(v.y));
}

// sine and cosine of the carrier phase, paired: Cody-Waite reduction (1980) by 2 pi with a
// two-part constant to |r| <= pi, then the hardware sine and cosine (absolute error below
// 2^-21.4 on [-pi, pi]; 20 instructions per pair fewer than the polynomial form)
__device__ __forceinline__ void sincos2(float2 v, float2& s_out, float2& c_out) {
    const float kMagic = 0x1.8p23f;
    const float2 t = fma2(v, P2(0.159154943091895336f), P2(kMagic));    // 2 pi k + ..., k = rint(v / 2 pi)
    const float2 nk = sub2(P2(kMagic), t);                              // -k, exact
    float2 r = fma2(nk, P2(6.28318548202514648f), v);                   // 2 pi, nearest float
    r = fma2(nk, P2(-1.74845553e-7f), r);                               // 2 pi - its nearest float
    s_out = make_float2(__sinf(r.x), __sinf(r.y));
    c_out = make_float2(__cosf(r.x), __cosf(r.y));
}

// two electrons; per-electron activity, optical-depth pairs and event fingerprints
struct Pair {
    float2 x, x_lo, u0, u1, u2, tau, tau_lo;
    uint32_t ev_cnt[2], ev_hash[2];
    uint32_t wait[2];
    bool act[2];
};

__device__ __forceinline__ Particle<float> unpack(const Pair& Q, int k) {
    Particle<float> P;
    P.x = comp(Q.x, k); P.x_lo = comp(Q.x_lo, k);
    P.y = 0.0f; P.y_lo = 0.0f;
    P.u[0] = comp(Q.u0, k); P.u[1] = comp(Q.u1, k); P.u[2] = comp(Q.u2, k);
    P.tau = comp(Q.tau, k); P.tau_lo = comp(Q.tau_lo, k);
    P.ev_cnt = Q.ev_cnt[k]; P.ev_hash = Q.ev_hash[k];
    P.wait = Q.wait[k];
    return P;
}
__device__ __forceinline__ void repack(Pair& Q, int k, const Particle<float>& P) {
    set_comp(Q.x, k, P.x); set_comp(Q.x_lo, k, P.x_lo);
    set_comp(Q.u0, k, P.u[0]); set_comp(Q.u1, k, P.u[1]); set_comp(Q.u2, k, P.u[2]);
    set_comp(Q.tau, k, P.tau); set_comp(Q.tau_lo, k, P.tau_lo);
    Q.ev_cnt[k] = P.ev_cnt; Q.ev_hash[k] = P.ev_hash;
    Q.wait[k] = P.wait;
}

// one step of two electrons (plane wave, G = FK_PLANE_LP or FK_PLANE_CP)
template <int G>
__device__ __forceinline__ void step_pair(const TablesDev& t, const RunDevT<float>& r, const float* h_tab,
                                          const float* sig_tab, const uint32_t id[2], uint32_t n, float nf, Pair& Q,
                                          bool st_ncs[2], Photon pn[2], bool st_br[2], Photon pb[2],
                                          unsigned long long* hist, unsigned long long* tally, uint32_t& n_above) {
    const StepC<float>& c = r.c;
    const TabC<float>& tc = t.cf;
    const float2 dt = P2(c.dt), h = P2(0.5f * c.dt);
    // fields at (x^n, t^n): phase, envelope, carrier
    const float2 nf2 = P2(nf);
    float2 phi = fma2(nf2, P2(c.dt_lo), sub2(mul2(nf2, P2(c.dt_hi)), Q.x));
    phi = sub2(phi, Q.x_lo);
    // envelope g = sin^2(k psi), psi the phase distance to the nearer end of the pulse, k psi
    // clamped to [0, pi/2] (0 outside the pulse, pi/2 on the flat top); dg/dphi = +-k sin(2 k psi),
    // + before the middle of the pulse and - after it (it vanishes on the flat top and outside)
    const float2 rem = sub2(P2(2.0f * c.phi_r + c.phi_f), phi);
    const float2 psi = make_float2(fminf(phi.x, rem.x), fminf(phi.y, rem.y));
    const float2 arg = clamp2(mul2(P2(c.k_env), psi), 0.0f, 1.57079632679489662f);
    float2 rs, rc;
    ramp_sincos2(arg, rs, rc);
    const float2 g = mul2(rs, rs);
    const float2 kts = mul2(P2(2.0f * c.k_env), mul2(rs, rc));
    const float2 side = sub2(rem, phi);
    const float2 dg = make_float2(copysignf(kts.x, side.x), copysignf(kts.y, side.y));
    float2 st, ct;
    sincos2(phi, st, ct);
    const float2 ma0 = P2(-c.a0);
    float2 ey = mul2(ma0, fma2(dg, st, mul2(g, ct)));          // -a0 (g' sin + g cos)
    float2 ez = P2(0.0f);
    if (G == FK_PLANE_CP) ez = mul2(P2(c.a0), sub2(mul2(dg, ct), mul2(g, st)));   // a0 (g' cos - g sin)
    // Boris push with E = (0, ey, ez), B = (0, -ez, ey)
    const float2 mhey = mul2(P2(-0.5f * c.dt), ey);                    // -h E_y (the sign is exact)
    float2 um0 = Q.u0;
    float2 um1 = add2(Q.u1, mhey);
    float2 um2 = (G == FK_PLANE_CP) ? sub2(Q.u2, mul2(h, ez)) : Q.u2;
    float2 q = fma2(um2, um2, fma2(um1, um1, fma2(um0, um0, P2(1.0f))));
    float2 ig = rsqrt2(q);
    float2 t1 = (G == FK_PLANE_CP) ? mul2(mul2(h, ez), ig) : P2(0.0f);   // -h B_y / gamma
    float2 t2 = mul2(mhey, ig);                                        // -h B_z / gamma
    float2 f = mul2(P2(2.0f), rcp2(fma2(t2, t2, fma2(t1, t1, P2(1.0f)))));
    float2 s1 = mul2(f, t1), s2 = mul2(f, t2);
    float2 p0 = add2(um0, sub2(mul2(um1, t2), mul2(um2, t1)));
    float2 p1 = sub2(um1, mul2(um0, t2));
    float2 p2 = add2(um2, mul2(um0, t1));
    Q.u0 = add2(um0, sub2(mul2(p1, s2), mul2(p2, s1)));
    Q.u1 = add2(sub2(um1, mul2(p0, s2)), mhey);
    Q.u2 = (G == FK_PLANE_CP) ? sub2(add2(um2, mul2(p0, s1)), mul2(h, ez)) : um2;
    // gamma and 1/gamma from one reciprocal square root (1/gamma serves the rate and the
    // position update; emitting lanes refresh it from their new gamma)
    const float2 g2 = fma2(Q.u2, Q.u2, fma2(Q.u1, Q.u1, fma2(Q.u0, Q.u0, P2(1.0f))));
    float2 inv_g = rsqrt2(g2);
    float2 gamma = mul2(g2, inv_g);
    const float2 xn = Q.x;
    float gam[2] = {gamma.x, gamma.y};

    if (r.enable_ncs) {
        // eta = (gamma - u_x) |E| / E_S for the plane wave
        float2 up = fma2(Q.u2, Q.u2, fma2(Q.u1, Q.u1, P2(1.0f)));
        float2 gm = sel2(Q.u0.x > 0.0f, Q.u0.y > 0.0f, mul2(up, rcp2(add2(gamma, Q.u0))), sub2(gamma, Q.u0));
        float2 Emag = (G == FK_PLANE_CP) ? sqrt2(fma2(ez, ez, mul2(ey, ey))) : make_float2(fabsf(ey.x), fabsf(ey.y));
        float2 eta = mul2(mul2(gm, Emag), P2(c.inv_ES));
        // h(eta): row interpolation in log eta (log2 scaled to the row position by one FMA), the
        // classical limit below the table; above it the last row, counted (the position is clamped
        // just below the top node, so the split needs no correction there)
        const float2 tp = fma2(log2v(eta), P2(tc.inv_dln_eta * 0.693147180559945309f),
                               P2(-tc.ln_eta_min * tc.inv_dln_eta));
        n_above += (uint32_t)(Q.act[0] && tp.x >= tc.eta_last) + (uint32_t)(Q.act[1] && tp.y >= tc.eta_last);
        const float2 tpc = clamp2(tp, 0.0f, tc.eta_last - 0x1.0p-10f);
        const float2 tt = add2(sub2(tpc, P2(0.5f)), P2(0x1.8p23f));
        const int ix = __float_as_int(tt.x) - 0x4B400000, iy = __float_as_int(tt.y) - 0x4B400000;
        const float2 w = sub2(tpc, sub2(tt, P2(0x1.8p23f)));
        const float2 h0 = make_float2(h_tab[ix], h_tab[iy]), h1 = make_float2(h_tab[ix + 1], h_tab[iy + 1]);
        float2 hv = fma2(w, sub2(h1, h0), h0);
        hv = sel2(eta.x >= tc.eta_min, eta.y >= tc.eta_min, hv, P2(tc.h_classical));
        // tau -= ncs_coef (eta / gamma) h(eta), compensated by Dekker's Fast2Sum (exact for
        // |tau| >= |dtau|, which holds on every step but the one where tau crosses zero, and
        // that step emits and resets tau)
        const float2 ndtau = mul2(mul2(P2(-c.ncs_coef), mul2(eta, inv_g)), hv);
        const float2 s = add2(Q.tau, ndtau);
        const float2 e = sub2(ndtau, sub2(s, Q.tau));
        Q.tau = s;
        Q.tau_lo = add2(Q.tau_lo, e);
        float2 tsum = add2(Q.tau, Q.tau_lo);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (Q.act[k] && comp(tsum, k) <= 0.0f) {
                Particle<float> P = unpack(Q, k);
                take(ncs_emit<float>(t, r, id[k], n, P, gam[k], comp(eta, k), comp(xn, k), 0.0f, hist, tally), P,
                     gam[k], st_ncs[k], pn[k]);
                repack(Q, k, P);
                set_comp(inv_g, k, 1.0f / gam[k]);
            }
        }
    }

    if (r.enable_brems) {
        if (r.brems_method == PE_BREMS_NULL) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (!Q.act[k]) continue;
                if (Q.wait[k] == 0u) {
                    const float x = comp(xn, k);
                    Particle<float> P = unpack(Q, k);
                    take(brems_candidate<float>(t, r, sig_tab, id[k], n, P, gam[k], x >= c.x0 && x <= c.x1, x, 0.0f,
                                                hist, tally),
                         P, gam[k], st_br[k], pb[k]);
                    repack(Q, k, P);
                    set_comp(inv_g, k, 1.0f / gam[k]);
                } else if (Q.wait[k] != PE_WAIT_NEVER) {
                    --Q.wait[k];
                }
            }
        } else {
            // Eq. 4 for both electrons: x_b = K sigma_Z(gamma) beta on the paired instructions (row
            // position in log gamma from log2 by one FMA, clamped below the top node as for h(eta);
            // beta = |u| / gamma), then per electron in the target its draw and the integer test
            bool in[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float x = comp(xn, k);
                in[k] = Q.act[k] && x >= c.x0 && x <= c.x1 && gam[k] > 1.0f + tc.photon_min;
            }
            if (in[0] || in[1]) {
                const float2 gv = make_float2(gam[0], gam[1]);
                const float2 tg = fma2(log2v(gv), P2(tc.inv_dln_g * 0.693147180559945309f),
                                       P2(-tc.ln_g_min * tc.inv_dln_g));
#pragma unroll
                for (int k = 0; k < 2; ++k)
                    if (in[k] && comp(tg, k) >= tc.g_last) atomicAdd(tally + PE_T_N_GAMMA_ABOVE, 1ull);
                const float2 tgc = clamp2(tg, 0.0f, tc.g_last - 0x1.0p-10f);
                const float2 tt = add2(sub2(tgc, P2(0.5f)), P2(0x1.8p23f));
                const int gx = __float_as_int(tt.x) - 0x4B400000, gy = __float_as_int(tt.y) - 0x4B400000;
                const float2 w = sub2(tgc, sub2(tt, P2(0x1.8p23f)));
                const float2 s0 = make_float2(sig_tab[gx], sig_tab[gy]);
                const float2 s1 = make_float2(sig_tab[gx + 1], sig_tab[gy + 1]);
                const float2 sig = fma2(w, sub2(s1, s0), s0);
                const float2 um = sqrt2(fma2(Q.u2, Q.u2, fma2(Q.u1, Q.u1, mul2(Q.u0, Q.u0))));
                const float2 xb = mul2(mul2(P2(c.K_br), sig), mul2(um, inv_g));
                // 1 - e^{-x_b} by its Taylor series x (1 - x/2 + x^2/6 - x^3/24) below 2^-5 (truncation
                // under 2^-26 relative), the library expm1f above
                const float2 ser = mul2(xb, fma2(xb, fma2(xb, fma2(xb, P2(-1.0f / 24.0f), P2(1.0f / 6.0f)),
                                                           P2(-0.5f)), P2(1.0f)));
                float pb_[2] = {ser.x, ser.y};
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (!in[k]) continue;
                    if (!(comp(xb, k) < 0x1.0p-5f)) pb_[k] = -expm1f(-comp(xb, k));
                    const uint4 wd = draw(r, id[k], n, PUR_BREMS);
                    if (brems_event(pb_[k], wd)) {
                        Particle<float> P = unpack(Q, k);
                        take(brems_emit<float>(t, r, id[k], n, P, gam[k], comp(xn, k), 0.0f, wd, hist, tally), P,
                             gam[k], st_br[k], pb[k]);
                        repack(Q, k, P);
                        set_comp(inv_g, k, 1.0f / gam[k]);
                    }
                }
            }
        }
    }

    // x^{n+1} = x^n + dt u_x / gamma, compensated
    float2 d = mul2(mul2(dt, Q.u0), inv_g);
    float2 s, e;
    two_sum2(Q.x, d, s, e);
    Q.x = s;
    Q.x_lo = add2(Q.x_lo, e);
    if (r.box_enable) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (!Q.act[k]) continue;
            Particle<float> P = unpack(Q, k);
            box_check<float>(r, P, n, tally);
            repack(Q, k, P);
        }
    }
}

__device__ __forceinline__ void load_one(const RunDevT<float>& r, int64_t i, Pair& Q, int k) {
    Particle<float> P;
    load_particle<float>(r, i, P);
    repack(Q, k, P);
    Q.act[k] = !isnan(P.x);
}

// K steps of the pair Q (electrons i0 and i1) with warp-aggregated photon appends
template <int G>
__device__ __forceinline__ void pair_loop(const TablesDev& t, const RunDevT<float>& r, const float* s_h,
                                          const float* sig_z, int64_t i0, int64_t i1, Pair& Q, int steps,
                                          unsigned long long* s_hist, unsigned long long* s_tally) {
    const uint32_t id[2] = {(uint32_t)i0, (uint32_t)i1};
    const uint32_t n0 = (uint32_t)r.step0;
    float nf = (float)n0;
    uint32_t n_above = 0;                               // particle-steps with eta above the table
    for (int s = 0; s < steps; ++s, nf += 1.0f) {
        bool st_ncs[2] = {false, false}, st_br[2] = {false, false};
        Photon pn[2], pb[2];
        if (Q.act[0] || Q.act[1]) {
            step_pair<G>(t, r, s_h, sig_z, id, n0 + (uint32_t)s, nf, Q, st_ncs, pn, st_br, pb, s_hist, s_tally,
                         n_above);
            if (r.box_enable) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (Q.act[k] && isnan(comp(Q.x, k))) {
                        Q.act[k] = false;
                        store_particle<float>(r, k ? i1 : i0, unpack(Q, k));
                    }
                }
            }
        }
        if (__any_sync(0xffffffffu, st_ncs[0] || st_br[0] || st_ncs[1] || st_br[1])) {
            warp_append(r, st_ncs[0], pn[0]);
            warp_append(r, st_br[0], pb[0]);
            warp_append(r, st_ncs[1], pn[1]);
            warp_append(r, st_br[1], pb[1]);
        }
    }
    if (n_above) atomicAdd(s_tally + PE_T_N_ETA_ABOVE, (unsigned long long)n_above);
}

__device__ __forceinline__ void pair_clear(Pair& Q) {
    Q.x = Q.x_lo = Q.u0 = Q.u1 = Q.u2 = Q.tau = Q.tau_lo = P2(0.0f);
    Q.ev_cnt[0] = Q.ev_cnt[1] = Q.ev_hash[0] = Q.ev_hash[1] = 0;
    Q.wait[0] = Q.wait[1] = PE_WAIT_NEVER;
    Q.act[0] = Q.act[1] = false;
}

// K steps of the two electrons i0 = base + tid and i1 = base + tid + blockDim
template <int G>
__device__ __forceinline__ void tile_steps_pair(const TablesDev& t, const RunDevT<float>& r, const float* s_h,
                                                const float* sig_z, int64_t i0, int64_t i1, int steps,
                                                unsigned long long* s_hist, unsigned long long* s_tally) {
    Pair Q;
    pair_clear(Q);
    if (i0 < r.n) load_one(r, i0, Q, 0);
    if (i1 < r.n) load_one(r, i1, Q, 1);
    const bool live0 = i0 < r.n, live1 = i1 < r.n;
    pair_loop<G>(t, r, s_h, sig_z, i0, i1, Q, steps, s_hist, s_tally);
    if (live0 && Q.act[0]) store_particle<float>(r, i0, unpack(Q, 0));
    if (live1 && Q.act[1]) store_particle<float>(r, i1, unpack(Q, 1));
}

#ifndef PE_PAIR_MIN_CTAS
#define PE_PAIR_MIN_CTAS 5   // resident CTAs of 128 threads per SM the register budget is sized for (96 registers)
#endif
// Persistent kernel of the paired form: 128 threads cover a tile of 256 electrons.
template <bool kSingle, int G>
__global__ void __launch_bounds__(128, PE_PAIR_MIN_CTAS) k_step_pair(TablesDev t, BatchDevT<float> b, int steps) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ RunDevT<float> s_run;
    unsigned long long* s_hist = reinterpret_cast<unsigned long long*>(smem);
    unsigned long long* s_tally = s_hist + PE_HIST_WORDS;
    float* s_h = reinterpret_cast<float*>(s_tally + PE_TALLY_WORDS);
    float* s_sig = s_h + t.n_eta;

    for (int k = threadIdx.x; k < PE_HIST_WORDS + PE_TALLY_WORDS; k += blockDim.x) s_hist[k] = 0;
    for (int k = threadIdx.x; k < t.n_eta; k += blockDim.x) s_h[k] = t.h32[k];
    for (int k = threadIdx.x; k < t.n_Z * t.n_E; k += blockDim.x) s_sig[k] = t.sig32[k];
    __syncthreads();

    const int64_t n_tiles = b.tile_start[b.n_runs];
    int cur = -1;
    int run_idx = 0;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        if (!kSingle) {
            while (run_idx + 1 < b.n_runs && b.tile_start[run_idx + 1] <= tile) ++run_idx;
            if (run_idx != cur) {
                if (cur >= 0) flush_shared<float>(s_hist, s_tally, s_run);
                constexpr int kWords = sizeof(RunDevT<float>) / 4;
                for (int w = threadIdx.x; w < kWords; w += blockDim.x)
                    reinterpret_cast<uint32_t*>(&s_run)[w] = reinterpret_cast<const uint32_t*>(&b.runs[run_idx])[w];
                __syncthreads();
                cur = run_idx;
            }
        }
        const RunDevT<float>& r = kSingle ? b.runs[0] : s_run;
        const int64_t base = (tile - b.tile_start[run_idx]) * b.tile;
        const int64_t i0 = base + threadIdx.x, i1 = base + threadIdx.x + blockDim.x;
        tile_steps_pair<G>(t, r, s_h, s_sig + (size_t)r.iz * t.n_E, i0, i1, steps, s_hist, s_tally);
    }
    if (kSingle) {
        if (n_tiles > 0) flush_shared<float>(s_hist, s_tally, b.runs[0]);
    } else if (cur >= 0) {
        flush_shared<float>(s_hist, s_tally, s_run);
    }
}


// ---------------------------------------------------------------------------
// Streaming form for launches of a few steps (the state round-trips HBM): each CTA
// prefetches the state of its next tile into shared memory with bulk copies (TMA,
// cp.async.bulk) that complete on an mbarrier while it steps the current tile, so the
// loads of one tile overlap the arithmetic of the previous one.  Single run; tiles
// of 256 electrons (x pairs 2 KB, u 3 x 1 KB, tau pairs 2 KB per tile); the ragged
// last tile and the optional event / wait words use plain loads.
// ---------------------------------------------------------------------------
constexpr int kStreamTile = 256;
constexpr int kStageBytes = kStreamTile * (8 + 4 + 4 + 4 + 8);

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// wait for the phase of the given parity to complete; gives up after about 2 s (returns false)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255u) == 255u && global_ns() - t0 > 2000000000ull) return false;
    }
    return false;
}

// thread 0: bulk copies of the full tile `tile` into stage buffer `buf`
__device__ __forceinline__ void stream_issue(const RunDevT<float>& r, int64_t tile, unsigned char* buf, uint32_t bar) {
    const int64_t base = tile * kStreamTile;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier generic reads of buf first
    mbar_expect_tx(bar, kStageBytes);
    const uint32_t d = smem_addr(buf);
    bulk_g2s(d, (const float2*)r.x + base, kStreamTile * 8, bar);
    bulk_g2s(d + kStreamTile * 8, (const float*)r.ux + base, kStreamTile * 4, bar);
    bulk_g2s(d + kStreamTile * 12, (const float*)r.uy + base, kStreamTile * 4, bar);
    bulk_g2s(d + kStreamTile * 16, (const float*)r.uz + base, kStreamTile * 4, bar);
    bulk_g2s(d + kStreamTile * 20, (const float2*)r.tau + base, kStreamTile * 8, bar);
}

// electron j of a staged tile into pair slot k (the optional words from global memory)
__device__ __forceinline__ void stream_take(const RunDevT<float>& r, const unsigned char* buf, int j, int64_t i,
                                            Pair& Q, int k) {
    const float2 x = reinterpret_cast<const float2*>(buf)[j];
    const float* u = reinterpret_cast<const float*>(buf + kStreamTile * 8);
    const float2 tau = reinterpret_cast<const float2*>(buf + kStreamTile * 20)[j];
    set_comp(Q.x, k, x.x); set_comp(Q.x_lo, k, x.y);
    set_comp(Q.u0, k, u[j]); set_comp(Q.u1, k, u[kStreamTile + j]); set_comp(Q.u2, k, u[2 * kStreamTile + j]);
    set_comp(Q.tau, k, tau.x); set_comp(Q.tau_lo, k, tau.y);
    Q.wait[k] = r.wait ? r.wait[i] : PE_WAIT_NEVER;
    if (r.events) {
        unsigned long long e = r.events[i];
        Q.ev_cnt[k] = (uint32_t)e;
        Q.ev_hash[k] = (uint32_t)(e >> 32);
    }
    Q.act[k] = !isnan(x.x);
}

template <int G>
__global__ void __launch_bounds__(128, PE_PAIR_MIN_CTAS) k_step_pair_stream(TablesDev t, BatchDevT<float> b, int steps) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* s_hist = reinterpret_cast<unsigned long long*>(smem);
    unsigned long long* s_tally = s_hist + PE_HIST_WORDS;
    float* s_h = reinterpret_cast<float*>(s_tally + PE_TALLY_WORDS);
    float* s_sig = s_h + t.n_eta;
    // stage buffers on a 128-byte boundary of the shared window after the tables
    const uint32_t s0 = smem_addr(smem);
    const uint32_t table_end = s0 + 8 * (PE_HIST_WORDS + PE_TALLY_WORDS) + 4 * (t.n_eta + t.n_Z * t.n_E);
    unsigned char* stage_buf = smem + (((table_end + 127u) & ~127u) - s0);
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(stage_buf + 2 * kStageBytes);
    const RunDevT<float>& r = b.runs[0];

    for (int k = threadIdx.x; k < PE_HIST_WORDS + PE_TALLY_WORDS; k += blockDim.x) s_hist[k] = 0;
    for (int k = threadIdx.x; k < t.n_eta; k += blockDim.x) s_h[k] = t.h32[k];
    for (int k = threadIdx.x; k < t.n_Z * t.n_E; k += blockDim.x) s_sig[k] = t.sig32[k];
    const uint32_t bar0 = smem_addr(&bars[0]), bar1 = smem_addr(&bars[1]);
    if (threadIdx.x == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int64_t n_tiles = b.tile_start[1];
    const int64_t n_full = r.n / kStreamTile;          // tiles with all 256 electrons present
    const float* sig_z = s_sig + (size_t)r.iz * t.n_E;
    uint32_t parity[2] = {0u, 0u};
    bool pending[2] = {false, false};                   // a copy into the stage awaits its wait
    bool stuck[2] = {false, false};                     // its wait ran out: the stage is not reused
    bool broken = false;                                // after a timeout: plain loads only
    int stage = 0;
    int64_t tile = blockIdx.x;
    if (threadIdx.x == 0 && tile < n_full) stream_issue(r, tile, stage_buf, bar0);
    pending[0] = tile < n_full;
    for (; tile < n_tiles; tile += gridDim.x) {
        const int64_t next = tile + gridDim.x;
        if (!broken && next < n_full) {
            if (threadIdx.x == 0) stream_issue(r, next, stage_buf + (stage ^ 1) * kStageBytes, stage ? bar0 : bar1);
            pending[stage ^ 1] = true;
        }
        const int64_t i0 = tile * kStreamTile + threadIdx.x, i1 = i0 + blockDim.x;
        Pair Q;
        pair_clear(Q);
        bool staged = false;
        if (pending[stage]) {
            staged = mbar_wait(stage ? bar1 : bar0, parity[stage]);
            pending[stage] = false;
            if (staged) {
                parity[stage] ^= 1u;
            } else {
                stuck[stage] = true;
                broken = true;
                if (threadIdx.x == 0) atomicAdd(s_tally + PE_T_N_WAIT_TIMEOUT, 1ull);
            }
        }
        if (staged) {
            const unsigned char* buf = stage_buf + stage * kStageBytes;
            stream_take(r, buf, threadIdx.x, i0, Q, 0);
            stream_take(r, buf, threadIdx.x + blockDim.x, i1, Q, 1);
        } else {                                        // ragged last tile (or a timed-out copy)
            if (i0 < r.n) load_one(r, i0, Q, 0);
            if (i1 < r.n) load_one(r, i1, Q, 1);
        }
        const bool live0 = i0 < r.n, live1 = i1 < r.n;
        pair_loop<G>(t, r, s_h, sig_z, i0, i1, Q, steps, s_hist, s_tally);
        if (live0 && Q.act[0]) store_particle<float>(r, i0, unpack(Q, 0));
        if (live1 && Q.act[1]) store_particle<float>(r, i1, unpack(Q, 1));
        __syncthreads();                                // the stage is read before it is refilled
        stage ^= 1;
    }
    // copies still in flight after a timeout must land before the CTA exits (bounded again)
    for (int k = 0; k < 2; ++k)
        if (pending[k] || stuck[k]) mbar_wait(k ? bar1 : bar0, parity[k]);
    if (n_tiles > 0) flush_shared<float>(s_hist, s_tally, r);
}

}  // namespace pe
