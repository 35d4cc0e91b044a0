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
// the hardware's approximate square root, written out (the translation unit that instantiates the
// paired kernels rounds its own divisions and square roots as IEEE operations)
__device__ __forceinline__ float2 sqrt2(float2 a) {
    float2 r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r.x) : "f"(a.x));
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r.y) : "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 rsqrt2(float2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }
// -1/d for d >= 1 (both uses below): the hardware reciprocal estimate of -d refined by one
// Newton-Raphson step, r' = r + r (1 + d r), which squares its relative error (about 1 ulp after
// it); it replaces an IEEE division, whose special-case check and branch cost more than the
// estimate and two FMAs.  The sign is taken by the estimate's operand (free) rather than by a
// paired multiply by -1 (a whole instruction: paired arithmetic has no negated operands), and the
// callers absorb it into a constant factor.
__device__ __forceinline__ float2 nrcp2(float2 d) {
    float2 r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(-d.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(-d.y));
    const float2 e = fma2(d, r, P2(1.0f));
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

// 1 - e^{-x} by the Taylor series x (1 - x/2 + x^2/6 - x^3/24) (for x < 2^-5), paired; the
// same operations in the same order as one_minus_exp_neg_f32
__device__ __forceinline__ float2 brems_series2(float2 x) {
    return mul2(x, fma2(x, fma2(x, fma2(x, P2(-1.0f / 24.0f), P2(1.0f / 6.0f)), P2(-0.5f)), P2(1.0f)));
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

// e^{-v} for v >= 0, paired: the hardware base-2 exponential of -v log2(e) (relative error a few
// ulp; underflows to 0)
__device__ __forceinline__ float2 exp_neg2(float2 v) {
    const float2 a = mul2(v, P2(-1.44269504088896341f));
    float2 r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(a.x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(a.y));
    return r;
}

// Amplitude and Gouy phase of the 2D paraxial focus at a = (x - x_f) / z_R, without an
// arctangent: sqrt(w0 / w) e^{i atan(a) / 2} = (1 + i a)^{1/2} / |1 + i a|, and with
// n = |1 + i a| = sqrt(1 + a^2) the square root of 1 + i a is R + i I, R = sqrt((n + 1) / 2),
// I = a / (2 R) (the half-angle formulas; I written without the cancelling n - 1).  Returns
// Rn = R / n and In = I / n, and 1 / n^2 = w0^2 / w^2.
__device__ __forceinline__ void gouy2(float2 a, float2& Rn, float2& In, float2& inv_n2) {
    const float2 q1 = fma2(a, a, P2(1.0f));                    // n^2
    const float2 inv_n = rsqrt2(q1);
    inv_n2 = mul2(inv_n, inv_n);
    const float2 hh = fma2(mul2(q1, inv_n), P2(0.5f), P2(0.5f));   // (n + 1) / 2
    const float2 inv_r = rsqrt2(hh);
    Rn = mul2(mul2(hh, inv_r), inv_n);
    In = mul2(mul2(P2(0.5f), a), mul2(inv_r, inv_n));
}

// envelope g = sin^2(k psi) of a pulse at phase phi, psi the phase distance to the nearer end of
// the pulse, k psi clamped to [0, pi/2] (0 outside the pulse, pi/2 on the flat top); dg/dphi =
// +-k sin(2 k psi), + before the middle of the pulse and - after it (it vanishes on the flat top
// and outside)
__device__ __forceinline__ void envelope2(const StepC<float>& c, float2 phi, float2& g, float2& dg) {
    const float2 rem = sub2(P2(2.0f * c.phi_r + c.phi_f), phi);
    const float2 psi = make_float2(fminf(phi.x, rem.x), fminf(phi.y, rem.y));
    const float2 arg = clamp2(mul2(P2(c.k_env), psi), 0.0f, 1.57079632679489662f);
    float2 rs, rc;
    ramp_sincos2(arg, rs, rc);
    g = mul2(rs, rs);
    const float2 kts = mul2(P2(2.0f * c.k_env), mul2(rs, rc));
    const float2 side = sub2(rem, phi);
    dg = make_float2(copysignf(kts.x, side.x), copysignf(kts.y, side.y));
}

// two electrons; per-electron activity, optical-depth pairs and event fingerprints
struct Pair {
    float2 x, x_lo, u0, u1, u2, tau, tau_lo;
    float2 y, y_lo;                     // 2D focus only (zero and unused in 1D)
    uint32_t ev_cnt[2], ev_hash[2];
    uint32_t wait[2];
    bool act[2];
};

__device__ __forceinline__ Particle<float> unpack(const Pair& Q, int k) {
    Particle<float> P;
    P.x = comp(Q.x, k); P.x_lo = comp(Q.x_lo, k);
    P.y = comp(Q.y, k); P.y_lo = comp(Q.y_lo, k);
    P.u[0] = comp(Q.u0, k); P.u[1] = comp(Q.u1, k); P.u[2] = comp(Q.u2, k);
    P.tau = comp(Q.tau, k); P.tau_lo = comp(Q.tau_lo, k);
    // selects, not Q.ev_cnt[k]: an index unknown at compile time (the reflected wave's emission
    // loop) would move the arrays to local memory
    P.ev_cnt = k ? Q.ev_cnt[1] : Q.ev_cnt[0]; P.ev_hash = k ? Q.ev_hash[1] : Q.ev_hash[0];
    P.wait = k ? Q.wait[1] : Q.wait[0];
    return P;
}
__device__ __forceinline__ void repack(Pair& Q, int k, const Particle<float>& P) {
    set_comp(Q.x, k, P.x); set_comp(Q.x_lo, k, P.x_lo);
    set_comp(Q.y, k, P.y); set_comp(Q.y_lo, k, P.y_lo);
    set_comp(Q.u0, k, P.u[0]); set_comp(Q.u1, k, P.u[1]); set_comp(Q.u2, k, P.u[2]);
    set_comp(Q.tau, k, P.tau); set_comp(Q.tau_lo, k, P.tau_lo);
    if (k) { Q.ev_cnt[1] = P.ev_cnt; Q.ev_hash[1] = P.ev_hash; Q.wait[1] = P.wait; }
    else { Q.ev_cnt[0] = P.ev_cnt; Q.ev_hash[0] = P.ev_hash; Q.wait[0] = P.wait; }
}

// one step of two electrons (G = FK_PLANE_LP, FK_PLANE_CP: the 1D plane wave; FK_REFL_LP,
// FK_REFL_CP: the plane wave and its mirror image; FK_GAUSS_LP, FK_GAUSS_CP: the 2D paraxial focus;
// FK_CONST: constant fields).  An inactive half of the pair (a removed electron, or an
// empty slot past the end of the run) has x = NaN, so its fields, momenta, eta and optical depth
// are NaN from its first step on, and the eta count, the optical depth's crossing and the target
// test are false for it without reading the activity flags.  kCommon: the run has NCS on, direct brems and no
// absorbing box (the paper's setup), known at compile time, so the step carries no test of the
// run's flags; otherwise they are read from the run.
template <int G, bool kCommon>
__device__ __forceinline__ void step_pair(const TablesDev& t, const RunDevT<float>& r, const float* h_tab,
                                          const float* sig_tab, const uint32_t id[2], uint32_t n, float nf, Pair& Q,
                                          unsigned long long* hist, unsigned long long* tally, float2& n_above) {
    const StepC<float>& c = r.c;
    const TabC<float>& tc = t.cf;
    const float2 dt = P2(c.dt), h = P2(0.5f * c.dt);
    // fields at (x^n, t^n): phase, envelope, carrier
    const float2 nf2 = P2(nf);
    float2 phi = fma2(nf2, P2(c.dt_lo), sub2(mul2(nf2, P2(c.dt_hi)), Q.x));
    phi = sub2(phi, Q.x_lo);
    float2 g, dg;
    envelope2(c, phi, g, dg);
    constexpr bool kPlane = G == FK_PLANE_LP || G == FK_PLANE_CP;
    constexpr bool kRefl = G == FK_REFL_LP || G == FK_REFL_CP;
    constexpr bool kConst = G == FK_CONST;
    constexpr bool kOneD = kPlane || kRefl || kConst;   // no transverse position
    constexpr bool kCP = G == FK_PLANE_CP || G == FK_GAUSS_CP || G == FK_REFL_CP;
    float2 by = P2(0.0f), bz = P2(0.0f);                // B_y, B_z of the reflected kinds
    const float2 ma0 = P2(-c.a0);
    float2 ey, ez = P2(0.0f), ex = P2(0.0f), bx = P2(0.0f);
    if constexpr (kPlane) {
    float2 st, ct;
    sincos2(phi, st, ct);
    ey = mul2(ma0, fma2(dg, st, mul2(g, ct)));                 // -a0 (g' sin + g cos)
    if (G == FK_PLANE_CP) ez = mul2(P2(c.a0), sub2(mul2(dg, ct), mul2(g, st)));   // a0 (g' cos - g sin)
    // Boris push with E = (0, ey, ez), B = (0, -ez, ey)
    const float2 mhey = mul2(P2(-0.5f * c.dt), ey);                    // -h E_y (the sign is exact)
    float2 um0 = Q.u0;
    float2 um1 = add2(Q.u1, mhey);
    float2 um2 = (G == FK_PLANE_CP) ? sub2(Q.u2, mul2(h, ez)) : Q.u2;
    float2 q = fma2(um2, um2, fma2(um1, um1, fma2(um0, um0, P2(1.0f))));
    float2 ig = rsqrt2(q);
    float2 t2 = mul2(mhey, ig);                                        // -h B_z / gamma
    if constexpr (G == FK_PLANE_CP) {
        float2 t1 = mul2(mul2(h, ez), ig);                             // -h B_y / gamma
        float2 f = mul2(P2(-2.0f), nrcp2(fma2(t2, t2, fma2(t1, t1, P2(1.0f)))));
        float2 s1 = mul2(f, t1), s2 = mul2(f, t2);
        float2 p0 = add2(um0, sub2(mul2(um1, t2), mul2(um2, t1)));
        float2 p1 = sub2(um1, mul2(um0, t2));
        float2 p2 = add2(um2, mul2(um0, t1));
        Q.u0 = add2(um0, sub2(mul2(p1, s2), mul2(p2, s1)));
        Q.u1 = add2(sub2(um1, mul2(p0, s2)), mhey);
        Q.u2 = sub2(add2(um2, mul2(p0, s1)), mul2(h, ez));
    } else {
        // LP: B = (0, 0, E_y), so t and s lie along z and the rotation leaves u_z alone; the
        // terms with t_y (exact zeros) are left out, which changes no rounding
        float2 f = mul2(P2(-2.0f), nrcp2(fma2(t2, t2, P2(1.0f))));
        float2 s2 = mul2(f, t2);
        float2 p0 = add2(um0, mul2(um1, t2));
        float2 p1 = sub2(um1, mul2(um0, t2));
        Q.u0 = add2(um0, mul2(p1, s2));
        Q.u1 = add2(sub2(um1, mul2(p0, s2)), mhey);
    }
    } else if constexpr (kConst) {
        // constant fields (the Sec. 2.2 bunch: fields off), the general Boris push
        ex = P2(c.E_const[0]);
        ey = P2(c.E_const[1]);
        ez = P2(c.E_const[2]);
        bx = P2(c.B_const[0]);
        by = P2(c.B_const[1]);
        bz = P2(c.B_const[2]);
        const float2 mh = P2(-0.5f * c.dt);
        const float2 um0 = fma2(mh, ex, Q.u0), um1 = fma2(mh, ey, Q.u1), um2 = fma2(mh, ez, Q.u2);
        const float2 ig = rsqrt2(fma2(um2, um2, fma2(um1, um1, fma2(um0, um0, P2(1.0f)))));
        const float2 mhig = mul2(mh, ig);
        const float2 t0 = mul2(bx, mhig), t1 = mul2(by, mhig), t2 = mul2(bz, mhig);   // -h B / gamma
        const float2 f = mul2(P2(-2.0f), nrcp2(fma2(t2, t2, fma2(t1, t1, fma2(t0, t0, P2(1.0f))))));
        const float2 s0_ = mul2(f, t0), s1 = mul2(f, t1), s2 = mul2(f, t2);
        const float2 p0 = add2(um0, sub2(mul2(um1, t2), mul2(um2, t1)));
        const float2 p1 = add2(um1, sub2(mul2(um2, t0), mul2(um0, t2)));
        const float2 p2 = add2(um2, sub2(mul2(um0, t1), mul2(um1, t0)));
        Q.u0 = fma2(mh, ex, add2(um0, sub2(mul2(p1, s2), mul2(p2, s1))));
        Q.u1 = fma2(mh, ey, add2(um1, sub2(mul2(p2, s0_), mul2(p0, s2))));
        Q.u2 = fma2(mh, ez, add2(um2, sub2(mul2(p0, s1), mul2(p1, s0_))));
    } else if constexpr (kRefl) {
        // incident pulse (B = x^ x E) plus the mirror image -r e(psi) at the reflected phase
        // t + x - 2 x_m, moving along -x (B = -x^ x E): E = (0, e_y + r_y, e_z + r_z),
        // B = (0, r_z - e_z, e_y - r_y)
        float2 st, ct;
        sincos2(phi, st, ct);
        const float2 eiy = mul2(ma0, fma2(dg, st, mul2(g, ct)));
        const float2 eiz = kCP ? mul2(P2(c.a0), sub2(mul2(dg, ct), mul2(g, st))) : P2(0.0f);
        const float2 pr = add2(add2(fma2(nf2, P2(c.dt_hi), P2(-c.xm2_hi)), Q.x),
                               fma2(nf2, P2(c.dt_lo), sub2(Q.x_lo, P2(c.xm2_lo))));
        float2 gr, dgr, sr, cr;
        envelope2(c, pr, gr, dgr);
        sincos2(pr, sr, cr);
        const float2 ry = mul2(P2(c.refl_r * c.a0), fma2(dgr, sr, mul2(gr, cr)));    // -r (-a0 (...))
        ey = add2(eiy, ry);
        bz = sub2(eiy, ry);
        if constexpr (kCP) {
            const float2 rz = mul2(P2(-c.refl_r * c.a0), sub2(mul2(dgr, cr), mul2(gr, sr)));
            ez = add2(eiz, rz);
            by = sub2(rz, eiz);
        }
        // Boris push with E = (0, E_y, E_z), B = (0, B_y, B_z)
        const float2 mh = P2(-0.5f * c.dt);
        const float2 um0 = Q.u0;
        const float2 um1 = fma2(mh, ey, Q.u1);
        const float2 um2 = kCP ? fma2(mh, ez, Q.u2) : Q.u2;
        const float2 ig = rsqrt2(fma2(um2, um2, fma2(um1, um1, fma2(um0, um0, P2(1.0f)))));
        const float2 mhig = mul2(mh, ig);
        const float2 t2 = mul2(bz, mhig);                              // -h B_z / gamma
        if constexpr (kCP) {
            const float2 t1 = mul2(by, mhig);                          // -h B_y / gamma
            const float2 f = mul2(P2(-2.0f), nrcp2(fma2(t2, t2, fma2(t1, t1, P2(1.0f)))));
            const float2 s1 = mul2(f, t1), s2 = mul2(f, t2);
            const float2 p0 = add2(um0, sub2(mul2(um1, t2), mul2(um2, t1)));
            const float2 p1 = sub2(um1, mul2(um0, t2));
            const float2 p2 = fma2(um0, t1, um2);
            Q.u0 = add2(um0, sub2(mul2(p1, s2), mul2(p2, s1)));
            Q.u1 = fma2(mh, ey, sub2(um1, mul2(p0, s2)));
            Q.u2 = fma2(mh, ez, fma2(p0, s1, um2));
        } else {
            const float2 f = mul2(P2(-2.0f), nrcp2(fma2(t2, t2, P2(1.0f))));
            const float2 s2 = mul2(f, t2);
            const float2 p0 = fma2(um1, t2, um0);
            const float2 p1 = sub2(um1, mul2(um0, t2));
            Q.u0 = fma2(p1, s2, um0);
            Q.u1 = fma2(mh, ey, sub2(um1, mul2(p0, s2)));
        }
    } else {
        // 2D paraxial focus (fields() in physics.cuh), amplitude and Gouy phase by gouy2: with
        // S = sqrt(w0 / w) e^{-y^2 / w^2} and theta = phi - y^2 / (2 R_c) + atan(a) / 2,
        // E_y = -a0 S (g' sin + g cos), E_x = a0 g S (y / R_c cos + 2 y / w^2 sin), for CP
        // E_z = a0 S (g' cos - g sin) and B_x = a0 g S (2 y / w^2 cos - y / R_c sin); B = (B_x, -E_z, E_y)
        const float2 a = mul2(sub2(Q.x, P2(c.xf)), P2(c.inv_zr));
        float2 Rn, In, inv_n2;
        gouy2(a, Rn, In, inv_n2);
        const float2 yy = mul2(Q.y, Q.y);
        const float2 inv_w2 = mul2(inv_n2, P2(c.inv_w0sq));
        const float2 inv_R = mul2(mul2(a, inv_n2), P2(c.inv_zr));
        const float2 G_ = exp_neg2(mul2(yy, inv_w2));
        float2 s0, c0;
        sincos2(fma2(mul2(yy, inv_R), P2(-0.5f), phi), s0, c0);
        const float2 Sc = mul2(G_, sub2(mul2(Rn, c0), mul2(In, s0)));    // S cos(theta)
        const float2 Ss = mul2(G_, fma2(Rn, s0, mul2(In, c0)));          // S sin(theta)
        ey = mul2(ma0, fma2(dg, Ss, mul2(g, Sc)));
        const float2 yR = mul2(Q.y, inv_R), y2w = mul2(mul2(P2(2.0f), Q.y), inv_w2);
        const float2 a0g = mul2(P2(c.a0), g);
        ex = mul2(a0g, fma2(yR, Sc, mul2(y2w, Ss)));
        if constexpr (kCP) {
            ez = mul2(P2(c.a0), sub2(mul2(dg, Sc), mul2(g, Ss)));
            bx = mul2(a0g, sub2(mul2(y2w, Sc), mul2(yR, Ss)));
        }
        // Boris push, u^- = u - h E, rotation by t = -h B / gamma^-, u^+ = u^- + (u^- + u^- x t) x s
        // - h E (terms of the exact zeros left out: B_y = B_x = E_z = 0 for LP)
        const float2 mh = P2(-0.5f * c.dt);
        const float2 um0 = fma2(mh, ex, Q.u0);
        const float2 um1 = fma2(mh, ey, Q.u1);
        const float2 um2 = kCP ? fma2(mh, ez, Q.u2) : Q.u2;
        const float2 ig = rsqrt2(fma2(um2, um2, fma2(um1, um1, fma2(um0, um0, P2(1.0f)))));
        const float2 mhig = mul2(mh, ig);
        const float2 t2 = mul2(ey, mhig);                              // -h B_z / gamma
        if constexpr (kCP) {
            const float2 t0 = mul2(bx, mhig);                          // -h B_x / gamma
            const float2 t1 = mul2(ez, mul2(P2(0.5f * c.dt), ig));     // -h B_y / gamma, B_y = -E_z
            const float2 f = mul2(P2(-2.0f), nrcp2(fma2(t2, t2, fma2(t1, t1, fma2(t0, t0, P2(1.0f))))));
            const float2 s0_ = mul2(f, t0), s1 = mul2(f, t1), s2 = mul2(f, t2);
            const float2 p0 = add2(um0, sub2(mul2(um1, t2), mul2(um2, t1)));
            const float2 p1 = add2(um1, sub2(mul2(um2, t0), mul2(um0, t2)));
            const float2 p2 = add2(um2, sub2(mul2(um0, t1), mul2(um1, t0)));
            Q.u0 = fma2(mh, ex, add2(um0, sub2(mul2(p1, s2), mul2(p2, s1))));
            Q.u1 = fma2(mh, ey, add2(um1, sub2(mul2(p2, s0_), mul2(p0, s2))));
            Q.u2 = fma2(mh, ez, add2(um2, sub2(mul2(p0, s1), mul2(p1, s0_))));
        } else {
            const float2 f = mul2(P2(-2.0f), nrcp2(fma2(t2, t2, P2(1.0f))));
            const float2 s2 = mul2(f, t2);
            const float2 p0 = fma2(um1, t2, um0);
            const float2 p1 = sub2(um1, mul2(um0, t2));
            Q.u0 = fma2(mh, ex, fma2(p1, s2, um0));
            Q.u1 = fma2(mh, ey, sub2(um1, mul2(p0, s2)));
        }
    }
    // gamma and 1/gamma from one reciprocal square root (1/gamma serves the rate and the
    // position update; emitting lanes refresh it from their new gamma)
    const float2 g2 = fma2(Q.u2, Q.u2, fma2(Q.u1, Q.u1, fma2(Q.u0, Q.u0, P2(1.0f))));
    float2 inv_g = rsqrt2(g2);
    float2 gamma = mul2(g2, inv_g);
    const float2 xn = Q.x, yn = Q.y;
    float gam[2] = {gamma.x, gamma.y};

    if (kCommon || r.enable_ncs) {
        // eta = (gamma - u_x) |E| / E_S for the plane wave; ngm = u_x - gamma, for u_x > 0 as
        // -(1 + u_y^2 + u_z^2) / (gamma + u_x) (no cancellation), its sign taken by the last factor
        float2 up = fma2(Q.u2, Q.u2, fma2(Q.u1, Q.u1, P2(1.0f)));
        float2 ngm = sel2(Q.u0.x > 0.0f, Q.u0.y > 0.0f, mul2(up, nrcp2(add2(gamma, Q.u0))), sub2(Q.u0, gamma));
        float2 eta;
        if constexpr (kPlane) {
            float2 Emag = (G == FK_PLANE_CP) ? sqrt2(fma2(ez, ez, mul2(ey, ey))) : make_float2(fabsf(ey.x), fabsf(ey.y));
            eta = mul2(mul2(ngm, Emag), P2(-c.inv_ES));
        } else if constexpr (kConst) {
            // eta = |V^2 + 2 V_x (u.E)|^{1/2} / E_S with V = (gamma - u_x) E + u x d, d = B - x^ x E =
            // (B_x, B_y + E_z, B_z - E_y); nV = -V
            const float2 d1 = add2(by, ez), d2 = sub2(bz, ey);
            const float2 nV0 = sub2(mul2(ngm, ex), sub2(mul2(Q.u1, d2), mul2(Q.u2, d1)));
            const float2 nV1 = sub2(mul2(ngm, ey), sub2(mul2(Q.u2, bx), mul2(Q.u0, d2)));
            const float2 nV2 = sub2(mul2(ngm, ez), sub2(mul2(Q.u0, d1), mul2(Q.u1, bx)));
            const float2 uE = fma2(Q.u2, ez, fma2(Q.u1, ey, mul2(Q.u0, ex)));
            const float2 qv = sub2(fma2(nV2, nV2, fma2(nV1, nV1, mul2(nV0, nV0))), mul2(mul2(P2(2.0f), nV0), uE));
            const float2 rq = sqrt2(make_float2(fmaxf(qv.x, 0.0f), fmaxf(qv.y, 0.0f)));
            eta = mul2(rq, P2(c.inv_ES));
        } else if constexpr (kRefl) {
            // eta = |V^2 + 2 V_x (u.E)|^{1/2} / E_S with V = (gamma - u_x) E + u x d, d = B - x^ x E =
            // (0, B_y + E_z, B_z - E_y); nV1, nV2 = -V_y, -V_z
            const float2 d2 = sub2(bz, ey);
            const float2 d1 = kCP ? add2(by, ez) : P2(0.0f);
            const float2 V0 = kCP ? sub2(mul2(Q.u1, d2), mul2(Q.u2, d1)) : mul2(Q.u1, d2);
            const float2 nV1 = fma2(ngm, ey, mul2(Q.u0, d2));
            const float2 nV2 = kCP ? sub2(mul2(ngm, ez), mul2(Q.u0, d1)) : P2(0.0f);
            const float2 uE = kCP ? fma2(Q.u2, ez, mul2(Q.u1, ey)) : mul2(Q.u1, ey);
            const float2 qv = fma2(mul2(P2(2.0f), V0), uE, fma2(nV2, nV2, fma2(nV1, nV1, mul2(V0, V0))));
            const float2 rq = sqrt2(make_float2(fmaxf(qv.x, 0.0f), fmaxf(qv.y, 0.0f)));
            eta = mul2(rq, P2(c.inv_ES));
        } else {
            // eta = |V^2 + 2 V_x (u.E)|^{1/2} / E_S with V = (gamma - u_x) E + u x (B - x^ x E): here
            // B_y + E_z = B_z - E_y = 0, so u x (...) = (0, u_z B_x, -u_y B_x); nV = -V except in y
            const float2 nV0 = mul2(ngm, ex);
            const float2 uE = fma2(Q.u1, ey, fma2(Q.u0, ex, kCP ? mul2(Q.u2, ez) : P2(0.0f)));
            float2 V1 = mul2(ngm, ey), V2 = P2(0.0f);
            if constexpr (kCP) {
                V1 = sub2(mul2(Q.u2, bx), V1);                         // u_z B_x + (gamma - u_x) E_y
                V2 = fma2(Q.u1, bx, mul2(ngm, ez));                    // -(V_z)
            }
            const float2 qv = sub2(fma2(V2, V2, fma2(V1, V1, mul2(nV0, nV0))), mul2(mul2(P2(2.0f), nV0), uE));
            const float2 rq = sqrt2(make_float2(fmaxf(qv.x, 0.0f), fmaxf(qv.y, 0.0f)));
            eta = mul2(rq, P2(c.inv_ES));
        }
        // h(eta): row interpolation in log eta (log2 scaled to the row position by one FMA), the
        // classical limit below the table; above it the last row, counted (the position is clamped
        // just below the top node, so the split needs no correction there)
        const float2 tp = fma2(log2v(eta), P2(tc.inv_dln_eta * 0.693147180559945309f),
                               P2(-tc.ln_eta_min * tc.inv_dln_eta));
        n_above = add2(n_above, make_float2(tp.x >= tc.eta_last ? 1.0f : 0.0f, tp.y >= tc.eta_last ? 1.0f : 0.0f));
        const float2 tpc = clamp2(tp, 0.0f, tc.eta_last - 0x1.0p-10f);
        const float2 tt = add2(sub2(tpc, P2(0.5f)), P2(0x1.8p23f));
        const int ix = dbg_idx(t.dbg, __float_as_int(tt.x) - 0x4B400000, t.n_eta - 1);
        const int iy = dbg_idx(t.dbg, __float_as_int(tt.y) - 0x4B400000, t.n_eta - 1);
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
        if (kRefl && (tsum.x <= 0.0f || tsum.y <= 0.0f)) {
            // frequent emissions (about 4 % of the particle-steps in the reflected pulse): the crossings
            // of a lane go one at a time through one inlined branch, so lanes whose crossing is in
            // different halves of their pairs take it together
            unsigned m = (unsigned)(tsum.x <= 0.0f) | ((unsigned)(tsum.y <= 0.0f) << 1);
            while (m) {
                const int k = (m & 1u) ? 0 : 1;
                m &= m - 1u;
                Particle<float> P = unpack(Q, k);
                float gk = k ? gam[1] : gam[0];
                bool st;
                Photon ph;
                take(ncs_emit_body<float>(t, r, k ? id[1] : id[0], n, P, gk, comp(eta, k), comp(xn, k), 0.0f, hist,
                                          tally),
                     P, gk, st, ph);
                if (st) append_now(r, ph);
                repack(Q, k, P);
                set_comp(inv_g, k, __frcp_rn(gk));
                if (k) gam[1] = gk; else gam[0] = gk;
            }
        } else if (tsum.x <= 0.0f || tsum.y <= 0.0f) {  // one test of the pair on the common path
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (comp(tsum, k) <= 0.0f) {
                    Particle<float> P = unpack(Q, k);
                    bool st;
                    Photon ph;
                    take(ncs_emit_body<float>(t, r, id[k], n, P, gam[k], comp(eta, k), comp(xn, k), comp(yn, k), hist,
                                              tally),
                         P, gam[k], st, ph);
                    if (st) append_now(r, ph);
                    repack(Q, k, P);
                    // 1/gamma by the correctly rounded reciprocal: with the branch inlined, a plain
                    // division of its sqrt result is open to per-kernel rewriting (1/sqrt as rsqrt),
                    // and every paired kernel must round it alike
                    set_comp(inv_g, k, __frcp_rn(gam[k]));
                }
            }
        }
    }

    if (kCommon || r.enable_brems) {
        if (!kCommon && r.brems_method == PE_BREMS_NULL) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (!Q.act[k]) continue;
                if (Q.wait[k] == 0u) {
                    const float x = comp(xn, k);
                    Particle<float> P = unpack(Q, k);
                    bool st;
                    Photon ph;
                    const bool in_slab = x >= c.x0 && x <= c.x1 && (kOneD || fabsf(comp(yn, k)) <= c.yh);
                    take(brems_candidate<float>(t, r, sig_tab, id[k], n, P, gam[k], in_slab, x, comp(yn, k), hist,
                                                tally),
                         P, gam[k], st, ph);
                    if (st) append_now(r, ph);
                    repack(Q, k, P);
                    set_comp(inv_g, k, __frcp_rn(gam[k]));
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
                in[k] = x >= c.x0 && x <= c.x1 && (kOneD || fabsf(comp(yn, k)) <= c.yh) &&
                        gam[k] > 1.0f + tc.photon_min;
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
                const int gx = dbg_idx(t.dbg, __float_as_int(tt.x) - 0x4B400000, t.n_E - 1);
                const int gy = dbg_idx(t.dbg, __float_as_int(tt.y) - 0x4B400000, t.n_E - 1);
                const float2 w = sub2(tgc, sub2(tt, P2(0x1.8p23f)));
                const float2 s0 = make_float2(sig_tab[gx], sig_tab[gy]);
                const float2 s1 = make_float2(sig_tab[gx + 1], sig_tab[gy + 1]);
                const float2 sig = fma2(w, sub2(s1, s0), s0);
                const float2 um = sqrt2(fma2(Q.u2, Q.u2, fma2(Q.u1, Q.u1, mul2(Q.u0, Q.u0))));
                const float2 xb = mul2(mul2(P2(c.K_br), sig), mul2(um, inv_g));
                // 1 - e^{-x_b} by its Taylor series below 2^-5 (truncation under 2^-26 relative), the
                // library expm1f above: one_minus_exp_neg_f32 on the paired instructions
                const float2 ser = brems_series2(xb);
                float pb_[2] = {ser.x, ser.y};
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (!in[k]) continue;
                    if (!(comp(xb, k) < 0x1.0p-5f)) pb_[k] = -expm1f(-comp(xb, k));
                    const uint4 wd = draw(r, id[k], n, PUR_BREMS);
                    if (brems_event(pb_[k], wd)) {
                        Particle<float> P = unpack(Q, k);
                        bool st;
                        Photon ph;
                        take(brems_emit_body<float>(t, r, id[k], n, P, gam[k], comp(xn, k), comp(yn, k), wd, hist, tally), P,
                             gam[k], st, ph);
                        if (st) append_now(r, ph);
                        repack(Q, k, P);
                        set_comp(inv_g, k, __frcp_rn(gam[k]));
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
    if constexpr (!kOneD) {                             // y^{n+1} = y^n + dt u_y / gamma, compensated
        two_sum2(Q.y, mul2(mul2(dt, Q.u1), inv_g), s, e);
        Q.y = s;
        Q.y_lo = add2(Q.y_lo, e);
    }
    if (!kCommon && r.box_enable) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (!Q.act[k]) continue;
            Particle<float> P = unpack(Q, k);
            box_check<float>(r, P, n, tally);
            repack(Q, k, P);
        }
    }
}

__device__ __forceinline__ void load_one(const RunDevT<float>& r, int64_t i, Pair& Q, int k,
                                         unsigned long long* tally) {
    Particle<float> P;
    load_particle<float>(r, i, P);
    Q.act[k] = live_or_kill<float>(r, i, P, (uint32_t)r.step0, tally);
    repack(Q, k, P);
}

// K steps of the pair Q (electrons i0 and i1); photons are appended inside the emission branches
// (append_now), so none is held across the step
template <int G, bool kCommon>
__device__ __forceinline__ void pair_loop(const TablesDev& t, const RunDevT<float>& r, const float* s_h,
                                          const float* sig_z, int64_t i0, int64_t i1, Pair& Q, int steps,
                                          unsigned long long* s_hist, unsigned long long* s_tally) {
    const uint32_t id[2] = {r.id0 + (uint32_t)i0, r.id0 + (uint32_t)i1};
    const uint32_t n0 = (uint32_t)r.step0;
    float nf = (float)n0;
    float2 n_above = P2(0.0f);                          // particle-steps with eta above the table (exact to 2^24)
    for (int s = 0; s < steps; ++s, nf += 1.0f) {
        if (Q.act[0] || Q.act[1]) {
            step_pair<G, kCommon>(t, r, s_h, sig_z, id, n0 + (uint32_t)s, nf, Q, s_hist, s_tally, n_above);
            if (!kCommon && r.box_enable) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (Q.act[k] && isnan(comp(Q.x, k))) {
                        Q.act[k] = false;
                        store_particle<float>(r, k ? i1 : i0, unpack(Q, k));
                    }
                }
            }
        }
    }
    const unsigned int na = __float2uint_rz(n_above.x) + __float2uint_rz(n_above.y);
    if (na) atomicAdd(s_tally + PE_T_N_ETA_ABOVE, (unsigned long long)na);
}

__device__ __forceinline__ void pair_clear(Pair& Q) {
    Q.x_lo = Q.y = Q.y_lo = Q.u0 = Q.u1 = Q.u2 = Q.tau_lo = P2(0.0f);
    Q.x = Q.tau = P2(__int_as_float(0x7fc00000));       // an empty slot is NaN, as a removed electron
    Q.ev_cnt[0] = Q.ev_cnt[1] = Q.ev_hash[0] = Q.ev_hash[1] = 0;
    Q.wait[0] = Q.wait[1] = PE_WAIT_NEVER;
    Q.act[0] = Q.act[1] = false;
}

// K steps of the two electrons i0 = base + tid and i1 = base + tid + blockDim
template <int G, bool kCommon>
__device__ __forceinline__ void tile_steps_pair(const TablesDev& t, const RunDevT<float>& r, const float* s_h,
                                                const float* sig_z, int64_t i0, int64_t i1, int steps,
                                                unsigned long long* s_hist, unsigned long long* s_tally) {
    Pair Q;
    pair_clear(Q);
    if (i0 < r.n) load_one(r, i0, Q, 0, s_tally);
    if (i1 < r.n) load_one(r, i1, Q, 1, s_tally);
    if constexpr (G != FK_GAUSS_LP && G != FK_GAUSS_CP) Q.y = Q.y_lo = P2(0.0f);   // 1D: y is not state
    const bool live0 = i0 < r.n, live1 = i1 < r.n;
    pair_loop<G, kCommon>(t, r, s_h, sig_z, i0, i1, Q, steps, s_hist, s_tally);
    if (live0 && Q.act[0]) store_particle<float>(r, i0, unpack(Q, 0));
    if (live1 && Q.act[1]) store_particle<float>(r, i1, unpack(Q, 1));
}

// Resident CTAs of 128 threads per SM the register budget is sized for.  Measured on the headline job
// with the run's flags as compile-time constants (particle-steps/s): 4 CTAs (128 registers) 1.59e11,
// 5 (96) 1.74e11, 6 (80) 1.78e11, 7 (72) 1.79e11, 8 (64) 1.77e11; the grid of three resident waves
// (21 CTAs per SM) stays the best at 7 (7: 1.63e11, 14: 1.77e11, 21: 1.79e11, 28 and 35: 1.79e11).
// With the emission branches inlined (no call in the loop, no spill at 72 registers): 6 CTAs
// 2.005e11, 7 2.058e11, 8 2.066e11 (at 64 registers the batch instance spills).
#ifndef PE_PAIR_MIN_CTAS
#define PE_PAIR_MIN_CTAS 7
#endif
// The 2D focus (config 3, one run, particle-steps/s): 4 CTAs (128 registers) 1.25e11, 5 (96)
// 1.30e11, 6 (80) 1.31e11; at 80 registers the batch instance (served requests) spills, at 96 none.
#ifndef PE_PAIR_MIN_CTAS_2D
#define PE_PAIR_MIN_CTAS_2D 5
#endif
// The reflected wave (1e6 electrons x 4000 steps of the a0 = 270 job with the mirror at the slab
// rear): 6 CTAs 4.97e10, 7 5.02e10, 8 4.63e10 (one electron per thread at 8 CTAs of 256 threads:
// 4.78e10); 7 CTAs 5.50e10 once the emission loop's pair-half selects kept the per-electron words
// out of local memory.
#ifndef PE_PAIR_MIN_CTAS_REFL
#define PE_PAIR_MIN_CTAS_REFL 7
#endif
// The general instances (flags read at run time: the null-collision method, a process switched
// off, the box boundary) carry more live state than the common ones, but more registers for them
// measured slower on the 1 GeV Au bunch (1e6 electrons, fields off, dt = T; direct / null-collision
// particle-steps/s): 7 CTAs (72 registers) 9.88e10 / 7.09e10, 6 (80) 9.55e10 / 6.70e10, 5 (96)
// 9.34e10 / 7.01e10.
#ifndef PE_PAIR_MIN_CTAS_GENERAL
#define PE_PAIR_MIN_CTAS_GENERAL 7
#endif
template <int G, bool kCommon>
constexpr int pair_min_ctas() {
    constexpr int kind = (G == FK_GAUSS_LP || G == FK_GAUSS_CP) ? PE_PAIR_MIN_CTAS_2D
                         : (G == FK_REFL_LP || G == FK_REFL_CP) ? PE_PAIR_MIN_CTAS_REFL : PE_PAIR_MIN_CTAS;
    return kCommon || kind < PE_PAIR_MIN_CTAS_GENERAL ? kind : PE_PAIR_MIN_CTAS_GENERAL;
}
// Persistent kernel of the paired form: 128 threads cover a tile of 256 electrons.
template <bool kSingle, int G, bool kCommon>
__global__ void __launch_bounds__(128, (pair_min_ctas<G, kCommon>())) k_step_pair(TablesDev t, BatchDevT<float> b, int steps) {
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
        tile_steps_pair<G, kCommon>(t, r, s_h, s_sig + (size_t)r.iz * t.n_E, i0, i1, steps, s_hist, s_tally);
    }
    if (kSingle) {
        if (n_tiles > 0) flush_shared<float>(s_hist, s_tally, b.runs[0]);
    } else if (cur >= 0) {
        flush_shared<float>(s_hist, s_tally, s_run);
    }
}


// ---------------------------------------------------------------------------
// Streaming form for launches of a few steps (the state round-trips HBM every launch).
// Each thread takes two adjacent electrons (2j, 2j + 1) of a 256-electron tile, so one
// 16-byte vector covers both position pairs (and both optical-depth pairs) and one 8-byte
// vector both values of each momentum component.  Each thread prefetches its two
// electrons of the CTA's next tile into its own slots of a shared-memory stage with
// per-thread asynchronous copies (cp.async, 16 and 8 bytes) while it steps the current
// tile, and waits only for its own copies (cp.async.wait_group): no barrier, no spin-wait.
// Results go back with streaming vector stores.  The arithmetic is that of the resident
// kernel (the paired step is elementwise in its two electrons), so the results are the
// same bit for bit.  Single run; the ragged end (an odd last electron) and the optional
// event / wait words use plain loads.
// ---------------------------------------------------------------------------
constexpr int kStreamTile = 256;                       // electrons per tile (128 threads x 2)
constexpr int kStreamThreads = kStreamTile / 2;
// Measured on the 3e7-electron, 4000-step one-step job (stages x CTAs per SM, TB/s at 56 B per
// particle-step), with the emission calls of the step: 2 x 4 4.83, 3 x 3 4.77, 3 x 4 4.60, 2 x 5
// 4.52, 4 x 4 4.12, 3 x 5 4.14, 2 x 6 3.87 (128 registers took the step without spills, and larger
// stages shrink the L1 that holds the remaining local memory).  With the emission branches inlined
// and photons appended in place the step needs 104 registers: 2 x 4 5.48, 2 x 5 5.80, 2 x 6 4.71.
#ifndef PE_STREAM_STAGES
#define PE_STREAM_STAGES 2    // stages per CTA: tiles in flight = stages - 1
#endif
#ifndef PE_STREAM_MIN_CTAS
#define PE_STREAM_MIN_CTAS 5  // resident CTAs of 128 threads per SM the registers are sized for
#endif
constexpr int kStreamStages = PE_STREAM_STAGES;
// one stage: x pairs (float4 per thread), tau pairs (float4), ux, uy, uz (float2 each)
constexpr int kStageBytes = kStreamThreads * (16 + 16 + 8 + 8 + 8);

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// all of this thread's copy groups but the most recent `n` have landed
template <int n>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(n) : "memory"); }

// this thread's slots of a stage
struct StageSlots {
    uint32_t x, tau, ux, uy, uz;       // shared addresses (for the copies)
    const float4* px;                  // generic pointers (for the reads)
    const float4* ptau;
    const float2 *pux, *puy, *puz;
};
__device__ __forceinline__ StageSlots stage_slots(unsigned char* stage, int t) {
    StageSlots q;
    unsigned char* b = stage;
    q.px = reinterpret_cast<const float4*>(b) + t;
    q.ptau = reinterpret_cast<const float4*>(b + kStreamThreads * 16) + t;
    q.pux = reinterpret_cast<const float2*>(b + kStreamThreads * 32) + t;
    q.puy = reinterpret_cast<const float2*>(b + kStreamThreads * 40) + t;
    q.puz = reinterpret_cast<const float2*>(b + kStreamThreads * 48) + t;
    q.x = smem_addr(q.px); q.tau = smem_addr(q.ptau);
    q.ux = smem_addr(q.pux); q.uy = smem_addr(q.puy); q.uz = smem_addr(q.puz);
    return q;
}
// copies of electrons 2j, 2j + 1 (both present) into the slots
__device__ __forceinline__ void stage_issue(const RunDevT<float>& r, int64_t j, const StageSlots& q) {
    cp_async16(q.x, reinterpret_cast<const float4*>(r.x) + j);
    cp_async16(q.tau, reinterpret_cast<const float4*>(r.tau) + j);
    cp_async8(q.ux, reinterpret_cast<const float2*>(r.ux) + j);
    cp_async8(q.uy, reinterpret_cast<const float2*>(r.uy) + j);
    cp_async8(q.uz, reinterpret_cast<const float2*>(r.uz) + j);
}
// a particle is removed (x NaN, finite momenta), live, or has a non-finite momentum
__device__ __forceinline__ bool finite3(float a, float b, float c) { return isfinite(a) && isfinite(b) && isfinite(c); }

// electrons 2j, 2j + 1 from the slots (the optional words from global memory)
__device__ __forceinline__ void stage_take(const RunDevT<float>& r, int64_t j, const StageSlots& q, Pair& Q,
                                           unsigned long long* tally) {
    const float4 x = *q.px, tau = *q.ptau;
    Q.x = make_float2(x.x, x.z);
    Q.x_lo = make_float2(x.y, x.w);
    Q.tau = make_float2(tau.x, tau.z);
    Q.tau_lo = make_float2(tau.y, tau.w);
    Q.u0 = *q.pux;
    Q.u1 = *q.puy;
    Q.u2 = *q.puz;
    if (r.wait) {
        const uint2 w = reinterpret_cast<const uint2*>(r.wait)[j];
        Q.wait[0] = w.x;
        Q.wait[1] = w.y;
    } else {
        Q.wait[0] = Q.wait[1] = PE_WAIT_NEVER;
    }
    if (r.events) {
        const ulonglong2 e = reinterpret_cast<const ulonglong2*>(r.events)[j];
        Q.ev_cnt[0] = (uint32_t)e.x; Q.ev_hash[0] = (uint32_t)(e.x >> 32);
        Q.ev_cnt[1] = (uint32_t)e.y; Q.ev_hash[1] = (uint32_t)(e.y >> 32);
    } else {
        Q.ev_cnt[0] = Q.ev_cnt[1] = Q.ev_hash[0] = Q.ev_hash[1] = 0;
    }
    Q.act[0] = !isnan(Q.x.x);
    Q.act[1] = !isnan(Q.x.y);
    if (!finite3(Q.u0.x, Q.u1.x, Q.u2.x) || !finite3(Q.u0.y, Q.u1.y, Q.u2.y)) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {             // rare: remove and count (as live_or_kill)
            Particle<float> P = unpack(Q, k);
            Q.act[k] = live_or_kill<float>(r, 2 * j + k, P, (uint32_t)r.step0, tally);
            repack(Q, k, P);
        }
    }
}

// electrons 2j, 2j + 1 back to memory (both present; removed ones were stored when removed)
__device__ __forceinline__ void pair_store(const RunDevT<float>& r, int64_t j, const Pair& Q, bool st0, bool st1) {
    if (st0 && st1) {
        __stcs(reinterpret_cast<float4*>(r.x) + j, make_float4(Q.x.x, Q.x_lo.x, Q.x.y, Q.x_lo.y));
        __stcs(reinterpret_cast<float4*>(r.tau) + j, make_float4(Q.tau.x, Q.tau_lo.x, Q.tau.y, Q.tau_lo.y));
        __stcs(reinterpret_cast<float2*>(r.ux) + j, Q.u0);
        __stcs(reinterpret_cast<float2*>(r.uy) + j, Q.u1);
        __stcs(reinterpret_cast<float2*>(r.uz) + j, Q.u2);
        if (r.wait) reinterpret_cast<uint2*>(r.wait)[j] = make_uint2(Q.wait[0], Q.wait[1]);
        if (r.events)
            reinterpret_cast<ulonglong2*>(r.events)[j] =
                make_ulonglong2(((unsigned long long)Q.ev_hash[0] << 32) | Q.ev_cnt[0],
                                ((unsigned long long)Q.ev_hash[1] << 32) | Q.ev_cnt[1]);
    } else {
        if (st0) store_particle<float>(r, 2 * j, unpack(Q, 0));
        if (st1) store_particle<float>(r, 2 * j + 1, unpack(Q, 1));
    }
}

template <int G, bool kCommon>
__global__ void __launch_bounds__(kStreamThreads, PE_STREAM_MIN_CTAS) k_step_pair_stream(TablesDev t, BatchDevT<float> b,
                                                                                         int steps) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* s_hist = reinterpret_cast<unsigned long long*>(smem);
    unsigned long long* s_tally = s_hist + PE_HIST_WORDS;
    float* s_h = reinterpret_cast<float*>(s_tally + PE_TALLY_WORDS);
    float* s_sig = s_h + t.n_eta;
    // the stages on a 16-byte boundary after the tables
    const uint32_t table_bytes = 8 * (PE_HIST_WORDS + PE_TALLY_WORDS) + 4 * (t.n_eta + t.n_Z * t.n_E);
    unsigned char* stage_buf = smem + ((table_bytes + 15u) & ~15u);
    const RunDevT<float>& r = b.runs[0];

    for (int k = threadIdx.x; k < PE_HIST_WORDS + PE_TALLY_WORDS; k += blockDim.x) s_hist[k] = 0;
    for (int k = threadIdx.x; k < t.n_eta; k += blockDim.x) s_h[k] = t.h32[k];
    for (int k = threadIdx.x; k < t.n_Z * t.n_E; k += blockDim.x) s_sig[k] = t.sig32[k];
    __syncthreads();

    const int64_t n_tiles = b.tile_start[1];
    const int64_t n_pairs = r.n >> 1;                   // j < n_pairs: electrons 2j and 2j + 1 both present
    const int64_t stride = (int64_t)gridDim.x * kStreamThreads;
    const float* sig_z = s_sig + (size_t)r.iz * t.n_E;
    // tile k of this CTA (k = 0, 1, ...) is tile blockIdx.x + k gridDim.x, staged in stage k mod S;
    // the copies of tiles k + 1 .. k + S - 1 are in flight while tile k is stepped
    const int64_t j0 = (int64_t)blockIdx.x * kStreamThreads + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kStreamStages - 1; ++k) {
        const int64_t jk = j0 + k * stride;
        if (jk < n_pairs) stage_issue(r, jk, stage_slots(stage_buf + k * kStageBytes, threadIdx.x));
        cp_async_commit();
    }
    int stage = 0;
    for (int64_t j = j0; j - threadIdx.x < n_tiles * kStreamThreads; j += stride) {
        const int64_t jn = j + (kStreamStages - 1) * stride;
        const int sn = stage == 0 ? kStreamStages - 1 : stage - 1;       // (stage + S - 1) mod S
        if (jn < n_pairs) stage_issue(r, jn, stage_slots(stage_buf + sn * kStageBytes, threadIdx.x));
        cp_async_commit();
        cp_async_wait<kStreamStages - 1>();             // this thread's copies of the current tile
        Pair Q;
        const bool full = j < n_pairs;
        if (full) {
            stage_take(r, j, stage_slots(stage_buf + stage * kStageBytes, threadIdx.x), Q, s_tally);
        } else {
            pair_clear(Q);
            if (2 * j < r.n) load_one(r, 2 * j, Q, 0, s_tally);   // the odd last electron
        }
        const bool live0 = 2 * j < r.n, live1 = full;
        pair_loop<G, kCommon>(t, r, s_h, sig_z, 2 * j, 2 * j + 1, Q, steps, s_hist, s_tally);
        pair_store(r, j, Q, live0 && Q.act[0], live1 && Q.act[1]);
        stage = stage + 1 == kStreamStages ? 0 : stage + 1;
    }
    cp_async_wait<0>();
    if (n_tiles > 0) flush_shared<float>(s_hist, s_tally, r);
}

}  // namespace pe
