// physics.cuh -- per-particle arithmetic of the emission step, templated on
// the floating type R (float for the fast path, double for the plain path).
// Every constant a step reads is stored in R, so the float path issues no
// FP64 instruction per step.  Each function cites the part of the method it
// implements.
#pragma once
#include <cuda_runtime.h>
#include <type_traits>
#include <stdint.h>

#include "internal.h"

namespace pe {

// ---- math wrappers (CUDA's own functions for both types) --------------------
__device__ __forceinline__ float m_sqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double m_sqrt(double v) { return sqrt(v); }
__device__ __forceinline__ float m_exp(float v) { return expf(v); }
__device__ __forceinline__ double m_exp(double v) { return exp(v); }
__device__ __forceinline__ float m_log(float v) { return __logf(v); }
__device__ __forceinline__ double m_log(double v) { return log(v); }
__device__ __forceinline__ float m_log_acc(float v) { return logf(v); }
__device__ __forceinline__ double m_log_acc(double v) { return log(v); }
__device__ __forceinline__ float m_expm1(float v) { return expm1f(v); }
__device__ __forceinline__ double m_expm1(double v) { return expm1(v); }
__device__ __forceinline__ float m_atan(float v) { return atanf(v); }
__device__ __forceinline__ double m_atan(double v) { return atan(v); }
// Single-precision sine and cosine: Cody-Waite reduction (1980) by 2 pi with a
// two-part constant to |r| <= pi (the multiple by magic-number rounding, no int/float
// conversion), then the hardware sine and cosine (absolute error below 2^-21.4 on
// [-pi, pi]).  Valid for |v| < 2^24.
__device__ __forceinline__ void m_sincos(float v, float* s_out, float* c_out) {
    const float kMagic = 0x1.8p23f;                       // 1.5 * 2^23
    const float k = fmaf(v, 0.159154943091895336f, kMagic) - kMagic;   // rint(v / 2 pi)
    float r = fmaf(-k, 6.28318548202514648f, v);          // 2 pi, nearest float
    r = fmaf(-k, -1.74845553e-7f, r);                     // 2 pi - its nearest float
    *s_out = __sinf(r);
    *c_out = __cosf(r);
}
__device__ __forceinline__ void m_sincos(double v, double* s, double* c) { sincos(v, s, c); }

// sin and cos of 0 <= v <= pi/2 (the envelope ramps): the hardware units, no reduction
__device__ __forceinline__ void ramp_sincos(float v, float* s_out, float* c_out) {
    *s_out = __sinf(v);
    *c_out = __cosf(v);
}
__device__ __forceinline__ void ramp_sincos(double v, double* s, double* c) { sincos(v, s, c); }
__device__ __forceinline__ float m_atan2(float a, float b) { return atan2f(a, b); }
__device__ __forceinline__ double m_atan2(double a, double b) { return atan2(a, b); }
__device__ __forceinline__ float m_floor(float v) { return floorf(v); }
__device__ __forceinline__ double m_floor(double v) { return floor(v); }

template <typename R> __device__ __forceinline__ const TabC<R>& tabc(const TablesDev& t);
template <> __device__ __forceinline__ const TabC<float>& tabc<float>(const TablesDev& t) { return t.cf; }
template <> __device__ __forceinline__ const TabC<double>& tabc<double>(const TablesDev& t) { return t.cd; }

// ---- range checks of debug builds --------------------------------------------------
// With -DPE_DEBUG every table row or column, guide entry and histogram bin a kernel is
// about to index is checked against its array: an index outside [0, n) is counted in the
// table set's violation word (pe_debug_count) and clamped into range, so the access stays
// in bounds and nothing traps.  A release build compiles the checks away.
__device__ __forceinline__ int dbg_idx(unsigned long long* word, int i, int n) {
#ifdef PE_DEBUG
    if ((unsigned)i >= (unsigned)n) {
        atomicAdd(word, 1ull);
        return i < 0 ? 0 : n - 1;
    }
#else
    (void)word; (void)n;
#endif
    return i;
}

// ---- Philox4x32-10 (Salmon et al., SC'11) ------------------------------------
// Counter (particle id, run id, step, purpose), key (seed lo, seed hi).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}
enum { PUR_BREMS = 0, PUR_NCS = 1, PUR_TAU0 = 2, PUR_POS = 3, PUR_MJ = 4, PUR_WAIT = 256 };

template <typename R>
__device__ __forceinline__ uint4 draw(const RunDevT<R>& r, uint32_t id, uint32_t step, uint32_t purpose) {
    return philox4x32_10(make_uint4(id, r.run_id, step, purpose), r.seed_lo, r.seed_hi);
}
__device__ __forceinline__ uint64_t w64(uint32_t lo, uint32_t hi) { return ((uint64_t)hi << 32) | lo; }
// uniforms in (0,1) with 53 and 32 random bits
__device__ __forceinline__ double uni53(uint64_t v) { return ((double)(v >> 11) + 0.5) * 0x1.0p-53; }
__device__ __forceinline__ double uni32(uint32_t v) { return ((double)v + 0.5) * 0x1.0p-32; }

// Brems test of Eq. (4): event iff the 64-bit uniform (hi:lo) is below floor(P 2^64).
__device__ __forceinline__ bool below_threshold(double P, uint32_t lo, uint32_t hi) {
    uint64_t T = P >= 1.0 ? 0xFFFFFFFFFFFFFFFFull : __double2ull_rz(P * 0x1.0p64);
    return w64(lo, hi) < T;
}
// float P: floor(P 2^64) = th 2^32 + floor(frac(P 2^32) 2^32), both parts exact in
// float, so the comparison runs on 32-bit integers.
__device__ __forceinline__ bool below_threshold(float P, uint32_t lo, uint32_t hi) {
    if (!(P > 0.0f)) return false;
    if (P >= 1.0f) return true;
    float p32 = P * 0x1.0p32f;
    float fth = floorf(p32);
    uint32_t th = (uint32_t)fth;
    if (hi != th) return hi < th;
    uint32_t tl = (uint32_t)floorf((p32 - fth) * 0x1.0p32f);
    return lo < tl;
}

// ---- prescribed laser fields (Sec. 3 setup) ------------------------------------
// Pulse through its vector potential A(phi), phi = t - x: sin^2 ramps of
// phi_r and a flat top phi_f; E = -dA/dt, B = x^ cross E for the plane wave.
template <typename R>
__device__ __forceinline__ void envelope(const StepC<R>& c, R phi, R& g, R& dg) {
    const R pr = c.phi_r, pf = c.phi_f, k = c.k_env;
    if (!(phi > (R)0) || phi >= (R)2 * pr + pf) { g = 0; dg = 0; return; }
    if (phi < pr) {
        R s, cc;
        ramp_sincos(k * phi, &s, &cc);
        g = s * s;
        dg = k * (R)2 * s * cc;
        return;
    }
    if (phi <= pr + pf) { g = 1; dg = 0; return; }
    R s, cc;
    ramp_sincos(k * (phi - pr - pf), &s, &cc);
    g = cc * cc;
    dg = -k * (R)2 * s * cc;
}

// Float version without branches (lanes of a warp sit in different parts of the
// pulse): g = sin^2(k psi) with psi the phase distance to the nearer end of the pulse,
// k psi clamped to [0, pi/2] (0 outside, pi/2 on the flat top; the falling ramp
// through cos^2(k q) = sin^2(pi/2 - k q)); dg/dphi = +-k sin(2 k psi), + before the
// middle of the pulse and - after it.
__device__ __forceinline__ void envelope_sel(const StepC<float>& c, float phi, float& g, float& dg) {
    const float rem = (2.0f * c.phi_r + c.phi_f) - phi;
    const float arg = fminf(fmaxf(c.k_env * fminf(phi, rem), 0.0f), 1.57079632679489662f);
    float s, cc;
    ramp_sincos(arg, &s, &cc);
    g = s * s;
    dg = copysignf(2.0f * c.k_env * s * cc, rem - phi);
}

// phase t^n - x with t^n = n dt.  In float, n * dt_hi is exact (dt_hi has 11
// significant bits, n < 2^13), the small remainder n * dt_lo is added, and the
// position enters as the unevaluated sum x + x_lo kept by the compensated update.
// nf is the step index n held as a float (exact for n < 2^24).
__device__ __forceinline__ double phase(const StepC<double>& c, double nf, double x, double) {
    return nf * c.dt - x;
}
__device__ __forceinline__ float phase(const StepC<float>& c, float nf, float x, float x_lo) {
    return fmaf(nf, c.dt_lo, nf * c.dt_hi - x) - x_lo;
}

// x += d.  In float the rounding error of every add is kept in x_lo (Knuth's
// TwoSum), so positions stay exact to ~1e-12 over the steps done in registers.
__device__ __forceinline__ void advance(float& x, float& x_lo, float d) {
    float s = x + d;
    float bb = s - x;
    float e = (x - (s - bb)) + (d - bb);
    x = s;
    x_lo += e;
}
__device__ __forceinline__ void advance(double& x, double&, double d) { x += d; }

// phase of the reflected wave t^n + x - 2 x_m, with the same care as phase():
// n * dt_hi - 2 x_m,hi is exact in float (2 x_m,hi lies on dt_hi's grid), then x,
// then the small remainders.
__device__ __forceinline__ double phase_refl(const StepC<double>& c, double nf, double x, double) {
    return nf * c.dt + x - (c.xm2_hi + c.xm2_lo);
}
__device__ __forceinline__ float phase_refl(const StepC<float>& c, float nf, float x, float x_lo) {
    float a = fmaf(nf, c.dt_hi, -c.xm2_hi);
    return (a + x) + fmaf(nf, c.dt_lo, x_lo - c.xm2_lo);
}

// Field kind of a run, a compile-time parameter of the step so that each geometry
// and polarisation gets its own straight-line code.
enum { FK_PLANE_LP = 0, FK_PLANE_CP = 1, FK_GAUSS_LP = 2, FK_GAUSS_CP = 3, FK_CONST = 4, FK_REFL_LP = 5,
       FK_REFL_CP = 6, FK_PIC = 7 };
constexpr int kFieldKinds = 7;        // kinds of the prescribed-field kernels (FK_PIC has its own path)
__host__ __device__ __forceinline__ int field_kind(int geometry, int polarisation, bool reflected) {
    if (geometry == PE_CONST) return FK_CONST;
    if (geometry == PE_PIC_1D) return FK_PIC;
    int cp = polarisation == PE_CP ? 1 : 0;
    if (geometry == PE_PLANE_1D && reflected) return FK_REFL_LP + cp;
    return (geometry == PE_GAUSS_2D ? 2 : 0) + cp;
}

// host dispatch of a runtime field kind to f(std::integral_constant<int, G>{})
template <typename F>
inline void with_field_kind(int fk, F&& f) {
    switch (fk) {
        case FK_PLANE_LP: f(std::integral_constant<int, FK_PLANE_LP>{}); break;
        case FK_PLANE_CP: f(std::integral_constant<int, FK_PLANE_CP>{}); break;
        case FK_GAUSS_LP: f(std::integral_constant<int, FK_GAUSS_LP>{}); break;
        case FK_GAUSS_CP: f(std::integral_constant<int, FK_GAUSS_CP>{}); break;
        case FK_REFL_LP: f(std::integral_constant<int, FK_REFL_LP>{}); break;
        case FK_REFL_CP: f(std::integral_constant<int, FK_REFL_CP>{}); break;
        default: f(std::integral_constant<int, FK_CONST>{}); break;
    }
}

// transverse E of the 1D plane pulse at phase p: E_y = -a0 (g' sin p + g cos p),
// and for CP E_z = a0 (g' cos p - g sin p)
template <typename R, bool kCP>
__device__ __forceinline__ void plane_e(const StepC<R>& c, R p, R& ey, R& ez) {
    R g, dg;
    if constexpr (sizeof(R) == 4) envelope_sel(c, p, g, dg);
    else envelope<R>(c, p, g, dg);
    R st, ct;
    m_sincos(p, &st, &ct);
    ey = -c.a0 * (dg * st + g * ct);
    ez = kCP ? c.a0 * (dg * ct - g * st) : (R)0;
}

// 1D PIC: fields at x from the grid, linear weights of the nodes (transverse fields
// from the wave variants F+- = E_y +- B_z, G+- = E_z -+ B_y) and of the half nodes (E_x);
// zero beyond the grid
template <typename R>
__device__ __forceinline__ void pic_gather(const RunDevT<R>& r, R x, R E[3], R B[3]) {
    const int n = r.n_cells;
    const R* ex = static_cast<const R*>(r.grid);
    const R* fp = ex + n;
    const R* fm = fp + n + 1;
    const R* gp = fm + n + 1;
    const R* gm = gp + n + 1;
    const R s = x / r.c.dt;                          // dx = c dt
    const R fl = floor(s);
    const int i = (int)fl;
    const R f = s - fl;
    R v[4][2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int m = i + k;
        const bool in = m >= 0 && m <= n;
        v[0][k] = in ? fp[m] : (R)0;
        v[1][k] = in ? fm[m] : (R)0;
        v[2][k] = in ? gp[m] : (R)0;
        v[3][k] = in ? gm[m] : (R)0;
    }
    const R Fp = ((R)1 - f) * v[0][0] + f * v[0][1], Fm = ((R)1 - f) * v[1][0] + f * v[1][1];
    const R Gp = ((R)1 - f) * v[2][0] + f * v[2][1], Gm = ((R)1 - f) * v[3][0] + f * v[3][1];
    E[1] = (R)0.5 * (Fp + Fm);
    B[2] = (R)0.5 * (Fp - Fm);
    E[2] = (R)0.5 * (Gp + Gm);
    B[1] = (R)0.5 * (Gm - Gp);
    B[0] = 0;
    const R sh = s - (R)0.5;
    const R flh = floor(sh);
    const int j = (int)flh;
    const R fh = sh - flh;
    const R h0 = (j >= 0 && j < n) ? ex[j] : (R)0, h1 = (j + 1 >= 0 && j + 1 < n) ? ex[j + 1] : (R)0;
    E[0] = ((R)1 - fh) * h0 + fh * h1;
}

template <typename R, int G>
__device__ __forceinline__ void fields(const RunDevT<R>& r, R x, R x_lo, R y, R nf, R E[3], R B[3]) {
    const StepC<R>& c = r.c;
    E[0] = E[1] = E[2] = 0;
    B[0] = B[1] = B[2] = 0;
    if (G == FK_PIC) {
        pic_gather<R>(r, x + x_lo, E, B);
        return;
    }
    if (G == FK_CONST) {
        for (int k = 0; k < 3; ++k) { E[k] = c.E_const[k]; B[k] = c.B_const[k]; }
        return;
    }
    if (G == FK_REFL_LP || G == FK_REFL_CP) {
        // incident pulse (B = x^ cross E) plus the mirror image -r e(psi) moving
        // along -x (B = -x^ cross E)
        constexpr bool kCP = G == FK_REFL_CP;
        R ey, ez, fy, fz;
        plane_e<R, kCP>(c, phase(c, nf, x, x_lo), ey, ez);
        plane_e<R, kCP>(c, phase_refl(c, nf, x, x_lo), fy, fz);
        const R ry = -c.refl_r * fy, rz = -c.refl_r * fz;
        E[1] = ey + ry;
        E[2] = ez + rz;
        B[1] = rz - ez;
        B[2] = ey - ry;
        return;
    }
    R phi = phase(c, nf, x, x_lo);
    R g, dg;
    if constexpr (sizeof(R) == 4) {
        envelope_sel(c, phi, g, dg);      // no early exit either: zero fields fall out of g = dg = 0
    } else {
        envelope<R>(c, phi, g, dg);
        if (g == (R)0 && dg == (R)0) return;
    }
    const R a0 = c.a0;
    R S = 1, theta = phi, inv_R = 0, inv_w2 = 0;
    if (G == FK_GAUSS_LP || G == FK_GAUSS_CP) {
        // paraxial 2D focus: amplitude sqrt(w0/w) exp(-y^2/w^2), curvature and Gouy phase
        const R w0 = c.w0, zr = c.zr;
        R xi = x - c.xf;
        R w2 = w0 * w0 * ((R)1 + xi * xi / (zr * zr));
        inv_w2 = (R)1 / w2;
        inv_R = xi / (xi * xi + zr * zr);
        S = m_sqrt(w0 / m_sqrt(w2)) * m_exp(-y * y * inv_w2);
        theta = phi - (R)0.5 * y * y * inv_R + (R)0.5 * m_atan(xi / zr);
    }
    R st, ct;
    m_sincos(theta, &st, &ct);
    R ey = -a0 * S * (dg * st + g * ct);
    E[1] = ey;
    B[2] = ey;
    if (G == FK_GAUSS_LP || G == FK_GAUSS_CP) E[0] = a0 * g * S * (y * inv_R * ct + (R)2 * y * inv_w2 * st);
    if (G == FK_PLANE_CP || G == FK_GAUSS_CP) {
        R ez = a0 * S * (dg * ct - g * st);
        E[2] = ez;
        B[1] = -ez;
        if (G == FK_GAUSS_CP) B[0] = a0 * g * S * ((R)2 * y * inv_w2 * ct - y * inv_R * st);
    }
}

// ---- Boris push, charge -e (particle pusher, Sec. 2.2) -------------------------
template <typename R>
__device__ __forceinline__ void boris(R u[3], const R E[3], const R B[3], R dt) {
    const R h = (R)0.5 * dt;
    R um0 = u[0] - h * E[0], um1 = u[1] - h * E[1], um2 = u[2] - h * E[2];
    R ig;                                           // 1/gamma at the half step
    if constexpr (sizeof(R) == 4) ig = rsqrtf(1.0f + um0 * um0 + um1 * um1 + um2 * um2);
    else ig = (R)1 / m_sqrt((R)1 + um0 * um0 + um1 * um1 + um2 * um2);
    R t0 = -h * B[0] * ig, t1 = -h * B[1] * ig, t2 = -h * B[2] * ig;
    R f = (R)2 / ((R)1 + t0 * t0 + t1 * t1 + t2 * t2);
    R s0 = f * t0, s1 = f * t1, s2 = f * t2;
    R p0 = um0 + (um1 * t2 - um2 * t1);
    R p1 = um1 + (um2 * t0 - um0 * t2);
    R p2 = um2 + (um0 * t1 - um1 * t0);
    u[0] = um0 + (p1 * s2 - p2 * s1) - h * E[0];
    u[1] = um1 + (p2 * s0 - p0 * s2) - h * E[1];
    u[2] = um2 + (p0 * s1 - p1 * s0) - h * E[2];
}

// ---- quantum parameter (Sec. 2.1) ------------------------------------------------
// eta E_S = sqrt((gamma E + u x B)^2 - (u.E)^2), rewritten without the
// cancellation of electrons riding a wave along x: with dB = B - x^ cross E
// and V = (gamma - u_x) E + u x dB, the radicand is |V|^2 + 2 V_x (u.E).
// For the plane wave (B = x^ cross E, E_x = 0) dB and V_x vanish and the radicand is
// exactly (gamma - u_x)^2 |E|^2.
template <typename R, int G>
__device__ __forceinline__ R eta_of(const R u[3], R gamma, const R E[3], const R B[3], R inv_ES) {
    R gm = (u[0] > (R)0) ? ((R)1 + u[1] * u[1] + u[2] * u[2]) / (gamma + u[0]) : gamma - u[0];
    if (G == FK_PLANE_LP) return gm * fabs(E[1]) * inv_ES;
    if (G == FK_PLANE_CP) return gm * m_sqrt(E[1] * E[1] + E[2] * E[2]) * inv_ES;
    R d0 = B[0], d1 = B[1] + E[2], d2 = B[2] - E[1];
    R V0 = gm * E[0] + (u[1] * d2 - u[2] * d1);
    R V1 = gm * E[1] + (u[2] * d0 - u[0] * d2);
    R V2 = gm * E[2] + (u[0] * d1 - u[1] * d0);
    R uE = u[0] * E[0] + u[1] * E[1] + u[2] * E[2];
    R q = V0 * V0 + V1 * V1 + V2 * V2 + (R)2 * V0 * uE;
    return q > (R)0 ? m_sqrt(q) * inv_ES : (R)0;
}

// ---- table lookups (rows linear in log eta / log gamma) -----------------------
// Row of a position 0 <= tp < 2^22 without int/float conversion instructions: the
// nearest integer to tp - 1/2 is read off the mantissa after adding 1.5 * 2^23 (where
// floats are spaced by 1).  This is floor(tp), or floor(tp) - 1 with weight 1 when tp
// is an exact integer; both give the same interpolated value.
__device__ __forceinline__ void split_pos(float tp, int& i, float& w) {
    float t = (tp - 0.5f) + 0x1.8p23f;
    i = __float_as_int(t) - 0x4B400000;
    w = tp - (t - 0x1.8p23f);
}
__device__ __forceinline__ void split_pos(double tp, int& i, double& w) {
    double f = floor(tp);
    i = (int)f;
    w = tp - f;
}

template <typename R>
__device__ __forceinline__ void row_pos(R v, R lnlo, R inv, R last, int n, int& i, R& w, int& flag) {
    R tp = (m_log(v) - lnlo) * inv;
    flag = 0;
    if (tp >= last) { i = n - 2; w = 1; flag = 1; return; }
    if (!(tp >= (R)0)) { i = 0; w = 0; flag = -1; return; }
    split_pos(tp, i, w);
}

// h(eta) by row interpolation; below the table: classical limit 5 pi / 3
template <typename R>
__device__ __forceinline__ R h_of_eta(const TablesDev& t, const R* h, R eta, int& flag) {
    const TabC<R>& c = tabc<R>(t);
    if constexpr (sizeof(R) == 4) {
        // clamps and selects instead of branches; flag = 1 above the table.  The row position
        // comes from log2 by one FMA and is clamped just below the top node, so the split
        // needs no correction there (above the table: the last row).
        const float tp = fmaf(__log2f(eta), c.inv_dln_eta * 0.693147180559945309f, -c.ln_eta_min * c.inv_dln_eta);
        flag = tp >= c.eta_last ? 1 : 0;
        const float tpc = fminf(fmaxf(tp, 0.0f), c.eta_last - 0x1.0p-10f);
        int i;
        float w;
        split_pos(tpc, i, w);
        i = dbg_idx(t.dbg, i, t.n_eta - 1);
        const float v = fmaf(w, h[i + 1] - h[i], h[i]);
        return (eta >= c.eta_min) ? v : c.h_classical;
    } else {
        if (!(eta >= c.eta_min)) { flag = -1; return c.h_classical; }
        int i; R w;
        row_pos<R>(eta, c.ln_eta_min, c.inv_dln_eta, c.eta_last, t.n_eta, i, w, flag);
        i = dbg_idx(t.dbg, i, t.n_eta - 1);
        return ((R)1 - w) * h[i] + w * h[i + 1];
    }
}

// inverse of the row-interpolated CDF: largest j with c_j <= R, linear between nodes
template <typename R>
__device__ __forceinline__ R invert_rows(const R* ra, const R* rb, R w, int n, R Rv, int& j_out) {
    R c0 = ((R)1 - w) * ra[0] + w * rb[0];
    if (Rv < c0) { j_out = -1; return Rv / c0; }
    R cn = ((R)1 - w) * ra[n - 1] + w * rb[n - 1];
    if (Rv >= cn) { j_out = n - 1; return (R)0; }
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        R cm = ((R)1 - w) * ra[mid] + w * rb[mid];
        if (cm <= Rv) lo = mid; else hi = mid;
    }
    R cl = ((R)1 - w) * ra[lo] + w * rb[lo];
    R ch = ((R)1 - w) * ra[hi] + w * rb[hi];
    j_out = lo;
    return ch > cl ? (Rv - cl) / (ch - cl) : (R)0;
}

// NCS photon energy fraction delta for given eta and uniform Rv (Sec. 2.2)
template <typename R>
__device__ __forceinline__ R sample_ncs_delta(const TablesDev& t, const R* cdf, R eta, R Rv, bool& below) {
    const TabC<R>& c = tabc<R>(t);
    const R *ra, *rb;
    R w;
    below = false;
    if (!(eta >= c.eta_min)) {
        ra = rb = cdf + (size_t)t.n_eta * t.n_y;
        w = 0;
        below = true;
    } else {
        int i, fl;
        row_pos<R>(eta, c.ln_eta_min, c.inv_dln_eta, c.eta_last, t.n_eta, i, w, fl);
        i = dbg_idx(t.dbg, i, t.n_eta - 1);
        ra = cdf + (size_t)i * t.n_y;
        rb = ra + t.n_y;
    }
    int j;
    R fr = invert_rows<R>(ra, rb, w, t.n_y, Rv, j);
    R y;
    if (j < 0) y = c.y_min * fr * fr * fr;            // CDF ~ y^(1/3) below the grid
    else if (j >= t.n_y - 1) y = c.y_max;
    else y = m_exp(c.ln_y_min + ((R)j + fr) * c.dln_y);
    R q = (R)3 * eta * y;
    return q / ((R)2 + q);
}

// sigma_Z(gamma) by row interpolation in log gamma
template <typename R>
__device__ __forceinline__ R sigma_of(const TablesDev& t, const R* sig, R gamma, bool& above) {
    const TabC<R>& c = tabc<R>(t);
    int i, fl; R w;
    row_pos<R>(gamma, c.ln_g_min, c.inv_dln_g, c.g_last, t.n_E, i, w, fl);
    i = dbg_idx(t.dbg, i, t.n_E - 1);
    above = (fl == 1);
    return ((R)1 - w) * sig[i] + w * sig[i + 1];
}

// brems photon energy fraction y from sigma(y, E) = sigma(E) R2 (text after Eq. 4)
template <typename R>
__device__ __forceinline__ R sample_brems_y(const TablesDev& t, const R* bcdf_z, R gamma, R Rv) {
    const TabC<R>& c = tabc<R>(t);
    int i, fl; R w;
    row_pos<R>(gamma, c.ln_g_min, c.inv_dln_g, c.g_last, t.n_E, i, w, fl);
    i = dbg_idx(t.dbg, i, t.n_E - 1);
    const R* ra = bcdf_z + (size_t)i * t.n_s;
    const R* rb = ra + t.n_s;
    int j;
    R fr = invert_rows<R>(ra, rb, w, t.n_s, Rv, j);
    R s;
    if (j < 0) s = 0;
    else if (j >= t.n_s - 1) s = 1;
    else s = ((R)j + fr) / (R)(t.n_s - 1);
    R ycut = c.photon_min / gamma, ymax = (R)1 - (R)1 / gamma;
    return ycut * m_exp(s * m_log(ymax / ycut));
}

// energy-conserving recoil along u (photon direction k = v/|v|, Sec. 2.2)
template <typename R>
__device__ __forceinline__ void recoil(R u[3], R gamma, R w, R k[3]) {
    R um = m_sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (um > (R)0) { R iu = (R)1 / um; k[0] = u[0] * iu; k[1] = u[1] * iu; k[2] = u[2] * iu; }
    else { k[0] = 1; k[1] = 0; k[2] = 0; }
    R g2 = gamma - w;
    R un = g2 > (R)1 ? m_sqrt(g2 * g2 - (R)1) : (R)0;
    u[0] = k[0] * un; u[1] = k[1] * un; u[2] = k[2] * un;
}

}  // namespace pe
