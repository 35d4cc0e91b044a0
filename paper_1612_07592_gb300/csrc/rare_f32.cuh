// rare_f32.cuh -- the emission branch of the FP32 path without FP64 or int/float
// conversion instructions (both run on GB300's narrow FP64 pipe, where a
// divergent warp pays for them whenever any lane emits).
//
// Precision is kept where it matters for per-particle agreement with the FP64
// reference: the CDF tables are stored as float pairs (hi + lo, ~48 bits), the
// 53-bit uniform is assembled as a float pair from its bits, and the inverse
// CDF compares and interpolates in double-float arithmetic (error-free sums
// and products of floats), so both tails of the photon spectrum are resolved.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "physics.cuh"

namespace pe {

// ---- exact small-integer <-> float without conversion instructions -------------
// 0 <= i < 2^22: the float with value i, built in the mantissa of 1.5 * 2^23
__device__ __forceinline__ float int_to_float_small(int i) {
    return __int_as_float(0x4B400000 + i) - 0x1.8p23f;
}
// 0 <= v < 2^22: floor(v) as an integer, exact (nearest of v - 1/2 read off the
// mantissa of 1.5 * 2^23, then corrected by one when that fell below)
__device__ __forceinline__ uint32_t floor_small(float v) {
    float t = (v - 0.5f) + 0x1.8p23f;
    int i = __float_as_int(t) - 0x4B400000;
    if (int_to_float_small(i + 1) <= v) ++i;
    return (uint32_t)i;
}

// ---- double-float helpers --------------------------------------------------------
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    return DF{s, (a - (s - bb)) + (b - bb)};
}
// uniform in (0, 1) with 53 random bits of (hi:lo) as a float pair: the bits above
// bit 11 plus one half unit, (2^53 - 1 - those bits) plus one half when complemented
__device__ __forceinline__ DF uni53_pair(uint32_t lo, uint32_t hi) {
    uint32_t p1 = hi >> 9;                            // bits 63..41
    uint32_t p2 = ((hi & 0x1FFu) << 14) | (lo >> 18); // bits 40..18
    uint32_t p3 = (lo >> 11) & 0x7Fu;                 // bits 17..11
    float f1 = __int_as_float(0x4B000000 | (int)p1) - 0x1.0p23f;
    float f2 = __int_as_float(0x4B000000 | (int)p2) - 0x1.0p23f;
    float f3 = __int_as_float(0x4B000000 | (int)p3) - 0x1.0p23f + 0.5f;
    return DF{f1 * 0x1.0p-23f, fmaf(f3, 0x1.0p-53f, f2 * 0x1.0p-46f)};
}
// row-interpolated CDF value (1 - w) A + w B of one pair-row entry e = (A_hi, A_lo, B_hi, B_lo)
__device__ __forceinline__ DF pair_value(float4 e, float w) {
    if (w == 0.0f) return DF{e.x, e.y};
    DF d = two_sum(e.z, -e.x);                        // B_hi - A_hi exactly
    float dl = d.lo + (e.w - e.y);
    float p = w * d.hi;
    float ep = fmaf(w, d.hi, -p);                     // exact error of the product
    DF c = two_sum(e.x, p);
    return DF{c.hi, c.lo + (e.y + fmaf(w, dl, ep))};
}
// sign of a - b for float pairs
__device__ __forceinline__ float df_diff(DF a, DF b) { return (a.hi - b.hi) + (a.lo - b.lo); }

// Inverse of the row-interpolated CDF of pair-row q (n columns, guide g of M entries)
// at the uniform R: the largest j with c_j <= R (j = -1 below the first node, n - 1 at or
// above the last) and the fraction (R - c_j) / (c_{j+1} - c_j), or R / c_0 below the
// first node.  The guide brackets j to a few columns, so the binary search that follows
// takes one or two probes instead of log2(n) (a wider search window loaded at once
// measured slower: its registers crowd the step loop).
__device__ __forceinline__ float invert_pair_df(const float4* q, const short4* g, float w, int n, int M, float fM,
                                                DF R, int& j_out, unsigned long long* dbg) {
    // m with m / M <= R < (m + 1) / M (R.hi M is exact, M a power of two)
    float rm = R.hi * fM;
    int m = (int)floor_small(rm);
    if (R.lo < 0.0f && int_to_float_small(m) == rm) --m;
    m = m < M - 1 ? m : M - 1;
    m = dbg_idx(dbg, m, M);
    const float4 e0 = __ldg(q), en = __ldg(q + n - 1);
    const short4 gg = __ldg(g + m);
    DF c0 = pair_value(e0, w);
    if (df_diff(R, c0) < 0.0f) { j_out = -1; return (R.hi + R.lo) / (c0.hi + c0.lo); }
    DF cn = pair_value(en, w);
    if (df_diff(R, cn) >= 0.0f) { j_out = n - 1; return 0.0f; }
    // bracket from the two rows' inverses, widened by one column for rounding
    int a = min((int)gg.x, (int)gg.y) - 1, b = max((int)gg.z, (int)gg.w) + 1;
    a = a > 0 ? a : 0;
    b = b < n - 2 ? b : n - 2;
    int lo = a, hi = b + 1;                           // c_lo <= R < c_hi
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (df_diff(R, pair_value(__ldg(q + mid), w)) >= 0.0f) lo = mid; else hi = mid;
    }
    const int j = lo;
    const DF cl = pair_value(__ldg(q + lo), w), ch = pair_value(__ldg(q + hi), w);
    j_out = j;
    float num = df_diff(R, cl), den = df_diff(ch, cl);
    return den > 0.0f ? num / den : 0.0f;
}

// NCS photon energy fraction (Sec. 2.2) from the pair tables
__device__ __forceinline__ float sample_ncs_delta_f32(const TablesDev& t, float eta, uint32_t wlo, uint32_t whi,
                                                      bool& below) {
    const TabC<float>& c = t.cf;
    float w;
    int pr;
    below = false;
    if (!(eta >= c.eta_min)) {
        pr = t.n_eta - 1;                              // (classical, classical)
        w = 0.0f;
        below = true;
    } else {
        int fl;
        row_pos<float>(eta, c.ln_eta_min, c.inv_dln_eta, c.eta_last, t.n_eta, pr, w, fl);
    }
    pr = dbg_idx(t.dbg, pr, t.n_eta);
    int j;
    float fr = invert_pair_df(t.cdfq + (size_t)pr * t.n_y, t.gq + (size_t)pr * t.M_y, w, t.n_y, t.M_y, t.fM_y,
                              uni53_pair(wlo, whi), j, t.dbg);
    float y;
    if (j < 0) y = c.y_min * fr * fr * fr;           // CDF ~ y^(1/3) below the grid
    else if (j >= t.n_y - 1) y = c.y_max;
    else y = __expf(c.ln_y_min + (int_to_float_small(j) + fr) * c.dln_y);
    float q = 3.0f * eta * y;
    return q / (2.0f + q);
}

// brems photon energy fraction y from sigma(y, E) = sigma(E) R2 (text after Eq. 4)
__device__ __forceinline__ float sample_brems_y_f32(const TablesDev& t, int iz, float gamma, uint32_t wlo,
                                                    uint32_t whi) {
    const TabC<float>& c = t.cf;
    int i, fl;
    float w;
    row_pos<float>(gamma, c.ln_g_min, c.inv_dln_g, c.g_last, t.n_E, i, w, fl);
    i = dbg_idx(t.dbg, i, t.n_E - 1);
    const size_t pr = (size_t)dbg_idx(t.dbg, iz, t.n_Z) * (t.n_E - 1) + i;
    int j;
    float fr = invert_pair_df(t.bcdfq + pr * t.n_s, t.bgq + pr * t.M_s, w, t.n_s, t.M_s, t.fM_s,
                              uni53_pair(wlo, whi), j, t.dbg);
    float s;
    if (j < 0) s = 0.0f;
    else if (j >= t.n_s - 1) s = 1.0f;
    else s = (int_to_float_small(j) + fr) * c.s_step;
    float ycut = c.photon_min / gamma, ymax = 1.0f - 1.0f / gamma;
    return ycut * __expf(s * __logf(ymax / ycut));
}

// new optical depth -ln U from the 53-bit uniform, to first order in the low part of the
// pair: for U >= 1/2 through log1p of the complement (built exactly from the complemented
// bits; the correction lo / (1 - hi) is below 2^-22), else -ln hi - lo / hi.  hi carries
// the top 23 bits of U as a fixed-point number, so below 2^-10 it holds few of U's leading
// bits (none below 2^-23, where it is 0): there the pair is first renormalised (exactly,
// TwoSum), which bounds lo / hi by 2^-24.  Relative error about one ulp of the result.
__device__ __forceinline__ float tau_draw_f32(uint32_t wlo, uint32_t whi) {
    if (whi & 0x80000000u) {
        DF q = uni53_pair(~wlo, ~whi);                  // 1 - U
        return -log1pf(-q.hi) + q.lo / (1.0f - q.hi);
    }
    DF u = uni53_pair(wlo, whi);
    if (u.hi < 0x1.0p-10f) u = two_sum(u.hi, u.lo);
    return -logf(u.hi) - u.lo / u.hi;
}

// 128-bit fixed-point add of a float v >= 0 (m c^2) with integer operations only:
// v 2^64 = m 2^(e - 86) for the 24-bit significand m and biased exponent e
__device__ __forceinline__ void fx_add_f32(unsigned long long* w, float v) {
    if (!(v > 0.0f)) return;
    uint32_t b = __float_as_uint(v);
    int e = (int)(b >> 23);
    unsigned long long m = (b & 0x7FFFFFu) | (e ? 0x800000u : 0u);
    if (e == 0) e = 1;
    int s = e - 86;
    unsigned long long lo, hi;
    if (s >= 64) { lo = 0; hi = m << (s - 64); }
    else if (s > 0) { lo = m << s; hi = (s > 40) ? (m >> (64 - s)) : 0ull; }
    else { lo = (s > -64) ? (m >> (-s)) : 0ull; hi = 0; }
    unsigned long long old = atomicAdd(w, lo);
    if (old + lo < old) hi += 1;
    if (hi) atomicAdd(w + 1, hi);
}

// energy and angle bins of a stored photon (floor by the exact small-integer route)
__device__ __forceinline__ void hist_bins_f32(float e, float kx, float ky, float inv_log_emax, int& eb, int& tb,
                                              bool& over) {
    float fe = (float)PE_HIST_E_BINS * __logf(e) * inv_log_emax;
    over = fe >= (float)PE_HIST_E_BINS;
    eb = over ? PE_HIST_E_BINS - 1 : (fe > 0.0f ? (int)floor_small(fe) : 0);
    float ft = (atan2f(ky, kx) + 3.14159265358979f) * (float)(PE_HIST_T_BINS / (2.0 * 3.14159265358979323846));
    tb = ft > 0.0f ? (int)floor_small(ft) : 0;
    if (tb >= PE_HIST_T_BINS) tb = PE_HIST_T_BINS - 1;
}

// brems test of Eq. (4) for float P: event iff the 64-bit uniform (hi:lo) is below
// floor(P 2^64) = th 2^32 + floor(frac(P 2^32) 2^32); exact integer comparison
__device__ __forceinline__ bool below_threshold_f32(float P, uint32_t lo, uint32_t hi) {
    if (!(P > 0.0f)) return false;
    if (P >= 1.0f) return true;
    float p32 = P * 0x1.0p32f;
    if (p32 >= 0x1.0p22f) return below_threshold(P, lo, hi);   // P >= 2^-10: conversion route
    uint32_t th = floor_small(p32);
    if (hi != th) return hi < th;
    // equal high words (probability 2^-32): compare the low words exactly
    float frac = (p32 - int_to_float_small((int)th)) * 0x1.0p32f;
    uint32_t tl = (uint32_t)frac;
    return lo < tl;
}

}  // namespace pe
