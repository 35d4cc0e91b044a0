// kernels_bw.cu -- Breit-Wheeler conversion of photon records in the run's prescribed fields.
//
// Sec. 1 names pair production by a photon in the laser field; its rate is taken, like the
// NCS module's (Sec. 2.2), as that of a locally constant crossed field: a photon of energy k
// (m c^2) with quantum parameter chi makes pairs at W = alpha E_S T(chi) / k per unit time
// (1/omega_L).  Each photon record moves at c along its direction from its emission point;
// at step m (n_e < m < step_end) it is at x_e + k^ (m - n_e) c dt, the run's fields there at
// t = m dt give chi, and an optical depth tau_0 = -ln U falls by W dt per step; at the first
// step with tau <= 0 the photon converts, the positron's share x from the tabulated CDF.
//
// One thread per photon, with the step loop flattened: every pass of the loop takes one
// step of each lane's current photon, and a lane whose photon is done (converted, at
// step_end, or out of reach of every pulse for good) takes its next photon, so the lanes of
// a warp stay busy whatever the spread of path lengths.  A pulse is out of reach of a photon
// when it is behind it -- its fields vanish identically once its phase t - x (for the
// reflected wave t + x - 2 x_m) is past the pulse's end, and both phases only grow along a
// photon's path -- or when it can never give chi above the table: a plane wave gives
// chi = (k -+ k_x) |E| / E_S exactly (- for the incident pulse, + for its mirror image) with
// |E| <= r a0 sqrt(1 + k_env^2) (Cauchy-Schwarz on g' sin + g cos), so with a factor 2 of
// margin the bound below chi_min means T = 0 at every step (photons co-moving with the
// incident pulse, for instance).  From then on chi < chi_min, T = 0 and the
// optical depth stays, so the photon stops with its remaining steps counted as taken (the
// tally equals stepping them).
//
// FP64 runs step in double (parity with the oracle: the same pair list).  FP32 runs step in
// float -- positions, fields, chi and T -- with the optical depth as a compensated float
// pair, tau_0 drawn in float-pair arithmetic; the once-per-conversion sampling of x runs in
// double in both.
#include "kernels.cuh"

namespace pe {
namespace {

constexpr uint32_t kPurBWTau = 0x60000000u;   // tau_0: counter (id_mech, run id, n_e, kPurBWTau + n_e)
constexpr uint32_t kPurBWX = 0x70000000u;     // x at conversion step m: (id_mech, run id, m, kPurBWX + n_e)

// T(chi): 0 below the table (flag -1), the last node above (flag 1), else L linear in ln chi
__device__ __forceinline__ double bw_T(const BwDev& b, double chi, int& flag) {
    if (!(chi >= b.chi_min)) { flag = -1; return 0.0; }
    double tp = (log(chi) - b.ln_chi_min) * b.inv_dln_chi;
    if (tp >= (double)(b.n_chi - 1)) { flag = 1; return b.T_last; }
    flag = 0;
    if (tp < 0.0) tp = 0.0;
    int i = (int)floor(tp);
    if (i > b.n_chi - 2) i = b.n_chi - 2;
    const double w = tp - (double)i;
    i = dbg_idx(b.dbg, i, b.n_chi - 1);
    return exp((1.0 - w) * b.L64[i] + w * b.L64[i + 1] - 8.0 / (3.0 * chi));
}
__device__ __forceinline__ float bw_T(const BwDev& b, float chi, int& flag) {
    if (!(chi >= b.fchi_min)) { flag = -1; return 0.0f; }
    const float tp = (__logf(chi) - b.fln_chi_min) * b.finv_dln_chi;
    if (tp >= b.f_last) { flag = 1; return b.fT_last; }
    flag = 0;
    // row by the magic-number split (no int/float conversion: GB300 runs those on its FP64 pipe)
    int i;
    float w;
    split_pos(fmaxf(tp, 0.0f), i, w);
    i = dbg_idx(b.dbg, i, b.n_chi - 1);
    // T below ~1e-38 (chi below ~0.03) underflows to 0: a rate 1e-36 times the unit
    return __expf((1.0f - w) * b.L32[i] + w * b.L32[i + 1] - 8.0f / (3.0f * chi));
}

// positron share x at uniform R: the CDF rows interpolated in ln chi (chi clamped to the
// table), inverted linearly in s between the nodes, x = (1 - cos(pi s)) / 2
__device__ __forceinline__ double bw_sample_x(const BwDev& b, double chi, double R) {
    if (!(chi >= b.chi_min)) chi = b.chi_min;
    const double tp = (log(chi) - b.ln_chi_min) * b.inv_dln_chi;
    int i;
    double w;
    if (tp >= (double)(b.n_chi - 1)) { i = b.n_chi - 2; w = 1.0; }
    else if (!(tp >= 0.0)) { i = 0; w = 0.0; }
    else { i = min((int)floor(tp), b.n_chi - 2); w = tp - (double)i; }
    i = dbg_idx(b.dbg, i, b.n_chi - 1);
    const double* ra = b.cdf64 + (size_t)i * b.n_x;
    int j;
    const double fr = invert_rows<double>(ra, ra + b.n_x, w, b.n_x, R, j);
    double s;
    if (j < 0) s = 0.0;
    else if (j >= b.n_x - 1) s = 1.0;
    else s = ((double)j + fr) / (double)(b.n_x - 1);
    return 0.5 * (1.0 - cos(kPi * s));
}

// the photon's chi: the electron's eta with u -> kvec and gamma -> |kvec|, in the same
// cancellation-safe arrangement (|kvec| - k_x = k_perp^2 / (|kvec| + k_x) for k_x > 0);
// kk = |kvec| and gm depend on the photon only
template <typename R>
__device__ __forceinline__ R chi_photon(const R kv[3], R gm, const R E[3], const R B[3], R inv_ES) {
    const R d0 = B[0], d1 = B[1] + E[2], d2 = B[2] - E[1];
    const R V0 = gm * E[0] + (kv[1] * d2 - kv[2] * d1);
    const R V1 = gm * E[1] + (kv[2] * d0 - kv[0] * d2);
    const R V2 = gm * E[2] + (kv[0] * d1 - kv[1] * d0);
    const R kE = kv[0] * E[0] + kv[1] * E[1] + kv[2] * E[2];
    const R q = V0 * V0 + V1 * V1 + V2 * V2 + (R)2 * V0 * kE;
    return q > (R)0 ? m_sqrt(q) * inv_ES : (R)0;
}

// optical depth: double, or a compensated float pair
template <typename R> struct Depth;
template <> struct Depth<double> {
    double v;
    __device__ void set(double t) { v = t; }
    __device__ void sub(double d) { v -= d; }
    __device__ bool crossed() const { return v <= 0.0; }
};
template <> struct Depth<float> {
    float v, lo;
    __device__ void set(double t) { v = (float)t; lo = (float)(t - (double)v); }
    __device__ void set(float t) { v = t; lo = 0.0f; }
    __device__ void sub(float d) {       // TwoSum: v + lo stays exact to ~2^-48
        const float s = v - d, bb = s - v;
        lo += (v - (s - bb)) + (-d - bb);
        v = s;
    }
    __device__ bool crossed() const { return v + lo <= 0.0f; }
};

// position at step m: e + d ((m - n_e) dt) with sf = m - n_e held as a floating-point counter
// (advanced by exact + 1, so no integer-to-float conversion per step: GB300 runs conversions on
// its narrow FP64 pipe); one rounding for the product and one for the FMA
__device__ __forceinline__ double bw_pos(const StepC<double>& c, double d, double e, double sf) {
    return __fma_rn(d, __dmul_rn(sf, c.dt), e);
}
__device__ __forceinline__ float bw_pos(const StepC<float>& c, float d, float e, float sf) {
    return fmaf(d, sf * c.dt, e);
}

#ifndef PE_BW_MIN_CTAS
#define PE_BW_MIN_CTAS 4
#endif

template <typename R, int G>
__global__ void __launch_bounds__(256, PE_BW_MIN_CTAS) k_bw_transport(BwDev bw, RunDevT<R> r, const Photon* ph,
                                                                     int64_t n_ph, int64_t step_end, PairRec* out,
                                                                     int64_t cap, unsigned long long* tally) {
    const StepC<R>& c = r.c;
    const bool two_d = r.geometry == PE_GAUSS_2D;
    constexpr bool kLeave = G != FK_CONST;                 // a prescribed pulse: fields vanish behind it
    constexpr bool kRefl = G == FK_REFL_LP || G == FK_REFL_CP;
    constexpr bool kPlane = G == FK_PLANE_LP || G == FK_PLANE_CP || kRefl;   // chi bounded as for a plane wave
    // 2 E_max / E_S of the incident pulse: twice the bound on chi / (k - k_x)
    const R reach = (R)2 * c.a0 * m_sqrt((R)1 + c.k_env * c.k_env) * c.inv_ES;
    const R chi_min = sizeof(R) == 8 ? (R)bw.chi_min : (R)bw.fchi_min;
    const R L_end = (R)2 * c.phi_r + c.phi_f + (sizeof(R) == 8 ? (R)1e-6 : (R)1e-3);   // pulse end + margin
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    unsigned long long n_followed = 0, n_tests = 0, n_above = 0;
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - stride;
    bool have = false;
    Photon p{};
    R k = 0, kv[3] = {0, 0, 0}, gm = 0, kx = 0, ky = 0, xe = 0, ye = 0, kdt = 0;
    int64_t ne = 0, m = 0;
    R sf = 0, mf = 0;                              // m - n_e and m as exact floating-point counters
    bool inc_never = false, ref_never = true;     // a pulse can never raise chi above the table
    Depth<R> tau;
    tau.set(1.0);
    while (true) {
        if (!have) {
            // this lane's next photon to step: k > 2 m c^2, a step left before step_end, and a pulse
            // that can raise its chi into the table; the others are only counted (no draw)
            while (true) {
                j += stride;
                if (j >= n_ph) break;
                p = ph[j];
                if (!(p.e > 2.0f)) continue;               // the same decision as (double) k > 2
                ++n_followed;
                ne = (int64_t)p.step;
                m = ne + 1;
                k = (R)p.e;
                kx = (R)p.kx; ky = (R)p.ky; xe = (R)p.x; ye = (R)p.y;
                kv[0] = k * kx; kv[1] = k * ky; kv[2] = k * (R)p.kz;
                const R kk = m_sqrt(kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2]);
                gm = (kv[0] > (R)0) ? (kv[1] * kv[1] + kv[2] * kv[2]) / (kk + kv[0]) : kk - kv[0];
                if (kPlane) {
                    // k - k_x is gm (formed without cancellation); k + k_x likewise for backward photons
                    const R gp = (kv[0] < (R)0) ? (kv[1] * kv[1] + kv[2] * kv[2]) / (kk - kv[0]) : kk + kv[0];
                    inc_never = gm * reach < chi_min;
                    ref_never = !kRefl || gp * c.refl_r * reach < chi_min;
                    if (inc_never && ref_never) {        // no pulse can convert it: every step counted, none taken
                        n_tests += (unsigned long long)(step_end > m ? step_end - m : 0);
                        continue;
                    }
                }
                if (m >= step_end) continue;
                const uint4 w = philox4x32_10(make_uint4(p.id_mech, r.run_id, (uint32_t)ne, kPurBWTau + p.step),
                                              r.seed_lo, r.seed_hi);
                kdt = c.bw_coef / k;
                sf = (R)1;
                if constexpr (sizeof(R) == 8) {
                    tau.set(-log(uni53(w64(w.x, w.y))));
                    mf = (R)m;
                } else {
                    // -ln U from the same 53 bits in float-pair arithmetic, and the step as a float
                    // without a conversion instruction (m < 8192): no FP64-pipe work per photon
                    tau.set(tau_draw_f32(w.x, w.y));
                    mf = int_to_float_small((int)m);
                }
                have = true;
                break;
            }
            if (!have) break;                          // no photon left for this lane
        }
        // step m of the lane's photon
        const R px = bw_pos(c, kx, xe, sf);
        const R py = bw_pos(c, ky, ye, sf);
        R E[3], B[3];
        fields<R, G>(r, px, (R)0, py, mf, E, B);
        const R chi = chi_photon<R>(kv, gm, E, B, c.inv_ES);
        int fl;
        const R T = bw_T(bw, chi, fl);
        ++n_tests;
        n_above += fl == 1;
        if constexpr (sizeof(R) == 8) tau.sub(c.bw_coef * T / k);    // (alpha E_S dt) T / k, the oracle's order
        else tau.sub(kdt * T);
        bool conv = false;
        PairRec q;
        if (tau.crossed()) {
            const uint4 w = philox4x32_10(make_uint4(p.id_mech, r.run_id, (uint32_t)m, kPurBWX + p.step),
                                          r.seed_lo, r.seed_hi);
            const double kd = (double)p.e;
            const double x = bw_sample_x(bw, (double)chi, uni53(w64(w.x, w.y)));
            const double ep = x * kd;
            q.x = (float)px;
            q.y = (float)(two_d ? py : (R)0);
            q.e_minus = (float)(kd - ep);
            q.e_plus = (float)ep;
            q.kx = p.kx; q.ky = p.ky; q.kz = p.kz;
            q.step = (uint32_t)m;
            q.photon = (uint32_t)j;
            q.id_mech = p.id_mech;
            fx_add(tally + PE_PT_E_PAIRS, kd);
            fx_add(tally + PE_PT_E_POSITRONS, ep);
            conv = true;
            have = false;
        } else {
            ++m;
            if (m >= step_end) {
                have = false;
            } else if (kLeave) {
                // every pulse behind the photon for good, or never strong enough for it: the
                // remaining steps see chi below the table
                bool gone = inc_never || phase(c, mf, px, (R)0) > L_end;
                if (kRefl) gone = gone && (ref_never || phase_refl(c, mf, px, (R)0) > L_end);
                if (gone) {
                    n_tests += (unsigned long long)(step_end - m);
                    have = false;
                }
            }
            sf += (R)1;
            mf += (R)1;
        }
        // conversions of this pass, one counter atomic per converging group of lanes
        const unsigned act = __activemask();
        const unsigned mask = __ballot_sync(act, conv);
        if (conv) {
            const int leader = __ffs(mask) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(tally + PE_PT_N_PAIRS, (unsigned long long)__popc(mask));
            base = __shfl_sync(mask, base, leader);
            const unsigned long long idx = base + __popc(mask & ((1u << lane) - 1u));
            if (idx < (unsigned long long)cap) out[idx] = q;
        }
    }
    // counters: one warp sum each
    for (int o = 16; o > 0; o >>= 1) {
        n_followed += __shfl_xor_sync(0xffffffffu, n_followed, o);
        n_tests += __shfl_xor_sync(0xffffffffu, n_tests, o);
        n_above += __shfl_xor_sync(0xffffffffu, n_above, o);
    }
    if (lane == 0) {
        if (n_followed) atomicAdd(tally + PE_PT_N_ENTERED, n_followed);
        if (n_tests) atomicAdd(tally + PE_PT_N_TESTS, n_tests);
        if (n_above) atomicAdd(tally + PE_PT_N_K_ABOVE, n_above);
    }
}

template <typename R, int G>
void launch_kind(const BwDev& b, const RunDevT<R>& r, const void* photons, int64_t n, int64_t step_end, void* pairs,
                 int64_t cap, unsigned long long* tally, cudaStream_t s) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bw_transport<R, G>, 256, 0) != cudaSuccess || occ < 1)
        occ = 1;
    const int64_t blocks = (n + 255) / 256;
    const int grid = (int)(blocks < (int64_t)sms * occ ? (blocks > 0 ? blocks : 1) : (int64_t)sms * occ);
    k_bw_transport<R, G><<<grid, 256, 0, s>>>(b, r, static_cast<const Photon*>(photons), n, step_end,
                                              static_cast<PairRec*>(pairs), cap, tally);
}

}  // namespace

void launch_bw_transport(const BwDev& b, const RunDev& r, int precision, const void* photons, int64_t n_photons,
                         int64_t step_end, void* pairs, int64_t capacity, unsigned long long* tally, cudaStream_t s) {
    with_field_kind(r.fk, [&](auto g) {
        constexpr int G = decltype(g)::value;
        if (precision == PE_F32)
            launch_kind<float, G>(b, to_float(r), photons, n_photons, step_end, pairs, capacity, tally, s);
        else
            launch_kind<double, G>(b, r, photons, n_photons, step_end, pairs, capacity, tally, s);
    });
}

}  // namespace pe
