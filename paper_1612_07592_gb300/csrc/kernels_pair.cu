// kernels_pair.cu -- Bethe-Heitler conversion of photon records in the target.
//
// Sec. 2.2 implements pair production by photons in the field of the nuclei like the
// bremsstrahlung: a direct MC collision of Eq. (4), here with the pair cross section
// sigma_BH(k) of the photon energy k.  A photon moves at c along its direction from its
// emission point; at every step inside the target it takes the test, and on a conversion
// the positron fraction x is drawn from the tabulated CDF of Tsai's pair DCS.
//
// Two methods of the same law: the per-step tests of Eq. 4 (the paper's direct collision),
// and the free path (the trials of one crossing share P, so the first success is geometric:
// one draw per photon, the random-free-path sampling Sec. 2.2 mentions).
//
// Rounds of 32 photons per warp.  Each lane first finds its photon's run of consecutive
// steps inside the target by binary search on the FP64 position computed exactly as the
// definition computes it at each step (GB300's FP64 pipe is narrow: the literal per-step
// position kept it 84 % busy).  Then the warp takes the tests of the round's photons one
// photon at a time, 32 steps at once (the draws are counter-based, so the first passing
// step is found from a ballot): the per-step work is a Philox draw and a 64-bit integer
// compare on every lane, whatever the spread of path lengths.  Conversions are appended
// per warp (one atomic per warp and round).
#include "kernels.cuh"

namespace pe {
namespace {

constexpr uint32_t kPurBH = 0x40000000u;      // per-step tests: counter word 3 = kPurBH + emission step
constexpr uint32_t kPurBHFree = 0x50000000u;  // free path: counter word 3 = kPurBHFree + emission step


// sigma_BH(k) by row interpolation in log k over [2, gamma_max] (0 for k <= 2); the row
// position (i, w) is kept for the sampling of x
__device__ __forceinline__ double bh_sigma_of(const TablesDev& t, const double* sig, double k, bool& above, int& i,
                                              double& w) {
    const TabC<double>& c = t.cd;
    above = false;
    if (!(k > 2.0)) return 0.0;
    int fl;
    row_pos<double>(k, c.ln_k_min, c.inv_dln_k, c.g_last, t.n_E, i, w, fl);
    i = dbg_idx(t.dbg, i, t.n_E - 1);
    above = (fl == 1);
    return (1.0 - w) * sig[i] + w * sig[i + 1];
}

// positron fraction x in [1/k, 1 - 1/k] from the CDF interpolated at row position (i, w) of k,
// at uniform Rv (2/k is formed as 2 (1/k), the same double)
__device__ __forceinline__ double bh_sample_x(const TablesDev& t, const double* cdf_z, double k, int i, double w,
                                              double Rv) {
    const double* ra = cdf_z + (size_t)i * t.n_s;
    const double* rb = ra + t.n_s;
    int j;
    const double fr = invert_rows<double>(ra, rb, w, t.n_s, Rv, j);
    double s;
    if (j < 0) s = 0.0;
    else if (j >= t.n_s - 1) s = 1.0;
    else s = ((double)j + fr) / (double)(t.n_s - 1);
    const double ik = 1.0 / k;
    return ik + s * (1.0 - 2.0 * ik);
}


#ifndef PE_PAIR_MIN_CTAS_SM
#define PE_PAIR_MIN_CTAS_SM 3      // resident CTAs of 256 threads per SM the registers are sized for
#endif

// kFree: the free-path method (one geometric draw per photon) instead of the per-step tests
template <bool kFree>
__global__ void __launch_bounds__(256, PE_PAIR_MIN_CTAS_SM) k_pair_transport(TablesDev t, RunDev r, const Photon* ph,
                                                                           int64_t n_ph, int64_t step_end,
                                                                           PairRec* out, int64_t cap,
                                                                           unsigned long long* tally) {
    __shared__ unsigned long long s_t[PE_PAIR_TALLY_WORDS];
    if (threadIdx.x < PE_PAIR_TALLY_WORDS) s_t[threadIdx.x] = 0;
    __syncthreads();
    const StepC<double>& c = r.c;
    const double* sig = t.bhsig64 + (size_t)r.iz * t.n_E;
    const double* cdf = t.bhcdf64 + (size_t)r.iz * t.n_E * t.n_s;
    const bool two_d = r.geometry == PE_GAUSS_2D;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform rounds of 32 photons, so that every lane reaches the shuffles and the append
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_ph; base += stride) {
        const int64_t j = base + lane;
        bool conv = false;
        unsigned long long tests = 0;
        PairRec q;
        // lane's photon: the run [a, b] of steps inside the target and the threshold of the test
        Photon p{};
        int64_t a = 1, b = 0;
        uint64_t thr = 0;
        double k = 0.0, lam = 0.0, wk = 0.0;       // lam = n_i sigma_BH c dt = -ln(1 - P)
        int ik = 0;
        if (j < n_ph) {
            p = ph[j];
            k = (double)p.e;
            if (k > 2.0) {
                const double kx = p.kx, ky = p.ky, xe = p.x, ye = p.y;
                const int64_t ne = p.step;
                bool above;
                lam = c.K_br * bh_sigma_of(t, sig, k, above, ik, wk);
                if constexpr (!kFree) {
                    const double P = -expm1(-lam);
                    thr = P >= 1.0 ? 0xFFFFFFFFFFFFFFFFull : __double2ull_rz(P * 0x1.0p64);
                }
                // The steps with the photon inside the target form one run [a, b] (its position
                // is monotone in the step and the target convex): bound it with each face by
                // binary search on the position exactly as the step computes it, so the tests
                // run on integers only.
                a = ne + 1;
                b = step_end - 1;
                auto clip = [&](double d, double e, double lo, double hi) {
                    if (a > b) return;
                    if (d == 0.0) {
                        const double v = photon_pos(c, d, e, ne, a);
                        if (!(v >= lo && v <= hi)) b = a - 1;
                        return;
                    }
                    // the entry face is reached (d > 0: pos >= lo; d < 0: pos <= hi) ...
                    auto entered = [&](int64_t m) {
                        const double v = photon_pos(c, d, e, ne, m);
                        return d > 0.0 ? v >= lo : v <= hi;
                    };
                    // ... and the exit face not yet passed
                    auto before_exit = [&](int64_t m) {
                        const double v = photon_pos(c, d, e, ne, m);
                        return d > 0.0 ? v <= hi : v >= lo;
                    };
                    if (!entered(b)) { b = a - 1; return; }
                    if (!entered(a)) {
                        int64_t u = a, v = b;              // entered(u) false, entered(v) true
                        while (v - u > 1) {
                            const int64_t mid = u + (v - u) / 2;
                            if (entered(mid)) v = mid; else u = mid;
                        }
                        a = v;
                    }
                    if (!before_exit(a)) { b = a - 1; return; }
                    if (!before_exit(b)) {
                        int64_t u = a, v = b;              // before_exit(u) true, before_exit(v) false
                        while (v - u > 1) {
                            const int64_t mid = u + (v - u) / 2;
                            if (before_exit(mid)) u = mid; else v = mid;
                        }
                        b = u;
                    }
                };
                clip(kx, xe, c.x0, c.x1);
                if (two_d) clip(ky, ye, -c.yh, c.yh);
                if (a <= b) {
                    atomicAdd(&s_t[PE_PT_N_ENTERED], 1ull);
                    if (above) atomicAdd(&s_t[PE_PT_N_K_ABOVE], 1ull);
                }
            }
        }
        // the lane's pair record for a conversion at step `hit` with the fraction word (wz, ww)
        auto record = [&](int64_t hit, uint32_t wz, uint32_t ww) {
            const double x = bh_sample_x(t, cdf, k, ik, wk, uni53(w64(wz, ww)));
            const double ep = x * k;
            q.x = (float)photon_pos(c, p.kx, p.x, p.step, hit);
            q.y = (float)(two_d ? photon_pos(c, p.ky, p.y, p.step, hit) : 0.0);
            q.e_minus = (float)(k - ep);
            q.e_plus = (float)ep;
            q.kx = p.kx; q.ky = p.ky; q.kz = p.kz;
            q.step = (uint32_t)hit;
            q.photon = (uint32_t)j;
            q.id_mech = p.id_mech;
            fx_add(&s_t[PE_PT_E_PAIRS], k);
            fx_add(&s_t[PE_PT_E_POSITRONS], ep);
            conv = true;
        };
        if constexpr (kFree) {
            // the trials of the crossing all have probability P = 1 - exp(-lam): the number of
            // failures before the first success is geometric, floor(-ln U / lam); one draw per photon
            if (a <= b && lam > 0.0) {
                const uint4 w = philox4x32_10(make_uint4(p.id_mech, r.run_id, (uint32_t)a, kPurBHFree + p.step),
                                              r.seed_lo, r.seed_hi);
                tests = 1;
                const double jf = floor(-log(uni53(w64(w.x, w.y))) / lam);
                if (jf <= (double)(b - a)) record(a + (int64_t)jf, w.z, w.w);
            }
        }
        // The warp takes the tests of each photon of the round in turn, 32 steps at a time
        // (lane l tests step m0 + l); the conversion is at the first step whose draw passes.
        for (int src = 0; src < 32 && !kFree; ++src) {
            const int64_t as = __shfl_sync(0xffffffffu, a, src), bs = __shfl_sync(0xffffffffu, b, src);
            if (as > bs) continue;
            const uint32_t idm = __shfl_sync(0xffffffffu, p.id_mech, src);
            const uint32_t ne = __shfl_sync(0xffffffffu, p.step, src);
            const uint64_t th = __shfl_sync(0xffffffffu, thr, src);
            int64_t hit = -1;
            uint32_t hz = 0, hw = 0;
            for (int64_t m0 = as; m0 <= bs; m0 += 32) {
                const int64_t m = m0 + lane;
                bool ok = false;
                uint4 w = make_uint4(0, 0, 0, 0);
                if (m <= bs) {
                    w = philox4x32_10(make_uint4(idm, r.run_id, (uint32_t)m, kPurBH + ne), r.seed_lo, r.seed_hi);
                    ok = w64(w.x, w.y) < th;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, ok);
                if (bal) {
                    const int first = __ffs(bal) - 1;
                    hit = m0 + first;
                    hz = __shfl_sync(0xffffffffu, w.z, first);
                    hw = __shfl_sync(0xffffffffu, w.w, first);
                    break;
                }
            }
            if (lane == src) {
                tests += (unsigned long long)((hit >= 0 ? hit : bs) - as + 1);
                if (hit >= 0) record(hit, hz, hw);
            }
        }
        // tests of the warp's round, one shared atomic per warp
        for (int o = 16; o > 0; o >>= 1) tests += __shfl_xor_sync(0xffffffffu, tests, o);
        if (lane == 0 && tests) atomicAdd(&s_t[PE_PT_N_TESTS], tests);
        const unsigned mask = __ballot_sync(0xffffffffu, conv);
        if (mask) {
            const int leader = __ffs(mask) - 1;
            unsigned long long b = 0;
            if (lane == leader) b = atomicAdd(tally + PE_PT_N_PAIRS, (unsigned long long)__popc(mask));
            b = __shfl_sync(0xffffffffu, b, leader);
            if (conv) {
                const unsigned long long idx = b + __popc(mask & ((1u << lane) - 1u));
                if (idx < (unsigned long long)cap) out[idx] = q;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_t[PE_PT_N_ENTERED]) atomicAdd(tally + PE_PT_N_ENTERED, s_t[PE_PT_N_ENTERED]);
        if (s_t[PE_PT_N_K_ABOVE]) atomicAdd(tally + PE_PT_N_K_ABOVE, s_t[PE_PT_N_K_ABOVE]);
        if (s_t[PE_PT_N_TESTS]) atomicAdd(tally + PE_PT_N_TESTS, s_t[PE_PT_N_TESTS]);
        for (int k = PE_PT_E_PAIRS; k <= PE_PT_E_POSITRONS; k += 2) {
            unsigned long long lo = s_t[k], hi = s_t[k + 1];
            if (lo || hi) {
                const unsigned long long old = atomicAdd(tally + k, lo);
                if (old + lo < old) hi += 1;
                if (hi) atomicAdd(tally + k + 1, hi);
            }
        }
    }
}

}  // namespace

void launch_pair_transport(const TablesDev& t, const RunDev& r, const void* photons, int64_t n_photons,
                           int64_t step_end, void* pairs, int64_t capacity, unsigned long long* tally, int method,
                           cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t blocks = (n_photons + 255) / 256;
    const int grid = (int)(blocks < (int64_t)sms * 8 ? (blocks > 0 ? blocks : 1) : (int64_t)sms * 8);
    if (method == PE_PAIR_FREE_PATH)
        k_pair_transport<true><<<grid, 256, 0, s>>>(t, r, static_cast<const Photon*>(photons), n_photons, step_end,
                                                    static_cast<PairRec*>(pairs), capacity, tally);
    else
        k_pair_transport<false><<<grid, 256, 0, s>>>(t, r, static_cast<const Photon*>(photons), n_photons, step_end,
                                                     static_cast<PairRec*>(pairs), capacity, tally);
}

}  // namespace pe
