// kernels_pair.cu -- Bethe-Heitler conversion of photon records in the target.
//
// Sec. 2.2 implements pair production by photons in the field of the nuclei like the
// bremsstrahlung: a direct MC collision of Eq. (4), here with the pair cross section
// sigma_BH(k) of the photon energy k.  A photon moves at c along its direction from its
// emission point; at every step inside the target it takes the test, and on a conversion
// the positron fraction x is drawn from the tabulated CDF of Tsai's pair DCS.
//
// One thread per photon (FP64: the arithmetic per step is one position, two compares and
// the Philox draw); the steps before the photon can reach the target are skipped, then
// the steps are taken one by one exactly as the definition states them.  Conversions
// are appended per warp (one atomic per warp and round of photons).
#include "kernels.cuh"

namespace pe {
namespace {

constexpr uint32_t kPurBH = 0x40000000u;   // counter word 3 = kPurBH + emission step

struct PairRec {
    float x, y, e_minus, e_plus, kx, ky, kz;
    uint32_t step, photon, id_mech;
};
static_assert(sizeof(PairRec) == 40, "pe_pair layout");
static_assert(sizeof(Photon) == 32, "photon record layout");

// sigma_BH(k) by row interpolation in log k over [2, gamma_max] (0 for k <= 2)
__device__ __forceinline__ double bh_sigma_of(const TablesDev& t, const double* sig, double k, bool& above) {
    const TabC<double>& c = t.cd;
    above = false;
    if (!(k > 2.0)) return 0.0;
    int i, fl;
    double w;
    row_pos<double>(k, c.ln_k_min, c.inv_dln_k, c.g_last, t.n_E, i, w, fl);
    above = (fl == 1);
    return (1.0 - w) * sig[i] + w * sig[i + 1];
}

// positron fraction x in [1/k, 1 - 1/k] from the row-interpolated CDF at uniform Rv
__device__ __forceinline__ double bh_sample_x(const TablesDev& t, const double* cdf_z, double k, double Rv) {
    const TabC<double>& c = t.cd;
    int i, fl;
    double w;
    row_pos<double>(k, c.ln_k_min, c.inv_dln_k, c.g_last, t.n_E, i, w, fl);
    const double* ra = cdf_z + (size_t)i * t.n_s;
    const double* rb = ra + t.n_s;
    int j;
    const double fr = invert_rows<double>(ra, rb, w, t.n_s, Rv, j);
    double s;
    if (j < 0) s = 0.0;
    else if (j >= t.n_s - 1) s = 1.0;
    else s = ((double)j + fr) / (double)(t.n_s - 1);
    return 1.0 / k + s * (1.0 - 2.0 / k);
}

__global__ void __launch_bounds__(256) k_pair_transport(TablesDev t, RunDev r, const Photon* ph, int64_t n_ph,
                                                        int64_t step_end, PairRec* out, int64_t cap,
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
    // warp-uniform rounds of photons, so that every lane reaches the append
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_ph; base += stride) {
        const int64_t j = base + lane;
        bool conv = false;
        PairRec q;
        if (j < n_ph) {
            const Photon p = ph[j];
            const double k = (double)p.e;
            if (k > 2.0) {
                const double kx = p.kx, ky = p.ky, xe = p.x, ye = p.y;
                const int64_t ne = p.step;
                bool above;
                const double P = -expm1(-c.K_br * bh_sigma_of(t, sig, k, above));
                // skip the steps at which the photon is still at least two steps short of
                // the target along x (no test is taken there)
                int64_t m = ne + 1;
                const double vdt = kx * c.dt;
                const double margin = 1e-9 * (fabs(c.x0) + fabs(c.x1) + 1.0);
                double q_skip = 0.0;
                if (vdt > margin && xe < c.x0) q_skip = floor((c.x0 - xe) / vdt);
                else if (vdt < -margin && xe > c.x1) q_skip = floor((c.x1 - xe) / vdt);
                q_skip = fmin(q_skip, (double)(step_end - ne));
                if (q_skip > 2.0) m = ne + (int64_t)q_skip - 1;
                bool was_in = false;
                for (; m < step_end; ++m) {
                    const double tt = __dmul_rn((double)(m - ne), c.dt);
                    const double px = __fma_rn(kx, tt, xe), py = __fma_rn(ky, tt, ye);
                    bool in = px >= c.x0 && px <= c.x1;
                    if (two_d && fabs(py) > c.yh) in = false;
                    if (!in) {
                        if (was_in) break;                        // left the target
                        if ((px < c.x0 && kx <= 0.0) || (px > c.x1 && kx >= 0.0)) break;
                        if (two_d && fabs(py) > c.yh && py * ky >= 0.0) break;
                        continue;
                    }
                    if (!was_in) {
                        was_in = true;
                        atomicAdd(&s_t[PE_PT_N_ENTERED], 1ull);
                        if (above) atomicAdd(&s_t[PE_PT_N_K_ABOVE], 1ull);
                    }
                    const uint4 w = philox4x32_10(make_uint4(p.id_mech, r.run_id, (uint32_t)m, kPurBH + (uint32_t)ne),
                                                  r.seed_lo, r.seed_hi);
                    if (below_threshold(P, w.x, w.y)) {
                        const double x = bh_sample_x(t, cdf, k, uni53(w64(w.z, w.w)));
                        const double ep = x * k;
                        q.x = (float)px;
                        q.y = (float)(two_d ? py : 0.0);
                        q.e_minus = (float)(k - ep);
                        q.e_plus = (float)ep;
                        q.kx = p.kx; q.ky = p.ky; q.kz = p.kz;
                        q.step = (uint32_t)m;
                        q.photon = (uint32_t)j;
                        q.id_mech = p.id_mech;
                        fx_add(&s_t[PE_PT_E_PAIRS], k);
                        fx_add(&s_t[PE_PT_E_POSITRONS], ep);
                        conv = true;
                        break;
                    }
                }
            }
        }
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
                           int64_t step_end, void* pairs, int64_t capacity, unsigned long long* tally,
                           cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t blocks = (n_photons + 255) / 256;
    const int grid = (int)(blocks < (int64_t)sms * 8 ? (blocks > 0 ? blocks : 1) : (int64_t)sms * 8);
    k_pair_transport<<<grid, 256, 0, s>>>(t, r, static_cast<const Photon*>(photons), n_photons, step_end,
                                          static_cast<PairRec*>(pairs), capacity, tally);
}

}  // namespace pe
