// kernels.cu -- the init kernel, the diagnostics kernels and their launchers.  The
// step kernels are instantiated per precision in kernels_paired.cu (FP32) and kernels_f64.cu.
#include <algorithm>
#include <cmath>

#include "kernels.cuh"

namespace pe {

// ---------------------------------------------------------------------------
// init kernel
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_init(RunDevT<double> r, int init_dist, double theta, double beam_u) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= r.n) return;
    uint32_t id = r.id0 + (uint32_t)i;
    uint4 w = draw(r, id, 0, PUR_TAU0);
    double tau0 = -log(uni53(w64(w.x, w.y)));
    if (sizeof(R) == 4) {
        float hi = (float)tau0;
        ((float2*)r.tau)[i] = make_float2(hi, (float)(tau0 - (double)hi));
    } else {
        ((double*)r.tau)[i] = tau0;
    }
    if (r.wait) {
        uint4 v = draw(r, id, 0, PUR_WAIT);
        r.wait[i] = wait_draw(r.x_hat, v.x, v.y);
    }
    if (init_dist == PE_CALLER) return;
    uint4 p = draw(r, id, 0, PUR_POS);
    const StepC<double>& c = r.c;
    // a beam enters at the front face of the slab
    double x = (init_dist == PE_BEAM) ? c.x0 : c.x0 + (c.x1 - c.x0) * uni32(p.x);
    double y = (r.geometry == PE_GAUSS_2D) ? -c.yh + 2.0 * c.yh * uni32(p.y) : 0.0;
    double u0 = 0, u1 = 0, u2 = 0;
    if (init_dist == PE_MAXWELL_JUTTNER) {
        // Sobol (1976) rejection sampling of the Maxwell-Juttner momentum magnitude
        double um = 0.0;
        for (uint32_t round = 0; round < 64; ++round) {
            uint4 m = draw(r, id, 0, PUR_MJ + round);
            double X1 = uni32(m.x), X2 = uni32(m.y), X3 = uni32(m.z), X4 = uni32(m.w);
            double uu = -theta * log(X1 * X2 * X3);
            double ee = -theta * log(X1 * X2 * X3 * X4);
            if (ee * ee - uu * uu > 1.0) { um = uu; break; }
        }
        double X5 = uni32(p.z), X6 = uni32(p.w);
        double sn = 2.0 * sqrt(X5 * (1.0 - X5));
        double sphi, cphi;
        sincos(2.0 * kPi * X6, &sphi, &cphi);
        u0 = um * (2.0 * X5 - 1.0);
        u1 = um * sn * cphi;
        u2 = um * sn * sphi;
    } else if (init_dist == PE_BEAM) {
        u0 = beam_u;
    }
    if (sizeof(R) == 4) {
        float xh = (float)x, yh = (float)y;
        ((float2*)r.x)[i] = make_float2(xh, (float)(x - (double)xh));
        ((float2*)r.y)[i] = make_float2(yh, (float)(y - (double)yh));
    } else {
        ((double*)r.x)[i] = x;
        ((double*)r.y)[i] = y;
    }
    ((R*)r.ux)[i] = (R)u0;
    ((R*)r.uy)[i] = (R)u1;
    ((R*)r.uz)[i] = (R)u2;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_init(const RunDev& r, int precision, int init_dist, double theta, double beam_u, cudaStream_t s) {
    if (r.n == 0) return;
    int grid = (int)((r.n + 255) / 256);
    if (precision == PE_F32)
        k_init<float><<<grid, 256, 0, s>>>(r, init_dist, theta, beam_u);
    else
        k_init<double><<<grid, 256, 0, s>>>(r, init_dist, theta, beam_u);
}

int persistent_smem_bytes(const TablesDev& t, int precision) {
    size_t rs = precision == PE_F32 ? 4 : 8;
    return (int)(8 * (PE_HIST_WORDS + PE_TALLY_WORDS) + rs * (t.n_eta + (size_t)t.n_Z * t.n_E));
}

}  // namespace pe

namespace pe {

// ---------------------------------------------------------------------------
// diagnostics: electron energy spectrum (Fig. 5) and photon (x, energy) map (Fig. 4)
// ---------------------------------------------------------------------------
// bin of v in [lo, hi) on log bins: -1 below, n_bins at or above
__device__ __forceinline__ int log_bin(double v, double ln_lo, double inv_dln, int n_bins) {
    if (!(v > 0.0)) return -1;
    const double b = (log(v) - ln_lo) * inv_dln;
    if (b < 0.0) return -1;
    return b >= (double)n_bins ? n_bins : (int)b;
}

template <typename R>
__global__ void __launch_bounds__(256) k_electron_spectrum(RunDevT<double> r, double ln_lo, double inv_dln, int n_bins,
                                                           unsigned long long* out) {
    extern __shared__ unsigned long long s_bins[];
    for (int k = threadIdx.x; k < n_bins; k += blockDim.x) s_bins[k] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r.n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = sizeof(R) == 4 ? (double)((const float2*)r.x)[i].x : ((const double*)r.x)[i];
        if (isnan(x)) continue;
        const double u0 = ((const R*)r.ux)[i], u1 = ((const R*)r.uy)[i], u2 = ((const R*)r.uz)[i];
        const double ek = (sqrt(1.0 + u0 * u0 + u1 * u1 + u2 * u2) - 1.0) * kMec2MeV;   // kinetic energy, MeV
        const int b = log_bin(ek, ln_lo, inv_dln, n_bins);
        if (b >= 0 && b < n_bins) atomicAdd(&s_bins[b], 1ull);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_bins; k += blockDim.x)
        if (s_bins[k]) atomicAdd(out + k, s_bins[k]);
}

__global__ void __launch_bounds__(256) k_photon_map(const uint8_t* photons, const unsigned long long* tally,
                                                    int64_t capacity, double x_lo, double inv_dx, int nx,
                                                    double ln_lo, double inv_dln, int ne, unsigned long long* out) {
    const unsigned long long appended = tally[PE_T_N_PHOTONS];
    const int64_t count = appended < (unsigned long long)capacity ? (int64_t)appended : capacity;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = reinterpret_cast<const float4*>(photons + i * 32)[0];   // x, y, energy (m c^2), kx
        const double xb = ((double)a.x - x_lo) * inv_dx;
        if (!(xb >= 0.0) || xb >= (double)nx) continue;
        const int eb = log_bin((double)a.z * kMec2MeV, ln_lo, inv_dln, ne);
        if (eb < 0 || eb >= ne) continue;
        atomicAdd(out + (size_t)((int)xb) * ne + eb, 1ull);
    }
}

void launch_electron_spectrum(const RunDev& r, int precision, double e_lo, double e_hi, int n_bins,
                              unsigned long long* out, cudaStream_t s) {
    const double ln_lo = std::log(e_lo), inv_dln = n_bins / (std::log(e_hi) - std::log(e_lo));
    const int grid = (int)std::min<int64_t>((r.n + 255) / 256, 1024);
    if (grid <= 0) return;
    const size_t smem = sizeof(unsigned long long) * (size_t)n_bins;
    if (precision == PE_F32) k_electron_spectrum<float><<<grid, 256, smem, s>>>(r, ln_lo, inv_dln, n_bins, out);
    else k_electron_spectrum<double><<<grid, 256, smem, s>>>(r, ln_lo, inv_dln, n_bins, out);
}

void launch_photon_map(const RunDev& r, double x_lo, double x_hi, int nx, double e_lo, double e_hi, int ne,
                       unsigned long long* out, cudaStream_t s) {
    if (r.capacity <= 0) return;
    // the stored count is read on the device: a grid-stride launch sized for the capacity
    const int grid = (int)std::min<int64_t>((r.capacity + 255) / 256, 2048);
    k_photon_map<<<grid, 256, 0, s>>>(r.photons, r.tally, r.capacity, x_lo, nx / (x_hi - x_lo), nx, std::log(e_lo),
                                      ne / (std::log(e_hi) - std::log(e_lo)), ne, out);
}

}  // namespace pe
