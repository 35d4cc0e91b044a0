// kernels_pic.cu -- the 1D electromagnetic PIC around the emission step.
//
//  k_pic_particles  one thread per electron: fields gathered from the grid at
//                   x^n (linear weights), the emission step of Sec. 2.2 (push,
//                   NCS, brems, position), then the electron's current J^{n+1/2}
//                   by charge-conserving linear weighting, summed per CTA in
//                   shared memory and once per CTA into the run's accumulator;
//                   an electron that left [0, L] is removed after its deposit.
//                   The last CTA to finish (a count after the sums) then advances
//                   the grid: E_x -= dt J_x at the half nodes; the wave variants
//                   F+- = E_y +- B_z and G+- = E_z -+ B_y carried one cell along
//                   +-x with the current at the path's midpoint; the laser enters
//                   at x = 0; the sums and the count are cleared for the next step.
//                   One launch per step.
//  k_pic_rho        ion charge of the neutral start (the electrons' initial
//                   charge with the opposite sign), a diagnostic of Gauss's law.
//
// Currents are summed as dimensionless 2^-36 fixed-point integers, one rounding
// per contribution: exact and independent of the order of the atomic adds.
#include "kernels.cuh"

namespace pe {

namespace {

__device__ __forceinline__ long long fxq(double v) { return __double2ll_rn(v * 68719476736.0); }
__device__ __forceinline__ long long fxq(float v) { return __float2ll_rn(v * 68719476736.0f); }

// weight of grid point k (node, or half node with off = 1/2) for a particle at s = x/dx
template <typename R>
__device__ __forceinline__ R lin_w(R s, int k, R off) {
    R d = fabs(s - ((R)k + off));
    return d < (R)1 ? (R)1 - d : (R)0;
}

__device__ __forceinline__ void acc_add(unsigned long long* a, long long v) {
    if (v) atomicAdd(a, (unsigned long long)v);
}

// Shared-memory current sums as two 32-bit words per grid word (32-bit shared atomics
// run about four times faster than 64-bit ones on GB300): a contribution v (|v| <= 2^36)
// adds v >> 16 (|.| <= 2^20) to the high word and v & 0xffff to the low word, so
// v = hi 2^16 + lo exactly.  Up to kFlushTiles tiles of 256 electrons (each adds at
// most once per word per electron) the high sums stay below 2^31 in magnitude and the
// low sums below 2^32; the CTA then moves them into the run's 64-bit sums.
constexpr int kFlushTiles = 7;
struct SplitSums {
    unsigned int* hi;   // [3 n_cells], two's complement
    unsigned int* lo;   // [3 n_cells]
};
__device__ __forceinline__ void acc_add(const SplitSums& a, int k, long long v) {
    if (v) {
        atomicAdd(a.hi + k, (unsigned int)(int)(v >> 16));
        atomicAdd(a.lo + k, (unsigned int)(v & 0xffff));
    }
}
__device__ __forceinline__ void flush_split(const SplitSums& a, int nj, unsigned long long* acc) {
    for (int k = threadIdx.x; k < nj; k += blockDim.x) {
        const long long v = (long long)(int)a.hi[k] * 65536 + (long long)a.lo[k];
        if (v) atomicAdd(acc + k, (unsigned long long)v);
        a.hi[k] = 0;
        a.lo[k] = 0;
    }
}

// current of one electron moving from x_old to x_new (|x_new - x_old| < dx) with
// velocity (vy, vz): J_x at half nodes from the change of its node weights
// (cumulative, charge conserving); J_y, J_z at half nodes with the mean of its
// half-node weights at the two positions.  Dimensionless sums; the field kernel
// applies the weight and the charge sign.
template <typename R>
__device__ __forceinline__ void pic_deposit(R dx, int n, R x_old, R x_new, R vy, R vz, const SplitSums& sj) {
    const R so = x_old / dx, sn = x_new / dx;
    const int ia = (int)floor(so < sn ? so : sn);
    R cum = 0;
#pragma unroll
    for (int k = ia; k <= ia + 1; ++k) {
        cum += lin_w<R>(sn, k, (R)0) - lin_w<R>(so, k, (R)0);
        if (k >= 0 && k < n) acc_add(sj, k, fxq(cum));
    }
#pragma unroll
    for (int k = ia - 1; k <= ia + 1; ++k) {
        const R sbar = (R)0.5 * (lin_w<R>(so, k, (R)0.5) + lin_w<R>(sn, k, (R)0.5));
        if (sbar > (R)0 && k >= 0 && k < n) {
            acc_add(sj, n + k, fxq(vy * sbar));
            acc_add(sj, 2 * n + k, fxq(vz * sbar));
        }
    }
}

// The field update of one step by one CTA of any size: E_x -= dt J_x at the half nodes;
// F+ and G+ carried one cell along +x, F- and G- along -x, each with the current at the
// midpoint of its path; the laser enters at x = 0; the current sums are cleared.  Each
// thread updates one contiguous run of nodes in place (descending for the +x variants,
// ascending for the -x ones) after keeping the one value it needs from the neighbouring
// run.  The sums are read at L2 (they were built there by atomics).
template <typename R, bool kCP>
__device__ void pic_fields_block(const RunDevT<R>& r) {
    const int n = r.n_cells;
    const StepC<R>& c = r.c;
    R* ex = static_cast<R*>(r.grid);
    R* fp = ex + n;
    R* fm = fp + n + 1;
    R* gp = fm + n + 1;
    R* gm = gp + n + 1;
    unsigned long long* jx = r.jacc;
    unsigned long long* jy = jx + n;
    unsigned long long* jz = jy + n;
    const R dt = c.dt;
    const R kx = c.pic_kx, kyz = c.pic_kyz;   // J_x = kx sum, J_y,z = kyz sum (charge sign included)
    auto J = [](const unsigned long long* a, int i) { return (R)(long long)__ldcg(a + i); };
    const int chunk = (n + 1 + blockDim.x - 1) / blockDim.x;
    const int i0 = threadIdx.x * chunk, i1 = min(i0 + chunk, n + 1) - 1;   // this thread's nodes [i0, i1]
    R fp_in = 0, gp_in = 0, fm_in = 0, gm_in = 0;
    if (i0 <= i1) {
        if (i0 >= 1) { fp_in = fp[i0 - 1]; gp_in = gp[i0 - 1]; }
        if (i1 < n) { fm_in = fm[i1 + 1]; gm_in = gm[i1 + 1]; }
    }
    __syncthreads();
    if (i0 <= i1) {
        for (int i = i1; i >= i0; --i) {            // along +x from node i - 1 through half node i - 1
            const R f = i == i0 ? fp_in : fp[i - 1];
            const R g = i == i0 ? gp_in : gp[i - 1];
            fp[i] = i > 0 ? f - dt * kyz * J(jy, i - 1) : (R)0;
            gp[i] = i > 0 ? g - dt * kyz * J(jz, i - 1) : (R)0;
        }
        for (int i = i0; i <= i1; ++i) {            // along -x from node i + 1 through half node i
            const R f = i == i1 ? fm_in : fm[i + 1];
            const R g = i == i1 ? gm_in : gm[i + 1];
            fm[i] = i < n ? f - dt * kyz * J(jy, i) : (R)0;
            gm[i] = i < n ? g - dt * kyz * J(jz, i) : (R)0;
        }
        for (int i = i0; i <= i1 && i < n; ++i) ex[i] -= dt * kx * J(jx, i);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) jx[i] = 0;
    if (threadIdx.x == 0) {
        // the laser enters at x = 0: F+ = 2 g_y, G+ = 2 g_z at t^{n+1}
        R gy, gz;
        const R nf1 = (R)(r.step0 + 1);
        plane_e<R, kCP>(c, phase(c, nf1, (R)0, (R)0), gy, gz);
        fp[0] = (R)2 * gy;
        gp[0] = (R)2 * gz;
    }
}

// kCommon: NCS on and direct brems (a PIC run has no absorbing box), known at compile time
template <typename R, bool kCommon>
__global__ void __launch_bounds__(256, 4) k_pic_particles(TablesDev t, RunDevT<R> r) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* s_hist = reinterpret_cast<unsigned long long*>(smem);
    unsigned long long* s_tally = s_hist + PE_HIST_WORDS;
    unsigned long long* s_j = s_tally + PE_TALLY_WORDS;             // 3 n_cells current sums (split)
    const SplitSums sj{reinterpret_cast<unsigned int*>(s_j), reinterpret_cast<unsigned int*>(s_j) + 3 * r.n_cells};
    R* s_h = reinterpret_cast<R*>(s_j + 3 * r.n_cells);
    R* s_sig = s_h + t.n_eta;
    const R* g_h = (sizeof(R) == 4) ? (const R*)t.h32 : (const R*)t.h64;
    const R* g_sig = (sizeof(R) == 4) ? (const R*)t.sig32 : (const R*)t.sig64;
    const int nj = 3 * r.n_cells;
    for (int k = threadIdx.x; k < PE_HIST_WORDS + PE_TALLY_WORDS + nj; k += blockDim.x) s_hist[k] = 0;
    for (int k = threadIdx.x; k < t.n_eta; k += blockDim.x) s_h[k] = g_h[k];
    for (int k = threadIdx.x; k < t.n_Z * t.n_E; k += blockDim.x) s_sig[k] = g_sig[k];
    __syncthreads();

    const R* sig_z = s_sig + (size_t)r.iz * t.n_E;
    const uint32_t step = (uint32_t)r.step0;
    const R nf = (R)step;
    int tiles = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < r.n; base += (int64_t)gridDim.x * blockDim.x) {
        if (tiles == kFlushTiles) {                     // keep the split sums in range
            __syncthreads();
            flush_split(sj, nj, r.jacc);
            __syncthreads();
            tiles = 0;
        }
        ++tiles;
        const int64_t i = base + threadIdx.x;
        bool active = i < r.n;
        Particle<R> P;
        if (active) {
            load_particle<R>(r, i, P);
            active = live_or_kill<R>(r, i, P, step, s_tally);
        }
        if (active) {
            const R x_old = P.x + P.x_lo;
            step_one<R, FK_PIC, kCommon>(t, r, s_h, sig_z, r.id0 + (uint32_t)i, step, nf, P, s_hist, s_tally);
            const R gamma = m_sqrt((R)1 + P.u[0] * P.u[0] + P.u[1] * P.u[1] + P.u[2] * P.u[2]);
            const R x_new = P.x + P.x_lo;
            pic_deposit<R>(r.c.dt, r.n_cells, x_old, x_new, P.u[1] / gamma, P.u[2] / gamma, sj);
            if (x_new < (R)0 || x_new > r.c.box1) {   // it left through a boundary face, carrying its charge out
                P.x = (R)NAN;
                atomicAdd(s_tally + PE_T_N_KILLED, 1ull);
                atomicAdd(s_tally + PE_T_KILLED_STEPS, (unsigned long long)step + 1ull);
            }
            store_particle<R>(r, i, P);
        }
    }
    __syncthreads();
    flush_split(sj, nj, r.jacc);
    flush_shared<R>(s_hist, s_tally, r);
    // the last CTA to finish (its sums and every other CTA's are in the run's sums) advances
    // the fields; the count word after the sums goes back to zero for the next step
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    unsigned int* done = reinterpret_cast<unsigned int*>(r.jacc + 3 * r.n_cells);
    if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (r.polarisation == PE_CP) pic_fields_block<R, true>(r);
        else pic_fields_block<R, false>(r);
        if (threadIdx.x == 0) *done = 0;
    }
}

constexpr int kFieldThreads = 1024;

template <typename R>
__global__ void __launch_bounds__(256) k_pic_rho_deposit(RunDevT<R> r) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= r.n) return;
    Particle<R> P;
    load_pos(r, i, P);
    const R x = P.x + P.x_lo;
    if (isnan(x)) return;
    const R s = x / r.c.dt;
    const int i0 = (int)floor(s);
    for (int k = i0; k <= i0 + 1; ++k)
        if (k >= 0 && k <= r.n_cells) acc_add(r.jacc + k, fxq(lin_w<R>(s, k, (R)0)));
}

template <typename R>
__global__ void __launch_bounds__(kFieldThreads) k_pic_rho_store(RunDevT<R> r) {
    const int n = r.n_cells;
    R* rho = static_cast<R*>(r.grid) + n + 4 * (n + 1);
    for (int i = threadIdx.x; i <= n; i += blockDim.x) {
        rho[i] = -r.c.pic_kyz * (R)(long long)r.jacc[i];   // + (w/dx) sum of node weights
        r.jacc[i] = 0;
    }
}

}  // namespace

static int pic_smem_bytes(const TablesDev& t, int n_cells, int precision) {
    const size_t rs = precision == PE_F32 ? 4 : 8;
    return (int)(8 * (PE_HIST_WORDS + PE_TALLY_WORDS + 3 * (size_t)n_cells) + rs * (t.n_eta + (size_t)t.n_Z * t.n_E));
}

template <typename R>
static void pic_step(const TablesDev& t, const RunDevT<R>& r, int sms, cudaStream_t s) {
    const int smem = pic_smem_bytes(t, r.n_cells, sizeof(R) == 4 ? PE_F32 : PE_F64);
    const bool common = r.enable_ncs && r.enable_brems && r.brems_method == PE_BREMS_DIRECT;
    const void* f = common ? (const void*)k_pic_particles<R, true> : (const void*)k_pic_particles<R, false>;
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    // four resident CTAs of 256 threads per SM (64 registers): measured 90 us per step on 1e6
    // electrons against 112 us at two (each CTA adds one flush of its current sums)
    const int64_t blocks = (r.n + 255) / 256;
    const int grid = (int)(blocks < 4 * (int64_t)sms ? (blocks > 0 ? blocks : 1) : 4 * (int64_t)sms);
    if (common) k_pic_particles<R, true><<<grid, 256, smem, s>>>(t, r);
    else k_pic_particles<R, false><<<grid, 256, smem, s>>>(t, r);
}

void launch_pic_step(const TablesDev& t, const RunDev& r, int precision, int sms, cudaStream_t s) {
    if (precision == PE_F32) pic_step<float>(t, to_float(r), sms, s);
    else pic_step<double>(t, r, sms, s);
}

void launch_pic_rho(const RunDev& r, int precision, cudaStream_t s) {
    const int grid = (int)((r.n + 255) / 256);
    if (precision == PE_F32) {
        const RunDevT<float> f = to_float(r);
        if (grid > 0) k_pic_rho_deposit<float><<<grid, 256, 0, s>>>(f);
        k_pic_rho_store<float><<<1, kFieldThreads, 0, s>>>(f);
    } else {
        if (grid > 0) k_pic_rho_deposit<double><<<grid, 256, 0, s>>>(r);
        k_pic_rho_store<double><<<1, kFieldThreads, 0, s>>>(r);
    }
}

}  // namespace pe
