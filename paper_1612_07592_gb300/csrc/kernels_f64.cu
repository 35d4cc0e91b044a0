// kernels_f64.cu -- every FP64 step kernel: the plain per-run kernel and the
// instantiations of the persistent kernel for double.
//
// This translation unit is compiled with -fmad=false: no multiply and add is
// contracted into a fused multiply-add unless the source asks for one, so each
// FP64 operation of the step is one IEEE-rounded multiply or add whatever kernel
// it is inlined into.  The plain kernel (one step per launch, global atomics) and
// the persistent kernel (K steps per launch, shared-memory accumulators) therefore
// compute bit-identical particles, photons and tallies.  The FP64 oracle is built
// with the same rule (no contraction).
#include "kernels.cuh"

namespace pe {

// ---------------------------------------------------------------------------
// plain FP64 kernel: one step, one particle per thread
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_step_plain(TablesDev t, RunDevT<double> r) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool active = i < r.n;
    Particle<double> P;
    if (active) {
        load_particle<double>(r, i, P);
        active = live_or_kill<double>(r, i, P, (uint32_t)r.step0, r.tally);
    }
    if (active) {
        const double* sig = t.sig64 + (size_t)r.iz * t.n_E;
        const uint32_t n = (uint32_t)r.step0;
        const uint32_t id = r.id0 + (uint32_t)i;
        switch (r.fk) {
            case FK_PLANE_LP: step_one<double, FK_PLANE_LP>(t, r, t.h64, sig, id, n, (double)n, P, r.hist, r.tally); break;
            case FK_PLANE_CP: step_one<double, FK_PLANE_CP>(t, r, t.h64, sig, id, n, (double)n, P, r.hist, r.tally); break;
            case FK_GAUSS_LP: step_one<double, FK_GAUSS_LP>(t, r, t.h64, sig, id, n, (double)n, P, r.hist, r.tally); break;
            case FK_GAUSS_CP: step_one<double, FK_GAUSS_CP>(t, r, t.h64, sig, id, n, (double)n, P, r.hist, r.tally); break;
            case FK_REFL_LP: step_one<double, FK_REFL_LP>(t, r, t.h64, sig, id, n, (double)n, P, r.hist, r.tally); break;
            case FK_REFL_CP: step_one<double, FK_REFL_CP>(t, r, t.h64, sig, id, n, (double)n, P, r.hist, r.tally); break;
            default: step_one<double, FK_CONST>(t, r, t.h64, sig, id, n, (double)n, P, r.hist, r.tally); break;
        }
        store_particle<double>(r, i, P);
    }
}

void launch_step_plain_f64(const TablesDev& t, const RunDev& r, cudaStream_t s) {
    if (r.n == 0) return;
    int grid = (int)((r.n + 255) / 256);
    k_step_plain<<<grid, 256, 0, s>>>(t, r);
}

// ---------------------------------------------------------------------------
// persistent kernel for double
// ---------------------------------------------------------------------------
template <bool kSingle, int G>
static const void* kernel_f64() {
    return (const void*)k_step_persistent<double, kSingle, G>;
}

void launch_step_persistent_f64(const TablesDev& t, const BatchDevT<double>& b, int steps, int grid, int block,
                                cudaStream_t s) {
    const int smem = persistent_smem_bytes(t, PE_F64);
    // all runs of b share one field kind (the caller groups a batch by kind)
    with_field_kind(b.runs[0].fk, [&](auto g) {
        constexpr int G = decltype(g)::value;
        if (b.n_runs == 1) {
            if (smem > 48 * 1024) cudaFuncSetAttribute(kernel_f64<true, G>(), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            k_step_persistent<double, true, G><<<grid, block, smem, s>>>(t, b, steps);
        } else {
            if (smem > 48 * 1024) cudaFuncSetAttribute(kernel_f64<false, G>(), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            k_step_persistent<double, false, G><<<grid, block, smem, s>>>(t, b, steps);
        }
    });
}

// the kernel a launch of these runs uses (for graph nodes); sets the shared-memory attribute
const void* persistent_kernel_f64(const BatchDevT<double>& b, int smem, int block, int* threads) {
    *threads = block;
    const void* f = nullptr;
    with_field_kind(b.runs[0].fk, [&](auto g) {
        constexpr int G = decltype(g)::value;
        f = b.n_runs == 1 ? kernel_f64<true, G>() : kernel_f64<false, G>();
    });
    if (smem > 48 * 1024) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return f;
}

int persistent_occupancy_f64(int block, int smem) {
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step_persistent<double, false, FK_PLANE_LP>, block, smem);
    return e == cudaSuccess ? occ : 1;
}

}  // namespace pe
