// kernels_f64.cu -- instantiations of the persistent kernel for double.
#include "kernels.cuh"

namespace pe {

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
