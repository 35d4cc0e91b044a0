// kernels_f64.cu -- instantiations of the persistent kernel for double.
#include "kernels.cuh"

namespace pe {

template <bool kSingle, int G>
static void launch_one(const TablesDev& t, const BatchDevT<double>& b, int steps, int grid, int block, cudaStream_t s,
                       int smem) {
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_step_persistent<double, kSingle, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_step_persistent<double, kSingle, G><<<grid, block, smem, s>>>(t, b, steps);
}

void launch_step_persistent_f64(const TablesDev& t, const BatchDevT<double>& b, int steps, int grid, int block,
                                cudaStream_t s) {
    int smem = persistent_smem_bytes(t, PE_F64);
    // all runs of b share one field kind (the caller groups a batch by kind)
    const int fk = field_kind(b.runs[0].geometry, b.runs[0].polarisation);
    if (b.n_runs == 1) {
        switch (fk) {
            case FK_PLANE_LP: launch_one<true, FK_PLANE_LP>(t, b, steps, grid, block, s, smem); break;
            case FK_PLANE_CP: launch_one<true, FK_PLANE_CP>(t, b, steps, grid, block, s, smem); break;
            case FK_GAUSS_LP: launch_one<true, FK_GAUSS_LP>(t, b, steps, grid, block, s, smem); break;
            case FK_GAUSS_CP: launch_one<true, FK_GAUSS_CP>(t, b, steps, grid, block, s, smem); break;
            default: launch_one<true, FK_CONST>(t, b, steps, grid, block, s, smem); break;
        }
        return;
    }
    switch (fk) {
        case FK_PLANE_LP: launch_one<false, FK_PLANE_LP>(t, b, steps, grid, block, s, smem); break;
        case FK_PLANE_CP: launch_one<false, FK_PLANE_CP>(t, b, steps, grid, block, s, smem); break;
        case FK_GAUSS_LP: launch_one<false, FK_GAUSS_LP>(t, b, steps, grid, block, s, smem); break;
        case FK_GAUSS_CP: launch_one<false, FK_GAUSS_CP>(t, b, steps, grid, block, s, smem); break;
        default: launch_one<false, FK_CONST>(t, b, steps, grid, block, s, smem); break;
    }
}

// the kernel a launch of these runs uses (for graph nodes); sets the shared-memory attribute
const void* persistent_kernel_f64(const BatchDevT<double>& b, int smem, int block, int* threads) {
    *threads = block;
    const int fk = field_kind(b.runs[0].geometry, b.runs[0].polarisation);
    const void* f = nullptr;
    if (b.n_runs == 1) {
        switch (fk) {
            case FK_PLANE_LP: f = (const void*)k_step_persistent<double, true, FK_PLANE_LP>; break;
            case FK_PLANE_CP: f = (const void*)k_step_persistent<double, true, FK_PLANE_CP>; break;
            case FK_GAUSS_LP: f = (const void*)k_step_persistent<double, true, FK_GAUSS_LP>; break;
            case FK_GAUSS_CP: f = (const void*)k_step_persistent<double, true, FK_GAUSS_CP>; break;
            default: f = (const void*)k_step_persistent<double, true, FK_CONST>; break;
        }
    } else {
        switch (fk) {
            case FK_PLANE_LP: f = (const void*)k_step_persistent<double, false, FK_PLANE_LP>; break;
            case FK_PLANE_CP: f = (const void*)k_step_persistent<double, false, FK_PLANE_CP>; break;
            case FK_GAUSS_LP: f = (const void*)k_step_persistent<double, false, FK_GAUSS_LP>; break;
            case FK_GAUSS_CP: f = (const void*)k_step_persistent<double, false, FK_GAUSS_CP>; break;
            default: f = (const void*)k_step_persistent<double, false, FK_CONST>; break;
        }
    }
    if (smem > 48 * 1024) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return f;
}

int persistent_occupancy_f64(int block, int smem) {
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step_persistent<double, false, FK_PLANE_LP>, block, smem);
    return e == cudaSuccess ? occ : 1;
}

}  // namespace pe
