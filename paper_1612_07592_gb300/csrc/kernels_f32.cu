// kernels_f32.cu -- instantiations of the persistent kernel for float.
#include "kernels.cuh"
#include "pair_f32.cuh"

namespace pe {

// The 1D plane-wave kinds use the paired kernel (two electrons per thread, block/2
// threads per tile of `block` electrons); the others one electron per thread.
template <bool kSingle, int G>
static const void* kernel_of(int block, int& threads) {
    if constexpr (G == FK_PLANE_LP || G == FK_PLANE_CP) {
        threads = block / 2;
        return (const void*)k_step_pair<kSingle, G>;
    } else {
        threads = block;
        return (const void*)k_step_persistent<float, kSingle, G>;
    }
}

template <bool kSingle, int G>
static void launch_one(const TablesDev& t, const BatchDevT<float>& b, int steps, int grid, int block, cudaStream_t s,
                       int smem) {
    int threads;
    const void* f = kernel_of<kSingle, G>(block, threads);
    if (smem > 48 * 1024) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if constexpr (G == FK_PLANE_LP || G == FK_PLANE_CP)
        k_step_pair<kSingle, G><<<grid, threads, smem, s>>>(t, b, steps);
    else
        k_step_persistent<float, kSingle, G><<<grid, threads, smem, s>>>(t, b, steps);
}

void launch_step_persistent_f32(const TablesDev& t, const BatchDevT<float>& b, int steps, int grid, int block,
                                cudaStream_t s) {
    const int smem = persistent_smem_bytes(t, PE_F32);
    // all runs of b share one field kind (the caller groups a batch by kind)
    with_field_kind(b.runs[0].fk, [&](auto g) {
        if (b.n_runs == 1) launch_one<true, decltype(g)::value>(t, b, steps, grid, block, s, smem);
        else launch_one<false, decltype(g)::value>(t, b, steps, grid, block, s, smem);
    });
}

// the kernel a launch of these runs uses and its threads per CTA (for graph nodes);
// sets the shared-memory attribute
const void* persistent_kernel_f32(const BatchDevT<float>& b, int smem, int block, int* threads) {
    const void* f = nullptr;
    int th = block;
    with_field_kind(b.runs[0].fk, [&](auto g) {
        f = b.n_runs == 1 ? kernel_of<true, decltype(g)::value>(block, th)
                          : kernel_of<false, decltype(g)::value>(block, th);
    });
    if (smem > 48 * 1024) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    *threads = th;
    return f;
}

// default CTAs per SM of the grid: three waves of the paired kernel (plane-wave kinds;
// tiles differ in cost with their emission histories, and a CTA per one or two tiles lets
// the block scheduler balance them: measured +6 % over one wave, +2.5 % over two, on
// 1e6 electrons), twice the resident CTAs of the one-electron kernel otherwise
int default_ctas_per_sm_f32(int fk, int block, int smem) {
    if (fk == FK_PLANE_LP || fk == FK_PLANE_CP) {
        int occ = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step_pair<true, FK_PLANE_LP>, block / 2,
                                                                      smem);
        return 3 * (e == cudaSuccess && occ > 0 ? occ : 1);
    }
    return 2 * persistent_occupancy_f32(block, smem);
}

int persistent_occupancy_f32(int block, int smem) {
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step_persistent<float, false, FK_PLANE_LP>, block, smem);
    return e == cudaSuccess ? occ : 1;
}

}  // namespace pe
