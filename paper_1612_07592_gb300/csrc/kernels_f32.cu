// kernels_f32.cu -- the FP32 launches: the prescribed-field kinds (1D plane wave, its reflection,
// 2D focus) go to the paired kernels (kernels_paired.cu); constant fields to the one-electron
// persistent kernel instantiated here for float.
#include "kernels.cuh"

namespace pe {

template <bool kSingle, int G>
static const void* kernel_of(const BatchDevT<float>& b, int base_smem, int block, int& threads, int& smem) {
    smem = base_smem;
    threads = block;
    return common_flags_f32(b) ? (const void*)k_step_persistent<float, kSingle, G, true>
                               : (const void*)k_step_persistent<float, kSingle, G, false>;
}

template <bool kSingle, int G>
static void launch_one(const TablesDev& t, const BatchDevT<float>& b, int steps, int grid, int block, cudaStream_t s,
                       int base_smem) {
    int threads, smem;
    const void* f = kernel_of<kSingle, G>(b, base_smem, block, threads, smem);
    if (smem > 48 * 1024) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (f == (const void*)k_step_persistent<float, kSingle, G, true>)
        k_step_persistent<float, kSingle, G, true><<<grid, threads, smem, s>>>(t, b, steps);
    else
        k_step_persistent<float, kSingle, G, false><<<grid, threads, smem, s>>>(t, b, steps);
}

// the kinds of the one-electron FP32 kernel: constant fields
template <typename F>
static void with_one_electron_kind(int, F&& f) {
    f(std::integral_constant<int, FK_CONST>{});
}

void launch_step_persistent_f32(const TablesDev& t, const BatchDevT<float>& b, int steps, int grid, int block,
                                cudaStream_t s) {
    // all runs of b share one field kind (the caller groups a batch by kind)
    if (paired_kind_f32(b.runs[0].fk)) {
        launch_step_paired_f32(t, b, steps, grid, block, s);
        return;
    }
    const int smem = persistent_smem_bytes(t, PE_F32);
    with_one_electron_kind(b.runs[0].fk, [&](auto g) {
        if (b.n_runs == 1) launch_one<true, decltype(g)::value>(t, b, steps, grid, block, s, smem);
        else launch_one<false, decltype(g)::value>(t, b, steps, grid, block, s, smem);
    });
}

// the kernel a launch of these runs uses, its threads per CTA and dynamic shared memory
// (for graph nodes); sets the shared-memory attribute
const void* persistent_kernel_f32(const BatchDevT<float>& b, int steps, int base_smem, int block, int* threads,
                                  int* smem_out) {
    if (paired_kind_f32(b.runs[0].fk)) return paired_kernel_f32(b, steps, base_smem, block, threads, smem_out);
    const void* f = nullptr;
    int th = block, smem = base_smem;
    with_one_electron_kind(b.runs[0].fk, [&](auto g) {
        f = b.n_runs == 1 ? kernel_of<true, decltype(g)::value>(b, base_smem, block, th, smem)
                          : kernel_of<false, decltype(g)::value>(b, base_smem, block, th, smem);
    });
    if (smem > 48 * 1024) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    *threads = th;
    *smem_out = smem;
    return f;
}

// Default CTAs per SM of the grid: the paired kernels' rule (kernels_paired.cu) for their kinds;
// for the one-electron kernel twice its resident CTAs.
int default_ctas_per_sm_f32(int fk, int block, int smem, int steps_per_launch) {
    if (paired_kind_f32(fk)) return default_ctas_per_sm_paired_f32(fk, block, smem, steps_per_launch);
    int occ = 0;
    with_one_electron_kind(fk, [&](auto g) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step_persistent<float, false, decltype(g)::value, true>,
                                                          block, smem) != cudaSuccess)
            occ = 0;
    });
    return 2 * (occ > 0 ? occ : 1);
}

}  // namespace pe
