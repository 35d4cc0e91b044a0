// kernels_paired.cu -- the FP32 step: instantiations and dispatch of the paired kernels (two
// electrons per thread) for every prescribed-field kind (the 1D plane wave, its reflection, the 2D
// focus, constant fields), and the plane wave's one-step streaming form.
// This translation unit is built without multiply-add contraction and with IEEE division and
// square root: its kernels (single run, batch, streaming) inline the same emission branches, and
// with every rounding written in the source they agree bit for bit (the approximate forms the
// step needs are explicit instructions in pair_f32.cuh).
#include "kernels.cuh"
#include "pair_f32.cuh"

namespace pe {

// Launches of at most this many steps (the state round-trips memory) on a single run
// of a plane-wave kind use the streaming form of the paired kernel.
constexpr int kStreamMaxSteps = 4;

static bool plane_kind(int fk) { return fk == FK_PLANE_LP || fk == FK_PLANE_CP; }
static bool use_stream(const BatchDevT<float>& b, int steps, int block) {
    return b.n_runs == 1 && plane_kind(b.runs[0].fk) && steps <= kStreamMaxSteps && block == kStreamTile;
}
// tables, then 16-byte alignment slack and the stage buffers
static int stream_smem_bytes(int base) { return base + 16 + kStreamStages * kStageBytes; }

// The kernel of a launch, its threads per CTA (block/2: two electrons per thread) and dynamic
// shared memory: the resident paired kernel, or for the plane wave its streaming form.
template <bool kSingle, int G>
static const void* kernel_of(const BatchDevT<float>& b, int steps, int block, int base_smem, int& threads, int& smem) {
    smem = base_smem;
    threads = block / 2;
    const bool common = common_flags_f32(b);
    if constexpr (G == FK_PLANE_LP || G == FK_PLANE_CP) {
        if (kSingle && use_stream(b, steps, block)) {
            smem = stream_smem_bytes(base_smem);
            return common ? (const void*)k_step_pair_stream<G, true> : (const void*)k_step_pair_stream<G, false>;
        }
    }
    return common ? (const void*)k_step_pair<kSingle, G, true> : (const void*)k_step_pair<kSingle, G, false>;
}

template <bool kSingle, int G>
static void launch_one(const TablesDev& t, const BatchDevT<float>& b, int steps, int grid, int block, cudaStream_t s,
                       int base_smem) {
    int threads, smem;
    const void* f = kernel_of<kSingle, G>(b, steps, block, base_smem, threads, smem);
    if (smem > 48 * 1024) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if constexpr (G == FK_PLANE_LP || G == FK_PLANE_CP) {
        if (f == (const void*)k_step_pair_stream<G, true>) {
            k_step_pair_stream<G, true><<<grid, threads, smem, s>>>(t, b, steps);
            return;
        }
        if (f == (const void*)k_step_pair_stream<G, false>) {
            k_step_pair_stream<G, false><<<grid, threads, smem, s>>>(t, b, steps);
            return;
        }
    }
    if (f == (const void*)k_step_pair<kSingle, G, true>)
        k_step_pair<kSingle, G, true><<<grid, threads, smem, s>>>(t, b, steps);
    else
        k_step_pair<kSingle, G, false><<<grid, threads, smem, s>>>(t, b, steps);
}

template <typename F>
static void with_paired_kind(int fk, F&& f) {
    switch (fk) {
        case FK_PLANE_LP: f(std::integral_constant<int, FK_PLANE_LP>{}); break;
        case FK_PLANE_CP: f(std::integral_constant<int, FK_PLANE_CP>{}); break;
        case FK_GAUSS_LP: f(std::integral_constant<int, FK_GAUSS_LP>{}); break;
        case FK_GAUSS_CP: f(std::integral_constant<int, FK_GAUSS_CP>{}); break;
        case FK_REFL_LP: f(std::integral_constant<int, FK_REFL_LP>{}); break;
        case FK_REFL_CP: f(std::integral_constant<int, FK_REFL_CP>{}); break;
        default: f(std::integral_constant<int, FK_CONST>{}); break;
    }
}

void launch_step_persistent_f32(const TablesDev& t, const BatchDevT<float>& b, int steps, int grid, int block,
                                cudaStream_t s) {
    const int smem = persistent_smem_bytes(t, PE_F32);
    with_paired_kind(b.runs[0].fk, [&](auto g) {
        if (b.n_runs == 1) launch_one<true, decltype(g)::value>(t, b, steps, grid, block, s, smem);
        else launch_one<false, decltype(g)::value>(t, b, steps, grid, block, s, smem);
    });
}

// the kernel a launch of these runs uses, its threads per CTA and dynamic shared memory
// (for graph nodes); sets the shared-memory attribute
const void* persistent_kernel_f32(const BatchDevT<float>& b, int steps, int base_smem, int block, int* threads,
                                  int* smem_out) {
    const void* f = nullptr;
    int th = block, smem = base_smem;
    with_paired_kind(b.runs[0].fk, [&](auto g) {
        f = b.n_runs == 1 ? kernel_of<true, decltype(g)::value>(b, steps, block, base_smem, th, smem)
                          : kernel_of<false, decltype(g)::value>(b, steps, block, base_smem, th, smem);
    });
    if (smem > 48 * 1024) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    *threads = th;
    *smem_out = smem;
    return f;
}

// Default CTAs per SM of the grid: three resident waves of the resident paired kernel (tiles differ in
// cost with their emission histories, and a CTA per one or two tiles lets the block scheduler balance
// them: measured +6 % over one wave, +2.5 % over two, on 1e6 electrons); one wave for the streaming
// form (each CTA streams many tiles of equal cost).
int default_ctas_per_sm_f32(int fk, int block, int smem, int steps_per_launch) {
    int occ = 0;
    cudaError_t e;
    if (plane_kind(fk) && steps_per_launch <= kStreamMaxSteps && block == kStreamTile) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step_pair_stream<FK_PLANE_LP, true>, block / 2,
                                                          stream_smem_bytes(smem));
        return e == cudaSuccess && occ > 0 ? occ : 1;
    }
    with_paired_kind(fk, [&](auto g) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step_pair<true, decltype(g)::value, true>, block / 2,
                                                          smem);
    });
    return 3 * (e == cudaSuccess && occ > 0 ? occ : 1);
}

}  // namespace pe
