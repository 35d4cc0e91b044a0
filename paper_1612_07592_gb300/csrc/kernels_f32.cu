// kernels_f32.cu -- instantiations of the persistent kernel for float.
#include "kernels.cuh"
#include "pair_f32.cuh"

namespace pe {

// Launches of at most this many steps (the state round-trips memory) on a single run
// of a plane-wave kind use the streaming form of the paired kernel.
constexpr int kStreamMaxSteps = 4;

static bool plane_kind(int fk) { return fk == FK_PLANE_LP || fk == FK_PLANE_CP; }
// kinds stepped by the paired kernel (two electrons per thread): the 1D plane wave and the 2D focus.
// The reflected wave stays on the one-electron kernel: with an emission in about 4 % of its
// particle-steps, the paired form (both halves of a pair emitting in turn, 72 registers) measured
// 4.15e10 particle-steps/s against 4.78e10 for one electron per thread at 8 CTAs of 256 threads.
template <int G>
constexpr bool kPairedKind = G == FK_PLANE_LP || G == FK_PLANE_CP || G == FK_GAUSS_LP || G == FK_GAUSS_CP;
// every run of the launch has the paper's setup: NCS on, direct brems, no absorbing box (the paired
// kernels then take these flags as compile-time constants)
static bool common_flags(const BatchDevT<float>& b) {
    for (int k = 0; k < b.n_runs; ++k) {
        const RunDevT<float>& r = b.runs[k];
        if (!r.enable_ncs || !r.enable_brems || r.brems_method != PE_BREMS_DIRECT || r.box_enable) return false;
    }
    return true;
}
static bool use_stream(const BatchDevT<float>& b, int steps, int block) {
    return b.n_runs == 1 && plane_kind(b.runs[0].fk) && steps <= kStreamMaxSteps && block == kStreamTile;
}
// tables, then 16-byte alignment slack and the stage buffers
static int stream_smem_bytes(int base) { return base + 16 + kStreamStages * kStageBytes; }

// The kernel of a launch, its threads per CTA and dynamic shared memory: the plane-wave and 2D
// focus kinds use the paired kernel (two electrons per thread, block/2 threads per tile of `block`
// electrons), the plane wave also its streaming form; the others one electron per thread.
template <bool kSingle, int G>
static const void* kernel_of(const BatchDevT<float>& b, int steps, int block, int base_smem, int& threads, int& smem) {
    smem = base_smem;
    if constexpr (kPairedKind<G>) {
        threads = block / 2;
        const bool common = common_flags(b);
        if constexpr (G == FK_PLANE_LP || G == FK_PLANE_CP) {
            if (kSingle && use_stream(b, steps, block)) {
                smem = stream_smem_bytes(base_smem);
                return common ? (const void*)k_step_pair_stream<G, true> : (const void*)k_step_pair_stream<G, false>;
            }
        }
        return common ? (const void*)k_step_pair<kSingle, G, true> : (const void*)k_step_pair<kSingle, G, false>;
    } else {
        threads = block;
        return common_flags(b) ? (const void*)k_step_persistent<float, kSingle, G, true>
                               : (const void*)k_step_persistent<float, kSingle, G, false>;
    }
}

template <bool kSingle, int G>
static void launch_one(const TablesDev& t, const BatchDevT<float>& b, int steps, int grid, int block, cudaStream_t s,
                       int base_smem) {
    int threads, smem;
    const void* f = kernel_of<kSingle, G>(b, steps, block, base_smem, threads, smem);
    if (smem > 48 * 1024) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if constexpr (kPairedKind<G>) {
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
    } else {
        if (f == (const void*)k_step_persistent<float, kSingle, G, true>)
            k_step_persistent<float, kSingle, G, true><<<grid, threads, smem, s>>>(t, b, steps);
        else
            k_step_persistent<float, kSingle, G, false><<<grid, threads, smem, s>>>(t, b, steps);
    }
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

// the kernel a launch of these runs uses, its threads per CTA and dynamic shared memory
// (for graph nodes); sets the shared-memory attribute
const void* persistent_kernel_f32(const BatchDevT<float>& b, int steps, int base_smem, int block, int* threads,
                                  int* smem_out) {
    const void* f = nullptr;
    int th = block, smem = base_smem;
    with_field_kind(b.runs[0].fk, [&](auto g) {
        f = b.n_runs == 1 ? kernel_of<true, decltype(g)::value>(b, steps, block, base_smem, th, smem)
                          : kernel_of<false, decltype(g)::value>(b, steps, block, base_smem, th, smem);
    });
    if (smem > 48 * 1024) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    *threads = th;
    *smem_out = smem;
    return f;
}

// Default CTAs per SM of the grid.  Paired kernel (plane-wave and 2D focus kinds): three resident waves
// (tiles differ in cost with their emission histories, and a CTA per one or two tiles lets
// the block scheduler balance them: measured +6 % over one wave, +2.5 % over two, on 1e6
// electrons); one wave for the streaming form (each CTA streams many tiles of equal cost).
// One-electron kernel: twice its resident CTAs.
int default_ctas_per_sm_f32(int fk, int block, int smem, int steps_per_launch) {
    if (plane_kind(fk) && steps_per_launch <= kStreamMaxSteps && block == kStreamTile) {
        int occ = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step_pair_stream<FK_PLANE_LP, true>,
                                                                      block / 2, stream_smem_bytes(smem));
        return e == cudaSuccess && occ > 0 ? occ : 1;
    }
    // paired kinds: three resident waves of this kind's paired kernel; the others twice the
    // resident CTAs of the one-electron kernel
    int occ = 0, waves = 2;
    with_field_kind(fk, [&](auto g) {
        constexpr int G = decltype(g)::value;
        cudaError_t e;
        if constexpr (kPairedKind<G>) {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step_pair<true, G, true>, block / 2, smem);
            waves = 3;
        } else {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step_persistent<float, false, G, true>, block, smem);
        }
        if (e != cudaSuccess) occ = 0;
    });
    return waves * (occ > 0 ? occ : 1);
}

}  // namespace pe
