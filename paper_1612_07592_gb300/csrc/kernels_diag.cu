// kernels_diag.cu -- diagnostics for tests and the benchmark: the library's own FP32 device
// forms evaluated on given inputs (pe_math_probe), and FMA-loop kernels that measure the peak
// of the FP32 and FP64 pipes (pe_fma_peak).  Compiled with the step kernels' flags, so the
// forms here are the ones the step uses.
#include "pair_f32.cuh"

namespace pe {

__global__ void __launch_bounds__(256) k_math_probe(int fn, const float* in, float* out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = in[i];
    float r = 0.0f;
    switch (fn) {
        case PE_MATH_RCP: r = -nrcp2(P2(v)).x; break;
        case PE_MATH_SIN: { float2 s, c; sincos2(P2(v), s, c); r = s.x; } break;
        case PE_MATH_COS: { float2 s, c; sincos2(P2(v), s, c); r = c.x; } break;
        case PE_MATH_SIN1: { float s, c; m_sincos(v, &s, &c); r = s; } break;
        case PE_MATH_COS1: { float s, c; m_sincos(v, &s, &c); r = c; } break;
        case PE_MATH_BREMS_P: r = v < 0x1.0p-5f ? brems_series2(P2(v)).x : -expm1f(-v); break;
        case PE_MATH_BREMS_P1: r = one_minus_exp_neg_f32(v); break;
        case PE_MATH_CUDA_RCP: r = __frcp_rn(v); break;
        case PE_MATH_CUDA_SIN: r = sinf(v); break;
        case PE_MATH_CUDA_COS: r = cosf(v); break;
        case PE_MATH_CUDA_EXPM1: r = -expm1f(-v); break;
        case PE_MATH_GOUY_C: { float2 c, sn, q; gouy2(P2(v), c, sn, q); r = c.x; } break;
        case PE_MATH_GOUY_S: { float2 c, sn, q; gouy2(P2(v), c, sn, q); r = sn.x; } break;
        case PE_MATH_EXP_NEG: r = exp_neg2(P2(v)).x; break;
        case PE_MATH_TAU: r = tau_draw_f32(__float_as_uint(in[2 * i]), __float_as_uint(in[2 * i + 1])); break;
        default: r = 0.0f; break;
    }
    out[i] = r;
}

// 16 independent FMA chains per thread, `iters` rounds
constexpr int kChains = 16;
__global__ void __launch_bounds__(256) k_fma_f32(int iters, float m, float* out) {
    float a[kChains];
    const float c = 1e-7f * (float)threadIdx.x;
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void __launch_bounds__(256) k_fma_f32x2(int iters, float m, float* out) {
    float2 a[kChains];
    const float2 c = P2(1e-7f * (float)threadIdx.x), m2 = P2(m);
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = make_float2((float)(threadIdx.x + k), (float)(threadIdx.x - k));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma2(a[k], m2, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void __launch_bounds__(256) k_fma_f64(int iters, double m, double* out) {
    double a[kChains];
    const double c = 1e-7 * (double)threadIdx.x;
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

void launch_math_probe(int fn, const float* in, float* out, int64_t n, cudaStream_t s) {
    const int64_t grid = (n + 255) / 256;
    k_math_probe<<<(unsigned)grid, 256, 0, s>>>(fn, in, out, n);
}

int fma_chains() { return kChains; }

void launch_fma_peak(int kind, int blocks, int threads, int iters, void* out, cudaStream_t s) {
    if (kind == PE_FMA_F32) k_fma_f32<<<blocks, threads, 0, s>>>(iters, 0.9999999f, static_cast<float*>(out));
    else if (kind == PE_FMA_F32X2) k_fma_f32x2<<<blocks, threads, 0, s>>>(iters, 0.9999999f, static_cast<float*>(out));
    else k_fma_f64<<<blocks, threads, 0, s>>>(iters, 0.9999999, static_cast<double*>(out));
}

}  // namespace pe
