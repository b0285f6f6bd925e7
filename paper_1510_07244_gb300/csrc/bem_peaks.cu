// Arithmetic-pipe probes: the denominators of the quadrature kernels'
// rooflines, measured on the GPU the library runs on.
//
// Quadrature is not a contraction and moves few bytes, so its kernels are
// bound by the FP32 or FP64 FMA pipe and by the special-function unit
// (reciprocal square root; sine and cosine for the Helmholtz kernel).  Each
// probe runs independent dependency chains of one instruction class in every
// thread of a grid that fills the GPU, and stores a result that depends on all
// of them, so nothing is removed by the compiler.  The caller times one launch
// with CUDA events on the context's stream; the launch performs exactly
// bem_peak_probe's returned operation count.
#include <cuda_runtime.h>

#include "bem_internal.h"

namespace bem {

namespace {

constexpr int kChains = 8;       // independent chains per thread
constexpr int kUnroll = 16;      // operations per chain per loop trip

__global__ void __launch_bounds__(256) k_peak_ffma(int64_t trips, float a, float b, float *sink)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int64_t t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) sink[blockIdx.x] = s;     // never true for the probe's inputs
}

__global__ void __launch_bounds__(256) k_peak_dfma(int64_t trips, double a, double b, double *sink)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
    for (int64_t t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678) sink[blockIdx.x] = s;
}

// Special-function unit: the same reciprocal square root the float kernels use.
__global__ void __launch_bounds__(256) k_peak_rsqrt(int64_t trips, float *sink)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0f + (float)(threadIdx.x + c) * 1e-3f;
    for (int64_t t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                float y;
                asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[c]));
                x[c] = y;     // x -> x^(-1/2) stays in [1/2, 2]
            }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) sink[blockIdx.x] = s;
}

// Special-function unit: sine and cosine of one argument (two operations).
__global__ void __launch_bounds__(256) k_peak_sincos(int64_t trips, float *sink)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int64_t t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                float sn, cs;
                asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(sn) : "f"(x[c]));
                asm volatile("cos.approx.ftz.f32 %0, %1;" : "=f"(cs) : "f"(x[c]));
                x[c] = sn + cs;   // stays in [-sqrt 2, sqrt 2]
            }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) sink[blockIdx.x] = s;
}

// Packed FP32 pairs: one fma.rn.f32x2 is two FMAs on the two halves of a
// 64-bit register pair (sm_100 and later).
__device__ __forceinline__ unsigned long long pack_f32x2(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__global__ void __launch_bounds__(256) k_peak_ffma2(int64_t trips, float a, float b, float *sink)
{
    unsigned long long x[kChains];
    const unsigned long long aa = pack_f32x2(a, a), bb = pack_f32x2(b, b);
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        x[c] = pack_f32x2((float)(threadIdx.x + c) * 1e-3f, (float)(threadIdx.x + c) * 2e-3f);
    for (int64_t t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(aa), "l"(bb));
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    if (s == 12345.678f) sink[blockIdx.x] = s;
}

}  // namespace

}  // namespace bem

extern "C" int bem_peak_probe(bem_ctx *ctx, int32_t kind, int64_t trips, double *ops)
{
    using namespace bem;
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (!ops || kind < 0 || kind > 4 || trips < 1 || trips > (int64_t)1 << 30)
        return api_fail(ctx, BEM_ERR_INVALID_ARG, "bem_peak_probe: kind in [0, 4], trips in [1, 2^30]");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "cudaSetDevice");
    const int blocks = ctx->num_sms * 8, threads = 256;
    // the sink is never written for the probes' inputs; the tile-prefix
    // scratch is large enough for one value per block
    int rc = api_ensure_prefix(ctx, blocks);
    if (rc) return rc;
    void *sink = ctx->tile_prefix;
    const double per_thread = (double)trips * kUnroll * kChains;
    const double n = per_thread * blocks * threads;
    switch (kind) {
    case 0:
        k_peak_ffma<<<blocks, threads, 0, ctx->stream>>>(trips, 0.999f, 1e-3f, (float *)sink);
        *ops = 2.0 * n;          // an FMA is two floating-point operations
        break;
    case 1:
        k_peak_dfma<<<blocks, threads, 0, ctx->stream>>>(trips, 0.999, 1e-3, (double *)sink);
        *ops = 2.0 * n;
        break;
    case 2:
        k_peak_rsqrt<<<blocks, threads, 0, ctx->stream>>>(trips, (float *)sink);
        *ops = n;
        break;
    case 3:
        k_peak_sincos<<<blocks, threads, 0, ctx->stream>>>(trips, (float *)sink);
        *ops = 2.0 * n;          // sine and cosine
        break;
    default:
        k_peak_ffma2<<<blocks, threads, 0, ctx->stream>>>(trips, 0.999f, 1e-3f, (float *)sink);
        *ops = 4.0 * n;          // two FMAs per instruction
        break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "peak probe");
    return BEM_OK;
}
