// Touching-pair kernels (Sauter-Schwab rules, Section 2.2): one warp per pair,
// single-mesh and batched forms, FP64 and the float kernels of the mixed forms.
#include <cuda_runtime.h>

#include "bem_device.cuh"

namespace bem {

template <int KIND, int BASIS, int CAS>
__global__ void __launch_bounds__(256) k_touching(MeshView m, const int *__restrict__ list,
                                                  int64_t n, const double *__restrict__ rule,
                                                  int np, double kappa, double eta)
{
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid >= n) return;
    touch_pair<KIND, BASIS, CAS>(m, __ldg(list + wid), rule, np, kappa, threadIdx.x & 31, eta);
}

// Batched: items[k] = (job, touching index) over many meshes / kernels.
template <int KIND, int BASIS, int CAS>
__global__ void __launch_bounds__(256) k_touching_batch(const TouchJob *__restrict__ jobs,
                                                        const int2 *__restrict__ items, int64_t n,
                                                        const double *__restrict__ rule, int np)
{
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid >= n) return;
    const int2 it = items[wid];
    touch_pair<KIND, BASIS, CAS>(jobs[it.x].m, it.y, rule, np, jobs[it.x].kappa, threadIdx.x & 31,
                                 jobs[it.x].eta);
}

template <int CAS, int KIND, int BASIS>
__global__ void __launch_bounds__(256) k_touching_f32(MeshView m, const int *__restrict__ list,
                                                      int64_t n, const float *__restrict__ rule,
                                                      int np, float kappa)
{
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid >= n) return;
    touch_f32<CAS, KIND, BASIS>(m, __ldg(list + wid), rule, np, threadIdx.x & 31, kappa);
}

template <int CAS, int KIND, int BASIS>
__global__ void __launch_bounds__(256) k_touching_f32_batch(const TouchJob *__restrict__ jobs,
                                                            const int2 *__restrict__ items,
                                                            int64_t n,
                                                            const float *__restrict__ rule, int np)
{
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid >= n) return;
    const int2 it = items[wid];
    touch_f32<CAS, KIND, BASIS>(jobs[it.x].m, it.y, rule, np, threadIdx.x & 31,
                                (float)jobs[it.x].kappa);
}

cudaError_t launch_touching(const MeshView &m, int cas, const int *list, int64_t n,
                            const Rule4D &rule, int kind, double kappa, int f32, cudaStream_t st,
                            double eta)
{
    if (n <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n + 7) / 8);
    const bool p1 = m.basis == BEM_P1;
    if (f32 && rule.f && !kind_fp64_only(kind)) {
        const float kf = (float)kappa;
#define BEM_TV(K, B)                                                                          \
    do {                                                                                      \
        if (cas == kIdentical) k_touching_f32<kIdentical, K, B><<<blocks, 256, 0, st>>>(m, list, n, rule.f, rule.n, kf); \
        else if (cas == kEdge) k_touching_f32<kEdge, K, B><<<blocks, 256, 0, st>>>(m, list, n, rule.f, rule.n, kf);      \
        else k_touching_f32<kVertex, K, B><<<blocks, 256, 0, st>>>(m, list, n, rule.f, rule.n, kf);                      \
    } while (0)
        if (kind == BEM_LAPLACE_SLP) { if (p1) BEM_TV(BEM_LAPLACE_SLP, BEM_P1); else BEM_TV(BEM_LAPLACE_SLP, BEM_P0); }
        else if (kind == BEM_LAPLACE_DLP) { if (p1) BEM_TV(BEM_LAPLACE_DLP, BEM_P1); else BEM_TV(BEM_LAPLACE_DLP, BEM_P0); }
        else { if (p1) BEM_TV(BEM_HELMHOLTZ_SLP, BEM_P1); else BEM_TV(BEM_HELMHOLTZ_SLP, BEM_P0); }
#undef BEM_TV
        return cudaGetLastError();
    }
#define BEM_TOUCH(K, B, C) k_touching<K, B, C><<<blocks, 256, 0, st>>>(m, list, n, rule.d, rule.n, kappa, eta)
#define BEM_TOUCH_CASE(K, B)                                   \
    do {                                                       \
        if (cas == kIdentical) BEM_TOUCH(K, B, kIdentical);    \
        else if (cas == kEdge) BEM_TOUCH(K, B, kEdge);         \
        else BEM_TOUCH(K, B, kVertex);                         \
    } while (0)
    switch (kind) {
    case BEM_LAPLACE_SLP: if (p1) BEM_TOUCH_CASE(BEM_LAPLACE_SLP, BEM_P1); else BEM_TOUCH_CASE(BEM_LAPLACE_SLP, BEM_P0); break;
    case BEM_LAPLACE_DLP: if (p1) BEM_TOUCH_CASE(BEM_LAPLACE_DLP, BEM_P1); else BEM_TOUCH_CASE(BEM_LAPLACE_DLP, BEM_P0); break;
    case BEM_HELMHOLTZ_DLP: if (p1) BEM_TOUCH_CASE(BEM_HELMHOLTZ_DLP, BEM_P1); else BEM_TOUCH_CASE(BEM_HELMHOLTZ_DLP, BEM_P0); break;
    case BEM_HELMHOLTZ_BW: if (p1) BEM_TOUCH_CASE(BEM_HELMHOLTZ_BW, BEM_P1); else BEM_TOUCH_CASE(BEM_HELMHOLTZ_BW, BEM_P0); break;
    default: if (p1) BEM_TOUCH_CASE(BEM_HELMHOLTZ_SLP, BEM_P1); else BEM_TOUCH_CASE(BEM_HELMHOLTZ_SLP, BEM_P0); break;
    }
#undef BEM_TOUCH_CASE
#undef BEM_TOUCH
    return cudaGetLastError();
}

cudaError_t launch_touching_batch(const TouchJob *jobs, int basis, int kind, int cas, int f32,
                                  const int2 *items, int64_t n, const Rule4D &rule, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n + 7) / 8);
    const bool p1 = basis == BEM_P1;
    if (f32 && rule.f && !kind_fp64_only(kind)) {
#define BEM_TVB(K, B)                                                                          \
    do {                                                                                       \
        if (cas == kIdentical) k_touching_f32_batch<kIdentical, K, B><<<blocks, 256, 0, st>>>(jobs, items, n, rule.f, rule.n); \
        else if (cas == kEdge) k_touching_f32_batch<kEdge, K, B><<<blocks, 256, 0, st>>>(jobs, items, n, rule.f, rule.n);      \
        else k_touching_f32_batch<kVertex, K, B><<<blocks, 256, 0, st>>>(jobs, items, n, rule.f, rule.n);                      \
    } while (0)
        if (kind == BEM_LAPLACE_SLP) { if (p1) BEM_TVB(BEM_LAPLACE_SLP, BEM_P1); else BEM_TVB(BEM_LAPLACE_SLP, BEM_P0); }
        else if (kind == BEM_LAPLACE_DLP) { if (p1) BEM_TVB(BEM_LAPLACE_DLP, BEM_P1); else BEM_TVB(BEM_LAPLACE_DLP, BEM_P0); }
        else { if (p1) BEM_TVB(BEM_HELMHOLTZ_SLP, BEM_P1); else BEM_TVB(BEM_HELMHOLTZ_SLP, BEM_P0); }
#undef BEM_TVB
        return cudaGetLastError();
    }
#define BEM_TB(K, B, C) k_touching_batch<K, B, C><<<blocks, 256, 0, st>>>(jobs, items, n, rule.d, rule.n)
#define BEM_TB_CASE(K, B)                                  \
    do {                                                   \
        if (cas == kIdentical) BEM_TB(K, B, kIdentical);   \
        else if (cas == kEdge) BEM_TB(K, B, kEdge);        \
        else BEM_TB(K, B, kVertex);                        \
    } while (0)
    switch (kind) {
    case BEM_LAPLACE_SLP: if (p1) BEM_TB_CASE(BEM_LAPLACE_SLP, BEM_P1); else BEM_TB_CASE(BEM_LAPLACE_SLP, BEM_P0); break;
    case BEM_LAPLACE_DLP: if (p1) BEM_TB_CASE(BEM_LAPLACE_DLP, BEM_P1); else BEM_TB_CASE(BEM_LAPLACE_DLP, BEM_P0); break;
    case BEM_HELMHOLTZ_DLP: if (p1) BEM_TB_CASE(BEM_HELMHOLTZ_DLP, BEM_P1); else BEM_TB_CASE(BEM_HELMHOLTZ_DLP, BEM_P0); break;
    case BEM_HELMHOLTZ_BW: if (p1) BEM_TB_CASE(BEM_HELMHOLTZ_BW, BEM_P1); else BEM_TB_CASE(BEM_HELMHOLTZ_BW, BEM_P0); break;
    default: if (p1) BEM_TB_CASE(BEM_HELMHOLTZ_SLP, BEM_P1); else BEM_TB_CASE(BEM_HELMHOLTZ_SLP, BEM_P0); break;
    }
#undef BEM_TB_CASE
#undef BEM_TB
    return cudaGetLastError();
}

}  // namespace bem
