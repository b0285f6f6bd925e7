// Touching-pair kernels (Sauter-Schwab rules, Section 2.2): one warp per pair,
// single-mesh and batched forms, FP64 and the float kernels of the mixed forms.
// Rules with xi integrated out (Rule4D::xi, the Laplace kernels, and the
// float Helmholtz single layer with its xi sums) come from the host's choice.
#include <cuda_runtime.h>

#include "bem_device.cuh"

namespace bem {

template <int KIND, int BASIS, int CAS>
__global__ void __launch_bounds__(256) k_touching(MeshView m, const int *__restrict__ list,
                                                  int64_t n, const double *__restrict__ rule,
                                                  int np, double kappa, double eta, int xi)
{
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid >= n) return;
    touch_pair<KIND, BASIS, CAS>(m, __ldg(list + wid), rule, np, kappa, threadIdx.x & 31, eta, xi);
}

// Batched: items[k] = (job, touching index) over many meshes / kernels.
template <int KIND, int BASIS, int CAS>
__global__ void __launch_bounds__(256) k_touching_batch(const TouchJob *__restrict__ jobs,
                                                        const int2 *__restrict__ items, int64_t n,
                                                        const double *__restrict__ rule, int np,
                                                        int xi)
{
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid >= n) return;
    const int2 it = items[wid];
    touch_pair<KIND, BASIS, CAS>(jobs[it.x].m, it.y, rule, np, jobs[it.x].kappa, threadIdx.x & 31,
                                 jobs[it.x].eta, xi);
}

// Float kernels: a pair per group of LPP lanes (touch_f32).  The first group
// of a warp decides whether the warp has work, so every lane of a working
// warp takes part in the group reductions.
template <int CAS, int KIND, int BASIS, int LPP>
__global__ void __launch_bounds__(256) k_touching_f32(MeshView m, const int *__restrict__ list,
                                                      int64_t n, const float *__restrict__ rule,
                                                      int np, float kappa, int xi, XiRule xr)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t g = t / LPP;
    if ((t >> 5) * (32 / LPP) >= n) return;   // the warp's first group
    const bool valid = g < n;
    touch_f32<CAS, KIND, BASIS, LPP>(m, __ldg(list + (valid ? g : n - 1)), rule, np,
                                     (int)(t % LPP), kappa, xi, xr, valid);
}

template <int CAS, int KIND, int BASIS, int LPP>
__global__ void __launch_bounds__(256) k_touching_f32_batch(const TouchJob *__restrict__ jobs,
                                                            const int2 *__restrict__ items,
                                                            int64_t n,
                                                            const float *__restrict__ rule, int np,
                                                            int xi, XiRule xr)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t g = t / LPP;
    if ((t >> 5) * (32 / LPP) >= n) return;
    const bool valid = g < n;
    const int2 it = items[valid ? g : n - 1];
    touch_f32<CAS, KIND, BASIS, LPP>(jobs[it.x].m, it.y, rule, np, (int)(t % LPP),
                                     (float)jobs[it.x].kappa, xi, xr, valid);
}

// Lanes per pair of the float kernels: the xi-integrated Laplace rules are
// short (q^3 points per subdomain), the Helmholtz xi sums cost a few sines
// per point, the q^4 rules fill a warp.  Every lane of a group repeats the
// pair's set-up, so the shorter rules take fewer lanes.
static int lanes_per_pair(const Rule4D &rule, int kind, int basis)
{
    if (!rule.xi) return 32;
    if (basis == BEM_P1) return 16;
    return kind_complex(kind) ? 8 : 4;
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
        XiRule xr;
        if (rule.xi && kind == BEM_HELMHOLTZ_SLP && !make_xi_rule(rule.q, xr)) return cudaErrorInvalidValue;
#define BEM_TVL(K, B, LP)                                                                       \
    do {                                                                                        \
        const unsigned g = (unsigned)((n + 8 * (32 / LP) - 1) / (8 * (32 / LP)));               \
        if (cas == kIdentical) k_touching_f32<kIdentical, K, B, LP><<<g, 256, 0, st>>>(m, list, n, rule.f, rule.n, kf, rule.xi, xr); \
        else if (cas == kEdge) k_touching_f32<kEdge, K, B, LP><<<g, 256, 0, st>>>(m, list, n, rule.f, rule.n, kf, rule.xi, xr);      \
        else k_touching_f32<kVertex, K, B, LP><<<g, 256, 0, st>>>(m, list, n, rule.f, rule.n, kf, rule.xi, xr);                      \
    } while (0)
#define BEM_TV(K, B)                                                                            \
    do {                                                                                        \
        const int lp = lanes_per_pair(rule, K, B);                                              \
        if (lp == 4) BEM_TVL(K, B, (B == BEM_P0 ? 4 : 16));                                         \
        else if (lp == 8) BEM_TVL(K, B, (B == BEM_P0 ? 8 : 16));                                    \
        else if (lp == 16) BEM_TVL(K, B, 16);                                                   \
        else BEM_TVL(K, B, 32);                                                                 \
    } while (0)
        if (kind == BEM_LAPLACE_SLP) { if (p1) BEM_TV(BEM_LAPLACE_SLP, BEM_P1); else BEM_TV(BEM_LAPLACE_SLP, BEM_P0); }
        else if (kind == BEM_LAPLACE_DLP) { if (p1) BEM_TV(BEM_LAPLACE_DLP, BEM_P1); else BEM_TV(BEM_LAPLACE_DLP, BEM_P0); }
        else { if (p1) BEM_TV(BEM_HELMHOLTZ_SLP, BEM_P1); else BEM_TV(BEM_HELMHOLTZ_SLP, BEM_P0); }
#undef BEM_TV
#undef BEM_TVL
        return cudaGetLastError();
    }
#define BEM_TOUCH(K, B, C) k_touching<K, B, C><<<blocks, 256, 0, st>>>(m, list, n, rule.d, rule.n, kappa, eta, rule.xi)
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
        XiRule xr;
        if (rule.xi && kind == BEM_HELMHOLTZ_SLP && !make_xi_rule(rule.q, xr)) return cudaErrorInvalidValue;
#define BEM_TVBL(K, B, LP)                                                                      \
    do {                                                                                        \
        const unsigned g = (unsigned)((n + 8 * (32 / LP) - 1) / (8 * (32 / LP)));               \
        if (cas == kIdentical) k_touching_f32_batch<kIdentical, K, B, LP><<<g, 256, 0, st>>>(jobs, items, n, rule.f, rule.n, rule.xi, xr); \
        else if (cas == kEdge) k_touching_f32_batch<kEdge, K, B, LP><<<g, 256, 0, st>>>(jobs, items, n, rule.f, rule.n, rule.xi, xr);      \
        else k_touching_f32_batch<kVertex, K, B, LP><<<g, 256, 0, st>>>(jobs, items, n, rule.f, rule.n, rule.xi, xr);                      \
    } while (0)
#define BEM_TVB(K, B)                                                                           \
    do {                                                                                        \
        const int lp = lanes_per_pair(rule, K, B);                                              \
        if (lp == 4) BEM_TVBL(K, B, (B == BEM_P0 ? 4 : 16));                                        \
        else if (lp == 8) BEM_TVBL(K, B, (B == BEM_P0 ? 8 : 16));                                   \
        else if (lp == 16) BEM_TVBL(K, B, 16);                                                  \
        else BEM_TVBL(K, B, 32);                                                                \
    } while (0)
        if (kind == BEM_LAPLACE_SLP) { if (p1) BEM_TVB(BEM_LAPLACE_SLP, BEM_P1); else BEM_TVB(BEM_LAPLACE_SLP, BEM_P0); }
        else if (kind == BEM_LAPLACE_DLP) { if (p1) BEM_TVB(BEM_LAPLACE_DLP, BEM_P1); else BEM_TVB(BEM_LAPLACE_DLP, BEM_P0); }
        else { if (p1) BEM_TVB(BEM_HELMHOLTZ_SLP, BEM_P1); else BEM_TVB(BEM_HELMHOLTZ_SLP, BEM_P0); }
#undef BEM_TVB
#undef BEM_TVBL
        return cudaGetLastError();
    }
#define BEM_TB(K, B, C) k_touching_batch<K, B, C><<<blocks, 256, 0, st>>>(jobs, items, n, rule.d, rule.n, rule.xi)
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
