// Piecewise-linear block engine kernels for one precision (included by
// bem_block_p1_fp64.cu and bem_block_p1_mixed.cu with BEM_P1_MIXED set, so
// that the two heavy instantiation sets compile in parallel).
#include <cuda_runtime.h>

#include "bem_device.cuh"

#ifndef BEM_P1_MIXED
#error "define BEM_P1_MIXED before including this file"
#endif

namespace bem {

template <int KIND, int NP, bool MIXED>
__global__ void __launch_bounds__(p1_threads(MIXED), p1_min_blocks(MIXED))
k_block_p1(MeshView m, BlockLaunch L, Rule2D R, const int64_t *__restrict__ prefix, int *status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t total = L.n_blocks > 0 ? prefix[L.n_blocks - 1] : 0;
    for (int64_t tile = blockIdx.x; tile < total; tile += gridDim.x)
        p1_tile<KIND, NP, MIXED>(m, L, R, prefix, tile, status, smem_raw);
}

template <int KIND, int NP, bool MIXED>
__global__ void __launch_bounds__(p1_threads(MIXED), p1_min_blocks(MIXED))
k_batch_p1(const BatchJob *__restrict__ jobs, int n_jobs, const int64_t *__restrict__ job_end,
           Rule2D R, int *status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int64_t next_tile;
    const int64_t total = n_jobs > 0 ? job_end[n_jobs - 1] : 0;
    // tiles differ in cost (cluster and support sizes): each CTA takes the
    // next tile from the counter job_end[n_jobs] (zeroed before the launch)
    // instead of a fixed stride, so that all SMs finish together
    unsigned long long *counter =
        reinterpret_cast<unsigned long long *>(const_cast<int64_t *>(job_end + n_jobs));
    for (;;) {
        if (threadIdx.x == 0) next_tile = (int64_t)atomicAdd(counter, 1ull);
        __syncthreads();
        const int64_t tile = next_tile;
        __syncthreads();
        if (tile >= total) break;
        const int j = find_job(job_end, n_jobs, tile);
        const int64_t local = tile - (j > 0 ? job_end[j - 1] : 0);
        const BatchJob &J = jobs[j];
        p1_tile<KIND, NP, MIXED>(J.m, J.L, R, J.prefix, local, status, smem_raw);
    }
}

namespace {

template <int KIND, int NP>
cudaError_t single(const MeshView &m, const BlockLaunch &L, const Rule2D &R, const int64_t *prefix,
                   int *status, int grid, cudaStream_t st)
{
    constexpr bool MIXED = BEM_P1_MIXED;
    const size_t sm = p1_smem_bytes(kind_complex(KIND), MIXED, KIND == kFusedLaplace);
    cudaError_t e = cudaFuncSetAttribute(k_block_p1<KIND, NP, MIXED>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_block_p1<KIND, NP, MIXED><<<grid, p1_threads(MIXED), sm, st>>>(m, L, R, prefix, status);
    return cudaGetLastError();
}

template <int KIND, int NP>
cudaError_t batch(const BatchJob *jobs, int n_jobs, const int64_t *job_end, const Rule2D &R,
                  int *status, int grid, cudaStream_t st)
{
    constexpr bool MIXED = BEM_P1_MIXED;
    const size_t sm = p1_smem_bytes(kind_complex(KIND), MIXED, KIND == kFusedLaplace);
    // set once (outside any stream capture: plans issue once before capturing)
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_batch_p1<KIND, NP, MIXED>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    cudaError_t e = cudaMemsetAsync(const_cast<int64_t *>(job_end) + n_jobs, 0, sizeof(int64_t), st);
    if (e != cudaSuccess) return e;
    k_batch_p1<KIND, NP, MIXED><<<grid, p1_threads(MIXED), sm, st>>>(jobs, n_jobs, job_end, R, status);
    return cudaGetLastError();
}

template <int NP>
cudaError_t single_kind(int kind, const MeshView &m, const BlockLaunch &L, const Rule2D &R,
                        const int64_t *prefix, int *status, int grid, cudaStream_t st)
{
    if (kind == BEM_LAPLACE_SLP) return single<BEM_LAPLACE_SLP, NP>(m, L, R, prefix, status, grid, st);
    if (kind == BEM_LAPLACE_DLP) return single<BEM_LAPLACE_DLP, NP>(m, L, R, prefix, status, grid, st);
#if !BEM_P1_MIXED
    if (kind == BEM_HELMHOLTZ_DLP) return single<BEM_HELMHOLTZ_DLP, NP>(m, L, R, prefix, status, grid, st);
    if (kind == BEM_HELMHOLTZ_BW) return single<BEM_HELMHOLTZ_BW, NP>(m, L, R, prefix, status, grid, st);
    return single<BEM_HELMHOLTZ_SLP, NP>(m, L, R, prefix, status, grid, st);
#else
    return cudaErrorInvalidValue;
#endif
}

template <int NP>
cudaError_t batch_kind(int kind, const BatchJob *jobs, int n_jobs, const int64_t *job_end,
                       const Rule2D &R, int *status, int grid, cudaStream_t st)
{
    if (kind == BEM_LAPLACE_SLP) return batch<BEM_LAPLACE_SLP, NP>(jobs, n_jobs, job_end, R, status, grid, st);
    if (kind == BEM_LAPLACE_DLP) return batch<BEM_LAPLACE_DLP, NP>(jobs, n_jobs, job_end, R, status, grid, st);
#if !BEM_P1_MIXED
    if (kind == BEM_HELMHOLTZ_DLP) return batch<BEM_HELMHOLTZ_DLP, NP>(jobs, n_jobs, job_end, R, status, grid, st);
    if (kind == BEM_HELMHOLTZ_BW) return batch<BEM_HELMHOLTZ_BW, NP>(jobs, n_jobs, job_end, R, status, grid, st);
    return batch<BEM_HELMHOLTZ_SLP, NP>(jobs, n_jobs, job_end, R, status, grid, st);
#else
    if (kind == kFusedLaplace) return batch<kFusedLaplace, NP>(jobs, n_jobs, job_end, R, status, grid, st);
    return cudaErrorInvalidValue;
#endif
}

}  // namespace

#if BEM_P1_MIXED
#define BEM_P1_SINGLE launch_p1_single_mixed
#define BEM_P1_BATCH launch_p1_batch_mixed
#else
#define BEM_P1_SINGLE launch_p1_single_fp64
#define BEM_P1_BATCH launch_p1_batch_fp64
#endif

cudaError_t BEM_P1_SINGLE(int kind, int np, const MeshView &m, const BlockLaunch &L, const Rule2D &R,
                          const int64_t *prefix, int *status, int grid, cudaStream_t st)
{
    switch (np) {
    case 4: return single_kind<4>(kind, m, L, R, prefix, status, grid, st);
    case 7: return single_kind<7>(kind, m, L, R, prefix, status, grid, st);
    case 9: return single_kind<9>(kind, m, L, R, prefix, status, grid, st);
    case 16: return single_kind<16>(kind, m, L, R, prefix, status, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t BEM_P1_BATCH(int kind, int np, const BatchJob *jobs, int n_jobs, const int64_t *job_end,
                         const Rule2D &R, int *status, int grid, cudaStream_t st)
{
    switch (np) {
    case 4: return batch_kind<4>(kind, jobs, n_jobs, job_end, R, status, grid, st);
    case 7: return batch_kind<7>(kind, jobs, n_jobs, job_end, R, status, grid, st);
    case 9: return batch_kind<9>(kind, jobs, n_jobs, job_end, R, status, grid, st);
    case 16: return batch_kind<16>(kind, jobs, n_jobs, job_end, R, status, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bem
