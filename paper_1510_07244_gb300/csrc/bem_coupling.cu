// Coupling-block engine for the piecewise-linear basis, mixed form (Laplace
// kernels).  Coupling blocks G|t~ x s~ (Section 2.4) hold entries between
// pivot vertices of admissible cluster pairs, so every pair of support
// triangles is disjoint and the supports of different pivots rarely share a
// triangle: the shared-triangle reuse of the near-field tile engine buys
// nothing here, while its nine-moment pair results, shared-memory gather and
// barriers cost a lot.  This engine gives every lane one entry g_ij and sums
// over supp(phi_i) x supp(psi_j) directly, with only the one basis product
// lambda_i(x) lambda_j(y) of that entry:
//     g_ij = 1/(4 pi) sum_{A in supp i} sum_{B in supp j} sqrt(g_A g_B)
//            sum_p w_p lambda_i(x_p) sum_q w_q lambda_j(y_q) k(x_p - y_q)
// (Eq. 1 with the product rule of Section 2.2).  A warp takes a tile of 16
// rows x 2 columns of one block, so each half-warp shares its column index
// and walks supp(j) in lockstep.  Pair sums are float; the sum over pairs is
// Kahan-compensated.  A pair of support triangles that touches means the block
// was not admissible: the entry is set to 0 and the status word gets
// BEM_ERR_INVALID_ARG, as in the near-field engine without a touching table.
#include <cuda_runtime.h>

#include "bem_device.cuh"

namespace bem {

namespace {

constexpr int kCouplingThreads = 256;

// Sum over the product rule of one disjoint pair for the basis functions at
// local vertices la (test) and the precomputed trial side (yx, yy, yz, wy).
template <int KIND, int NP>
__device__ __forceinline__ float coupling_pair(const TriF &A, const TriF &B, int la,
                                               const Rule2D &R, const float *yx, const float *yy,
                                               const float *yz, const float *wy)
{
    float d0[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) d0[c] = dd_diff(A.vh[0][c], A.vl[0][c], B.vh[0][c], B.vl[0][c]);
    Height H = {};
    if (KIND == BEM_LAPLACE_DLP)
        H = make_height(A.vh[0], A.vl[0], A.vh[1], A.vl[1], A.vh[2], A.vl[2], B.vh[0], B.vl[0],
                        B.nh, B.nl);
    float sum = 0.0f;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const float s = R.sf[i], t = R.tf[i];
        const float xx = fmaf(s, A.e1[0], fmaf(t, A.e2[0], d0[0]));
        const float xy = fmaf(s, A.e1[1], fmaf(t, A.e2[1], d0[1]));
        const float xz = fmaf(s, A.e1[2], fmaf(t, A.e2[2], d0[2]));
        const float dn = KIND == BEM_LAPLACE_DLP ? height_at_far(H, s, t) : 0.0f;
        float inner = 0.0f;
#pragma unroll
        for (int j = 0; j < NP; ++j)
            inner = fmaf(wy[j], kvalf_r<KIND>(xx - yx[j], xy - yy[j], xz - yz[j]), inner);
        if (KIND == BEM_LAPLACE_DLP) inner *= dn;
        const float wx = la == 0 ? R.wl[0][i] : (la == 1 ? R.wl[1][i] : R.wl[2][i]);
        sum = fmaf(wx, inner, sum);
    }
    return sum;
}

// Both layers of one pair at once: the single-layer sum is computed exactly as
// coupling_pair<SLP> does and the double-layer sum exactly as coupling_pair<DLP>
// does, sharing the points, the distances and the reciprocal square roots.
template <int NP>
__device__ __forceinline__ void coupling_pair2(const TriF &A, const TriF &B, int la, const Rule2D &R,
                                               const float *yx, const float *yy, const float *yz,
                                               const float *wy, float &out_s, float &out_d)
{
    float d0[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) d0[c] = dd_diff(A.vh[0][c], A.vl[0][c], B.vh[0][c], B.vl[0][c]);
    const Height H = make_height(A.vh[0], A.vl[0], A.vh[1], A.vl[1], A.vh[2], A.vl[2], B.vh[0],
                                 B.vl[0], B.nh, B.nl);
    float sum_s = 0.0f, sum_d = 0.0f;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const float s = R.sf[i], t = R.tf[i];
        const float xx = fmaf(s, A.e1[0], fmaf(t, A.e2[0], d0[0]));
        const float xy = fmaf(s, A.e1[1], fmaf(t, A.e2[1], d0[1]));
        const float xz = fmaf(s, A.e1[2], fmaf(t, A.e2[2], d0[2]));
        const float dn = height_at_far(H, s, t);
        float in_s = 0.0f, in_d = 0.0f;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            const float dx = xx - yx[j], dy = xy - yy[j], dz = xz - yz[j];
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float ri = rsqrt_fast(r2);
            in_s = fmaf(wy[j], ri, in_s);
            in_d = fmaf(wy[j], ri * ri * ri, in_d);
        }
        in_d *= dn;
        const float wx = la == 0 ? R.wl[0][i] : (la == 1 ? R.wl[1][i] : R.wl[2][i]);
        sum_s = fmaf(wx, in_s, sum_s);
        sum_d = fmaf(wx, in_d, sum_d);
    }
    out_s = sum_s;
    out_d = sum_d;
}

__device__ __forceinline__ int local_of(int4 tv, int v) { return tv.x == v ? 0 : (tv.y == v ? 1 : 2); }

// One 16 x 2 tile of one block list, one entry per lane.
template <int KIND, int NP>
__device__ __forceinline__ void coupling_tile(const MeshView &m, const BlockLaunch &L,
                                              const Rule2D &R, const int64_t *__restrict__ prefix,
                                              int64_t tile, int lane, int *status)
{
    const BlockInfo bi = block_info(L, prefix, tile, status);
    if (!bi.ok) return;   // uniform across the warp
    const int ntr = (bi.nr + kCouplingRows - 1) / kCouplingRows;
    const int er = (bi.tile_in_blk % ntr) * kCouplingRows + (lane & (kCouplingRows - 1));
    const int ec = (bi.tile_in_blk / ntr) * kCouplingCols + lane / kCouplingRows;
    if (er >= bi.nr || ec >= bi.nc) return;
    const int i = __ldg(L.row_idx + bi.r_lo + er), j = __ldg(L.col_idx + bi.c_lo + ec);
    double *out = reinterpret_cast<double *>(L.out) + bi.off + er + (int64_t)ec * bi.nr;
    if (i < 0 || i >= m.nv || j < 0 || j >= m.nv) {
        set_status(status, BEM_ERR_INVALID_ARG);
        *out = 0.0;
        return;
    }
    const int alo = __ldg(m.vt_ptr + i), ahi = __ldg(m.vt_ptr + i + 1);
    const int blo = __ldg(m.vt_ptr + j), bhi = __ldg(m.vt_ptr + j + 1);
    float acc = 0.0f, cmp = 0.0f;
    bool touched = false;
    for (int kb = blo; kb < bhi; ++kb) {
        const int b = __ldg(m.vt_tri + kb);
        const int4 vb = __ldg(m.tvid + b);
        const int lb = local_of(vb, j);
        TriF B;
        load_trif(m.geomf, b, B);
        // trial side of the product rule, relative to B's vertex 0
        float yx[NP], yy[NP], yz[NP], wy[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const float s = R.sf[q], t = R.tf[q];
            yx[q] = fmaf(s, B.e1[0], t * B.e2[0]);
            yy[q] = fmaf(s, B.e1[1], t * B.e2[1]);
            yz[q] = fmaf(s, B.e1[2], t * B.e2[2]);
            wy[q] = lb == 0 ? R.wl[0][q] : (lb == 1 ? R.wl[1][q] : R.wl[2][q]);
        }
        for (int ka = alo; ka < ahi; ++ka) {
            const int a = __ldg(m.vt_tri + ka);
            const int4 va = __ldg(m.tvid + a);
            if (touching(va, vb)) {
                touched = true;
                continue;
            }
            TriF A;
            load_trif(m.geomf, a, A);
            const float p = coupling_pair<KIND, NP>(A, B, local_of(va, i), R, yx, yy, yz, wy) *
                            (A.sg * B.sg);
            const float y = p - cmp;
            const float t = acc + y;
            cmp = (t - acc) - y;
            acc = t;
        }
    }
    if (touched) {
        set_status(status, BEM_ERR_INVALID_ARG);
        *out = 0.0;
        return;
    }
    *out = ((double)acc - (double)cmp) * kInv4Pi;
}

// One 16 x 2 tile of a fused job: single layer into L.out, double layer into L.out2.
template <int NP>
__device__ __forceinline__ void coupling_tile_fused(const MeshView &m, const BlockLaunch &L,
                                                    const Rule2D &R,
                                                    const int64_t *__restrict__ prefix,
                                                    int64_t tile, int lane, int *status)
{
    const BlockInfo bi = block_info(L, prefix, tile, status);
    if (!bi.ok) return;   // uniform across the warp
    const int ntr = (bi.nr + kCouplingRows - 1) / kCouplingRows;
    const int er = (bi.tile_in_blk % ntr) * kCouplingRows + (lane & (kCouplingRows - 1));
    const int ec = (bi.tile_in_blk / ntr) * kCouplingCols + lane / kCouplingRows;
    if (er >= bi.nr || ec >= bi.nc) return;
    const int i = __ldg(L.row_idx + bi.r_lo + er), j = __ldg(L.col_idx + bi.c_lo + ec);
    const int64_t o = bi.off + er + (int64_t)ec * bi.nr;
    double *out_s = reinterpret_cast<double *>(L.out) + o;
    double *out_d = reinterpret_cast<double *>(L.out2) + o;
    if (i < 0 || i >= m.nv || j < 0 || j >= m.nv) {
        set_status(status, BEM_ERR_INVALID_ARG);
        *out_s = *out_d = 0.0;
        return;
    }
    const int alo = __ldg(m.vt_ptr + i), ahi = __ldg(m.vt_ptr + i + 1);
    const int blo = __ldg(m.vt_ptr + j), bhi = __ldg(m.vt_ptr + j + 1);
    float acc_s = 0.0f, cmp_s = 0.0f, acc_d = 0.0f, cmp_d = 0.0f;
    bool touched = false;
    for (int kb = blo; kb < bhi; ++kb) {
        const int b = __ldg(m.vt_tri + kb);
        const int4 vb = __ldg(m.tvid + b);
        const int lb = local_of(vb, j);
        TriF B;
        load_trif(m.geomf, b, B);
        float yx[NP], yy[NP], yz[NP], wy[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const float s = R.sf[q], t = R.tf[q];
            yx[q] = fmaf(s, B.e1[0], t * B.e2[0]);
            yy[q] = fmaf(s, B.e1[1], t * B.e2[1]);
            yz[q] = fmaf(s, B.e1[2], t * B.e2[2]);
            wy[q] = lb == 0 ? R.wl[0][q] : (lb == 1 ? R.wl[1][q] : R.wl[2][q]);
        }
        for (int ka = alo; ka < ahi; ++ka) {
            const int a = __ldg(m.vt_tri + ka);
            const int4 va = __ldg(m.tvid + a);
            if (touching(va, vb)) {
                touched = true;
                continue;
            }
            TriF A;
            load_trif(m.geomf, a, A);
            float ps, pd;
            coupling_pair2<NP>(A, B, local_of(va, i), R, yx, yy, yz, wy, ps, pd);
            const float sg = A.sg * B.sg;
            float y = ps * sg - cmp_s, t = acc_s + y;
            cmp_s = (t - acc_s) - y;
            acc_s = t;
            y = pd * sg - cmp_d;
            t = acc_d + y;
            cmp_d = (t - acc_d) - y;
            acc_d = t;
        }
    }
    if (touched) {
        set_status(status, BEM_ERR_INVALID_ARG);
        *out_s = *out_d = 0.0;
        return;
    }
    *out_s = ((double)acc_s - (double)cmp_s) * kInv4Pi;
    *out_d = ((double)acc_d - (double)cmp_d) * kInv4Pi;
}

template <int NP>
__global__ void __launch_bounds__(kCouplingThreads)
k_coupling_p1_fused_batch(const BatchJob *__restrict__ jobs, int n_jobs,
                          const int64_t *__restrict__ job_end, Rule2D R, int *status)
{
    const int64_t total = n_jobs > 0 ? job_end[n_jobs - 1] : 0;
    const int64_t warps = (int64_t)gridDim.x * (kCouplingThreads / 32);
    const int lane = threadIdx.x & 31;
    for (int64_t tile = ((int64_t)blockIdx.x * kCouplingThreads + threadIdx.x) >> 5; tile < total;
         tile += warps) {
        const int jb = find_job(job_end, n_jobs, tile);
        const int64_t local = tile - (jb > 0 ? job_end[jb - 1] : 0);
        const BatchJob &J = jobs[jb];
        coupling_tile_fused<NP>(J.m, J.L, R, J.prefix, local, lane, status);
    }
}

template <int KIND, int NP>
__global__ void __launch_bounds__(kCouplingThreads)
k_coupling_p1(MeshView m, BlockLaunch L, Rule2D R, const int64_t *__restrict__ prefix, int *status)
{
    const int64_t total = L.n_blocks > 0 ? prefix[L.n_blocks - 1] : 0;
    const int64_t warps = (int64_t)gridDim.x * (kCouplingThreads / 32);
    const int lane = threadIdx.x & 31;
    for (int64_t tile = ((int64_t)blockIdx.x * kCouplingThreads + threadIdx.x) >> 5; tile < total;
         tile += warps)
        coupling_tile<KIND, NP>(m, L, R, prefix, tile, lane, status);
}

template <int KIND, int NP>
__global__ void __launch_bounds__(kCouplingThreads)
k_coupling_p1_batch(const BatchJob *__restrict__ jobs, int n_jobs,
                    const int64_t *__restrict__ job_end, Rule2D R, int *status)
{
    const int64_t total = n_jobs > 0 ? job_end[n_jobs - 1] : 0;
    const int64_t warps = (int64_t)gridDim.x * (kCouplingThreads / 32);
    const int lane = threadIdx.x & 31;
    for (int64_t tile = ((int64_t)blockIdx.x * kCouplingThreads + threadIdx.x) >> 5; tile < total;
         tile += warps) {
        const int jb = find_job(job_end, n_jobs, tile);
        const int64_t local = tile - (jb > 0 ? job_end[jb - 1] : 0);
        const BatchJob &J = jobs[jb];
        coupling_tile<KIND, NP>(J.m, J.L, R, J.prefix, local, lane, status);
    }
}

template <int KIND>
cudaError_t single_kind(const MeshView &m, const BlockLaunch &L, const Rule2D &R,
                        const int64_t *prefix, int *status, int grid, cudaStream_t st)
{
    switch (R.np) {
    case 4: k_coupling_p1<KIND, 4><<<grid, kCouplingThreads, 0, st>>>(m, L, R, prefix, status); break;
    case 7: k_coupling_p1<KIND, 7><<<grid, kCouplingThreads, 0, st>>>(m, L, R, prefix, status); break;
    case 9: k_coupling_p1<KIND, 9><<<grid, kCouplingThreads, 0, st>>>(m, L, R, prefix, status); break;
    case 16: k_coupling_p1<KIND, 16><<<grid, kCouplingThreads, 0, st>>>(m, L, R, prefix, status); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int KIND>
cudaError_t batch_kind(const BatchJob *jobs, int n_jobs, const int64_t *job_end, const Rule2D &R,
                       int *status, int grid, cudaStream_t st)
{
#define BEM_CB(NP) k_coupling_p1_batch<KIND, NP><<<grid, kCouplingThreads, 0, st>>>(jobs, n_jobs, job_end, R, status)
    switch (R.np) {
    case 4: BEM_CB(4); break;
    case 7: BEM_CB(7); break;
    case 9: BEM_CB(9); break;
    case 16: BEM_CB(16); break;
    default: return cudaErrorInvalidValue;
    }
#undef BEM_CB
    return cudaGetLastError();
}

}  // namespace

bool use_coupling_engine(int basis, int kind, int mixed, int allow_touching)
{
    return basis == BEM_P1 && mixed && !allow_touching &&
           (kind == BEM_LAPLACE_SLP || kind == BEM_LAPLACE_DLP);
}

cudaError_t launch_coupling_p1(const MeshView &m, const BlockLaunch &L, const Rule2D &R,
                               const int64_t *prefix, int *status, int grid, cudaStream_t st)
{
    if (L.n_blocks <= 0) return cudaSuccess;
    return L.kind == BEM_LAPLACE_SLP
               ? single_kind<BEM_LAPLACE_SLP>(m, L, R, prefix, status, grid, st)
               : single_kind<BEM_LAPLACE_DLP>(m, L, R, prefix, status, grid, st);
}

cudaError_t launch_coupling_p1_fused_batch(const BatchJob *jobs, int n_jobs,
                                           const int64_t *job_end, const Rule2D &R, int *status,
                                           int grid, cudaStream_t st)
{
    if (n_jobs <= 0) return cudaSuccess;
#define BEM_CF(NP) k_coupling_p1_fused_batch<NP><<<grid, kCouplingThreads, 0, st>>>(jobs, n_jobs, job_end, R, status)
    switch (R.np) {
    case 4: BEM_CF(4); break;
    case 7: BEM_CF(7); break;
    case 9: BEM_CF(9); break;
    case 16: BEM_CF(16); break;
    default: return cudaErrorInvalidValue;
    }
#undef BEM_CF
    return cudaGetLastError();
}

cudaError_t launch_coupling_p1_batch(const BatchJob *jobs, int n_jobs, const int64_t *job_end,
                                     int kind, const Rule2D &R, int *status, int grid,
                                     cudaStream_t st)
{
    if (n_jobs <= 0) return cudaSuccess;
    return kind == BEM_LAPLACE_SLP
               ? batch_kind<BEM_LAPLACE_SLP>(jobs, n_jobs, job_end, R, status, grid, st)
               : batch_kind<BEM_LAPLACE_DLP>(jobs, n_jobs, job_end, R, status, grid, st);
}

}  // namespace bem
