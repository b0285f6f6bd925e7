// sm_103a kernels of the Galerkin quadrature path, FP64 form.
//
//  k_touching      one warp per touching triangle pair (Sauter-Schwab rules,
//                  Section 2.2): lanes stride the q^4 * n_sub points of the
//                  case's rule, warp-shuffle reduction, result stored in the
//                  mesh's touching table in the ORIGINAL local vertex order.
//  k_block_p0/p1   block engine for near-field, coupling and dense blocks
//                  (Section 2.3 blocks t x s; Section 3 per-case lists are
//                  replaced by classifying each pair on the fly): one CTA per
//                  tile (P1: 32 x 32 of a block; P0: 256 consecutive entries
//                  of the list), one thread per disjoint triangle pair
//                  (product rule of a 2D triangle rule, Section 2.2 Duffy),
//                  touching pairs read from the touching table.
//  k_pivot         one warp per requested entry g_ij (pivot rows/columns).
//
// Kernel values (Eq. 2): laplace 1/(4 pi r), double layer (x-y).n_y/(4 pi r^3),
// helmholtz exp(i kappa r)/(4 pi r).  sqrt(g_a g_b)/(4 pi) is applied once per
// pair.
#include <cuda_runtime.h>

#include "bem_device.cuh"

namespace bem {

// Tiles per block of blocks [first, end) -> inclusive prefix sums from `first`
// (one CTA, a contiguous run of blocks per thread).
__device__ void tile_prefix_range(const BlockLaunch &L, int tr, int tc, int64_t *prefix,
                                  int *status, int64_t *total, int64_t first, int64_t end)
{
    __shared__ int64_t part[1024];
    const int64_t n = end - first;
    const int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
    const int64_t lo = first + threadIdx.x * chunk, hi = min(end, lo + chunk);
    int64_t sum = 0;
    // U blocks at a time: their cluster and size loads do not depend on one
    // another, so they are in flight together
    constexpr int U = 8;
    for (int64_t b0 = lo; b0 < hi; b0 += U) {
        int t[U], s[U], nr[U], nc[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool in = b0 + u < hi;
            t[u] = in ? L.blk_row[b0 + u] : 0;
            s[u] = in ? L.blk_col[b0 + u] : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ok[u] = b0 + u < hi && t[u] >= 0 && t[u] < L.n_row_clusters && s[u] >= 0 &&
                    s[u] < L.n_col_clusters;
            nr[u] = ok[u] ? L.row_ptr[t[u] + 1] - L.row_ptr[t[u]] : 0;
            nc[u] = ok[u] ? L.col_ptr[s[u] + 1] - L.col_ptr[s[u]] : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (b0 + u >= hi) break;
            int64_t tiles = 0;
            if (!ok[u] || nr[u] < 0 || nc[u] < 0) set_status(status, BEM_ERR_INVALID_ARG);
            else tiles = (int64_t)((nr[u] + tr - 1) / tr) * ((nc[u] + tc - 1) / tc);
            sum += tiles;
            prefix[b0 + u] = sum;   // local inclusive sum, fixed below
        }
    }
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        int64_t v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    const int64_t base = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0;
    for (int64_t b = lo; b < hi; ++b) prefix[b] += base;
    if (total && threadIdx.x == blockDim.x - 1) *total = part[threadIdx.x];
    __syncthreads();
}

// Tiles per block -> inclusive prefix sums (single CTA).
__device__ void tile_prefix_cta(const BlockLaunch &L, int tr, int tc, int64_t *prefix,
                                int *status, int64_t *total)
{
    tile_prefix_range(L, tr, tc, prefix, status, total, 0, L.n_blocks);
}

__global__ void __launch_bounds__(1024) k_tile_prefix(BlockLaunch L, int tr, int tc,
                                                      int64_t *prefix, int *status)
{
    tile_prefix_cta(L, tr, tc, prefix, status, nullptr);
}

// one CTA per job: per-job block prefix sums and the job's tile total
__global__ void __launch_bounds__(1024) k_tile_prefix_batch(BatchJob *jobs, int tr, int tc,
                                                            int64_t *job_total, int *status)
{
    BatchJob &J = jobs[blockIdx.x];
    tile_prefix_cta(J.L, tr, tc, const_cast<int64_t *>(J.prefix), status, job_total + blockIdx.x);
}

// inclusive scan of the job totals in tiles of `unit` (single CTA): the
// piecewise-constant engine counts entries per job, kP0Tile to a tile
__global__ void __launch_bounds__(1024) k_job_scan(const int64_t *job_total, int n, int unit,
                                                   int64_t *job_end)
{
    __shared__ int64_t part[1024];
    const int chunk = (n + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * chunk, hi = min(n, lo + chunk);
    int64_t sum = 0;
    for (int k = lo; k < hi; ++k) {
        sum += (job_total[k] + unit - 1) / unit;
        job_end[k] = sum;
    }
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        int64_t v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    const int64_t base = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0;
    for (int k = lo; k < hi; ++k) job_end[k] += base;
}

// The float form is capped at 64 registers (four CTAs, 32 warps per SM): the
// tiles' dependent loads (block, cluster, index, geometry) want the warps.
template <int KIND, int NP, bool MIXED>
__global__ void __launch_bounds__(256, MIXED ? 4 : 1) k_block_p0(MeshView m, BlockLaunch L, Rule2D R,
                                                  const int64_t *__restrict__ prefix,
                                                  int *status)
{
    // prefix counts entries; a tile is kP0Tile of them.  Each CTA takes a
    // contiguous run of tiles, so every warp finds its next tile's blocks
    // from the previous one's (flat_entry's hint).
    const int64_t total = L.n_blocks > 0 ? (prefix[L.n_blocks - 1] + kP0Tile - 1) / kP0Tile : 0;
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * per, t1 = min(total, t0 + per);
    int64_t hint = -1;
    for (int64_t tile = t0; tile < t1; ++tile)
        p0_tile<KIND, NP, MIXED>(m, L, R, prefix, tile, status, hint);
}

// ---------------------------------------------------------------------------
// Batched (persistent) block engine: one launch drains the tiles of many
// block lists (jobs) that share kernel, basis, rule and precision, e.g. the
// near-field and coupling blocks of many meshes.  job_end[j] = tiles of jobs
// 0..j (inclusive); every tile finds its job by binary search and runs the
// same tile body as the single-list kernels, so the results are identical.
// ---------------------------------------------------------------------------
template <int KIND, int NP, bool MIXED>
__global__ void __launch_bounds__(256, MIXED ? 4 : 1) k_batch_p0(const BatchJob *__restrict__ jobs, int n_jobs,
                                                  const int64_t *__restrict__ job_end, Rule2D R,
                                                  int *status)
{
    // contiguous runs of tiles per CTA (see k_block_p0); the block hint is
    // kept while the run stays in one job
    const int64_t total = n_jobs > 0 ? job_end[n_jobs - 1] : 0;
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * per, t1 = min(total, t0 + per);
    int64_t hint = -1;
    int jprev = -1;
    for (int64_t tile = t0; tile < t1; ++tile) {
        const int j = find_job(job_end, n_jobs, tile);
        if (j != jprev) {
            hint = -1;
            jprev = j;
        }
        const int64_t local = tile - (j > 0 ? job_end[j - 1] : 0);
        const BatchJob &J = jobs[j];
        p0_tile<KIND, NP, MIXED>(J.m, J.L, R, J.prefix, local, status, hint);
    }
}

// ---------------------------------------------------------------------------
// Support records of the piecewise-linear tile engine, built once per run for
// every 32-index slice of a cluster list with the same p1_support the tiles
// run otherwise (identical records, so identical results).
// ---------------------------------------------------------------------------
// slice[c] = sum over clusters before c of ceil(|c| / 32); slice[n] = total
__global__ void __launch_bounds__(1024) k_slice_prefix(const int32_t *__restrict__ ptr, int32_t n,
                                                       int32_t *slice, int *status)
{
    __shared__ int32_t part[1024];
    const int32_t chunk = (n + blockDim.x - 1) / blockDim.x;
    const int32_t lo = min(n, (int32_t)threadIdx.x * chunk), hi = min(n, lo + chunk);
    int32_t sum = 0;
    for (int32_t c = lo; c < hi; ++c) {
        const int32_t size = ptr[c + 1] - ptr[c];
        if (size < 0) set_status(status, BEM_ERR_INVALID_ARG);
        slice[c] = sum;   // local exclusive sum, offset below
        sum += size > 0 ? (size + kTile - 1) / kTile : 0;
    }
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        const int32_t v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    const int32_t base = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0;
    for (int32_t c = lo; c < hi; ++c) slice[c] += base;
    if (threadIdx.x == blockDim.x - 1) slice[n] = part[threadIdx.x];
}

struct SupBuildSmem {
    int rows[kTile];
    int tri[kP1MaxTri];
    int cnt[kTile], off[kTile];
    int lists[kMaxDegP1][kTile];
    int list_n[kTile];
    int ntri, bad;
};

__global__ void __launch_bounds__(128) k_build_supports(MeshView m, const int32_t *__restrict__ ptr,
                                                        const int32_t *__restrict__ idx,
                                                        int32_t n_clusters,
                                                        const int32_t *__restrict__ slice,
                                                        int32_t *sup, int64_t cap, int *status)
{
    __shared__ SupBuildSmem S;
    const int tid = threadIdx.x;
    const int64_t total = slice[n_clusters];
    for (int64_t sl = blockIdx.x; sl < total; sl += gridDim.x) {
        if (sl >= cap) {
            if (tid == 0) set_status(status, BEM_ERR_INVALID_ARG);
            break;
        }
        // cluster of this slice: the last c with slice[c] <= sl
        int lo = 0, hi = n_clusters - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (slice[mid] <= sl) lo = mid;
            else hi = mid - 1;
        }
        const int c = lo;
        const int r0 = (int)(sl - slice[c]) * kTile;
        const int n = min(kTile, ptr[c + 1] - ptr[c] - r0);
        int32_t *rec = sup + sl * kSupInts;
        if (tid == 0) S.bad = 0;
        __syncthreads();
        if (tid < n) {
            const int v = idx[ptr[c] + r0 + tid];
            if (v < 0 || v >= m.nv) S.bad = 1;
            S.rows[tid] = v;
        }
        __syncthreads();
        if (S.bad) {
            if (tid == 0) {
                rec[kSupCount] = -1;
                set_status(status, BEM_ERR_INVALID_ARG);
            }
            __syncthreads();
            continue;
        }
        p1_support(m, S.rows, n, S.tri, S.cnt, S.off, S.lists, S.list_n, &S.ntri, status);
        for (int k = tid; k < kTile; k += blockDim.x) rec[kSupListN + k] = k < n ? S.list_n[k] : 0;
        for (int k = tid; k < kMaxDegP1 * kTile; k += blockDim.x)
            rec[kSupLists + k] = (&S.lists[0][0])[k];
        for (int k = tid; k < S.ntri; k += blockDim.x) rec[kSupTris + k] = S.tri[k];
        if (tid == 0) rec[kSupCount] = S.ntri;
        __syncthreads();
    }
}

cudaError_t launch_build_supports(const MeshView &m, const int32_t *ptr, const int32_t *idx,
                                  int32_t n_clusters, int32_t *slice, int32_t *sup, int64_t cap,
                                  int *status, int grid, cudaStream_t st)
{
    if (n_clusters <= 0) return cudaSuccess;
    k_slice_prefix<<<1, 1024, 0, st>>>(ptr, n_clusters, slice, status);
    k_build_supports<<<grid, 128, 0, st>>>(m, ptr, idx, n_clusters, slice, sup, cap, status);
    return cudaGetLastError();
}

size_t p1_smem_bytes(bool cplx, bool mixed, bool fused)
{
    // header, pair results of one chunk, staging sums (one or two results each)
    return ((sizeof(P1Smem) + 15) & ~size_t(15)) +
           ((size_t)p1_cap(mixed, fused) * 9 + (size_t)p1_chunk_rows(mixed, fused) * kP1StageLd * 3) *
               (mixed ? sizeof(float) : sizeof(double)) * (cplx || fused ? 2 : 1);
}

// ---------------------------------------------------------------------------
// Arbitrary entries: one warp per entry, lanes stride the points of each pair's rule.
// ---------------------------------------------------------------------------
// ABS: sum of the magnitudes of the quadrature terms instead of the terms
// (the forward-error scale of the sum), written as a real value.
template <int KIND, bool ABS>
__global__ void __launch_bounds__(256) k_pivot(MeshView m, const int32_t *__restrict__ rows,
                                               const int32_t *__restrict__ cols, int64_t n,
                                               void *out, RuleSet rs, double kappa, int *status,
                                               double eta)
{
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= n) return;
    const int i = rows[wid], j = cols[wid];
    const int64_t lim = m.basis == BEM_P0 ? m.nt : m.nv;
    if (i < 0 || i >= lim || j < 0 || j >= lim) {
        if (lane == 0) set_status(status, BEM_ERR_INVALID_ARG);
        return;
    }
    int alo, ahi, blo, bhi;
    if (m.basis == BEM_P0) {
        alo = 0; ahi = 1; blo = 0; bhi = 1;
    } else {
        alo = __ldg(m.vt_ptr + i); ahi = __ldg(m.vt_ptr + i + 1);
        blo = __ldg(m.vt_ptr + j); bhi = __ldg(m.vt_ptr + j + 1);
    }
    double sr = 0.0, si = 0.0;
    for (int ka = alo; ka < ahi; ++ka) {
        const int a = m.basis == BEM_P0 ? i : __ldg(m.vt_tri + ka);
        const int4 va = __ldg(m.tvid + a);
        const int la = m.basis == BEM_P0 ? -1 : (va.x == i ? 0 : (va.y == i ? 1 : 2));
        Tri A;
        load_tri(m.geom, a, A);
        for (int kb = blo; kb < bhi; ++kb) {
            const int b = m.basis == BEM_P0 ? j : __ldg(m.vt_tri + kb);
            const int4 vb = __ldg(m.tvid + b);
            const int lb = m.basis == BEM_P0 ? -1 : (vb.x == j ? 0 : (vb.y == j ? 1 : 2));
            int cas = kRegular, pc = 0;
            if (touching(va, vb)) {
                const int k = find_touching(m, a, b);
                cas = __ldg(m.nb_case + k);
                pc = __ldg(m.nb_perm + k);
            }
            const int *pa = c_perm[pc / 6], *pb = c_perm[pc % 6];
            int ca = -1, cb = -1;   // canonical positions of the basis vertices
            for (int q = 0; q < 3; ++q) {
                if (pa[q] == la) ca = q;
                if (pb[q] == lb) cb = q;
            }
            Tri B;
            load_tri(m.geom, b, B);
            double e1a[3], e2a[3], e1b[3], e2b[3], d0[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                e1a[c] = A.v[pa[1]][c] - A.v[pa[0]][c];
                e2a[c] = A.v[pa[2]][c] - A.v[pa[1]][c];
                e1b[c] = B.v[pb[1]][c] - B.v[pb[0]][c];
                e2b[c] = B.v[pb[2]][c] - B.v[pb[1]][c];
                d0[c] = A.v[pa[0]][c] - B.v[pb[0]][c];
            }
            const double *rule = rs.d[cas];
            const int np = rs.n[cas];
            double pr = 0.0, pi = 0.0;
            for (int p = lane; p < np; p += 32) {
                const double x1 = __ldg(rule + p), x2 = __ldg(rule + np + p),
                             y1 = __ldg(rule + 2 * np + p), y2 = __ldg(rule + 3 * np + p),
                             w = __ldg(rule + 4 * np + p);
                const double dx = d0[0] + x1 * e1a[0] + x2 * e2a[0] - y1 * e1b[0] - y2 * e2b[0];
                const double dy = d0[1] + x1 * e1a[1] + x2 * e2a[1] - y1 * e1b[1] - y2 * e2b[1];
                const double dz = d0[2] + x1 * e1a[2] + x2 * e2a[2] - y1 * e1b[2] - y2 * e2b[2];
                double kr, ki;
                kval<KIND>(dx, dy, dz, B.n, kappa, kr, ki, eta);
                double f = w;
                if (ca >= 0) f *= (ca == 0 ? 1.0 - x1 : (ca == 1 ? x1 - x2 : x2));
                if (cb >= 0) f *= (cb == 0 ? 1.0 - y1 : (cb == 1 ? y1 - y2 : y2));
                if (ABS) {
                    pr += fabs(f) * sqrt(kr * kr + ki * ki);
                } else {
                    pr += f * kr;
                    if (kind_complex(KIND)) pi += f * ki;
                }
            }
            const double scale = A.sg * B.sg * kInv4Pi;
            sr += pr * scale;
            si += pi * scale;
        }
    }
    sr = warp_sum(sr);
    if (kind_complex(KIND)) si = warp_sum(si);
    if (lane == 0) {
        if (kind_complex(KIND) && !ABS) reinterpret_cast<double2 *>(out)[wid] = make_double2(sr, si);
        else reinterpret_cast<double *>(out)[wid] = sr;
    }
}

cudaError_t launch_tile_prefix(const BlockLaunch &L, int tr, int tc, int64_t *prefix,
                               int *status, cudaStream_t st)
{
    if (L.n_blocks <= 0) return cudaSuccess;
    k_tile_prefix<<<1, 1024, 0, st>>>(L, tr, tc, prefix, status);
    return cudaGetLastError();
}

// Long block lists over many CTAs: CTA c scans blocks [c K, (c + 1) K) in place
// (K = kPrefixChunk) and leaves the chunk's total; then every later chunk adds
// the totals of the chunks before it.  Integer sums: the same prefix as the
// single-CTA pass.
__global__ void __launch_bounds__(1024) k_tile_prefix_chunk(BlockLaunch L, int tr, int tc,
                                                            int64_t *prefix, int64_t *chunk_total,
                                                            int *status)
{
    const int64_t lo = (int64_t)blockIdx.x * kPrefixChunk;
    tile_prefix_range(L, tr, tc, prefix, status, chunk_total + blockIdx.x, lo,
                      min(L.n_blocks, lo + kPrefixChunk));
}

// CTA c adds the totals of chunks 0 .. c to chunk c + 1
__global__ void __launch_bounds__(1024) k_tile_prefix_add(BlockLaunch L, int64_t *prefix,
                                                          const int64_t *__restrict__ chunk_total)
{
    __shared__ int64_t ws[32];
    const int c = blockIdx.x + 1;
    int64_t s = 0;
    for (int k = threadIdx.x; k < c; k += blockDim.x) s += chunk_total[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    int64_t base = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) base += ws[k];
    const int64_t lo = (int64_t)c * kPrefixChunk, hi = min(L.n_blocks, lo + kPrefixChunk);
    for (int64_t b = lo + threadIdx.x; b < hi; b += blockDim.x) prefix[b] += base;
}

cudaError_t launch_tile_prefix_wide(const BlockLaunch &L, int tr, int tc, int64_t *prefix,
                                    int64_t *chunk_total, int *status, cudaStream_t st)
{
    if (L.n_blocks <= kPrefixChunk) return launch_tile_prefix(L, tr, tc, prefix, status, st);
    const int64_t nch = prefix_chunks(L.n_blocks);
    k_tile_prefix_chunk<<<(unsigned)nch, 1024, 0, st>>>(L, tr, tc, prefix, chunk_total, status);
    k_tile_prefix_add<<<(unsigned)(nch - 1), 1024, 0, st>>>(L, prefix, chunk_total);
    return cudaGetLastError();
}

template <int KIND, int NP, bool MIXED>
static cudaError_t block_np(const MeshView &m, const BlockLaunch &L, const Rule2D &R,
                            const int64_t *prefix, int *status, int grid, cudaStream_t st)
{
    if (m.basis == BEM_P0) {
        k_block_p0<KIND, NP, MIXED><<<grid, 256, 0, st>>>(m, L, R, prefix, status);
    } else {
        return MIXED ? launch_p1_single_mixed(KIND, NP, m, L, R, prefix, status, grid * 2, st)
                     : launch_p1_single_fp64(KIND, NP, m, L, R, prefix, status, grid, st);
    }
    return cudaGetLastError();
}

template <int KIND, bool MIXED>
static cudaError_t block_kind(const MeshView &m, const BlockLaunch &L, const Rule2D &R,
                              const int64_t *prefix, int *status, int grid, cudaStream_t st)
{
    switch (R.np) {
    case 4: return block_np<KIND, 4, MIXED>(m, L, R, prefix, status, grid, st);
    case 7: return block_np<KIND, 7, MIXED>(m, L, R, prefix, status, grid, st);
    case 9: return block_np<KIND, 9, MIXED>(m, L, R, prefix, status, grid, st);
    case 16: return block_np<KIND, 16, MIXED>(m, L, R, prefix, status, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_block_engine(const MeshView &m, const BlockLaunch &L, const Rule2D &R,
                                const int64_t *prefix, int *status, int grid, cudaStream_t st)
{
    if (L.n_blocks <= 0) return cudaSuccess;
    // the mixed form covers the Laplace kernels; Helmholtz pairs stay FP64
    switch (L.kind) {
    case BEM_LAPLACE_SLP:
        return L.mixed ? block_kind<BEM_LAPLACE_SLP, true>(m, L, R, prefix, status, grid, st)
                       : block_kind<BEM_LAPLACE_SLP, false>(m, L, R, prefix, status, grid, st);
    case BEM_LAPLACE_DLP:
        return L.mixed ? block_kind<BEM_LAPLACE_DLP, true>(m, L, R, prefix, status, grid, st)
                       : block_kind<BEM_LAPLACE_DLP, false>(m, L, R, prefix, status, grid, st);
    case BEM_HELMHOLTZ_DLP:   // FP64 in every precision
        return block_kind<BEM_HELMHOLTZ_DLP, false>(m, L, R, prefix, status, grid, st);
    case BEM_HELMHOLTZ_BW:
        return block_kind<BEM_HELMHOLTZ_BW, false>(m, L, R, prefix, status, grid, st);
    default:
        // the mixed Helmholtz form covers piecewise-constant pairs
        return (L.mixed && m.basis == BEM_P0)
                   ? block_kind<BEM_HELMHOLTZ_SLP, true>(m, L, R, prefix, status, grid, st)
                   : block_kind<BEM_HELMHOLTZ_SLP, false>(m, L, R, prefix, status, grid, st);
    }
}

cudaError_t launch_pivot_entries(const MeshView &m, const int32_t *rows, const int32_t *cols,
                                 int64_t n, void *out, const Rule4D *rules, int kind,
                                 double kappa, int *status, cudaStream_t st, bool absolute,
                                 double eta)
{
    if (n <= 0) return cudaSuccess;
    RuleSet rs;
    for (int c = 0; c < 4; ++c) {
        rs.d[c] = rules[c].d;
        rs.n[c] = rules[c].n;
    }
    const int64_t blocks = (n + 7) / 8;
#define BEM_PIV(K, A) k_pivot<K, A><<<(unsigned)blocks, 256, 0, st>>>(m, rows, cols, n, out, rs, kappa, status, eta)
    switch (kind) {
    case BEM_LAPLACE_SLP: if (absolute) BEM_PIV(BEM_LAPLACE_SLP, true); else BEM_PIV(BEM_LAPLACE_SLP, false); break;
    case BEM_LAPLACE_DLP: if (absolute) BEM_PIV(BEM_LAPLACE_DLP, true); else BEM_PIV(BEM_LAPLACE_DLP, false); break;
    case BEM_HELMHOLTZ_DLP: if (absolute) BEM_PIV(BEM_HELMHOLTZ_DLP, true); else BEM_PIV(BEM_HELMHOLTZ_DLP, false); break;
    case BEM_HELMHOLTZ_BW: if (absolute) BEM_PIV(BEM_HELMHOLTZ_BW, true); else BEM_PIV(BEM_HELMHOLTZ_BW, false); break;
    default: if (absolute) BEM_PIV(BEM_HELMHOLTZ_SLP, true); else BEM_PIV(BEM_HELMHOLTZ_SLP, false); break;
    }
#undef BEM_PIV
    return cudaGetLastError();
}

cudaError_t launch_tile_prefix_batch(BatchJob *jobs, int n_jobs, int tr, int tc, int unit,
                                     int64_t *job_total, int64_t *job_end, int *status,
                                     cudaStream_t st)
{
    if (n_jobs <= 0) return cudaSuccess;
    k_tile_prefix_batch<<<n_jobs, 1024, 0, st>>>(jobs, tr, tc, job_total, status);
    k_job_scan<<<1, 1024, 0, st>>>(job_total, n_jobs, unit, job_end);
    return cudaGetLastError();
}

template <int KIND, int NP, bool MIXED>
static cudaError_t batch_np(const BatchJob *jobs, int n_jobs, const int64_t *job_end, int basis,
                            const Rule2D &R, int *status, int grid, cudaStream_t st)
{
    if (basis == BEM_P0) {
        k_batch_p0<KIND, NP, MIXED><<<grid, 256, 0, st>>>(jobs, n_jobs, job_end, R, status);
    } else {
        return MIXED ? launch_p1_batch_mixed(KIND, NP, jobs, n_jobs, job_end, R, status, grid, st)
                     : launch_p1_batch_fp64(KIND, NP, jobs, n_jobs, job_end, R, status, grid, st);
    }
    return cudaGetLastError();
}

template <int KIND, bool MIXED>
static cudaError_t batch_kind(const BatchJob *jobs, int n_jobs, const int64_t *job_end, int basis,
                              const Rule2D &R, int *status, int grid, cudaStream_t st)
{
    switch (R.np) {
    case 4: return batch_np<KIND, 4, MIXED>(jobs, n_jobs, job_end, basis, R, status, grid, st);
    case 7: return batch_np<KIND, 7, MIXED>(jobs, n_jobs, job_end, basis, R, status, grid, st);
    case 9: return batch_np<KIND, 9, MIXED>(jobs, n_jobs, job_end, basis, R, status, grid, st);
    case 16: return batch_np<KIND, 16, MIXED>(jobs, n_jobs, job_end, basis, R, status, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_block_batch(const BatchJob *jobs, int n_jobs, const int64_t *job_end, int basis,
                               int kind, int mixed, const Rule2D &R, int *status, int grid,
                               cudaStream_t st)
{
    if (n_jobs <= 0) return cudaSuccess;
    if (kind == kFusedLaplace)   // piecewise-linear float form only
        return (basis == BEM_P1 && mixed)
                   ? launch_p1_batch_mixed(kFusedLaplace, R.np, jobs, n_jobs, job_end, R, status, grid, st)
                   : cudaErrorInvalidValue;
    switch (kind) {
    case BEM_LAPLACE_SLP:
        return mixed ? batch_kind<BEM_LAPLACE_SLP, true>(jobs, n_jobs, job_end, basis, R, status, grid, st)
                     : batch_kind<BEM_LAPLACE_SLP, false>(jobs, n_jobs, job_end, basis, R, status, grid, st);
    case BEM_LAPLACE_DLP:
        return mixed ? batch_kind<BEM_LAPLACE_DLP, true>(jobs, n_jobs, job_end, basis, R, status, grid, st)
                     : batch_kind<BEM_LAPLACE_DLP, false>(jobs, n_jobs, job_end, basis, R, status, grid, st);
    case BEM_HELMHOLTZ_DLP:   // FP64 in every precision
        return batch_kind<BEM_HELMHOLTZ_DLP, false>(jobs, n_jobs, job_end, basis, R, status, grid, st);
    case BEM_HELMHOLTZ_BW:
        return batch_kind<BEM_HELMHOLTZ_BW, false>(jobs, n_jobs, job_end, basis, R, status, grid, st);
    default:
        return (mixed && basis == BEM_P0)
                   ? batch_kind<BEM_HELMHOLTZ_SLP, true>(jobs, n_jobs, job_end, basis, R, status, grid, st)
                   : batch_kind<BEM_HELMHOLTZ_SLP, false>(jobs, n_jobs, job_end, basis, R, status, grid, st);
    }
}

}  // namespace bem
