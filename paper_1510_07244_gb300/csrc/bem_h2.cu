// H2-matrix-vector product and conjugate gradients on the device (Sections
// 2.4 and 4).
//
// The matrix is G ~ sum over near blocks N_ts + sum over admissible blocks
// V_t S_ts V_s^T with nested cluster bases: V_t of a leaf is its
// interpolation matrix, V_t of a cluster with sons is diag(V_t1, V_t2) V^_t
// (transfer matrix V^_t, rows = the sons' pivots).  y = G x runs as
//   near     y|t = sum_s N_ts x|s                 one CTA per leaf, row per lane
//   forward  x^_s = V_s^T x|s (leaf) or V^_s^T (x^_s1; x^_s2), deepest level first
//   coupling y^_t = sum_s S_ts x^_s               one CTA per cluster
//   backward (y^_t1; y^_t2) += V^_t y^_t, y|t += V_t y^_t (leaf), top level first
// Every output element is written by one lane in a fixed order (no atomics),
// so products are bitwise reproducible.  The near field runs on a second
// stream beside the forward and coupling passes.  All arithmetic is FP64.  The matrix
// is memory- and latency-bound: per product it reads every near-field and
// coupling entry once (8 bytes each) and does 2 flops per entry.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "bem_internal.h"

struct bem_h2 {
    int64_t n = 0;
    int32_t nc = 0, max_rank = 0;
    std::vector<void *> allocs;
    // per cluster (device): rows of its basis matrix, pivots, offsets
    int32_t *rows = nullptr;       // basis rows R_c
    int32_t *rank = nullptr;       // K_c
    int64_t *v_off = nullptr;      // offset of the R_c x K_c row-major matrix in vals
    int64_t *src_off = nullptr;    // offset of the R_c row sources in src
    int64_t *hat_off = nullptr;    // offset of x^_c / y^_c in the hat vectors
    int32_t *leaf = nullptr;       // 1 for leaves
    int32_t *src = nullptr;        // row sources: vector index (leaf) or hat index (else)
    double *vals = nullptr;        // basis matrices
    double *valsT = nullptr;       // the same, each transposed (K_c x R_c row-major)
    // near blocks by leaf row cluster (CSR over nc), far blocks by row cluster
    int32_t *near_ptr = nullptr, *near_col = nullptr;
    int64_t *near_off = nullptr;
    int32_t *far_ptr = nullptr, *far_col = nullptr;
    int64_t *far_off = nullptr;
    const double *near_vals = nullptr, *far_vals = nullptr;
    int32_t *cl_ptr = nullptr, *cl_idx = nullptr;   // cluster index sets
    // levels (host lists of device cluster arrays), deepest last
    std::vector<int32_t *> level;
    std::vector<int32_t> level_n;
    std::vector<int32_t> leaves_h;
    int32_t *leaves = nullptr;
    int32_t n_leaves = 0;
    double *xhat = nullptr, *yhat = nullptr;
    int64_t n_hat = 0;
    double *diag = nullptr;        // added to the diagonal (null: none)
    // conjugate gradients: vectors and scalars
    double *r = nullptr, *p = nullptr, *q = nullptr, *part = nullptr, *scal = nullptr;
    // the near field runs on a second stream beside the forward and coupling
    // passes (it writes y, the backward pass then adds to it)
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

namespace bem {

namespace {

constexpr int kDotBlocks = 512;

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct H2View {
    const int32_t *rows, *rank, *leaf, *src;
    const int64_t *v_off, *src_off, *hat_off;
    const double *vals, *valsT;
    const int32_t *near_ptr, *near_col, *far_ptr, *far_col, *cl_ptr, *cl_idx;
    const int64_t *near_off, *far_off;
    const double *near_vals, *far_vals;
    const double *diag;
};

// near field: one CTA per leaf row cluster; its 8 warps take every 8th near
// block, lane i = row i (rows in passes of 32), and the warps' partial sums
// are added in warp order (fixed, so the result is reproducible)
constexpr int kH2Warps = 8;

__global__ void __launch_bounds__(256) k_h2_near(H2View H, const int32_t *leaves, int n_leaves,
                                                 const double *__restrict__ x, double *y)
{
    __shared__ double part[kH2Warps][32];
    const int t = leaves[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = H.cl_ptr[t], nr = H.cl_ptr[t + 1] - r0;
    for (int i0 = 0; i0 < nr; i0 += 32) {
        const int i = i0 + lane;
        double acc = 0.0;
        if (i < nr)
            for (int b = H.near_ptr[t] + warp; b < H.near_ptr[t + 1]; b += kH2Warps) {
                const int s = H.near_col[b];
                const int c0 = H.cl_ptr[s], ncl = H.cl_ptr[s + 1] - c0;
                const double *N = H.near_vals + H.near_off[b] + i;
#pragma unroll 4
                for (int j = 0; j < ncl; ++j) acc = fma(N[(int64_t)j * nr], x[H.cl_idx[c0 + j]], acc);
            }
        part[warp][lane] = acc;
        __syncthreads();
        if (warp == 0 && i < nr) {
            double sum = 0.0;
#pragma unroll
            for (int k = 0; k < kH2Warps; ++k) sum += part[k][lane];
            const int gi = H.cl_idx[r0 + i];
            if (H.diag) sum = fma(H.diag[gi], x[gi], sum);
            y[gi] = sum;
        }
        __syncthreads();
    }
}

// forward transformation of one level: x^_c = V_c^T v, v = x at the leaf's
// indices or the sons' x^ entries.  One CTA per cluster: lane k = column k
// (K_c <= 32), the 8 warps take every 8th row, and their partial sums are
// added in warp order (fixed, so the result is reproducible).  A level is
// latency-bound (a few rows per warp), so the rows are spread over warps.
__global__ void __launch_bounds__(256) k_h2_forward(H2View H, const int32_t *level, int n,
                                                    const double *__restrict__ x, double *xhat)
{
    __shared__ double part[kH2Warps][32];
    const int c = level[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int R = H.rows[c], K = H.rank[c];
    if (K == 0) return;                 // uniform across the CTA
    const double *V = H.vals + H.v_off[c];
    const int32_t *src = H.src + H.src_off[c];
    const double *v = H.leaf[c] ? x : xhat;
    double acc = 0.0;
    if (lane < K) {
#pragma unroll 4
        for (int i = warp; i < R; i += kH2Warps)
            acc = fma(V[(int64_t)i * K + lane], __ldg(v + __ldg(src + i)), acc);
    }
    part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && lane < K) {
        double sum = 0.0;
#pragma unroll
        for (int k = 0; k < kH2Warps; ++k) sum += part[k][lane];
        xhat[H.hat_off[c] + lane] = sum;
    }
}

// coupling: y^_t = sum over t's admissible blocks of S_ts x^_s (column-major
// K_t x K_s); one CTA per cluster, its 8 warps over every 8th block, lane =
// row, partial sums added in warp order; every cluster's y^ is written here,
// zero without blocks
__global__ void __launch_bounds__(256) k_h2_coupling(H2View H, int nc, const double *__restrict__ xhat,
                                                     double *yhat)
{
    __shared__ double part[kH2Warps][32];
    const int t = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int K = H.rank[t];
    if (K == 0) return;                 // uniform across the CTA
    double acc = 0.0;
    if (lane < K)
        for (int b = H.far_ptr[t] + warp; b < H.far_ptr[t + 1]; b += kH2Warps) {
            const int s = H.far_col[b], Ks = H.rank[s];
            const double *S = H.far_vals + H.far_off[b] + lane;
            const double *xs = xhat + H.hat_off[s];
#pragma unroll 4
            for (int l = 0; l < Ks; ++l) acc = fma(S[(int64_t)l * K], xs[l], acc);
        }
    part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && lane < K) {
        double sum = 0.0;
#pragma unroll
        for (int k = 0; k < kH2Warps; ++k) sum += part[k][lane];
        yhat[H.hat_off[t] + lane] = sum;
    }
}

// backward transformation of one level: every row i of V_c adds (V_c y^_c)_i
// to its target, the vector y at a leaf's index, the son's y^ entry otherwise.
// One CTA per cluster; rows of at most 64 take four threads each (columns
// k = part mod 4, combined by two fixed shuffles), longer ones one thread per
// row.  The transposed basis makes consecutive rows consecutive words.
__global__ void __launch_bounds__(256) k_h2_backward(H2View H, const int32_t *level, int n,
                                                     double *yhat, double *y)
{
    const int c = level[blockIdx.x];
    const int R = H.rows[c], K = H.rank[c];
    if (K == 0) return;                 // uniform across the CTA
    const double *VT = H.valsT + H.v_off[c];
    const int32_t *src = H.src + H.src_off[c];
    const double *yc = yhat + H.hat_off[c];
    double *dst = H.leaf[c] ? y : yhat;
    if (R <= 64) {
        const int i = threadIdx.x >> 2, part = threadIdx.x & 3;
        double acc = 0.0;
        if (i < R) {
#pragma unroll 4
            for (int k = part; k < K; k += 4) acc = fma(VT[(int64_t)k * R + i], yc[k], acc);
        }
        // the four parts of a row sit in four consecutive lanes
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (i < R && part == 0) dst[src[i]] += acc;
    } else {
        for (int i = threadIdx.x; i < R; i += blockDim.x) {
            double acc = 0.0;
#pragma unroll 8
            for (int k = 0; k < K; ++k) acc = fma(VT[(int64_t)k * R + i], yc[k], acc);
            dst[src[i]] += acc;
        }
    }
}

// deterministic dot product: fixed grid, per-block partial sums, then one
// block adds the partials in order
__global__ void __launch_bounds__(256) k_dot_part(const double *__restrict__ a,
                                                  const double *__restrict__ b, int64_t n,
                                                  double *part)
{
    __shared__ double sh[8];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        acc = fma(a[i], b[i], acc);
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
        part[blockIdx.x] = s;
    }
}

__global__ void k_dot_final(const double *part, int np, double *out)
{
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
        *out = s;
    }
}

// scal: [0] r.r, [1] p.q, [2] new r.r
__global__ void __launch_bounds__(256) k_cg_step(int64_t n, const double *scal, double *x,
                                                 double *r, const double *p, const double *q)
{
    const double alpha = scal[0] / scal[1];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        r[i] = fma(-alpha, q[i], r[i]);
    }
}

__global__ void __launch_bounds__(256) k_cg_dir(int64_t n, double *scal, const double *r, double *p)
{
    const double beta = scal[2] / scal[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], r[i]);
}

__global__ void k_cg_roll(double *scal) { scal[0] = scal[2]; }

H2View view(const bem_h2 *h)
{
    H2View v;
    v.rows = h->rows;
    v.rank = h->rank;
    v.leaf = h->leaf;
    v.src = h->src;
    v.v_off = h->v_off;
    v.src_off = h->src_off;
    v.hat_off = h->hat_off;
    v.vals = h->vals;
    v.valsT = h->valsT;
    v.near_ptr = h->near_ptr;
    v.near_col = h->near_col;
    v.near_off = h->near_off;
    v.far_ptr = h->far_ptr;
    v.far_col = h->far_col;
    v.far_off = h->far_off;
    v.near_vals = h->near_vals;
    v.far_vals = h->far_vals;
    v.cl_ptr = h->cl_ptr;
    v.cl_idx = h->cl_idx;
    v.diag = h->diag;
    return v;
}


cudaError_t matvec(const bem_h2 *h, const double *x, double *y, cudaStream_t st)
{
    const H2View H = view(h);
    // fork: the near field on the side stream, joined before the backward pass
    cudaError_t e = cudaEventRecord(h->fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->fork, 0);
    if (e != cudaSuccess) return e;
    if (h->n_leaves > 0) k_h2_near<<<h->n_leaves, 256, 0, h->side>>>(H, h->leaves, h->n_leaves, x, y);
    if ((e = cudaEventRecord(h->join, h->side)) != cudaSuccess) return e;
    for (int d = (int)h->level.size() - 1; d >= 0; --d)
        if (h->level_n[d] > 0)
            k_h2_forward<<<h->level_n[d], 256, 0, st>>>(H, h->level[d], h->level_n[d], x, h->xhat);
    k_h2_coupling<<<h->nc, 256, 0, st>>>(H, h->nc, h->xhat, h->yhat);
    if ((e = cudaStreamWaitEvent(st, h->join, 0)) != cudaSuccess) return e;
    for (size_t d = 0; d < h->level.size(); ++d)
        if (h->level_n[d] > 0)
            k_h2_backward<<<h->level_n[d], 256, 0, st>>>(H, h->level[d], h->level_n[d], h->yhat, y);
    return cudaGetLastError();
}

cudaError_t dot(const bem_h2 *h, const double *a, const double *b, double *out, cudaStream_t st)
{
    k_dot_part<<<kDotBlocks, 256, 0, st>>>(a, b, h->n, h->part);
    k_dot_final<<<1, 1024, 0, st>>>(h->part, kDotBlocks, out);
    return cudaGetLastError();
}

template <class T>
cudaError_t h2_upload(bem_h2 *h, T **d, const std::vector<T> &v)
{
    cudaError_t e = cudaMalloc((void **)d, std::max<size_t>(1, v.size()) * sizeof(T));
    if (e != cudaSuccess) return e;
    h->allocs.push_back(*d);
    if (!v.empty()) e = cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

template <class T>
cudaError_t h2_alloc(bem_h2 *h, T **d, size_t n)
{
    cudaError_t e = cudaMalloc((void **)d, std::max<size_t>(1, n) * sizeof(T));
    if (e == cudaSuccess) h->allocs.push_back(*d);
    return e;
}

void h2_free(bem_h2 *h)
{
    for (void *a : h->allocs) cudaFree(a);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->join) cudaEventDestroy(h->join);
    if (h->side) cudaStreamDestroy(h->side);
    delete h;
}

}  // namespace

}  // namespace bem

extern "C" {

int bem_h2_create(bem_ctx *ctx, int64_t n, int32_t n_clusters, const int32_t *cl_ptr,
                  const int32_t *cl_idx, const int32_t *cl_son, const int32_t *piv_ptr,
                  const int32_t *piv_idx, const int64_t *v_off, const double *V, int64_t n_near,
                  const int32_t *near_row, const int32_t *near_col, const int64_t *near_off,
                  const double *near_vals, int64_t n_far, const int32_t *far_row,
                  const int32_t *far_col, const int64_t *far_off, const double *far_vals,
                  const double *diag, bem_h2 **out)
{
    using namespace bem;
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (!out || n < 1 || n_clusters < 1 || !cl_ptr || !cl_idx || !cl_son || !piv_ptr ||
        !piv_idx || !v_off || !V || n_near < 0 || n_far < 0 ||
        (n_near > 0 && (!near_row || !near_col || !near_off || !near_vals)) ||
        (n_far > 0 && (!far_row || !far_col || !far_off || !far_vals)))
        return api_fail(ctx, BEM_ERR_INVALID_ARG, "bem_h2_create: bad arguments");
    *out = nullptr;
    const int nc = n_clusters;
    // host checks of the tree, the index sets and the bases' shapes
    if (cl_ptr[0] != 0 || piv_ptr[0] != 0 || v_off[0] != 0)
        return api_fail(ctx, BEM_ERR_INVALID_ARG, "bem_h2_create: CSR arrays must start at 0");
    std::vector<int> parent(nc, -1), depth(nc, 0);
    for (int c = 0; c < nc; ++c) {
        if (cl_ptr[c + 1] < cl_ptr[c] || piv_ptr[c + 1] < piv_ptr[c] || v_off[c + 1] < v_off[c])
            return api_fail(ctx, BEM_ERR_INVALID_ARG, "bem_h2_create: decreasing CSR pointers");
        if (piv_ptr[c + 1] - piv_ptr[c] > 32)
            return api_fail(ctx, BEM_ERR_UNSUPPORTED, "bem_h2_create: more than 32 pivots in a cluster");
        for (int s = 0; s < 2; ++s) {
            const int x = cl_son[2 * c + s];
            if (x < -1 || x >= nc || x == c || (x >= 0 && parent[x] >= 0))
                return api_fail(ctx, BEM_ERR_INVALID_ARG, "bem_h2_create: bad son");
            if (x >= 0) parent[x] = c;
        }
    }
    for (int64_t k = 0; k < cl_ptr[nc]; ++k)
        if (cl_idx[k] < 0 || cl_idx[k] >= n)
            return api_fail(ctx, BEM_ERR_INVALID_ARG, "bem_h2_create: index out of range");
    int max_depth = 0;
    for (int c = 0; c < nc; ++c) {
        int d = 0, x = c;
        while (parent[x] >= 0) {
            x = parent[x];
            if (++d > nc) return api_fail(ctx, BEM_ERR_INVALID_ARG, "bem_h2_create: cycle");
        }
        depth[c] = d;
        max_depth = std::max(max_depth, d);
    }
    bem_h2 *h = new bem_h2();
    h->n = n;
    h->nc = nc;
    std::vector<int32_t> rows(nc), rank(nc), leaf(nc), src;
    std::vector<int64_t> voff(nc), soff(nc), hoff(nc);
    int64_t hat = 0;
    for (int c = 0; c < nc; ++c) {
        rank[c] = piv_ptr[c + 1] - piv_ptr[c];
        hoff[c] = hat;
        hat += rank[c];
    }
    for (int c = 0; c < nc; ++c) {
        const int s0 = cl_son[2 * c], s1 = cl_son[2 * c + 1];
        leaf[c] = (s0 < 0 && s1 < 0) ? 1 : 0;
        soff[c] = (int64_t)src.size();
        if (leaf[c]) {
            for (int32_t k = cl_ptr[c]; k < cl_ptr[c + 1]; ++k) src.push_back(cl_idx[k]);
        } else {
            for (int s : {s0, s1})
                if (s >= 0)
                    for (int k = 0; k < rank[s]; ++k) src.push_back((int32_t)(hoff[s] + k));
        }
        rows[c] = (int32_t)((int64_t)src.size() - soff[c]);
        voff[c] = v_off[c];
        if (v_off[c + 1] - v_off[c] != (int64_t)rows[c] * rank[c]) {
            h2_free(h);
            return api_fail(ctx, BEM_ERR_INVALID_ARG, "bem_h2_create: basis matrix of the wrong size");
        }
        if (leaf[c] && rows[c] > 32 * 64) {
            h2_free(h);
            return api_fail(ctx, BEM_ERR_UNSUPPORTED, "bem_h2_create: leaf of more than 2048 indices");
        }
    }
    // blocks by row cluster
    auto by_row = [&](int64_t nb, const int32_t *br, const int32_t *bc, const int64_t *bo,
                      std::vector<int32_t> &ptr, std::vector<int32_t> &col,
                      std::vector<int64_t> &off) -> bool {
        ptr.assign(nc + 1, 0);
        for (int64_t b = 0; b < nb; ++b) {
            if (br[b] < 0 || br[b] >= nc || bc[b] < 0 || bc[b] >= nc || bo[b] < 0) return false;
            ptr[br[b] + 1]++;
        }
        for (int c = 0; c < nc; ++c) ptr[c + 1] += ptr[c];
        col.assign(nb, 0);
        off.assign(nb, 0);
        std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
        for (int64_t b = 0; b < nb; ++b) {   // block order kept within a row cluster
            col[fill[br[b]]] = bc[b];
            off[fill[br[b]]++] = bo[b];
        }
        return true;
    };
    std::vector<int32_t> nptr, ncol, fptr, fcol;
    std::vector<int64_t> noff, foff;
    if (!by_row(n_near, near_row, near_col, near_off, nptr, ncol, noff) ||
        !by_row(n_far, far_row, far_col, far_off, fptr, fcol, foff)) {
        h2_free(h);
        return api_fail(ctx, BEM_ERR_INVALID_ARG, "bem_h2_create: bad block list");
    }
    for (int c = 0; c < nc; ++c)
        if (!leaf[c] && nptr[c + 1] > nptr[c]) {
            h2_free(h);
            return api_fail(ctx, BEM_ERR_INVALID_ARG, "bem_h2_create: near block on a non-leaf row cluster");
        }
    std::vector<std::vector<int32_t>> lev(max_depth + 1);
    for (int c = 0; c < nc; ++c) {
        lev[depth[c]].push_back(c);
        if (leaf[c]) h->leaves_h.push_back(c);
    }
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaSuccess;
    std::vector<int32_t> cp(cl_ptr, cl_ptr + nc + 1), ci(cl_idx, cl_idx + cl_ptr[nc]);
    std::vector<double> vals(V, V + v_off[nc]), valsT(vals.size());
    for (int c = 0; c < nc; ++c)
        for (int i = 0; i < rows[c]; ++i)
            for (int k = 0; k < rank[c]; ++k)
                valsT[voff[c] + (int64_t)k * rows[c] + i] = vals[voff[c] + (int64_t)i * rank[c] + k];
    if ((e = h2_upload(h, &h->rows, rows)) || (e = h2_upload(h, &h->rank, rank)) ||
        (e = h2_upload(h, &h->leaf, leaf)) || (e = h2_upload(h, &h->src, src)) ||
        (e = h2_upload(h, &h->v_off, voff)) || (e = h2_upload(h, &h->src_off, soff)) ||
        (e = h2_upload(h, &h->hat_off, hoff)) || (e = h2_upload(h, &h->vals, vals)) ||
        (e = h2_upload(h, &h->valsT, valsT)) ||
        (e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking)) ||
        (e = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming)) ||
        (e = cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming)) ||
        (e = h2_upload(h, &h->near_ptr, nptr)) || (e = h2_upload(h, &h->near_col, ncol)) ||
        (e = h2_upload(h, &h->near_off, noff)) || (e = h2_upload(h, &h->far_ptr, fptr)) ||
        (e = h2_upload(h, &h->far_col, fcol)) || (e = h2_upload(h, &h->far_off, foff)) ||
        (e = h2_upload(h, &h->cl_ptr, cp)) || (e = h2_upload(h, &h->cl_idx, ci)) ||
        (e = h2_upload(h, &h->leaves, h->leaves_h)) || (e = h2_alloc(h, &h->xhat, hat)) ||
        (e = h2_alloc(h, &h->yhat, hat)) || (e = h2_alloc(h, &h->r, n)) ||
        (e = h2_alloc(h, &h->p, n)) || (e = h2_alloc(h, &h->q, n)) ||
        (e = h2_alloc(h, &h->part, kDotBlocks)) || (e = h2_alloc(h, &h->scal, 4))) {
        h2_free(h);
        return api_cuda_fail(ctx, e, "bem_h2_create");
    }
    if (diag) {
        std::vector<double> dg(diag, diag + n);
        if ((e = h2_upload(h, &h->diag, dg)) != cudaSuccess) {
            h2_free(h);
            return api_cuda_fail(ctx, e, "bem_h2_create");
        }
    }
    for (auto &l : lev) {
        int32_t *d = nullptr;
        if ((e = h2_upload(h, &d, l)) != cudaSuccess) {
            h2_free(h);
            return api_cuda_fail(ctx, e, "bem_h2_create");
        }
        h->level.push_back(d);
        h->level_n.push_back((int32_t)l.size());
    }
    h->n_leaves = (int32_t)h->leaves_h.size();
    h->n_hat = hat;
    h->near_vals = near_vals;
    h->far_vals = far_vals;
    *out = h;
    return BEM_OK;
}

int bem_h2_matvec(bem_ctx *ctx, bem_h2 *h, const double *x, double *y)
{
    using namespace bem;
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (!h || !x || !y || x == y) return api_fail(ctx, BEM_ERR_INVALID_ARG, "bem_h2_matvec: bad arguments");
    cudaError_t e = matvec(h, x, y, ctx->stream);
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "bem_h2_matvec");
    return BEM_OK;
}

int bem_h2_cg(bem_ctx *ctx, bem_h2 *h, const double *b, double *x, double tol, int32_t maxit,
              int32_t *iters, double *rel_res)
{
    using namespace bem;
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (!h || !b || !x || b == x || !(tol > 0.0) || maxit < 0 || !iters || !rel_res)
        return api_fail(ctx, BEM_ERR_INVALID_ARG, "bem_h2_cg: bad arguments");
    cudaStream_t st = ctx->stream;
    const size_t bytes = (size_t)h->n * sizeof(double);
    // x0 = 0, r = p = b, r.r and b.b
    cudaError_t e = cudaMemsetAsync(x, 0, bytes, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->r, b, bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->p, b, bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = dot(h, h->r, h->r, h->scal + 0, st);
    double rr = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&rr, h->scal + 0, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "bem_h2_cg");
    const double bb = rr;
    const unsigned grid = (unsigned)std::min<int64_t>((h->n + 255) / 256, 4 * 1024);
    int it = 0;
    while (it < maxit && rr > tol * tol * bb && bb > 0.0) {
        e = matvec(h, h->p, h->q, st);                          // q = A p
        if (e == cudaSuccess) e = dot(h, h->p, h->q, h->scal + 1, st);
        if (e == cudaSuccess) {
            k_cg_step<<<grid, 256, 0, st>>>(h->n, h->scal, x, h->r, h->p, h->q);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = dot(h, h->r, h->r, h->scal + 2, st);
        if (e == cudaSuccess) {
            k_cg_dir<<<grid, 256, 0, st>>>(h->n, h->scal, h->r, h->p);
            k_cg_roll<<<1, 1, 0, st>>>(h->scal);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&rr, h->scal + 0, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return api_cuda_fail(ctx, e, "bem_h2_cg");
        if (!std::isfinite(rr)) return api_fail(ctx, BEM_ERR_DEGENERATE, "bem_h2_cg: breakdown");
        ++it;
    }
    *iters = it;
    *rel_res = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
    return BEM_OK;
}

int bem_h2_destroy(bem_ctx *ctx, bem_h2 *h)
{
    if (!ctx || !h) return BEM_ERR_INVALID_ARG;
    cudaStreamSynchronize(ctx->stream);
    bem::h2_free(h);
    return BEM_OK;
}

}  // extern "C"
