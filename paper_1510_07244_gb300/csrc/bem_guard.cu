// Cancellation guard of the float forms (piecewise-constant double layer).
//
// A double-layer entry integrates (x - y).n_y / r^3 over a triangle pair; when
// the test triangle straddles the trial triangle's plane, positive and
// negative terms cancel and the entry can be far below the sum of the
// magnitudes of its terms, A = sum |w k|.  A float evaluation has a forward
// error of a few float ulps of A, which can then exceed 1e-6 of the entry (or
// of a thousandth of its row's largest entry, the relative-error measure of the
// configurations).  The guard makes the float forms meet that measure:
//
//   1. the float kernels of a guarded job write each entry as a float pair
//      (value, A) into its 8-byte output slot (touching pairs carry A in the
//      unused imaginary part of the touching table);
//   2. k_guard_rowmax takes, per job and row, the largest |value|;
//   3. k_guard_select writes every entry whose error bound
//      kGuardRel * A stays within 1e-6 * max(|value|, 1e-3 * row max) as a
//      double, and appends the others to a list;
//   4. the listed entries are evaluated again with the FP64 form's rules in
//      double-float arithmetic (float pairs hi + lo carry about 44 bits, far
//      more than the listed entries need, at the float pipe's rate): a
//      disjoint pair by k_guard_redo_dd (one thread per entry), a touching
//      pair by k_guard_redo_touch (one warp per entry over the Sauter-Schwab
//      rule).
//
// The list has a fixed capacity; a full list is reported through the status
// word (BEM_ERR_OOM) and its surplus entries keep their float values.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "bem_device.cuh"

namespace bem {

namespace {

constexpr float kRelBound = 1e-6f;         // the relative-error bar
constexpr float kRowFloor = 1e-3f;         // fraction of the row maximum

__device__ __forceinline__ int find_guard_job(const int64_t *blk_end, int n_jobs, int64_t b)
{
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (blk_end[mid] > b) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// Block b of the guard bucket: its job, clusters and output offset.
struct GBlock {
    int job, nr, nc, r_lo, c_lo;
    int64_t off;
    bool ok;
};

__device__ __forceinline__ GBlock guard_block(const GuardJob *jobs, const int64_t *blk_end,
                                              int n_jobs, int64_t b)
{
    GBlock g;
    g.job = find_guard_job(blk_end, n_jobs, b);
    const BlockLaunch &L = jobs[g.job].L;
    const int64_t lb = b - (g.job > 0 ? blk_end[g.job - 1] : 0);
    const int t = L.blk_row[lb], s = L.blk_col[lb];
    g.ok = t >= 0 && t < L.n_row_clusters && s >= 0 && s < L.n_col_clusters;
    if (!g.ok) return g;
    g.r_lo = L.row_ptr[t];
    g.nr = L.row_ptr[t + 1] - g.r_lo;
    g.c_lo = L.col_ptr[s];
    g.nc = L.col_ptr[s + 1] - g.c_lo;
    g.off = L.blk_off[lb];
    g.ok = g.nr > 0 && g.nc > 0;
    return g;
}

// One warp per block (blocks hold a few hundred entries, so a CTA per block
// would leave the passes waiting on each block's index loads): lanes take
// the block's rows, the maximum over the row's columns goes out with one
// atomic per (block, row).
__global__ void __launch_bounds__(256) k_guard_rowmax(const GuardJob *__restrict__ jobs,
                                                      const int64_t *__restrict__ blk_end,
                                                      int n_jobs)
{
    const int64_t nb = blk_end[n_jobs - 1];
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nb; b += nw) {
        const GBlock g = guard_block(jobs, blk_end, n_jobs, b);
        if (!g.ok) continue;
        const GuardJob &G = jobs[g.job];
        const float2 *o = reinterpret_cast<const float2 *>(G.L.out) + g.off;
        for (int r = lane; r < g.nr; r += 32) {
            const int row = G.L.row_idx[g.r_lo + r];
            float m0 = 0.0f, m1 = 0.0f;
            int c = 0;
            for (; c + 1 < g.nc; c += 2) {
                m0 = fmaxf(m0, fabsf(o[r + (int64_t)c * g.nr].x));
                m1 = fmaxf(m1, fabsf(o[r + (int64_t)(c + 1) * g.nr].x));
            }
            if (c < g.nc) m0 = fmaxf(m0, fabsf(o[r + (int64_t)c * g.nr].x));
            // |value| >= 0, so its bit pattern orders like the value
            if (row >= 0 && row < G.n_rows)
                atomicMax(G.rowmax + row, __float_as_uint(fmaxf(m0, m1)));
        }
    }
}

// One warp per block, lanes over its entries (column-major, coalesced), four
// entries per lane in flight.
__global__ void __launch_bounds__(256) k_guard_select(const GuardJob *__restrict__ jobs,
                                                      const int64_t *__restrict__ blk_end,
                                                      int n_jobs, GuardItem *list,
                                                      GuardItem *list_t,
                                                      unsigned long long *count, int64_t cap,
                                                      int64_t cap_t, float rel, int *status)
{
    // disjoint pairs go to list (count[0], capacity cap), touching pairs to
    // list_t (count[1], capacity cap_t: every touching pair of the jobs)
    const int64_t nb = blk_end[n_jobs - 1];
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nb; b += nw) {
        const GBlock g = guard_block(jobs, blk_end, n_jobs, b);
        if (!g.ok) continue;   // uniform across the warp
        const GuardJob &G = jobs[g.job];
        float2 *o2 = reinterpret_cast<float2 *>(G.L.out) + g.off;
        double *od = reinterpret_cast<double *>(G.L.out) + g.off;
        const int n = g.nr * g.nc;
        // four entries per lane and trip, their loads issued together; the
        // whole warp iterates together, so the ballots below see every lane
        constexpr int U = 4;
        for (int e0 = 0; e0 < n; e0 += 32 * U) {
            float2 v[U];
            int row[U], col[U];
            bool redo[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + 32 * u + lane;
                v[u] = e < n ? o2[e] : make_float2(0.0f, 0.0f);
                const int c = e < n ? e / g.nr : 0;
                row[u] = e < n ? G.L.row_idx[g.r_lo + e - c * g.nr] : 0;
                col[u] = e < n ? G.L.col_idx[g.c_lo + c] : 0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + 32 * u + lane;
                redo[u] = false;
                if (e < n) {
                    float rmax = 0.0f;
                    if (row[u] >= 0 && row[u] < G.n_rows) rmax = __uint_as_float(G.rowmax[row[u]]);
                    const float scale = fmaxf(fabsf(v[u].x), kRowFloor * rmax);
                    redo[u] = rel * v[u].y > kRelBound * scale;
                    // entries kept in float are widened in place; the listed
                    // ones keep the pair until the recomputation overwrites them
                    if (!redo[u]) od[e] = (double)v[u].x;
                }
            }
            if (!__any_sync(0xffffffffu, redo[0] || redo[1] || redo[2] || redo[3])) continue;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + 32 * u + lane;
                // touching pairs (shared vertex index) go to their own list
                bool touch = false;
                if (redo[u]) touch = touching(__ldg(G.m.tvid + row[u]), __ldg(G.m.tvid + col[u]));
                for (int side = 0; side < 2; ++side) {
                    const bool mine = redo[u] && (side == 1) == touch;
                    const unsigned mask = __ballot_sync(0xffffffffu, mine);
                    if (!mask) continue;
                    unsigned long long base = 0;
                    const int leader = __ffs(mask) - 1;
                    if (lane == leader) base = atomicAdd(count + side, (unsigned long long)__popc(mask));
                    base = __shfl_sync(0xffffffffu, base, leader);
                    if (mine) {
                        const unsigned long long k = base + __popc(mask & ((1u << lane) - 1u));
                        if ((int64_t)k < (side == 0 ? cap : cap_t)) {
                            GuardItem it;
                            it.job = g.job;
                            it.row = row[u];
                            it.col = col[u];
                            it.off = g.off + e;
                            (side == 0 ? list : list_t)[k] = it;
                        } else {
                            set_status(status, BEM_ERR_OOM);
                            od[e] = (double)v[u].x;
                        }
                    }
                }
            }
        }
    }
}

// ---- double-float arithmetic for the disjoint pairs ----------------------
// An unevaluated pair (h, l) stands for h + l; products use FMA for their
// exact rounding error, sums Knuth's TwoSum (two_sum, dd_add, dd_sub, dd_mul in
// bem_device.cuh).

// (a - b) . (a - b) for pairs a - b given per component
__device__ __forceinline__ void dd_norm2(const float *dh, const float *dl, float &h, float &l)
{
    h = 0.0f;
    l = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float p = dh[c] * dh[c];
        const float pe = fmaf(dh[c], dh[c], -p) + 2.0f * dh[c] * dl[c];
        dd_add(h, l, p, pe, h, l);
    }
}

// 1 / sqrt(h + l): the hardware estimate refined by one Newton step evaluated
// in double-float (relative error about 1.5 times the square of the
// estimate's, ~2e-14)
__device__ __forceinline__ void dd_rsqrt(float h, float l, float &yh, float &yl)
{
    const float y0 = rsqrt_fast(h);
    const float q = y0 * y0, qe = fmaf(y0, y0, -q);
    const float t = h * q;
    const float te = fmaf(h, q, -t) + fmaf(h, qe, l * q);
    const float e = (1.0f - t) - te;          // 1 - t is exact: t is within 2^-22 of 1
    two_sum(y0, 0.5f * y0 * e, yh, yl);
}

// The rule of the disjoint pairs with every node and weight as a float pair.

struct GuardRule {
    int np;
    float sh[kMaxNp], sl[kMaxNp], th[kMaxNp], tl[kMaxNp], wh[kMaxNp], wl[kMaxNp];
};

// The Sauter-Schwab rules of the touching cases as double-float columns.
struct TouchRules {
    const float *h[4], *l[4];   // [case]: kRuleCols n floats each, hi and lo parts
    int n[4];
    int xi[4];                  // 1: xi integrated out (the double layer's factor 1/2)
};

// One warp per listed touching entry (common vertex or common edge; a flat
// identical pair has no double layer): the FP64 form's Sauter-Schwab rule of
// the pair's case and canonical vertex order, evaluated in double-float.  The
// test triangle's vertex heights above the trial plane come from the FP64
// records (as in the float touching kernels), the rest from the float
// records' hi + lo vertices.
__global__ void __launch_bounds__(256) k_guard_redo_touch(const GuardJob *__restrict__ jobs,
                                                          const GuardItem *__restrict__ list,
                                                          const unsigned long long *count,
                                                          int64_t cap, TouchRules R, int *status)
{
    const int64_t n = min((int64_t)*count, cap);
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n; w += warps) {
        const GuardItem it = list[w];
        const GuardJob &G = jobs[it.job];
        const MeshView &m = G.m;
        const int a = it.row, b = it.col;
        if (a < 0 || a >= m.nt || b < 0 || b >= m.nt) {
            if (lane == 0) set_status(status, BEM_ERR_INVALID_ARG);
            continue;
        }
        const int k = find_touching(m, a, b);
        if (k < 0) {
            if (lane == 0) set_status(status, BEM_ERR_INVALID_ARG);
            continue;
        }
        const int cas = __ldg(m.nb_case + k), pc = __ldg(m.nb_perm + k);
        float gh = 0.0f, gl = 0.0f;
        if (cas == kVertex || cas == kEdge) {
            const int *pa = c_perm[pc / 6], *pb = c_perm[pc % 6];
            TriF A, B;
            load_trif(m.geomf, a, A);
            load_trif(m.geomf, b, B);
            float e1ah[3], e1al[3], e2ah[3], e2al[3], e1bh[3], e1bl[3], e2bh[3], e2bl[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int a0 = pa[0], a1 = pa[1], a2 = pa[2], b0 = pb[0], b1 = pb[1], b2 = pb[2];
                dd_sub(A.vh[a1][c], A.vl[a1][c], A.vh[a0][c], A.vl[a0][c], e1ah[c], e1al[c]);
                dd_sub(A.vh[a2][c], A.vl[a2][c], A.vh[a1][c], A.vl[a1][c], e2ah[c], e2al[c]);
                dd_sub(B.vh[b1][c], B.vl[b1][c], B.vh[b0][c], B.vl[b0][c], e1bh[c], e1bl[c]);
                dd_sub(B.vh[b2][c], B.vl[b2][c], B.vh[b1][c], B.vl[b1][c], e2bh[c], e2bl[c]);
            }
            // heights of a's canonical vertices 1, 2 above b's plane (vertex 0 is
            // shared and lies in it), from the FP64 records
            double d1 = 0.0, d2 = 0.0;
            {
                const double *ga = m.geom + (int64_t)a * kGeomStride;
                const double *gb = m.geom + (int64_t)b * kGeomStride;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const double q0 = __ldg(gb + 3 * pb[0] + c), nn = __ldg(gb + 9 + c);
                    d1 = fma(__ldg(ga + 3 * pa[1] + c) - q0, nn, d1);
                    d2 = fma(__ldg(ga + 3 * pa[2] + c) - q0, nn, d2);
                }
            }
            // h(x) = x1 h1 + x2 (h2 - h1) on the canonical parametrisation; for
            // a common edge h1 = 0
            const double h21 = d2 - d1;
            const float h1h = (float)d1, h1l = (float)(d1 - (double)h1h);
            const float h21h = (float)h21, h21l = (float)(h21 - (double)h21h);
            const int np = R.n[cas];
            const float *Xh = R.h[cas], *Xl = R.l[cas];
            for (int p = lane; p < np; p += 32) {
                const float x1h = Xh[p], x1l = Xl[p], x2h = Xh[np + p], x2l = Xl[np + p];
                const float y1h = Xh[2 * np + p], y1l = Xl[2 * np + p];
                const float y2h = Xh[3 * np + p], y2l = Xl[3 * np + p];
                const float wh = Xh[4 * np + p], wl = Xl[4 * np + p];
                float dh[3], dl[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float th, tl, uh, ul;
                    if (cas == kVertex) {
                        // x1 e1a + x2 e2a - y1 e1b - y2 e2b
                        dd_mul(x1h, x1l, e1ah[c], e1al[c], th, tl);
                        dd_mul(x2h, x2l, e2ah[c], e2al[c], uh, ul);
                        dd_add(th, tl, uh, ul, th, tl);
                        dd_mul(y1h, y1l, e1bh[c], e1bl[c], uh, ul);
                        dd_sub(th, tl, uh, ul, th, tl);
                        dd_mul(y2h, y2l, e2bh[c], e2bl[c], uh, ul);
                        dd_sub(th, tl, uh, ul, dh[c], dl[c]);
                    } else {
                        // (x1 - y1) e1a + x2 e2a - y2 e2b, x1 - y1 from the rule
                        const float d1h = Xh[5 * np + p], d1l = Xl[5 * np + p];
                        dd_mul(d1h, d1l, e1ah[c], e1al[c], th, tl);
                        dd_mul(x2h, x2l, e2ah[c], e2al[c], uh, ul);
                        dd_add(th, tl, uh, ul, th, tl);
                        dd_mul(y2h, y2l, e2bh[c], e2bl[c], uh, ul);
                        dd_sub(th, tl, uh, ul, dh[c], dl[c]);
                    }
                }
                float hh, hl, uh, ul;
                dd_mul(x2h, x2l, h21h, h21l, hh, hl);
                if (cas == kVertex) {
                    dd_mul(x1h, x1l, h1h, h1l, uh, ul);
                    dd_add(hh, hl, uh, ul, hh, hl);
                }
                float r2h, r2l, rih, ril, r3h, r3l;
                dd_norm2(dh, dl, r2h, r2l);
                dd_rsqrt(r2h, r2l, rih, ril);
                dd_mul(rih, ril, rih, ril, uh, ul);
                dd_mul(uh, ul, rih, ril, r3h, r3l);
                dd_mul(r3h, r3l, hh, hl, uh, ul);
                dd_mul(uh, ul, wh, wl, uh, ul);
                dd_add(gh, gl, uh, ul, gh, gl);
            }
            warp_sum2f(gh, gl);
        }
        if (lane == 0) {
            const double sa = __ldg(m.geom + (int64_t)a * kGeomStride + 12);
            const double sb = __ldg(m.geom + (int64_t)b * kGeomStride + 12);
            const double xs = cas >= kVertex && R.xi[cas] ? xi_moment(BEM_LAPLACE_DLP, 0, 0) : 1.0;
            reinterpret_cast<double *>(G.L.out)[it.off] =
                ((double)gh + (double)gl) * (sa * sb * kInv4Pi) * xs;
        }
    }
}

// (s, t) -> s e1 + t e2 in double-float, per component
__device__ __forceinline__ void dd_affine(float sh, float sl, float th, float tl, const float *e1h,
                                          const float *e1l, const float *e2h, const float *e2l,
                                          float *oh, float *ol)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float ah, al, bh, bl;
        dd_mul(sh, sl, e1h[c], e1l[c], ah, al);
        dd_mul(th, tl, e2h[c], e2l[c], bh, bl);
        dd_add(ah, al, bh, bl, oh[c], ol[c]);
    }
}

// One thread per listed disjoint entry: the tensor product of the 2D rule with
// itself (the FP64 form's regular rule) in double-float.  Vertices come as the
// float records' hi + lo pairs (exact to ~2^-48), differences and the trial
// normal in double-float; the trial points' offsets stay in registers when
// the rule is small.
template <int NP>
__global__ void __launch_bounds__(128) k_guard_redo_dd(const GuardJob *__restrict__ jobs,
                                                       const GuardItem *__restrict__ list,
                                                       const unsigned long long *count,
                                                       int64_t cap, GuardRule R, int *status)
{
    constexpr bool CACHE = NP <= 9;
    const int64_t n = min((int64_t)*count, cap);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const GuardItem it = list[k];
        const GuardJob &G = jobs[it.job];
        const MeshView &m = G.m;
        const int a = it.row, b = it.col;
        if (a < 0 || a >= m.nt || b < 0 || b >= m.nt) {
            set_status(status, BEM_ERR_INVALID_ARG);
            continue;
        }
        TriF A, B;
        load_trif(m.geomf, a, A);
        load_trif(m.geomf, b, B);
        float d0h[3], d0l[3], e1ah[3], e1al[3], e2ah[3], e2al[3], e1bh[3], e1bl[3], e2bh[3],
            e2bl[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dd_sub(A.vh[0][c], A.vl[0][c], B.vh[0][c], B.vl[0][c], d0h[c], d0l[c]);
            dd_sub(A.vh[1][c], A.vl[1][c], A.vh[0][c], A.vl[0][c], e1ah[c], e1al[c]);
            dd_sub(A.vh[2][c], A.vl[2][c], A.vh[1][c], A.vl[1][c], e2ah[c], e2al[c]);
            dd_sub(B.vh[1][c], B.vl[1][c], B.vh[0][c], B.vl[0][c], e1bh[c], e1bl[c]);
            dd_sub(B.vh[2][c], B.vl[2][c], B.vh[1][c], B.vl[1][c], e2bh[c], e2bl[c]);
        }
        float yh[CACHE ? NP : 1][3], yl[CACHE ? NP : 1][3];
        if (CACHE) {
#pragma unroll
            for (int j = 0; j < NP; ++j)
                dd_affine(R.sh[j], R.sl[j], R.th[j], R.tl[j], e1bh, e1bl, e2bh, e2bl, yh[j], yl[j]);
        }
        float gh = 0.0f, gl = 0.0f;
#pragma unroll 1
        for (int i = 0; i < NP; ++i) {
            // x - y_0 at the test point, and its height above the trial plane
            float xh[3], xl[3];
            dd_affine(R.sh[i], R.sl[i], R.th[i], R.tl[i], e1ah, e1al, e2ah, e2al, xh, xl);
            float hh = 0.0f, hl = 0.0f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dd_add(xh[c], xl[c], d0h[c], d0l[c], xh[c], xl[c]);
                float ph, pl;
                dd_mul(xh[c], xl[c], B.nh[c], B.nl[c], ph, pl);
                dd_add(hh, hl, ph, pl, hh, hl);
            }
            float sh = 0.0f, sl = 0.0f;      // sum_j w_j / r^3
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                float ojh[3], ojl[3];
                if (CACHE) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        ojh[c] = yh[j][c];
                        ojl[c] = yl[j][c];
                    }
                } else {
                    dd_affine(R.sh[j], R.sl[j], R.th[j], R.tl[j], e1bh, e1bl, e2bh, e2bl, ojh, ojl);
                }
                float dh[3], dl[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) dd_sub(xh[c], xl[c], ojh[c], ojl[c], dh[c], dl[c]);
                float r2h, r2l, rih, ril, r3h, r3l, th2, tl2;
                dd_norm2(dh, dl, r2h, r2l);
                dd_rsqrt(r2h, r2l, rih, ril);
                dd_mul(rih, ril, rih, ril, th2, tl2);
                dd_mul(th2, tl2, rih, ril, r3h, r3l);
                dd_mul(R.wh[j], R.wl[j], r3h, r3l, th2, tl2);
                dd_add(sh, sl, th2, tl2, sh, sl);
            }
            float ph, pl;
            dd_mul(hh, hl, sh, sl, ph, pl);
            dd_mul(R.wh[i], R.wl[i], ph, pl, ph, pl);
            dd_add(gh, gl, ph, pl, gh, gl);
        }
        const double sa = __ldg(m.geom + (int64_t)a * kGeomStride + 12);
        const double sb = __ldg(m.geom + (int64_t)b * kGeomStride + 12);
        reinterpret_cast<double *>(G.L.out)[it.off] =
            ((double)gh + (double)gl) * (sa * sb * kInv4Pi);
    }
}

}  // namespace

namespace {

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

}  // namespace

cudaError_t guard_add(GuardSet &g, const MeshView &m, const BlockLaunch &L, cudaStream_t st)
{
    // entries of the job: sum over its blocks of |row cluster| * |column cluster|
    // (the caller's arrays, read in stream order)
    std::vector<int32_t> rp((size_t)L.n_row_clusters + 1), cp((size_t)L.n_col_clusters + 1);
    std::vector<int32_t> br((size_t)L.n_blocks), bc((size_t)L.n_blocks);
    cudaError_t e = cudaMemcpyAsync(rp.data(), L.row_ptr, rp.size() * sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cp.data(), L.col_ptr, cp.size() * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && L.n_blocks > 0)
        e = cudaMemcpyAsync(br.data(), L.blk_row, br.size() * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && L.n_blocks > 0)
        e = cudaMemcpyAsync(bc.data(), L.blk_col, bc.size() * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    int64_t n = 0;
    for (int64_t k = 0; k < L.n_blocks; ++k) {
        const int t = br[k], s = bc[k];
        if (t < 0 || t >= L.n_row_clusters || s < 0 || s >= L.n_col_clusters) continue;
        n += (int64_t)std::max(0, rp[t + 1] - rp[t]) * std::max(0, cp[s + 1] - cp[s]);
    }
    GuardJob j;
    j.m = m;
    j.L = L;
    j.rowmax = nullptr;
    j.n_rows = m.nt;
    g.host.push_back(j);
    g.blk_end.push_back((g.blk_end.empty() ? 0 : g.blk_end.back()) + L.n_blocks);
    g.rows += m.nt;
    g.entries += n;
    if (L.allow_touching) g.cap_t += m.ntouch;   // each touching pair at most once
    // room for one entry in 16 (measured: about 2% of the double-layer
    // entries of jittered meshes need the FP64 pass)
    g.cap = g.entries / 16 + 4096;
    return cudaSuccess;
}

size_t guard_bytes(const GuardSet &g)
{
    return align256(g.host.size() * sizeof(GuardJob)) + align256(g.blk_end.size() * sizeof(int64_t)) +
           align256((size_t)g.rows * sizeof(unsigned)) + align256(2 * sizeof(unsigned long long)) +
           align256((size_t)g.cap * sizeof(GuardItem)) + align256((size_t)g.cap_t * sizeof(GuardItem));
}

cudaError_t guard_layout(GuardSet &g, void *buf, cudaStream_t st)
{
    char *p = static_cast<char *>(buf);
    g.d_jobs = reinterpret_cast<GuardJob *>(p);
    p += align256(g.host.size() * sizeof(GuardJob));
    g.d_blk_end = reinterpret_cast<int64_t *>(p);
    p += align256(g.blk_end.size() * sizeof(int64_t));
    g.d_rowmax = reinterpret_cast<unsigned *>(p);
    p += align256((size_t)g.rows * sizeof(unsigned));
    g.d_count = reinterpret_cast<unsigned long long *>(p);
    p += align256(2 * sizeof(unsigned long long));
    g.d_list = reinterpret_cast<GuardItem *>(p);
    p += align256((size_t)g.cap * sizeof(GuardItem));
    g.d_list_t = reinterpret_cast<GuardItem *>(p);
    int64_t at = 0;
    for (auto &j : g.host) {
        j.rowmax = g.d_rowmax + at;
        at += j.n_rows;
    }
    // stream-ordered behind earlier guard passes that read the same buffer;
    // from pageable memory the call returns once the source has been staged
    cudaError_t e = cudaMemcpyAsync(g.d_jobs, g.host.data(), g.host.size() * sizeof(GuardJob),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g.d_blk_end, g.blk_end.data(), g.blk_end.size() * sizeof(int64_t),
                            cudaMemcpyHostToDevice, st);
    return e;
}

cudaError_t guard_run(const GuardSet &g, int num_sms, int *status, cudaStream_t st)
{
    const int n_jobs = (int)g.host.size();
    if (n_jobs <= 0 || g.blk_end.back() == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(g.d_rowmax, 0, (size_t)g.rows * sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g.d_count, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_guard_rowmax<<<num_sms * 8, 256, 0, st>>>(g.d_jobs, g.d_blk_end, n_jobs);
    k_guard_select<<<num_sms * 8, 256, 0, st>>>(g.d_jobs, g.d_blk_end, n_jobs, g.d_list, g.d_list_t,
                                                g.d_count, g.cap, g.cap_t, kGuardRel, status);
    GuardRule R;
    R.np = g.r2.np;
    auto split = [](double v, float &h, float &l) {
        h = (float)v;
        l = (float)(v - (double)h);
    };
    for (int k = 0; k < g.r2.np; ++k) {
        split(g.r2.s[k], R.sh[k], R.sl[k]);
        split(g.r2.t[k], R.th[k], R.tl[k]);
        split(g.r2.w[k], R.wh[k], R.wl[k]);
    }
    const int grid = num_sms * 8;
    switch (g.r2.np) {
    case 4: k_guard_redo_dd<4><<<grid, 128, 0, st>>>(g.d_jobs, g.d_list, g.d_count, g.cap, R, status); break;
    case 7: k_guard_redo_dd<7><<<grid, 128, 0, st>>>(g.d_jobs, g.d_list, g.d_count, g.cap, R, status); break;
    case 9: k_guard_redo_dd<9><<<grid, 128, 0, st>>>(g.d_jobs, g.d_list, g.d_count, g.cap, R, status); break;
    case 16: k_guard_redo_dd<16><<<grid, 128, 0, st>>>(g.d_jobs, g.d_list, g.d_count, g.cap, R, status); break;
    case 25: k_guard_redo_dd<25><<<grid, 128, 0, st>>>(g.d_jobs, g.d_list, g.d_count, g.cap, R, status); break;
    default: k_guard_redo_dd<1><<<grid, 128, 0, st>>>(g.d_jobs, g.d_list, g.d_count, g.cap, R, status); break;
    }
    TouchRules tr;
    for (int c = 0; c < 4; ++c) {
        tr.h[c] = g.rules[c].f;
        tr.l[c] = g.rules[c].fl;
        tr.n[c] = g.rules[c].n;
        tr.xi[c] = g.rules[c].xi;
    }
    if (g.cap_t > 0)
        k_guard_redo_touch<<<num_sms * 4, 256, 0, st>>>(g.d_jobs, g.d_list_t, g.d_count + 1,
                                                        g.cap_t, tr, status);
    return cudaGetLastError();
}

}  // namespace bem
