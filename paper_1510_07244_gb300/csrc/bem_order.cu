// Learned quadrature-order selection for disjoint (regular) triangle pairs.
//
// The paper uses one fixed rule per Sauter-Schwab case (Section 2.2 and the
// "higher quadrature orders" study of Section 4).  Here a small MLP,
// 8 pair features -> 64 -> 64 -> 6 rule classes (ReLU), predicts for every
// disjoint pair the cheapest rule that meets an error target; the classes
// form a ladder of increasing accuracy and cost:
//     0: Duffy q=2 (16 points)   1: Radon 7x7 (49)   2: Duffy q=4 (256)
//     3: Duffy q=5 (625)         4: Duffy q=6 (1296) 5: Duffy q=8 (4096).
// A pair gets the cheapest class whose cumulative predicted probability
// reaches the confidence level (so uncertainty moves it up the ladder).
//
// Training runs on the GPU with the kernels below (FP32 forward, backward and
// Adam, batch sums in a fixed order, so a training step is deterministic);
// inference uses BF16 weights and activations on the tensor cores
// (mma.sync m16n8k16, FP32 accumulation).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "bem_device.cuh"

namespace bem {

// ---------------------------------------------------------------------------
// Pair features (8): log2(centroid distance / D), log2(closest vertex
// distance / D), cos(angle between normals), log2(area ratio), height of the
// test centroid above the trial plane / centroid distance, kernel id / 2,
// kappa D, log2(aspect ratio); D = the larger triangle diameter.  Normalised
// by the model's mean and standard deviation.  Float arithmetic (a feature
// only has to place the pair among the classes).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pair_features_rec(const TriF &A, const TriF &B, int kind,
                                                  double kappa, const float *mean,
                                                  const float *inv_std, float *f)
{
    // float arithmetic on the double-float records: vertex offsets from each
    // triangle's vertex 0, and the offset between the two vertices 0 formed from
    // the hi + lo pairs, so every difference keeps float precision
    float oa[3][3], ob[3][3], d0[3], na[3], nb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        oa[0][c] = 0.0f;
        oa[1][c] = A.e1[c];
        oa[2][c] = A.e1[c] + A.e2[c];
        ob[0][c] = 0.0f;
        ob[1][c] = B.e1[c];
        ob[2][c] = B.e1[c] + B.e2[c];
        d0[c] = dd_diff(A.vh[0][c], A.vl[0][c], B.vh[0][c], B.vl[0][c]);
        na[c] = A.nh[c] + A.nl[c];
        nb[c] = B.nh[c] + B.nl[c];
    }
    float da2 = 0.0f, db2 = 0.0f, dmin2 = 3.0e38f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3;
        float ea = 0.0f, eb = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ea = fmaf(oa[i][c] - oa[j][c], oa[i][c] - oa[j][c], ea);
            eb = fmaf(ob[i][c] - ob[j][c], ob[i][c] - ob[j][c], eb);
        }
        da2 = fmaxf(da2, ea);
        db2 = fmaxf(db2, eb);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float dd = 0.0f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float x = d0[c] + oa[i][c] - ob[k][c];
                dd = fmaf(x, x, dd);
            }
            dmin2 = fminf(dmin2, dd);
        }
    }
    const float D = sqrtf(fmaxf(da2, db2));
    float dc2 = 0.0f, h = 0.0f, cosang = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float dcv = d0[c] + (oa[1][c] + oa[2][c] - ob[1][c] - ob[2][c]) * (1.0f / 3.0f);
        dc2 = fmaf(dcv, dcv, dc2);
        h = fmaf(dcv, nb[c], h);
        cosang = fmaf(na[c], nb[c], cosang);
    }
    const float dc = sqrtf(dc2);
    const float area_a = 0.5f * A.sg, area_b = 0.5f * B.sg;
    const float ar = fmaxf(da2 / (2.0f * area_a), db2 / (2.0f * area_b));
    float raw[8];
    raw[0] = __log2f(fmaxf(dc / D, 1e-6f));
    raw[1] = __log2f(fmaxf(sqrtf(dmin2) / D, 1e-6f));
    raw[2] = cosang;
    raw[3] = __log2f(area_a / area_b);
    raw[4] = h / fmaxf(dc, 1e-30f);
    raw[5] = 0.5f * (float)kind;
    raw[6] = kind == BEM_HELMHOLTZ_SLP ? (float)kappa * D : 0.0f;
    raw[7] = __log2f(ar);
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] = (raw[k] - mean[k]) * inv_std[k];
}

__device__ __forceinline__ void pair_features(const MeshView &m, int a, int b, int kind,
                                              double kappa, const float *mean, const float *inv_std,
                                              float *f)
{
    TriF A, B;
    load_trif(m.geomf, a, A);
    load_trif(m.geomf, b, B);
    pair_features_rec(A, B, kind, kappa, mean, inv_std, f);
}

__global__ void k_features(MeshView m, const int32_t *__restrict__ a_idx,
                           const int32_t *__restrict__ b_idx, int64_t n, int kind, double kappa,
                           const float *mean, const float *inv_std, float *X)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    pair_features(m, a_idx[i], b_idx[i], kind, kappa, mean, inv_std, X + 8 * i);
}

// ---------------------------------------------------------------------------
// Training kernels (FP32).  Parameter layout (floats): W1[64][8] b1[64]
// W2[64][64] b2[64] W3[6][64] b3[6].
// ---------------------------------------------------------------------------
constexpr int kIn = 8, kHid = 64, kOut = 6;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid,
              kOffB2 = kOffW2 + kHid * kHid, kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kOut * kHid,
              kNParams = kOffB3 + kOut;

// z = in W^T + b (rows x outd), optional ReLU copy
__global__ void k_dense(const float *in, int rows, int ind, const float *W, const float *b, int outd,
                        float *z, float *h)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)rows * outd) return;
    const int64_t i = t / outd;
    const int o = (int)(t % outd);
    float s = b[o];
    for (int k = 0; k < ind; ++k) s = fmaf(in[i * ind + k], W[o * ind + k], s);
    z[t] = s;
    if (h) h[t] = fmaxf(s, 0.0f);
}

// softmax cross entropy: dz = (p - onehot) / n, per-row loss
__global__ void k_softmax_ce(const float *logits, const int32_t *y, int n, float *dz, float *loss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float mx = -1e30f;
    for (int o = 0; o < kOut; ++o) mx = fmaxf(mx, logits[i * kOut + o]);
    float se = 0.0f;
    for (int o = 0; o < kOut; ++o) se += expf(logits[i * kOut + o] - mx);
    const int yi = y[i];
    for (int o = 0; o < kOut; ++o) {
        const float p = expf(logits[i * kOut + o] - mx) / se;
        dz[i * kOut + o] = (p - (o == yi ? 1.0f : 0.0f)) / (float)n;
    }
    loss[i] = -(logits[i * kOut + yi] - mx - logf(se));
}

// dW[o][k] = sum_i dz[i][o] in[i][k], db[o] = sum_i dz[i][o]  (fixed order over i)
__global__ void k_weight_grad(const float *dz, const float *in, int rows, int outd, int ind,
                              float *dW, float *db)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < outd * ind) {
        const int o = t / ind, k = t % ind;
        float s = 0.0f;
        for (int i = 0; i < rows; ++i) s = fmaf(dz[(int64_t)i * outd + o], in[(int64_t)i * ind + k], s);
        dW[t] = s;
    } else if (t < outd * ind + outd) {
        const int o = t - outd * ind;
        float s = 0.0f;
        for (int i = 0; i < rows; ++i) s += dz[(int64_t)i * outd + o];
        db[o] = s;
    }
}

// dprev[i][k] = (sum_o dz[i][o] W[o][k]) * (zprev[i][k] > 0)
__global__ void k_back_act(const float *dz, const float *W, const float *zprev, int rows, int outd,
                           int ind, float *dprev)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)rows * ind) return;
    const int64_t i = t / ind;
    const int k = (int)(t % ind);
    float s = 0.0f;
    for (int o = 0; o < outd; ++o) s = fmaf(dz[i * outd + o], W[o * ind + k], s);
    dprev[t] = zprev[t] > 0.0f ? s : 0.0f;
}

__global__ void k_adam(float *p, const float *g, float *m1, float *m2, int n, float lr, float b1,
                       float b2, float eps, float c1, float c2)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    m1[t] = b1 * m1[t] + (1.0f - b1) * g[t];
    m2[t] = b2 * m2[t] + (1.0f - b2) * g[t] * g[t];
    p[t] -= lr * (m1[t] / c1) / (sqrtf(m2[t] / c2) + eps);
}

__global__ void k_sum_fixed(const float *x, int n, float *out)
{
    // one CTA, fixed-order strided partial sums then a tree
    __shared__ float part[256];
    float s = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0];
}

__global__ void k_to_bf16(const float *p, int n, __nv_bfloat16 *q)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) q[t] = __float2bfloat16_rn(p[t]);
}

// ---------------------------------------------------------------------------
// Inference on the tensor cores: one warp evaluates 16 feature rows per
// mma.sync.m16n8k16 (BF16 inputs, FP32 accumulators).  Fragment layouts of
// m16n8k16 (PTX ISA): A row-major 16x16, thread t holds rows t/4 and t/4+8,
// columns 2(t%4)+{0,1} and +8; B col-major 16x8, thread t holds k = 2(t%4)+{0,1}
// and +8 of column t/4; C 16x8, rows t/4 and t/4+8, columns 2(t%4)+{0,1}.
// The C fragments of two neighbouring 8-column tiles form the A fragment of
// the next layer's 16-wide k tile, so activations stay in registers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned *>(&v);
}

__device__ __forceinline__ void mma_bf16(float *c, const unsigned *a, const unsigned *b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// B fragment of W (out x in, row-major BF16) for output tile n0 (8 columns)
// and k tile k0 (16 inputs); inputs beyond `ind` and outputs beyond `outd` are 0.
__device__ __forceinline__ void load_b(const __nv_bfloat16 *W, int outd, int ind, int n0, int k0,
                                       int lane, unsigned *b)
{
    const int n = n0 + lane / 4, k = k0 + 2 * (lane % 4);
    __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
    auto at = [&](int kk) { return (n < outd && kk < ind) ? W[n * ind + kk] : z; };
    __nv_bfloat162 v0, v1;
    v0.x = at(k);
    v0.y = at(k + 1);
    v1.x = at(k + 8);
    v1.y = at(k + 9);
    b[0] = *reinterpret_cast<unsigned *>(&v0);
    b[1] = *reinterpret_cast<unsigned *>(&v1);
}

struct MlpDev {
    const __nv_bfloat16 *W1, *W2, *W3;
    const float *b1, *b2, *b3;
};

// The B operands of all three layers in mma fragment order, staged once per CTA
// in shared memory: each lane loads its fragment with one 8-byte read.
struct MlpFrag {
    uint2 w1[8][32];       // [n tile][lane]        (K = 8, padded to one 16-wide k tile)
    uint2 w2[8][4][32];    // [n tile][k tile][lane]
    uint2 w3[4][32];       // [k tile][lane]         (N = 6, padded to one 8-wide n tile)
    float b1[kHid], b2[kHid], b3[8];
};

// Called by every thread of the CTA (contains a barrier).
__device__ __forceinline__ void mlp_stage(const MlpDev &P, MlpFrag &F)
{
    for (int i = threadIdx.x; i < 8 * 32; i += blockDim.x) {
        unsigned b[2];
        load_b(P.W1, kHid, kIn, (i / 32) * 8, 0, i % 32, b);
        F.w1[i / 32][i % 32] = make_uint2(b[0], b[1]);
    }
    for (int i = threadIdx.x; i < 8 * 4 * 32; i += blockDim.x) {
        const int nt = i / 128, kt = (i / 32) % 4, ln = i % 32;
        unsigned b[2];
        load_b(P.W2, kHid, kHid, nt * 8, kt * 16, ln, b);
        F.w2[nt][kt][ln] = make_uint2(b[0], b[1]);
    }
    for (int i = threadIdx.x; i < 4 * 32; i += blockDim.x) {
        unsigned b[2];
        load_b(P.W3, kOut, kHid, 0, (i / 32) * 16, i % 32, b);
        F.w3[i / 32][i % 32] = make_uint2(b[0], b[1]);
    }
    for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
        F.b1[i] = P.b1[i];
        F.b2[i] = P.b2[i];
    }
    if (threadIdx.x < 8) F.b3[threadIdx.x] = threadIdx.x < kOut ? P.b3[threadIdx.x] : 0.0f;
    __syncthreads();
}

// 16 rows (features in X16, row-major 16 x 8 float) -> logits of rows t/4 and
// t/4 + 8 for this lane's two classes 2(t%4), 2(t%4)+1 (classes < 8).
__device__ __forceinline__ void mlp_tile(const MlpFrag &F, const float (*X16)[8], int lane,
                                         float *out_lo, float *out_hi)
{
    const int r = lane / 4, cq = 2 * (lane % 4);
    // layer 1: K = 8 (padded to 16)
    unsigned a[4];
    a[0] = pack_bf16(X16[r][cq], X16[r][cq + 1]);
    a[1] = pack_bf16(X16[r + 8][cq], X16[r + 8][cq + 1]);
    a[2] = 0u;   // columns 8..15 are padding
    a[3] = 0u;
    // layer 1, its ReLU outputs packed at once into layer 2's A fragments: n tile
    // 2kt fills registers 0 and 1 of k tile kt, n tile 2kt + 1 registers 2 and 3
    unsigned a1[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const uint2 bw = F.w1[nt][lane];
        const unsigned b[2] = {bw.x, bw.y};
        const int col = nt * 8 + cq;
        float h[4] = {F.b1[col], F.b1[col + 1], F.b1[col], F.b1[col + 1]};
        mma_bf16(h, a, b);
        a1[nt / 2][2 * (nt % 2)] = pack_bf16(fmaxf(h[0], 0.0f), fmaxf(h[1], 0.0f));
        a1[nt / 2][2 * (nt % 2) + 1] = pack_bf16(fmaxf(h[2], 0.0f), fmaxf(h[3], 0.0f));
    }
    // layer 2: K = 64 (4 k tiles), N = 64 (8 n tiles)
    float h2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int col = nt * 8 + cq;
        h2[nt][0] = F.b2[col];
        h2[nt][1] = F.b2[col + 1];
        h2[nt][2] = F.b2[col];
        h2[nt][3] = F.b2[col + 1];
    }
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const uint2 bw = F.w2[nt][kt][lane];
            const unsigned b[2] = {bw.x, bw.y};
            mma_bf16(h2[nt], a1[kt], b);
        }
    }
    // layer 3: K = 64, N = 6 (one 8-column tile)
    float o[4] = {F.b3[cq], F.b3[cq + 1], F.b3[cq], F.b3[cq + 1]};   // zero beyond kOut
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        unsigned ak[4];
        ak[0] = pack_bf16(fmaxf(h2[2 * kt][0], 0.0f), fmaxf(h2[2 * kt][1], 0.0f));
        ak[1] = pack_bf16(fmaxf(h2[2 * kt][2], 0.0f), fmaxf(h2[2 * kt][3], 0.0f));
        ak[2] = pack_bf16(fmaxf(h2[2 * kt + 1][0], 0.0f), fmaxf(h2[2 * kt + 1][1], 0.0f));
        ak[3] = pack_bf16(fmaxf(h2[2 * kt + 1][2], 0.0f), fmaxf(h2[2 * kt + 1][3], 0.0f));
        const uint2 bw = F.w3[kt][lane];
        const unsigned b[2] = {bw.x, bw.y};
        mma_bf16(o, ak, b);
    }
    out_lo[0] = o[0];
    out_lo[1] = o[1];
    out_hi[0] = o[2];
    out_hi[1] = o[3];
}

// Logits of n feature rows (n padded inside to multiples of 16): one warp per 16 rows.
__global__ void k_mlp_infer(MlpDev P, const float *__restrict__ X, int64_t n, float *logits)
{
    __shared__ float xs[8][16][8];
    __shared__ MlpFrag F;
    mlp_stage(P, F);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + w) * 16;
    if (row0 >= n) return;
    for (int k = lane; k < 128; k += 32) {
        const int rr = k / 8, cc = k % 8;
        xs[w][rr][cc] = row0 + rr < n ? X[(row0 + rr) * 8 + cc] : 0.0f;
    }
    __syncwarp();
    float lo[2], hi[2];
    mlp_tile(F, xs[w], lane, lo, hi);
    const int r = lane / 4, cq = 2 * (lane % 4);
    for (int q = 0; q < 2; ++q) {
        const int c = cq + q;
        if (c >= kOut) continue;
        if (row0 + r < n) logits[(row0 + r) * kOut + c] = lo[q];
        if (row0 + r + 8 < n) logits[(row0 + r + 8) * kOut + c] = hi[q];
    }
}

// ---------------------------------------------------------------------------
// Learned-order near field (piecewise constant).
//   select:  per tile entry (32 x 8 tiles as in the block engine): touching
//            pairs are written from the touching table; disjoint pairs get
//            features, the warp's 32 pairs go through the MLP on the tensor
//            cores (two 16-row tiles), and the class (argmax; the most
//            accurate class when the top softmax probability is below the
//            confidence threshold) is stored per entry and counted.
//   compact: a second walk writes (output position, a, b) records grouped by
//            class (within a class in any order; each record owns its output).
//   eval:    one warp per record with the class's rule.
// ---------------------------------------------------------------------------
constexpr int kClasses = 6;
// the classes' regular rules: (rule, q)
static const int kClassRule[kClasses][2] = {{BEM_RULE_DUFFY, 2}, {BEM_RULE_TRI7, 1},
                                            {BEM_RULE_DUFFY, 4}, {BEM_RULE_DUFFY, 5},
                                            {BEM_RULE_DUFFY, 6}, {BEM_RULE_DUFFY, 8}};

// Entry threadIdx.x of flat tile `tile` (flat_entry; every lane of the warp
// calls this), with both triangles' records.  The records are loaded beside
// the vertex ids and the features are formed before the touching test, so the
// loads of a tile wait once.  A touching pair is written from the touching
// table; its features are unused.
__device__ __forceinline__ void select_entry(const MeshView &m, const BlockLaunch &L,
                                             const int64_t *prefix, int64_t tile, int *status,
                                             const float *mean, const float *inv_std,
                                             int &a, int &b, int64_t &pos, int &state,
                                             int64_t &hint, float *f)
{
    // state: 0 = no entry, 1 = done (touching, written), 2 = regular pair
    state = 0;
    const FlatEntry fe = flat_entry(m, L, prefix, tile, status, hint);
    if (!fe.ok) return;
    a = fe.a;
    b = fe.b;
    pos = fe.pos;
    const int4 va = __ldg(m.tvid + a), vb = __ldg(m.tvid + b);
    TriF A, B;
    load_trif(m.geomf, a, A);
    load_trif(m.geomf, b, B);
    pair_features_rec(A, B, L.kind, L.kappa, mean, inv_std, f);
    if (touching(va, vb)) {
        // near field: the touching table's value; a touching pair in a coupling
        // block (no table) means the block was not admissible
        const int k = L.allow_touching ? find_touching(m, a, b) : -1;
        const double2 v = k >= 0 ? m.table[k] : make_double2(0.0, 0.0);
        if (k < 0) set_status(status, BEM_ERR_INVALID_ARG);
        if (L.kind == BEM_HELMHOLTZ_SLP) reinterpret_cast<double2 *>(L.out)[pos] = v;
        else reinterpret_cast<double *>(L.out)[pos] = v.x;
        state = 1;
        return;
    }
    state = 2;
}

struct LearnedArgs {
    MlpDev P;
    const float *mean, *inv_std;
    float conf;                  // confidence level of the cumulative class probability
    unsigned char *cls;          // per tile slot: class (255 = no regular pair)
    int *counts;                 // [kClasses]
    int64_t *offs;               // [kClasses + 1]
    int4 *rec;                   // records: (pos lo, pos hi, a, b)
    int *tcount;                 // [kClasses][8 ntile]: per warp of a tile, then its exclusive offset in the class
    int64_t ntile;               // tiles the scratch holds
};

// Tiles of a learned job: the list's entries in flat tiles of kP0Tile, at most
// the scratch's capacity (a list that outgrew it is reported by the selection).
__device__ __forceinline__ int64_t learned_tiles(const BlockLaunch &L, const int64_t *prefix,
                                                 int64_t cap)
{
    const int64_t t = L.n_blocks > 0 ? (prefix[L.n_blocks - 1] + kP0Tile - 1) / kP0Tile : 0;
    return t < cap ? t : cap;
}

// Capped at 64 registers (four CTAs, 32 warps per SM): the tiles' dependent
// loads want the warps, and the two MLP tiles run one after the other to fit.
__global__ void __launch_bounds__(256, 4) k_learned_select(MeshView m, BlockLaunch L,
                                                           const int64_t *__restrict__ prefix,
                                                           LearnedArgs A, int *status)
{
    // xs: per warp its 32 rows of features, then (same place) their logits
    __shared__ __align__(16) float xs[8][2][16][8];
    __shared__ float norm[2][8];
    __shared__ MlpFrag F;
    if (threadIdx.x < 16) norm[threadIdx.x / 8][threadIdx.x % 8] =
        threadIdx.x < 8 ? A.mean[threadIdx.x] : A.inv_std[threadIdx.x - 8];
    mlp_stage(A.P, F);   // ends with a barrier
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // prefix counts entries; a tile is kP0Tile of them
    const int64_t total = learned_tiles(L, prefix, A.ntile);
    if (blockIdx.x == 0 && threadIdx.x == 0 && L.n_blocks > 0 &&
        (prefix[L.n_blocks - 1] + kP0Tile - 1) / kP0Tile > A.ntile)
        set_status(status, BEM_ERR_INVALID_ARG);   // the lists outgrew the scratch
    // contiguous runs of tiles per CTA: the block search starts from the
    // previous tile's block
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * per, t1 = min(total, t0 + per);
    int64_t hint = -1;
    const int my_t = lane / 16, my_r = lane % 16;   // this lane's row: tile, row in tile
    const int r = lane / 4, cq = 2 * (lane % 4);    // mma fragment: row, class pair
    for (int64_t tile = t0; tile < t1; ++tile) {
        int a = 0, b = 0, state = 0;
        int64_t pos = 0;
        float f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        select_entry(m, L, prefix, tile, status, norm[0], norm[1], a, b, pos, state, hint, f);
#pragma unroll
        for (int k = 0; k < 8; ++k) xs[w][my_t][my_r][k] = state == 2 ? f[k] : 0.0f;
        __syncwarp();
        // logits of the warp's 32 rows: two 16-row tiles, one after the other,
        // each written back over its features once every lane has read them
#pragma unroll 1
        for (int t = 0; t < 2; ++t) {
            float lo[2], hi[2];
            mlp_tile(F, xs[w][t], lane, lo, hi);
            __syncwarp();
            *reinterpret_cast<float2 *>(&xs[w][t][r][cq]) = make_float2(lo[0], lo[1]);
            *reinterpret_cast<float2 *>(&xs[w][t][r + 8][cq]) = make_float2(hi[0], hi[1]);
        }
        __syncwarp();
        const float4 l0 = *reinterpret_cast<const float4 *>(&xs[w][my_t][my_r][0]);
        const float4 l1 = *reinterpret_cast<const float4 *>(&xs[w][my_t][my_r][4]);
        __syncwarp();   // the next tile's features overwrite xs
        const float logit[kClasses] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y};
        int cls = 255;
        if (state == 2) {
            float mx = logit[0];
#pragma unroll
            for (int cc = 1; cc < kClasses; ++cc) mx = fmaxf(mx, logit[cc]);
            float e[kClasses], se = 0.0f;
#pragma unroll
            for (int cc = 0; cc < kClasses; ++cc) {
                e[cc] = __expf(logit[cc] - mx);
                se += e[cc];
            }
            // cheapest class whose cumulative probability reaches the confidence
            cls = kClasses - 1;
            float cum = 0.0f;
#pragma unroll
            for (int cc = 0; cc < kClasses; ++cc) {
                cum += e[cc];
                if (cum >= A.conf * se) {
                    cls = cc;
                    break;
                }
            }
        }
        // the warp's class counts (no atomics and no barrier: a scan over the
        // tiles' warps follows)
#pragma unroll
        for (int cc = 0; cc < kClasses; ++cc) {
            const unsigned mk = __ballot_sync(0xffffffffu, cls == cc);
            if (lane == 0) A.tcount[cc * 8 * A.ntile + tile * 8 + w] = __popc(mk);
        }
        A.cls[tile * 256 + threadIdx.x] = (unsigned char)cls;
    }
}

// Exclusive scan of the warps' class counts (8 per tile, in entry order) in
// place, per class, in kScanSeg segments: segment sums (one CTA per class and
// segment, coalesced), the segments' offsets and the class totals (one warp
// per class), then each segment rescanned with its offset in chunks of 256
// (warp shuffles and the chunk's warp totals).  Integer sums, so the order of
// the additions does not matter.
constexpr int kScanSeg = 64;

__device__ __forceinline__ int64_t scan_len(const BlockLaunch &L, const int64_t *prefix,
                                            const LearnedArgs &A)
{
    return 8 * learned_tiles(L, prefix, A.ntile);
}

__global__ void __launch_bounds__(256) k_learned_seg_sum(BlockLaunch L,
                                                         const int64_t *__restrict__ prefix,
                                                         LearnedArgs A, int *seg)
{
    __shared__ int ws[8];
    const int c = blockIdx.x / kScanSeg, g = blockIdx.x % kScanSeg;
    const int64_t n = scan_len(L, prefix, A), len = (n + kScanSeg - 1) / kScanSeg;
    const int64_t lo = min(n, g * len), hi = min(n, lo + len);
    const int *t = A.tcount + c * 8 * A.ntile;
    int sum = 0;
    for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) sum += t[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int k = 0; k < 8; ++k) s += ws[k];
        seg[blockIdx.x] = s;
    }
}

// one warp per class: exclusive offsets of the segments, and the class total
__global__ void k_learned_seg_off(LearnedArgs A, int *seg)
{
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (c >= kClasses) return;
    int run = 0;
    for (int g0 = 0; g0 < kScanSeg; g0 += 32) {
        const int v = seg[c * kScanSeg + g0 + lane];
        int x = v;   // inclusive warp scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        seg[c * kScanSeg + g0 + lane] = run + x - v;
        run += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) A.counts[c] = run;
}

__global__ void __launch_bounds__(256) k_learned_seg_apply(BlockLaunch L,
                                                           const int64_t *__restrict__ prefix,
                                                           LearnedArgs A, const int *seg)
{
    __shared__ int ws[8];
    __shared__ int carry;
    const int c = blockIdx.x / kScanSeg, g = blockIdx.x % kScanSeg;
    const int64_t n = scan_len(L, prefix, A), len = (n + kScanSeg - 1) / kScanSeg;
    const int64_t lo = min(n, g * len), hi = min(n, lo + len);
    int *t = A.tcount + c * 8 * A.ntile;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = seg[blockIdx.x];
    __syncthreads();
    for (int64_t k0 = lo; k0 < hi; k0 += blockDim.x) {
        const int64_t k = k0 + threadIdx.x;
        const int v = k < hi ? t[k] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[w] = x;
        __syncthreads();
        int before = carry;
        for (int k2 = 0; k2 < w; ++k2) before += ws[k2];
        if (k < hi) t[k] = before + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + x;
        __syncthreads();
    }
}

__global__ void k_learned_offsets(LearnedArgs A)
{
    if (threadIdx.x == 0) {
        int64_t s = 0;
        for (int c = 0; c < kClasses; ++c) {
            A.offs[c] = s;
            s += A.counts[c];
        }
        A.offs[kClasses] = s;
    }
}

// Records by class at the scanned offsets: the warp's offset (k_learned_scan)
// + the lane's rank in its warp, so the records of a class come in entry order
// and no atomics or barriers are needed.
__global__ void __launch_bounds__(256) k_learned_compact(MeshView m, BlockLaunch L,
                                                         const int64_t *__restrict__ prefix,
                                                         LearnedArgs A)
{
    const int64_t total = learned_tiles(L, prefix, A.ntile);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * per, t1 = min(total, t0 + per);
    int64_t hint = -1;
    for (int64_t tile = t0; tile < t1; ++tile) {
        const int cls = A.cls[tile * 256 + threadIdx.x];
        // warp-uniform: flat_entry shuffles across the warp
        if (!__ballot_sync(0xffffffffu, cls < kClasses)) continue;
        unsigned mine = 0;
#pragma unroll
        for (int cc = 0; cc < kClasses; ++cc) {
            const unsigned mk = __ballot_sync(0xffffffffu, cls == cc);
            if (cls == cc) mine = mk;
        }
        // the selection pass already checked the indices (status not set twice)
        const FlatEntry fe = flat_entry(m, L, prefix, tile, nullptr, hint);
        if (cls < kClasses) {
            const int k = A.tcount[cls * 8 * A.ntile + tile * 8 + w] +
                          __popc(mine & ((1u << lane) - 1u));
            A.rec[A.offs[cls] + k] = make_int4((int)(fe.pos & 0xffffffff), (int)(fe.pos >> 32),
                                               fe.a, fe.b);
        }
    }
}

// Float form, classes whose rule is a product of a 2D rule with at most 25
// points: one thread per pair with the block engine's pair integrals.
template <int KIND, int NP>
__global__ void __launch_bounds__(256) k_learned_eval_tp(MeshView m, const int4 *__restrict__ rec,
                                                         const int64_t *__restrict__ offs, int cls,
                                                         Rule2D R, double kappa, void *out)
{
    const int64_t lo = offs[cls], hi = offs[cls + 1];
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < hi; k += nt) {
        const int4 Rk = rec[k];
        const int64_t pos = (int64_t)(unsigned)Rk.x | ((int64_t)Rk.y << 32);
        TriF A, B;
        load_trif(m.geomf, Rk.z, A);
        load_trif(m.geomf, Rk.w, B);
        if (KIND == BEM_HELMHOLTZ_SLP) {
            float fr, fi;
            regular_p0_f32_helm<NP>(A, B, R, kappa, fr, fi);
            reinterpret_cast<double2 *>(out)[pos] = make_double2((double)fr, (double)fi);
        } else {
            reinterpret_cast<double *>(out)[pos] = (double)regular_p0_f32<KIND, NP>(A, B, R);
        }
    }
}

// Float form, the larger product rules (Duffy q = 6, 8: 36, 64 points per
// triangle): one thread per pair, trial points taken CH at a time so that their
// coordinates fit in registers; the test-point loop stays rolled.
template <int NP>
struct RuleF {
    float s[NP], t[NP], w[NP];
};

template <int KIND, int NP, int CH>
__global__ void __launch_bounds__(256) k_learned_eval_big(MeshView m, const int4 *__restrict__ rec,
                                                          const int64_t *__restrict__ offs, int cls,
                                                          RuleF<NP> R, double kappa, void *out)
{
    static_assert(NP % CH == 0, "chunks must tile the rule");
    constexpr bool CPLX = KIND == BEM_HELMHOLTZ_SLP;
    const int64_t lo = offs[cls], hi = offs[cls + 1];
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < hi; k += nt) {
        const int4 Rk = rec[k];
        const int64_t pos = (int64_t)(unsigned)Rk.x | ((int64_t)Rk.y << 32);
        TriF A, B;
        load_trif(m.geomf, Rk.z, A);
        load_trif(m.geomf, Rk.w, B);
        // Laplace: positions relative to B's vertex 0; Helmholtz: to the centroids
        float d0[3] = {0.0f, 0.0f, 0.0f};
        Height H = {};
        HelmPhase P;
        if (CPLX) {
            P = helm_phase(A, B, kappa);
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c)
                d0[c] = dd_diff(A.vh[0][c], A.vl[0][c], B.vh[0][c], B.vl[0][c]);
            if (KIND == BEM_LAPLACE_DLP)
                H = make_height(A.vh[0], A.vl[0], A.vh[1], A.vl[1], A.vh[2], A.vl[2], B.vh[0],
                                B.vl[0], B.nh, B.nl);
        }
        const float sh = CPLX ? 0.666666687f : 0.0f, th = CPLX ? 0.333333343f : 0.0f;
        float sr = 0.0f, cr = 0.0f, si = 0.0f, ci = 0.0f;
#pragma unroll 1
        for (int jc = 0; jc < NP; jc += CH) {
            float yx[CH], yy[CH], yz[CH];
#pragma unroll
            for (int j = 0; j < CH; ++j) {
                const float a = R.s[jc + j] - sh, b = R.t[jc + j] - th;
                yx[j] = fmaf(a, B.e1[0], b * B.e2[0]);
                yy[j] = fmaf(a, B.e1[1], b * B.e2[1]);
                yz[j] = fmaf(a, B.e1[2], b * B.e2[2]);
            }
#pragma unroll 1
            for (int i = 0; i < NP; ++i) {
                const float a = R.s[i] - sh, b = R.t[i] - th;
                const float xx = fmaf(a, A.e1[0], fmaf(b, A.e2[0], d0[0]));
                const float xy = fmaf(a, A.e1[1], fmaf(b, A.e2[1], d0[1]));
                const float xz = fmaf(a, A.e1[2], fmaf(b, A.e2[2], d0[2]));
                const float dn = KIND == BEM_LAPLACE_DLP ? height_at(H, R.s[i], R.t[i]) : 0.0f;
                float ir = 0.0f, ii = 0.0f;
#pragma unroll
                for (int j = 0; j < CH; ++j) {
                    if (CPLX) {
                        float c, s, ri;
                        helm_offset(P, xx - yx[j], xy - yy[j], xz - yz[j], c, s, ri);
                        const float wr = R.w[jc + j] * ri;
                        ir = fmaf(c, wr, ir);
                        ii = fmaf(s, wr, ii);
                    } else {
                        ir = fmaf(R.w[jc + j], kvalf_r<KIND>(xx - yx[j], xy - yy[j], xz - yz[j]), ir);
                    }
                }
                if (KIND == BEM_LAPLACE_DLP) ir *= dn;
                // Kahan sums over the (test point, chunk) partial sums
                float y = fmaf(R.w[i], ir, -cr), t = sr + y;
                cr = (t - sr) - y;
                sr = t;
                if (CPLX) {
                    y = fmaf(R.w[i], ii, -ci);
                    t = si + y;
                    ci = (t - si) - y;
                    si = t;
                }
            }
        }
        const float sc = A.sg * B.sg * (float)kInv4Pi;
        if (CPLX) {
            float re, im;
            helm_rotate(P, sr, si, re, im);
            reinterpret_cast<double2 *>(out)[pos] = make_double2((double)(re * sc), (double)(im * sc));
        } else
            reinterpret_cast<double *>(out)[pos] = (double)(sr * sc);
    }
}

// Duffy product rule with q points per axis (q^2 points): s = x, t = x y, w = wx wy x
template <int NP>
bool duffy_rule_f(int q, RuleF<NP> &R)
{
    std::vector<double> g, gw;
    if (q * q != NP || !gauss_legendre_unit(q, g, gw)) return false;
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) {
            R.s[i * q + j] = (float)g[i];
            R.t[i * q + j] = (float)(g[i] * g[j]);
            R.w[i * q + j] = (float)(gw[i] * gw[j] * g[i]);
        }
    return true;
}

template <int KIND>
cudaError_t launch_learned_big(const MeshView &m, const int4 *rec, const int64_t *offs, int cls,
                               int q, double kappa, void *out, int grid, cudaStream_t st)
{
    if (q == 6) {
        RuleF<36> R;
        if (!duffy_rule_f(6, R)) return cudaErrorInvalidValue;
        k_learned_eval_big<KIND, 36, 12><<<grid, 256, 0, st>>>(m, rec, offs, cls, R, kappa, out);
    } else if (q == 8) {
        RuleF<64> R;
        if (!duffy_rule_f(8, R)) return cudaErrorInvalidValue;
        k_learned_eval_big<KIND, 64, 16><<<grid, 256, 0, st>>>(m, rec, offs, cls, R, kappa, out);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int KIND>
cudaError_t launch_learned_tp(const MeshView &m, const int4 *rec, const int64_t *offs, int cls,
                              const Rule2D &R, double kappa, void *out, int grid, cudaStream_t st)
{
    switch (R.np) {
    case 4: k_learned_eval_tp<KIND, 4><<<grid, 256, 0, st>>>(m, rec, offs, cls, R, kappa, out); break;
    case 7: k_learned_eval_tp<KIND, 7><<<grid, 256, 0, st>>>(m, rec, offs, cls, R, kappa, out); break;
    case 16: k_learned_eval_tp<KIND, 16><<<grid, 256, 0, st>>>(m, rec, offs, cls, R, kappa, out); break;
    case 25: k_learned_eval_tp<KIND, 25><<<grid, 256, 0, st>>>(m, rec, offs, cls, R, kappa, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// One warp per record of one class: disjoint pair with the class's 4D rule.
template <int KIND, bool MIXED>
__global__ void __launch_bounds__(256) k_learned_eval(MeshView m, const int4 *__restrict__ rec,
                                                      const int64_t *__restrict__ offs, int cls,
                                                      const double *__restrict__ rule,
                                                      const float *__restrict__ rulef, int np,
                                                      double kappa, void *out)
{
    const int lane = threadIdx.x & 31;
    const int64_t lo = offs[cls], hi = offs[cls + 1];
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = lo + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); k < hi; k += nw) {
        const int4 R = rec[k];
        const int64_t pos = (int64_t)(unsigned)R.x | ((int64_t)R.y << 32);
        const int a = R.z, b = R.w;
        double sr = 0.0, si = 0.0;
        if (MIXED) {
            TriF A, B;
            load_trif(m.geomf, a, A);
            load_trif(m.geomf, b, B);
            float d0[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) d0[c] = dd_diff(A.vh[0][c], A.vl[0][c], B.vh[0][c], B.vl[0][c]);
            Height H = {};
            if (KIND == BEM_LAPLACE_DLP)
                H = make_height(A.vh[0], A.vl[0], A.vh[1], A.vl[1], A.vh[2], A.vl[2], B.vh[0], B.vl[0],
                                B.nh, B.nl);
            float acc = 0.0f, acci = 0.0f;
            HelmPhase P;
            if (KIND == BEM_HELMHOLTZ_SLP) P = helm_phase(A, B, kappa);
            for (int p = lane; p < np; p += 32) {
                const float x1 = __ldg(rulef + p), x2 = __ldg(rulef + np + p),
                            y1 = __ldg(rulef + 2 * np + p), y2 = __ldg(rulef + 3 * np + p),
                            w = __ldg(rulef + 4 * np + p);
                if (KIND == BEM_HELMHOLTZ_SLP) {
                    // centroid-relative offsets (see helm_phase)
                    const float ax = x1 - 0.666666687f, at = x2 - 0.333333343f;
                    const float bx = y1 - 0.666666687f, bt = y2 - 0.333333343f;
                    float c, s, ri;
                    helm_offset(P, fmaf(ax, A.e1[0], at * A.e2[0]) - fmaf(bx, B.e1[0], bt * B.e2[0]),
                                fmaf(ax, A.e1[1], at * A.e2[1]) - fmaf(bx, B.e1[1], bt * B.e2[1]),
                                fmaf(ax, A.e1[2], at * A.e2[2]) - fmaf(bx, B.e1[2], bt * B.e2[2]), c, s, ri);
                    acc = fmaf(c, w * ri, acc);
                    acci = fmaf(s, w * ri, acci);
                } else {
                    const float dx = fmaf(x1, A.e1[0], fmaf(x2, A.e2[0], d0[0])) - fmaf(y1, B.e1[0], y2 * B.e2[0]);
                    const float dy = fmaf(x1, A.e1[1], fmaf(x2, A.e2[1], d0[1])) - fmaf(y1, B.e1[1], y2 * B.e2[1]);
                    const float dz = fmaf(x1, A.e1[2], fmaf(x2, A.e2[2], d0[2])) - fmaf(y1, B.e1[2], y2 * B.e2[2]);
                    const float dn = KIND == BEM_LAPLACE_DLP ? height_at(H, x1, x2) : 0.0f;
                    acc = fmaf(w, kvalf<KIND>(dx, dy, dz, dn), acc);
                }
            }
            acc = warp_sumf(acc);
            if (KIND == BEM_HELMHOLTZ_SLP) {
                acci = warp_sumf(acci);
                float re, im;
                helm_rotate(P, acc, acci, re, im);
                acc = re;
                acci = im;
            }
            const double sc = (double)A.sg * (double)B.sg * kInv4Pi;
            sr = (double)acc * sc;
            si = (double)acci * sc;
        } else {
            Tri A, B;
            load_tri(m.geom, a, A);
            load_tri(m.geom, b, B);
            double e1a[3], e2a[3], e1b[3], e2b[3], d0[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                e1a[c] = A.v[1][c] - A.v[0][c];
                e2a[c] = A.v[2][c] - A.v[1][c];
                e1b[c] = B.v[1][c] - B.v[0][c];
                e2b[c] = B.v[2][c] - B.v[1][c];
                d0[c] = A.v[0][c] - B.v[0][c];
            }
            double pr = 0.0, pi = 0.0;
            for (int p = lane; p < np; p += 32) {
                const double x1 = __ldg(rule + p), x2 = __ldg(rule + np + p), y1 = __ldg(rule + 2 * np + p),
                             y2 = __ldg(rule + 3 * np + p), w = __ldg(rule + 4 * np + p);
                const double dx = d0[0] + x1 * e1a[0] + x2 * e2a[0] - y1 * e1b[0] - y2 * e2b[0];
                const double dy = d0[1] + x1 * e1a[1] + x2 * e2a[1] - y1 * e1b[1] - y2 * e2b[1];
                const double dz = d0[2] + x1 * e1a[2] + x2 * e2a[2] - y1 * e1b[2] - y2 * e2b[2];
                double kr, ki;
                kval<KIND>(dx, dy, dz, B.n, kappa, kr, ki);
                pr += w * kr;
                pi += w * ki;
            }
            pr = warp_sum(pr);
            if (KIND == BEM_HELMHOLTZ_SLP) pi = warp_sum(pi);
            const double sc = A.sg * B.sg * kInv4Pi;
            sr = pr * sc;
            si = pi * sc;
        }
        if (lane == 0) {
            if (KIND == BEM_HELMHOLTZ_SLP) reinterpret_cast<double2 *>(out)[pos] = make_double2(sr, si);
            else reinterpret_cast<double *>(out)[pos] = sr;
        }
    }
}

}  // namespace bem

// ---------------------------------------------------------------------------
// Host side: the model object and its C entry points
// ---------------------------------------------------------------------------
using namespace bem;

struct bem_mlp {
    int device;
    float *params = nullptr, *grads = nullptr, *m1 = nullptr, *m2 = nullptr;
    __nv_bfloat16 *pbf = nullptr;
    float *norm = nullptr;     // mean[8], inv_std[8]
    int64_t step = 0;
    // training scratch
    float *xb = nullptr;       // minibatch of normalised features (bem_mlp_train_epoch)
    int32_t *yb = nullptr;
    float *loss_acc = nullptr;
    int64_t bcap = 0;
    int64_t cap = 0;
    float *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr, *z3 = nullptr, *dz3 = nullptr,
          *dz2 = nullptr, *dz1 = nullptr, *loss = nullptr, *loss_sum = nullptr;
};

namespace {

void mlp_free_scratch(bem_mlp *m)
{
    for (float *p : {m->z1, m->h1, m->z2, m->h2, m->z3, m->dz3, m->dz2, m->dz1, m->loss})
        cudaFree(p);
    m->z1 = m->h1 = m->z2 = m->h2 = m->z3 = m->dz3 = m->dz2 = m->dz1 = m->loss = nullptr;
    m->cap = 0;
}

cudaError_t mlp_scratch(bem_mlp *m, int64_t n)
{
    if (n <= m->cap) return cudaSuccess;
    mlp_free_scratch(m);
    cudaError_t e = cudaSuccess;
    auto al = [&](float **p, int64_t cnt) {
        if (e == cudaSuccess) e = cudaMalloc((void **)p, sizeof(float) * std::max<int64_t>(1, cnt));
    };
    al(&m->z1, n * kHid);
    al(&m->h1, n * kHid);
    al(&m->z2, n * kHid);
    al(&m->h2, n * kHid);
    al(&m->z3, n * kOut);
    al(&m->dz3, n * kOut);
    al(&m->dz2, n * kHid);
    al(&m->dz1, n * kHid);
    al(&m->loss, n);
    if (e == cudaSuccess) m->cap = n;
    return e;
}

unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// forward (training precision) + loss + gradients into m->grads
cudaError_t mlp_forward_backward(bem_mlp *m, const float *X, const int32_t *y, int n, cudaStream_t st)
{
    cudaError_t e = mlp_scratch(m, n);
    if (e != cudaSuccess) return e;
    const float *P = m->params;
    float *G = m->grads;
    k_dense<<<nblk((int64_t)n * kHid), 256, 0, st>>>(X, n, kIn, P + kOffW1, P + kOffB1, kHid, m->z1, m->h1);
    k_dense<<<nblk((int64_t)n * kHid), 256, 0, st>>>(m->h1, n, kHid, P + kOffW2, P + kOffB2, kHid, m->z2, m->h2);
    k_dense<<<nblk((int64_t)n * kOut), 256, 0, st>>>(m->h2, n, kHid, P + kOffW3, P + kOffB3, kOut, m->z3, nullptr);
    k_softmax_ce<<<nblk(n), 256, 0, st>>>(m->z3, y, n, m->dz3, m->loss);
    k_sum_fixed<<<1, 256, 0, st>>>(m->loss, n, m->loss_sum);
    k_weight_grad<<<nblk(kOut * kHid + kOut), 256, 0, st>>>(m->dz3, m->h2, n, kOut, kHid, G + kOffW3, G + kOffB3);
    k_back_act<<<nblk((int64_t)n * kHid), 256, 0, st>>>(m->dz3, P + kOffW3, m->z2, n, kOut, kHid, m->dz2);
    k_weight_grad<<<nblk(kHid * kHid + kHid), 256, 0, st>>>(m->dz2, m->h1, n, kHid, kHid, G + kOffW2, G + kOffB2);
    k_back_act<<<nblk((int64_t)n * kHid), 256, 0, st>>>(m->dz2, P + kOffW2, m->z1, n, kHid, kHid, m->dz1);
    k_weight_grad<<<nblk(kHid * kIn + kHid), 256, 0, st>>>(m->dz1, X, n, kHid, kIn, G + kOffW1, G + kOffB1);
    return cudaGetLastError();
}

// Per-feature mean and standard deviation (population) of X (n x 8) in FP64:
// one block per feature, fixed strided partial sums and a fixed tree, so the
// result does not depend on timing.  norm = (mean[8], 1 / std[8]), with std
// below 1e-6 taken as 1 (a constant feature).
__global__ void __launch_bounds__(256) k_norm_stats(const float *__restrict__ X, int64_t n,
                                                    float *norm)
{
    __shared__ double s1[256], s2[256];
    const int f = blockIdx.x;
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += (double)X[i * kIn + f];
    s1[threadIdx.x] = a;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s1[threadIdx.x] += s1[threadIdx.x + o];
        __syncthreads();
    }
    const double mean = s1[0] / (double)n;
    double b = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double d = (double)X[i * kIn + f] - mean;
        b += d * d;
    }
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s2[threadIdx.x] += s2[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double sd = sqrt(s2[0] / (double)n);
        norm[f] = (float)mean;
        norm[kIn + f] = (float)(sd > 1e-6 ? 1.0 / sd : 1.0);
    }
}

// rows perm[0..b) of the raw features, normalised with the model's (mean,
// 1/std), and their labels
__global__ void __launch_bounds__(256) k_gather_norm(const float *__restrict__ X,
                                                     const int32_t *__restrict__ y,
                                                     const int64_t *__restrict__ perm, int b,
                                                     const float *__restrict__ norm, float *xb,
                                                     int32_t *yb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b * kIn) return;
    const int r = i / kIn, f = i % kIn;
    const int64_t src = perm[r];
    xb[i] = (X[src * kIn + f] - norm[f]) * norm[kIn + f];
    if (f == 0) yb[r] = y[src];
}

__global__ void k_loss_acc(const float *loss_sum, float *acc, int reset)
{
    acc[0] = (reset ? 0.0f : acc[0]) + loss_sum[0];
}

// Order-class labels from the method's own errors (Section 2.2 rules against a
// high Duffy order): err_c = |v_c - v_ref| / A_ref for each class c (A_ref the
// sum of the magnitudes of the reference's terms), label = the cheapest class
// with err_c <= tol, else the most accurate one.
__global__ void __launch_bounds__(256) k_class_error(int64_t n, int cls, int cplx,
                                                     const double *__restrict__ v,
                                                     const double *__restrict__ ref,
                                                     const double *__restrict__ A, float *err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d;
    if (cplx) d = hypot(v[2 * i] - ref[2 * i], v[2 * i + 1] - ref[2 * i + 1]);
    else d = fabs(v[i] - ref[i]);
    err[i * kOut + cls] = (float)(d / fmax(A[i], 1e-300));
}

__global__ void __launch_bounds__(256) k_class_label(int64_t n, const float *__restrict__ err,
                                                     float tol, int32_t *label)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int l = kOut - 1;
    for (int c = kOut - 1; c >= 0; --c)
        if (err[i * kOut + c] <= tol) l = c;
    label[i] = l;
}

MlpDev mlp_dev(const bem_mlp *m)
{
    MlpDev d;
    d.W1 = m->pbf + kOffW1;
    d.W2 = m->pbf + kOffW2;
    d.W3 = m->pbf + kOffW3;
    d.b1 = m->params + kOffB1;
    d.b2 = m->params + kOffB2;
    d.b3 = m->params + kOffB3;
    return d;
}

}  // namespace

extern "C" {

int bem_mlp_create(bem_ctx *ctx, uint64_t seed, bem_mlp **out)
{
    if (!ctx || !out) return BEM_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    bem_mlp *m = new bem_mlp();
    m->device = ctx->device;
    cudaError_t e = cudaSuccess;
    auto al = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    al((void **)&m->params, sizeof(float) * kNParams);
    al((void **)&m->grads, sizeof(float) * kNParams);
    al((void **)&m->m1, sizeof(float) * kNParams);
    al((void **)&m->m2, sizeof(float) * kNParams);
    al((void **)&m->pbf, sizeof(__nv_bfloat16) * kNParams);
    al((void **)&m->norm, sizeof(float) * 16);
    al((void **)&m->loss_sum, sizeof(float));
    if (e != cudaSuccess) {
        delete m;
        return api_cuda_fail(ctx, e, "cudaMalloc(mlp)");
    }
    // He-style uniform init from a splitmix64 stream
    std::vector<float> h(kNParams, 0.0f);
    uint64_t s = seed;
    auto next = [&]() {
        s += 0x9E3779B97F4A7C15ull;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    auto fill = [&](int off, int cnt, int fan_in) {
        const double a = std::sqrt(6.0 / fan_in);
        for (int k = 0; k < cnt; ++k) h[off + k] = (float)((2.0 * next() - 1.0) * a);
    };
    fill(kOffW1, kHid * kIn, kIn);
    fill(kOffW2, kHid * kHid, kHid);
    fill(kOffW3, kOut * kHid, kHid);
    std::vector<float> norm(16, 0.0f);
    for (int k = 0; k < 8; ++k) norm[8 + k] = 1.0f;
    cudaMemcpy(m->params, h.data(), sizeof(float) * kNParams, cudaMemcpyHostToDevice);
    cudaMemset(m->m1, 0, sizeof(float) * kNParams);
    cudaMemset(m->m2, 0, sizeof(float) * kNParams);
    cudaMemcpy(m->norm, norm.data(), sizeof(float) * 16, cudaMemcpyHostToDevice);
    k_to_bf16<<<nblk(kNParams), 256>>>(m->params, kNParams, m->pbf);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        delete m;
        return api_cuda_fail(ctx, e, "mlp init");
    }
    *out = m;
    return BEM_OK;
}

int bem_mlp_destroy(bem_ctx *ctx, bem_mlp *m)
{
    if (!ctx || !m) return BEM_ERR_INVALID_ARG;
    cudaStreamSynchronize(ctx->stream);
    mlp_free_scratch(m);
    for (void *p : {(void *)m->params, (void *)m->grads, (void *)m->m1, (void *)m->m2, (void *)m->pbf,
                    (void *)m->norm, (void *)m->loss_sum, (void *)m->xb, (void *)m->yb,
                    (void *)m->loss_acc})
        cudaFree(p);
    delete m;
    return BEM_OK;
}

int bem_mlp_num_params(void) { return kNParams; }

int bem_mlp_set_params(bem_ctx *ctx, bem_mlp *m, const float *host_params, const float *host_norm)
{
    if (!ctx || !m) return BEM_ERR_INVALID_ARG;
    cudaError_t e = cudaSuccess;
    if (host_params) e = cudaMemcpy(m->params, host_params, sizeof(float) * kNParams, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && host_norm) e = cudaMemcpy(m->norm, host_norm, sizeof(float) * 16, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "mlp set");
    k_to_bf16<<<nblk(kNParams), 256, 0, ctx->stream>>>(m->params, kNParams, m->pbf);
    return BEM_OK;
}

int bem_mlp_get_params(bem_ctx *ctx, bem_mlp *m, float *host_params, float *host_norm)
{
    if (!ctx || !m) return BEM_ERR_INVALID_ARG;
    cudaStreamSynchronize(ctx->stream);
    cudaError_t e = cudaSuccess;
    if (host_params) e = cudaMemcpy(host_params, m->params, sizeof(float) * kNParams, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && host_norm) e = cudaMemcpy(host_norm, m->norm, sizeof(float) * 16, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "mlp get");
    return BEM_OK;
}

int bem_mlp_gradients(bem_ctx *ctx, bem_mlp *m, const float *X, const int32_t *y, int32_t n,
                      float *grads, float *loss)
{
    if (!ctx || !m || !X || !y || n < 1) return BEM_ERR_INVALID_ARG;
    cudaError_t e = mlp_forward_backward(m, X, y, n, ctx->stream);
    if (e == cudaSuccess && grads)
        e = cudaMemcpyAsync(grads, m->grads, sizeof(float) * kNParams, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess && loss) {
        float s = 0.0f;
        e = cudaMemcpyAsync(&s, m->loss_sum, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        *loss = s / (float)n;
    }
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "mlp gradients");
    return BEM_OK;
}

int bem_mlp_train_step(bem_ctx *ctx, bem_mlp *m, const float *X, const int32_t *y, int32_t n,
                       float lr, float *loss)
{
    if (!ctx || !m || !X || !y || n < 1) return BEM_ERR_INVALID_ARG;
    cudaError_t e = mlp_forward_backward(m, X, y, n, ctx->stream);
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "mlp step");
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)m->step), c2 = 1.0f - std::pow(b2, (float)m->step);
    k_adam<<<nblk(kNParams), 256, 0, ctx->stream>>>(m->params, m->grads, m->m1, m->m2, kNParams, lr,
                                                    b1, b2, 1e-8f, c1, c2);
    k_to_bf16<<<nblk(kNParams), 256, 0, ctx->stream>>>(m->params, kNParams, m->pbf);
    if (loss) {
        float s = 0.0f;
        e = cudaMemcpyAsync(&s, m->loss_sum, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        *loss = s / (float)n;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "mlp step");
    return BEM_OK;
}

int bem_mlp_fit_norm(bem_ctx *ctx, bem_mlp *m, const float *X, int64_t n)
{
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (!m || !X || n < 1) return api_fail(ctx, BEM_ERR_INVALID_ARG, "bem_mlp_fit_norm: bad arguments");
    k_norm_stats<<<kIn, 256, 0, ctx->stream>>>(X, n, m->norm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "bem_mlp_fit_norm");
    return BEM_OK;
}

int bem_mlp_train_epoch(bem_ctx *ctx, bem_mlp *m, const float *X, const int32_t *y, int64_t n,
                        const int64_t *perm, int32_t batch, float lr, float *mean_loss)
{
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (!m || !X || !y || !perm || n < 1 || batch < 1)
        return api_fail(ctx, BEM_ERR_INVALID_ARG, "bem_mlp_train_epoch: bad arguments");
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaSuccess;
    if (batch > m->bcap) {
        cudaStreamSynchronize(st);
        cudaFree(m->xb);
        cudaFree(m->yb);
        m->xb = nullptr;
        m->yb = nullptr;
        m->bcap = 0;
        e = cudaMalloc((void **)&m->xb, sizeof(float) * (size_t)batch * kIn);
        if (e == cudaSuccess) e = cudaMalloc((void **)&m->yb, sizeof(int32_t) * (size_t)batch);
        if (e != cudaSuccess) return api_cuda_fail(ctx, e, "cudaMalloc(minibatch)");
        m->bcap = batch;
    }
    if (!m->loss_acc) {
        e = cudaMalloc((void **)&m->loss_acc, sizeof(float));
        if (e != cudaSuccess) return api_cuda_fail(ctx, e, "cudaMalloc(loss)");
    }
    const float b1 = 0.9f, b2 = 0.999f;
    for (int64_t s = 0; s < n; s += batch) {
        const int b = (int)std::min<int64_t>(batch, n - s);
        k_gather_norm<<<nblk((int64_t)b * kIn), 256, 0, st>>>(X, y, perm + s, b, m->norm, m->xb, m->yb);
        e = mlp_forward_backward(m, m->xb, m->yb, b, st);
        if (e != cudaSuccess) return api_cuda_fail(ctx, e, "bem_mlp_train_epoch");
        m->step += 1;
        const float c1 = 1.0f - std::pow(b1, (float)m->step), c2 = 1.0f - std::pow(b2, (float)m->step);
        k_adam<<<nblk(kNParams), 256, 0, st>>>(m->params, m->grads, m->m1, m->m2, kNParams, lr,
                                               b1, b2, 1e-8f, c1, c2);
        k_to_bf16<<<nblk(kNParams), 256, 0, st>>>(m->params, kNParams, m->pbf);
        k_loss_acc<<<1, 1, 0, st>>>(m->loss_sum, m->loss_acc, s == 0 ? 1 : 0);
    }
    float tot = 0.0f;
    e = cudaMemcpyAsync(&tot, m->loss_acc, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "bem_mlp_train_epoch");
    if (mean_loss) *mean_loss = tot / (float)n;
    return BEM_OK;
}

int bem_mlp_infer(bem_ctx *ctx, bem_mlp *m, const float *X, int64_t n, float *logits)
{
    if (!ctx || !m || (n > 0 && (!X || !logits)) || n < 0) return BEM_ERR_INVALID_ARG;
    if (n == 0) return BEM_OK;
    const int64_t tiles = (n + 15) / 16;
    k_mlp_infer<<<(unsigned)((tiles + 7) / 8), 256, 0, ctx->stream>>>(mlp_dev(m), X, n, logits);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "mlp infer");
    return BEM_OK;
}

int bem_set_order_model(bem_ctx *ctx, bem_mlp *m, float confidence)
{
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (m && !(confidence >= 0.0f && confidence <= 1.0f))
        return api_fail(ctx, BEM_ERR_INVALID_ARG, "confidence must be in [0, 1]");
    ctx->order_model = m;
    ctx->order_conf = confidence;
    return BEM_OK;
}

int bem_learned_counts(bem_ctx *ctx, int64_t *counts)
{
    if (!ctx || !counts) return BEM_ERR_INVALID_ARG;
    for (int c = 0; c < kClasses; ++c) counts[c] = ctx->learned_counts[c];
    return BEM_OK;
}

int bem_order_labels(bem_ctx *ctx, int32_t mesh_id, const bem_kernel_desc *kernel,
                     const int32_t *a, const int32_t *b, int64_t n, float tol, int32_t q_ref,
                     int32_t *labels, float *errors)
{
    if (!ctx || !kernel) return BEM_ERR_INVALID_ARG;
    auto it = ctx->meshes.find(mesh_id);
    if (it == ctx->meshes.end()) return api_fail(ctx, BEM_ERR_INVALID_ARG, "unknown mesh id");
    const MeshView &mv = it->second->v;
    if (mv.basis != BEM_P0) return api_fail(ctx, BEM_ERR_UNSUPPORTED, "labels need a P0 mesh");
    if (kernel->kind < BEM_LAPLACE_SLP || kernel->kind > BEM_HELMHOLTZ_SLP || q_ref < 1 ||
        q_ref > 20 || !(tol > 0.0f) || n < 0)
        return api_fail(ctx, BEM_ERR_INVALID_ARG, "bem_order_labels: bad arguments");
    if (n == 0) return BEM_OK;
    if (!a || !b || !labels) return api_fail(ctx, BEM_ERR_INVALID_ARG, "null pointer");
    const int cplx = kernel->kind == BEM_HELMHOLTZ_SLP ? 1 : 0;
    Rule4D rules[4];
    for (int c = kVertex; c <= kIdentical; ++c) {
        int rc = api_get_rule4(ctx, c, 0, 5, rules[c]);
        if (rc) return rc;
    }
    cudaStream_t st = ctx->stream;
    double *ref = nullptr, *A = nullptr, *v = nullptr;
    float *err = nullptr;
    cudaError_t e = cudaMalloc((void **)&ref, sizeof(double) * n * (1 + cplx));
    if (e == cudaSuccess) e = cudaMalloc((void **)&A, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&v, sizeof(double) * n * (1 + cplx));
    if (e == cudaSuccess) e = cudaMalloc((void **)&err, sizeof(float) * n * kOut);
    int rc = BEM_OK;
    if (e == cudaSuccess) {
        // the reference: Duffy q_ref, its value and the sum of |terms|
        rc = api_get_rule4(ctx, kRegular, BEM_RULE_DUFFY, q_ref, rules[kRegular]);
        if (!rc) e = launch_pivot_entries(mv, a, b, n, ref, rules, kernel->kind, kernel->kappa,
                                          ctx->status, st, false);
        if (!rc && e == cudaSuccess)
            e = launch_pivot_entries(mv, a, b, n, A, rules, kernel->kind, kernel->kappa,
                                     ctx->status, st, true);
        for (int c = 0; c < kClasses && !rc && e == cudaSuccess; ++c) {
            rc = api_get_rule4(ctx, kRegular, kClassRule[c][0], kClassRule[c][1], rules[kRegular]);
            if (rc) break;
            e = launch_pivot_entries(mv, a, b, n, v, rules, kernel->kind, kernel->kappa,
                                     ctx->status, st, false);
            if (e == cudaSuccess) {
                k_class_error<<<nblk(n), 256, 0, st>>>(n, c, cplx, v, ref, A, err);
                e = cudaGetLastError();
            }
        }
        if (!rc && e == cudaSuccess) {
            k_class_label<<<nblk(n), 256, 0, st>>>(n, err, tol, labels);
            e = cudaGetLastError();
        }
        if (!rc && e == cudaSuccess && errors)
            e = cudaMemcpyAsync(errors, err, sizeof(float) * n * kOut, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    cudaFree(ref);
    cudaFree(A);
    cudaFree(v);
    cudaFree(err);
    if (rc) return rc;
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "bem_order_labels");
    return BEM_OK;
}

int bem_pair_features(bem_ctx *ctx, int32_t mesh_id, const bem_kernel_desc *kernel, bem_mlp *m,
                      const int32_t *a, const int32_t *b, int64_t n, float *X)
{
    if (!ctx || !kernel || n < 0) return BEM_ERR_INVALID_ARG;
    auto it = ctx->meshes.find(mesh_id);
    if (it == ctx->meshes.end()) return api_fail(ctx, BEM_ERR_INVALID_ARG, "unknown mesh id");
    if (it->second->v.basis != BEM_P0) return api_fail(ctx, BEM_ERR_UNSUPPORTED, "pair features need a P0 mesh");
    if (n == 0) return BEM_OK;
    if (!a || !b || !X) return api_fail(ctx, BEM_ERR_INVALID_ARG, "null pointer");
    static float *ident = nullptr;   // mean 0, inv_std 1 when no model is given
    const float *mean, *inv;
    if (m) {
        mean = m->norm;
        inv = m->norm + 8;
    } else {
        if (!ident) {
            std::vector<float> h(16, 0.0f);
            for (int k = 0; k < 8; ++k) h[8 + k] = 1.0f;
            cudaMalloc((void **)&ident, 16 * sizeof(float));
            cudaMemcpy(ident, h.data(), 16 * sizeof(float), cudaMemcpyHostToDevice);
        }
        mean = ident;
        inv = ident + 8;
    }
    k_features<<<nblk(n), 256, 0, ctx->stream>>>(it->second->v, a, b, n, kernel->kind, kernel->kappa,
                                                mean, inv, X);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "features");
    return BEM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Learned near-field job (called by bem_near_field for order_mode LEARNED;
// the touching table and the tile prefix sums are already on the stream).
// ---------------------------------------------------------------------------
namespace bem {


// Scratch of one learned job for `tiles` tiles: class per tile slot, records
// grouped by class, counters and class offsets.
cudaError_t learned_alloc(LearnedScratch &S, int64_t tiles)
{
    tiles = std::max<int64_t>(1, tiles);
    const int64_t slots = tiles * kP0Tile;
    cudaError_t e = cudaMalloc((void **)&S.cls, slots);
    if (e == cudaSuccess) e = cudaMalloc((void **)&S.rec, slots * sizeof(int4));
    // small: class counts (8 ints), offsets (8 + 1 int64), segment sums of the scan
    if (e == cudaSuccess) e = cudaMalloc((void **)&S.small, (16 + kClasses * kScanSeg) * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&S.tcount, tiles * 8 * kClasses * sizeof(int));
    if (e == cudaSuccess) S.cap = slots;
    return e;
}

void learned_free(LearnedScratch &S)
{
    cudaFree(S.cls);
    cudaFree(S.rec);
    cudaFree(S.small);
    cudaFree(S.tcount);
    S = LearnedScratch{};
}

// The launches of one learned job (the touching table and the tile prefix
// sums are already on the stream): select (features, MLP, class per entry),
// offsets, compaction by class, one evaluation per class.  `rules` holds the
// classes' FP64 4D rules (for the classes without a product-rule kernel).
// Errors are CUDA launch errors.
cudaError_t learned_launches(const MeshView &mv, const BlockLaunch &L, const int64_t *prefix,
                             const bem_mlp *model, float conf, const LearnedScratch &S,
                             const Rule4D *rules, int precision, int num_sms, int *status,
                             cudaStream_t st, bem_ctx *prof_ctx)
{
    LearnedArgs A;
    A.P = mlp_dev(model);
    A.mean = model->norm;
    A.inv_std = model->norm + 8;
    A.conf = conf;
    A.cls = S.cls;
    A.counts = reinterpret_cast<int *>(S.small);
    A.offs = S.small + 8;
    A.tcount = S.tcount;
    A.ntile = S.cap / kP0Tile;
    A.rec = reinterpret_cast<int4 *>(S.rec);
    cudaError_t e = cudaMemsetAsync(A.counts, 0, 16 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    const int grid = num_sms * 8;
    {
        ProfScope ps(prof_ctx, "learned_select");
        k_learned_select<<<grid, 256, 0, st>>>(mv, L, prefix, A, status);
        int *seg = reinterpret_cast<int *>(S.small + 16);   // kClasses * kScanSeg ints
        k_learned_seg_sum<<<kClasses * kScanSeg, 256, 0, st>>>(L, prefix, A, seg);
        k_learned_seg_off<<<1, 32 * kClasses, 0, st>>>(A, seg);
        k_learned_seg_apply<<<kClasses * kScanSeg, 256, 0, st>>>(L, prefix, A, seg);
        k_learned_offsets<<<1, 32, 0, st>>>(A);
        k_learned_compact<<<grid, 256, 0, st>>>(mv, L, prefix, A);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    static const char *kEvalName[kClasses] = {"learned_eval_duffy2", "learned_eval_tri7",
                                              "learned_eval_duffy4", "learned_eval_duffy5",
                                              "learned_eval_duffy6", "learned_eval_duffy8"};
    const bool mixed = is_mixed(precision);
    for (int c = 0; c < kClasses; ++c) {
        ProfScope ps(prof_ctx, kEvalName[c]);
        Rule2D r2;
        if (mixed && make_rule2d(kClassRule[c][0], kClassRule[c][1], r2) &&
            (r2.np == 4 || r2.np == 7 || r2.np == 16 || r2.np == 25)) {
            // thread per pair on the 2D product rule
            e = L.kind == BEM_LAPLACE_SLP
                    ? launch_learned_tp<BEM_LAPLACE_SLP>(mv, A.rec, A.offs, c, r2, L.kappa, L.out, grid, st)
                    : L.kind == BEM_LAPLACE_DLP
                          ? launch_learned_tp<BEM_LAPLACE_DLP>(mv, A.rec, A.offs, c, r2, L.kappa, L.out, grid, st)
                          : launch_learned_tp<BEM_HELMHOLTZ_SLP>(mv, A.rec, A.offs, c, r2, L.kappa, L.out, grid, st);
            if (e != cudaSuccess) return e;
            continue;
        }
        if (mixed && kClassRule[c][0] == BEM_RULE_DUFFY &&
            (kClassRule[c][1] == 6 || kClassRule[c][1] == 8)) {
            // thread per pair, trial points in chunks
            const int q = kClassRule[c][1];
            e = L.kind == BEM_LAPLACE_SLP
                    ? launch_learned_big<BEM_LAPLACE_SLP>(mv, A.rec, A.offs, c, q, L.kappa, L.out, grid, st)
                    : L.kind == BEM_LAPLACE_DLP
                          ? launch_learned_big<BEM_LAPLACE_DLP>(mv, A.rec, A.offs, c, q, L.kappa, L.out, grid, st)
                          : launch_learned_big<BEM_HELMHOLTZ_SLP>(mv, A.rec, A.offs, c, q, L.kappa, L.out, grid, st);
            if (e != cudaSuccess) return e;
            continue;
        }
        const Rule4D &r = rules[c];
        switch (L.kind) {
        case BEM_LAPLACE_SLP:
            if (mixed) k_learned_eval<BEM_LAPLACE_SLP, true><<<grid, 256, 0, st>>>(mv, A.rec, A.offs, c, r.d, r.f, r.n, L.kappa, L.out);
            else k_learned_eval<BEM_LAPLACE_SLP, false><<<grid, 256, 0, st>>>(mv, A.rec, A.offs, c, r.d, r.f, r.n, L.kappa, L.out);
            break;
        case BEM_LAPLACE_DLP:
            if (mixed) k_learned_eval<BEM_LAPLACE_DLP, true><<<grid, 256, 0, st>>>(mv, A.rec, A.offs, c, r.d, r.f, r.n, L.kappa, L.out);
            else k_learned_eval<BEM_LAPLACE_DLP, false><<<grid, 256, 0, st>>>(mv, A.rec, A.offs, c, r.d, r.f, r.n, L.kappa, L.out);
            break;
        default:
            if (mixed) k_learned_eval<BEM_HELMHOLTZ_SLP, true><<<grid, 256, 0, st>>>(mv, A.rec, A.offs, c, r.d, r.f, r.n, L.kappa, L.out);
            else k_learned_eval<BEM_HELMHOLTZ_SLP, false><<<grid, 256, 0, st>>>(mv, A.rec, A.offs, c, r.d, r.f, r.n, L.kappa, L.out);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int learned_rules(bem_ctx *ctx, Rule4D *rules)
{
    for (int c = 0; c < kClasses; ++c) {
        int rc = api_get_rule4(ctx, kRegular, kClassRule[c][0], kClassRule[c][1], rules[c]);
        if (rc) return rc;
    }
    return BEM_OK;
}

int run_learned_p0(bem_ctx *ctx, const MeshView &mv, const BlockLaunch &L, const int64_t *prefix,
                   int precision)
{
    bem_mlp *model = ctx->order_model;
    if (!model) return api_fail(ctx, BEM_ERR_INVALID_ARG, "order_mode LEARNED needs bem_set_order_model");
    // the number of entries sizes the scratch: one read back per call
    int64_t entries = 0;
    cudaError_t e = cudaMemcpyAsync(&entries, prefix + (L.n_blocks - 1), sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "learned: entry count");
    const int64_t tiles = (entries + kP0Tile - 1) / kP0Tile;
    if (std::max<int64_t>(1, tiles * 256) > ctx->learned.cap) {
        learned_free(ctx->learned);
        e = learned_alloc(ctx->learned, tiles);
        if (e != cudaSuccess) {
            learned_free(ctx->learned);
            return api_cuda_fail(ctx, e, "cudaMalloc(learned scratch)");
        }
    }
    Rule4D rules[kClasses];
    int rc = learned_rules(ctx, rules);
    if (rc) return rc;
    e = learned_launches(mv, L, prefix, model, ctx->order_conf, ctx->learned, rules, precision,
                         ctx->num_sms, ctx->status, ctx->stream, ctx);
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "learned evaluation");
    // class counts of this call (for reports): read after the launches
    int counts[8] = {0};
    e = cudaMemcpyAsync(counts, ctx->learned.small, 8 * sizeof(int), cudaMemcpyDeviceToHost,
                        ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "learned path");
    for (int c = 0; c < kClasses; ++c) ctx->learned_counts[c] = counts[c];
    return BEM_OK;
}

}  // namespace bem
