// Device-side building blocks shared by the kernel translation units:
// geometry records, kernel functions, double-float helpers, the regular
// pair integrals, and the tile bodies of the block engine.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "bem_internal.h"

namespace bem {

static __constant__ int c_perm[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {1, 0, 2}, {2, 1, 0}};

constexpr double kInv4Pi = 0.079577471545947667884441881686257181;

// First error wins; a null status word (passes that repeat a checked pass) drops it.
__device__ __forceinline__ void set_status(int *st, int code)
{
    if (st) atomicCAS(st, 0, code);
}

struct Tri {
    double v[3][3];
    double n[3];
    double sg;
};

__device__ __forceinline__ void load_tri(const double *__restrict__ geom, int64_t t, Tri &o)
{
    const double *g = geom + t * kGeomStride;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        o.v[k][0] = __ldg(g + 3 * k + 0);
        o.v[k][1] = __ldg(g + 3 * k + 1);
        o.v[k][2] = __ldg(g + 3 * k + 2);
    }
    o.n[0] = __ldg(g + 9);
    o.n[1] = __ldg(g + 10);
    o.n[2] = __ldg(g + 11);
    o.sg = __ldg(g + 12);
}

// Kernel value without the 1/(4 pi) factor; d = x - y, nb = trial normal.
template <int KIND>
__device__ __forceinline__ void kval(double dx, double dy, double dz, const double *nb,
                                     double kappa, double &re, double &im, double eta = 0.0)
{
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double ri = rsqrt(r2);
    if (KIND == BEM_LAPLACE_SLP) {
        re = ri;
        im = 0.0;
    } else if (KIND == BEM_LAPLACE_DLP) {
        const double dn = dx * nb[0] + dy * nb[1] + dz * nb[2];
        re = dn * ri * ri * ri;
        im = 0.0;
    } else if (KIND == BEM_HELMHOLTZ_SLP) {
        double s, c;
        sincos(kappa * (r2 * ri), &s, &c);
        re = c * ri;
        im = s * ri;
    } else {
        // (x-y).n_y (1 - i kappa r) exp(i kappa r) / r^3, and for the
        // Brakhage-Werner combination minus i eta exp(i kappa r) / r
        const double dn = dx * nb[0] + dy * nb[1] + dz * nb[2];
        const double kr = kappa * (r2 * ri);
        double s, c;
        sincos(kr, &s, &c);
        const double f = dn * ri * ri * ri;
        re = f * (c + kr * s);
        im = f * (s - kr * c);
        if (KIND == BEM_HELMHOLTZ_BW) {
            re += eta * s * ri;
            im -= eta * c * ri;
        }
    }
}

// Touching table index of the pair (a, b), or -1 if b is not a touching neighbour of a.
__device__ __forceinline__ int find_touching(const MeshView &m, int a, int b)
{
    const int lo = __ldg(m.nb_ptr + a), hi = __ldg(m.nb_ptr + a + 1);
    for (int k = lo; k < hi; ++k)
        if (__ldg(m.nb_tri + k) == b) return k;
    return -1;
}

__device__ __forceinline__ bool touching(int4 A, int4 B)
{
    return A.x == B.x || A.x == B.y || A.x == B.z || A.y == B.x || A.y == B.y || A.y == B.z ||
           A.z == B.x || A.z == B.y || A.z == B.z;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sumf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// 1/sqrt(x) in float as the single hardware approximation PTX calls
// rsqrt.approx.ftz.f32 (relative error about 2^-23).  Every argument here is a
// squared distance far above the subnormal range, so the flush changes
// nothing and the subnormal fix-up of rsqrtf is not needed.
__device__ __forceinline__ float rsqrt_fast(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------------------
// Mixed form: float arithmetic with double-float set-up.  Every vertex is held
// as hi + lo floats; differences of vertices and the heights of one
// triangle's vertices above another's plane are formed with error-free
// transformations (Knuth's TwoSum, FMA-based TwoProduct), so they carry full
// float precision even when they are tiny against the coordinates.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (ah + al) - (bh + bl) as an unevaluated hi + lo pair
__device__ __forceinline__ void dd_sub(float ah, float al, float bh, float bl, float &h, float &l)
{
    float s, e;
    two_sum(ah, -bh, s, e);
    e += al - bl;
    h = s + e;
    l = e - (h - s);
}

__device__ __forceinline__ float dd_diff(float ah, float al, float bh, float bl)
{
    float h, l;
    dd_sub(ah, al, bh, bl, h, l);
    return h + l;
}

// ((a - b) . n) as an unevaluated hi + lo pair, with a, b, n given as hi/lo triples
__device__ __forceinline__ void dd_height(const float *ah, const float *al, const float *bh,
                                          const float *bl, const float *nh, const float *nl,
                                          float &hh, float &hl)
{
    float S = 0.0f, E = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float dh, dl;
        dd_sub(ah[c], al[c], bh[c], bl[c], dh, dl);
        const float p = dh * nh[c];
        const float pe = fmaf(dh, nh[c], -p) + fmaf(dh, nl[c], dl * nh[c]);
        float s2, e2;
        two_sum(S, p, s2, e2);
        S = s2;
        E += e2 + pe;
    }
    hh = S + E;
    hl = E - (hh - S);
}

// Affine height h(s,t) = h0 + s h10 + t h21 of a point of the test triangle above
// the trial triangle's plane, from hi/lo coefficients, with compensated
// products and sums: its error is a few ulps of |h| even where h changes sign.
struct Height {
    float h0, h0l, h10, h10l, h21, h21l;
};

__device__ __forceinline__ float height_at(const Height &H, float s, float t)
{
    const float p1 = s * H.h10, p2 = t * H.h21;
    const float e1 = fmaf(s, H.h10, -p1), e2 = fmaf(t, H.h21, -p2);
    float a, ea, b, eb;
    two_sum(p1, p2, a, ea);
    two_sum(a, H.h0, b, eb);
    const float lo = ea + eb + e1 + e2 + H.h0l + fmaf(s, H.h10l, t * H.h21l);
    return b + lo;
}

// The same height in plain float from the rounded coefficients, for pairs of
// an admissible (far-field) block: the coefficients keep the precision of the
// double-float set-up (tiny for nearly coplanar triangles), and the rounding
// of the evaluation, a few ulps of |h0| + |h10| + |h21|, stays within a few
// ulps of the largest term of the pair's sum because the triangles lie at
// least a multiple of their size apart, so 1/r^3 varies by a bounded factor
// over the pair.  Near-field pairs, where the test triangle can cross the
// trial plane close to the trial triangle, use height_at.
__device__ __forceinline__ float height_at_far(const Height &H, float s, float t)
{
    return fmaf(s, H.h10, fmaf(t, H.h21, H.h0));
}

// Sum over the warp of the unevaluated pairs hi + lo of every lane: TwoSum at
// each butterfly level keeps the rounding error of the float additions.
__device__ __forceinline__ void warp_sum2f(float &hi, float &lo)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        float sh, e;
        two_sum(hi, h2, sh, e);
        hi = sh;
        lo = (lo + l2) + e;
    }
}

// The same over aligned groups of W lanes (W a power of two up to 32).
template <int W>
__device__ __forceinline__ void group_sum2f(float &hi, float &lo)
{
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        float sh, e;
        two_sum(hi, h2, sh, e);
        hi = sh;
        lo = (lo + l2) + e;
    }
}

template <int W>
__device__ __forceinline__ float group_sumf(float v)
{
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// heights of the test triangle's vertices k0, k1, k2 above the trial plane
// (through the trial vertex bh/bl with normal nh/nl) as affine coefficients
__device__ __forceinline__ Height make_height(const float *a0h, const float *a0l,
                                              const float *a1h, const float *a1l,
                                              const float *a2h, const float *a2l,
                                              const float *bh, const float *bl,
                                              const float *nh, const float *nl)
{
    float h0, l0, h1, l1, h2, l2;
    dd_height(a0h, a0l, bh, bl, nh, nl, h0, l0);
    dd_height(a1h, a1l, bh, bl, nh, nl, h1, l1);
    dd_height(a2h, a2l, bh, bl, nh, nl, h2, l2);
    Height H;
    H.h0 = h0;
    H.h0l = l0;
    dd_sub(h1, l1, h0, l0, H.h10, H.h10l);
    dd_sub(h2, l2, h1, l1, H.h21, H.h21l);
    return H;
}

struct TriF {
    float vh[3][3], vl[3][3];
    float e1[3], e2[3];
    float nh[3], nl[3];
    float sg;
};

__device__ __forceinline__ void load_trif(const float *__restrict__ geomf, int64_t t, TriF &o)
{
    const float4 *g = reinterpret_cast<const float4 *>(geomf + t * kGeomFStride);
    float f[32];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float4 v = __ldg(g + k);
        f[4 * k] = v.x;
        f[4 * k + 1] = v.y;
        f[4 * k + 2] = v.z;
        f[4 * k + 3] = v.w;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o.vh[k][c] = f[3 * k + c];
            o.vl[k][c] = f[9 + 3 * k + c];
        }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        o.e1[c] = f[18 + c];
        o.e2[c] = f[21 + c];
        o.nh[c] = f[24 + c];
        o.nl[c] = f[27 + c];
    }
    o.sg = f[30];
}

// Laplace kernel value in float: 1/r (single layer) or dn/r^3 (double layer)
template <int KIND>
__device__ __forceinline__ float kvalf(float dx, float dy, float dz, float dn)
{
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float ri = rsqrt_fast(r2);
    if (KIND == BEM_LAPLACE_SLP) return ri;
    return dn * (ri * ri * ri);
}

// The same without the double layer's height factor: 1/r (single layer) or
// 1/r^3 (double layer).  Product rules whose inner loop runs over trial points
// at one test point x multiply the inner sum by the height of x once instead.
template <int KIND>
__device__ __forceinline__ float kvalf_r(float dx, float dy, float dz)
{
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float ri = rsqrt_fast(r2);
    if (KIND == BEM_LAPLACE_SLP) return ri;
    return ri * ri * ri;
}

// ---------------------------------------------------------------------------
// Helmholtz in the mixed form.  exp(i kappa r) = exp(i kappa r0) exp(i kappa
// (r - r0)) with r0 = the distance of the two centroids: r0, kappa r0 and its
// reduction modulo 2 pi are formed in double-float arithmetic once per pair;
// per point only the small offset r - r0 (from q = (2 d_c + e) . e, with
// e = (x - x_c) - (y - y_c) from centroid-relative offsets, see helm_offset)
// is evaluated in float, so the phase keeps ~1e-7 absolute accuracy for
// kappa r of order 10^2.  The sums run over exp(i kappa (r - r0)) / r and are
// rotated by exp(i kappa r0) once per pair.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void dd_add(float ah, float al, float bh, float bl, float &h, float &l)
{
    float s, e;
    two_sum(ah, bh, s, e);
    e += al + bl;
    h = s + e;
    l = e - (h - s);
}

__device__ __forceinline__ void dd_mul(float ah, float al, float bh, float bl, float &h, float &l)
{
    const float p = ah * bh;
    const float e = fmaf(ah, bh, -p) + fmaf(ah, bl, al * bh);
    h = p + e;
    l = e - (h - p);
}

// phase data of a pair: cos/sin of kappa r0 and the float quantities per point
struct HelmPhase {
    float dcx, dcy, dcz;   // centroid difference d_c (float)
    float r0h, r0l;        // r0 as an unevaluated hi + lo pair
    float r0sqh, r0sql;    // r0^2 as an unevaluated hi + lo pair
    float m2r0l;           // -2 r0l
    float c0, s0;          // cos, sin of kappa r0
    float kap;
};

__device__ __forceinline__ HelmPhase helm_phase(const TriF &A, const TriF &B, double kappa)
{
    // centroid difference in double-float: (sum of vertices of A - of B) / 3
    float dh[3], dl[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float h = 0.0f, l = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            dd_add(h, l, A.vh[k][c], A.vl[k][c], h, l);
            dd_add(h, l, -B.vh[k][c], -B.vl[k][c], h, l);
        }
        // divide by 3: multiply by 1/3 in double-float
        const float th = 0.333333343267f, tl = -9.93410748e-09f;
        dd_mul(h, l, th, tl, dh[c], dl[c]);
    }
    // r0^2 = |d_c|^2 and r0 in double-float
    float sh = 0.0f, sl = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float ph, pl;
        dd_mul(dh[c], dl[c], dh[c], dl[c], ph, pl);
        dd_add(sh, sl, ph, pl, sh, sl);
    }
    const float rh0 = sqrtf(sh);
    // one Newton step in double-float: r = rh0 + (s - rh0^2) / (2 rh0)
    float qh, ql;
    dd_mul(rh0, 0.0f, rh0, 0.0f, qh, ql);
    float dh2, dl2;
    dd_add(sh, sl, -qh, -ql, dh2, dl2);
    const float corr = (dh2 + dl2) / (2.0f * rh0);
    float r0h, r0l;
    two_sum(rh0, corr, r0h, r0l);
    // kappa r0 in double-float, reduced modulo 2 pi
    const float kh = (float)kappa, kl = (float)(kappa - (double)kh);
    float ph, pl;
    dd_mul(kh, kl, r0h, r0l, ph, pl);
    const float n = rintf(ph * 0.159154943092f);
    const float two_pi_h = 6.28318548202514648f, two_pi_l = -1.74845553e-07f;
    float t = fmaf(-n, two_pi_h, ph);
    t = fmaf(-n, two_pi_l, t) + pl;
    HelmPhase P;
    sincosf(t, &P.s0, &P.c0);
    P.dcx = dh[0] + dl[0];
    P.dcy = dh[1] + dl[1];
    P.dcz = dh[2] + dl[2];
    P.r0h = r0h;
    P.r0l = r0l;
    P.m2r0l = -2.0f * r0l;
    P.r0sqh = sh;
    P.r0sql = sl;
    P.kap = kh;
    return P;
}

// At the offset e = d - d_c: cos and sin of kappa (r - r0), and 1/r.  The
// factor exp(i kappa r0) is common to every point of the pair and is applied
// to the pair's sum by helm_rotate.
//
// r - r0 without a division: q = r^2 - r0^2 = (2 d_c + e) . e is formed in
// float (accurate relative to q, not to r^2); r_a = r2 / sqrt(r2) from the
// rounded r2 = r0^2 + q carries the roundings of r2 and of the reciprocal
// square root, and the residual r^2 - r_a^2 = (r0sq_hi - r_a^2) + (r0sq_lo + q)
// (one FMA) corrects it to first order, r = r_a + res / (2 r_a).  r_a - r0_hi
// is exact while r_a is within a factor 2 of r0, so r - r0 keeps an error of
// a few float ulps of itself plus that of q.  Three special-function
// operations per point (rsqrt, sin, cos).
__device__ __forceinline__ void helm_offset(const HelmPhase &P, float ex, float ey, float ez,
                                            float &c, float &s, float &ri)
{
    const float q = fmaf(fmaf(2.0f, P.dcx, ex), ex,
                         fmaf(fmaf(2.0f, P.dcy, ey), ey, fmaf(2.0f, P.dcz, ez) * ez));
    const float r2 = P.r0sqh + q;
    ri = rsqrt_fast(r2);
    const float ra = r2 * ri;
    const float res = fmaf(-ra, ra, P.r0sqh) + (q + P.r0sql);
    const float delta = fmaf(0.5f, fmaf(res, ri, P.m2r0l), ra - P.r0h);
    __sincosf(P.kap * delta, &s, &c);
}

// (re, im) = exp(i kappa r0) (sr + i si)
__device__ __forceinline__ void helm_rotate(const HelmPhase &P, float sr, float si, float &re,
                                            float &im)
{
    re = P.c0 * sr - P.s0 * si;
    im = P.s0 * sr + P.c0 * si;
}

// Packed FP32 pairs (sm_100 and later): sub/add/mul/fma .f32x2 apply the scalar
// operation, with its rounding, to both halves of a 64-bit register pair in
// one instruction.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 f2_pack(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f32x2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// The float Helmholtz pair of regular_p0_f32_helm with two trial points per
// packed instruction: the same operations per point (helm_offset), each rounded
// as there; the reciprocal square roots, sines and cosines stay scalar.  The
// inner sums run as two partial sums (even and odd trial points) added per
// test point; an odd rule's last pair repeats its last point with weight 0.
template <int NP>
__device__ __forceinline__ void regular_p0_f32_helm_x2(const TriF &A, const TriF &B,
                                                       const Rule2D &R, double kappa,
                                                       float &out_re, float &out_im)
{
    constexpr int NQ = (NP + 1) / 2;
    const HelmPhase P = helm_phase(A, B, kappa);
    f32x2 yx[NQ], yy[NQ], yz[NQ], w2[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int j0 = 2 * q, j1 = 2 * q + 1 < NP ? 2 * q + 1 : NP - 1;
        const float a0 = R.sf[j0] - 0.666666687f, b0 = R.tf[j0] - 0.333333343f;
        const float a1 = R.sf[j1] - 0.666666687f, b1 = R.tf[j1] - 0.333333343f;
        yx[q] = f2_pack(fmaf(a0, B.e1[0], b0 * B.e2[0]), fmaf(a1, B.e1[0], b1 * B.e2[0]));
        yy[q] = f2_pack(fmaf(a0, B.e1[1], b0 * B.e2[1]), fmaf(a1, B.e1[1], b1 * B.e2[1]));
        yz[q] = f2_pack(fmaf(a0, B.e1[2], b0 * B.e2[2]), fmaf(a1, B.e1[2], b1 * B.e2[2]));
        w2[q] = f2_pack(R.wf[j0], 2 * q + 1 < NP ? R.wf[j1] : 0.0f);
    }
    const f32x2 tdx = f2_pack(2.0f * P.dcx, 2.0f * P.dcx), tdy = f2_pack(2.0f * P.dcy, 2.0f * P.dcy),
                tdz = f2_pack(2.0f * P.dcz, 2.0f * P.dcz);
    const f32x2 r0sqh = f2_pack(P.r0sqh, P.r0sqh), nr0sqh = f2_pack(-P.r0sqh, -P.r0sqh),
                r0sql = f2_pack(P.r0sql, P.r0sql), r0h = f2_pack(P.r0h, P.r0h),
                m2r0l = f2_pack(P.m2r0l, P.m2r0l), kap = f2_pack(P.kap, P.kap),
                half = f2_pack(0.5f, 0.5f);
    float sr = 0.0f, si = 0.0f, cr = 0.0f, ci = 0.0f;
#pragma unroll 1
    for (int i = 0; i < NP; ++i) {
        const float a = R.sf[i] - 0.666666687f, b = R.tf[i] - 0.333333343f;
        const float xx = fmaf(a, A.e1[0], b * A.e2[0]);
        const float xy = fmaf(a, A.e1[1], b * A.e2[1]);
        const float xz = fmaf(a, A.e1[2], b * A.e2[2]);
        const f32x2 X = f2_pack(xx, xx), Y = f2_pack(xy, xy), Z = f2_pack(xz, xz);
        f32x2 ir = f2_pack(0.0f, 0.0f), ii = ir;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const f32x2 ex = f2_sub(X, yx[q]), ey = f2_sub(Y, yy[q]), ez = f2_sub(Z, yz[q]);
            // q = (2 d_c + e) . e, r^2 = r0^2 + q (helm_offset)
            const f32x2 qq = f2_fma(f2_add(tdx, ex), ex,
                                    f2_fma(f2_add(tdy, ey), ey, f2_mul(f2_add(tdz, ez), ez)));
            const f32x2 r2 = f2_add(r0sqh, qq);
            float r2a, r2b;
            f2_unpack(r2, r2a, r2b);
            const f32x2 ri = f2_pack(rsqrt_fast(r2a), rsqrt_fast(r2b));
            const f32x2 ra = f2_mul(r2, ri);
            // (r0sq_hi - ra^2) + (q + r0sq_lo), with ra^2 - r0sq_hi from one FMA
            const f32x2 res = f2_sub(f2_add(qq, r0sql), f2_fma(ra, ra, nr0sqh));
            const f32x2 delta = f2_fma(half, f2_fma(res, ri, m2r0l), f2_sub(ra, r0h));
            float ta, tb;
            f2_unpack(f2_mul(kap, delta), ta, tb);
            float sa, ca, sb, cb;
            __sincosf(ta, &sa, &ca);
            __sincosf(tb, &sb, &cb);
            const f32x2 wr = f2_mul(w2[q], ri);
            ir = f2_fma(f2_pack(ca, cb), wr, ir);
            ii = f2_fma(f2_pack(sa, sb), wr, ii);
        }
        float ir0, ir1, ii0, ii1;
        f2_unpack(ir, ir0, ir1);
        f2_unpack(ii, ii0, ii1);
        // compensated outer sums
        float y = fmaf(R.wf[i], ir0 + ir1, -cr), t = sr + y;
        cr = (t - sr) - y;
        sr = t;
        y = fmaf(R.wf[i], ii0 + ii1, -ci);
        t = si + y;
        ci = (t - si) - y;
        si = t;
    }
    float re, im;
    helm_rotate(P, sr, si, re, im);
    const float sc = A.sg * B.sg * (float)kInv4Pi;
    out_re = re * sc;
    out_im = im * sc;
}

// Regular pair, piecewise constant, Helmholtz single layer, float.
template <int NP>
__device__ __forceinline__ void regular_p0_f32_helm(const TriF &A, const TriF &B, const Rule2D &R,
                                                    double kappa, float &out_re, float &out_im)
{
    const HelmPhase P = helm_phase(A, B, kappa);
    // centroid-relative offsets of the y points: y - y_c = (s - 2/3) e1 + (t - 1/3) e2
    float yx[NP], yy[NP], yz[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const float a = R.sf[j] - 0.666666687f, b = R.tf[j] - 0.333333343f;
        yx[j] = fmaf(a, B.e1[0], b * B.e2[0]);
        yy[j] = fmaf(a, B.e1[1], b * B.e2[1]);
        yz[j] = fmaf(a, B.e1[2], b * B.e2[2]);
    }
    float sr = 0.0f, si = 0.0f, cr = 0.0f, ci = 0.0f;
    auto outer = [&](int i) {
        const float a = R.sf[i] - 0.666666687f, b = R.tf[i] - 0.333333343f;
        const float xx = fmaf(a, A.e1[0], b * A.e2[0]);
        const float xy = fmaf(a, A.e1[1], b * A.e2[1]);
        const float xz = fmaf(a, A.e1[2], b * A.e2[2]);
        float ir = 0.0f, ii = 0.0f;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            float c, s, ri;
            helm_offset(P, xx - yx[j], xy - yy[j], xz - yz[j], c, s, ri);
            const float wr = R.wf[j] * ri;
            ir = fmaf(c, wr, ir);
            ii = fmaf(s, wr, ii);
        }
        // compensated outer sums
        float y = fmaf(R.wf[i], ir, -cr), t = sr + y;
        cr = (t - sr) - y;
        sr = t;
        y = fmaf(R.wf[i], ii, -ci);
        t = si + y;
        ci = (t - si) - y;
        si = t;
    };
    // the outer loop stays rolled from 9 points on: the unrolled body of
    // 81 points overflows the instruction cache
    if (NP >= 9) {
#pragma unroll 1
        for (int i = 0; i < NP; ++i) outer(i);
    } else {
#pragma unroll
        for (int i = 0; i < NP; ++i) outer(i);
    }
    float re, im;
    helm_rotate(P, sr, si, re, im);
    const float sc = A.sg * B.sg * (float)kInv4Pi;
    out_re = re * sc;
    out_im = im * sc;
}

// Regular pair, piecewise constant, float (Laplace kernels).  With ABS the
// double layer also returns in *abs_out the sum of the magnitudes of its terms
// (the scale of its rounding error, for the cancellation guard).
template <int KIND, int NP, bool ABS = false>
__device__ __forceinline__ float regular_p0_f32(const TriF &A, const TriF &B, const Rule2D &R,
                                                float *abs_out = nullptr)
{
    float d0[3], yx[NP], yy[NP], yz[NP];
#pragma unroll
    for (int c = 0; c < 3; ++c) d0[c] = dd_diff(A.vh[0][c], A.vl[0][c], B.vh[0][c], B.vl[0][c]);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        yx[j] = fmaf(R.sf[j], B.e1[0], R.tf[j] * B.e2[0]);
        yy[j] = fmaf(R.sf[j], B.e1[1], R.tf[j] * B.e2[1]);
        yz[j] = fmaf(R.sf[j], B.e1[2], R.tf[j] * B.e2[2]);
    }
    Height H = {};
    if (KIND == BEM_LAPLACE_DLP)
        H = make_height(A.vh[0], A.vl[0], A.vh[1], A.vl[1], A.vh[2], A.vl[2], B.vh[0], B.vl[0],
                        B.nh, B.nl);
    float sum = 0.0f, comp = 0.0f, asum = 0.0f;
    auto outer = [&](int i) {
        const float xx = fmaf(R.sf[i], A.e1[0], fmaf(R.tf[i], A.e2[0], d0[0]));
        const float xy = fmaf(R.sf[i], A.e1[1], fmaf(R.tf[i], A.e2[1], d0[1]));
        const float xz = fmaf(R.sf[i], A.e1[2], fmaf(R.tf[i], A.e2[2], d0[2]));
        const float dn = KIND == BEM_LAPLACE_DLP ? height_at(H, R.sf[i], R.tf[i]) : 0.0f;
        float inner = 0.0f;
#pragma unroll
        for (int j = 0; j < NP; ++j)
            inner = fmaf(R.wf[j], kvalf_r<KIND>(xx - yx[j], xy - yy[j], xz - yz[j]), inner);
        if (ABS) asum = fmaf(R.wf[i], inner * fabsf(dn), asum);
        if (KIND == BEM_LAPLACE_DLP) inner *= dn;
        // compensated outer sum (Kahan)
        const float y = fmaf(R.wf[i], inner, -comp);
        const float t = sum + y;
        comp = (t - sum) - y;
        sum = t;
    };
    // larger rules keep the outer loop rolled (code size)
    if (NP > 9) {
#pragma unroll 1
        for (int i = 0; i < NP; ++i) outer(i);
    } else {
#pragma unroll
        for (int i = 0; i < NP; ++i) outer(i);
    }
    if (ABS) *abs_out = asum * (A.sg * B.sg * (float)kInv4Pi);
    return sum * (A.sg * B.sg * (float)kInv4Pi);
}

// Regular pair, piecewise linear (3x3 local matrix), float (Laplace kernels).
template <int KIND, int NP>
__device__ __forceinline__ void regular_p1_f32(const TriF &A, const TriF &B, const Rule2D &R,
                                               float *acc)
{
    float d0[3], yx[NP], yy[NP], yz[NP];
#pragma unroll
    for (int c = 0; c < 3; ++c) d0[c] = dd_diff(A.vh[0][c], A.vl[0][c], B.vh[0][c], B.vl[0][c]);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        yx[j] = fmaf(R.sf[j], B.e1[0], R.tf[j] * B.e2[0]);
        yy[j] = fmaf(R.sf[j], B.e1[1], R.tf[j] * B.e2[1]);
        yz[j] = fmaf(R.sf[j], B.e1[2], R.tf[j] * B.e2[2]);
    }
    Height H = {};
    if (KIND == BEM_LAPLACE_DLP)
        H = make_height(A.vh[0], A.vl[0], A.vh[1], A.vl[1], A.vh[2], A.vl[2], B.vh[0], B.vl[0],
                        B.nh, B.nl);
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
    // outer points not unrolled: the unrolled inner loop alone keeps enough
    // independent work, and the loop body stays small in the instruction cache
#pragma unroll 1
    for (int i = 0; i < NP; ++i) {
        const float xx = fmaf(R.sf[i], A.e1[0], fmaf(R.tf[i], A.e2[0], d0[0]));
        const float xy = fmaf(R.sf[i], A.e1[1], fmaf(R.tf[i], A.e2[1], d0[1]));
        const float xz = fmaf(R.sf[i], A.e1[2], fmaf(R.tf[i], A.e2[2], d0[2]));
        const float dn = KIND == BEM_LAPLACE_DLP ? height_at(H, R.sf[i], R.tf[i]) : 0.0f;
        // trial moments: sum_j w_j lambda_q(y_j) k(x_i, y_j), weights from the rule
        float ir[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            const float k = kvalf_r<KIND>(xx - yx[j], xy - yy[j], xz - yz[j]);
            ir[0] = fmaf(R.wl[0][j], k, ir[0]);
            ir[1] = fmaf(R.wl[1][j], k, ir[1]);
            ir[2] = fmaf(R.wl[2][j], k, ir[2]);
        }
        if (KIND == BEM_LAPLACE_DLP) {
#pragma unroll
            for (int q = 0; q < 3; ++q) ir[q] *= dn;
        }
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const float f = R.wl[p][i];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                acc[p * 3 + q] = fmaf(f, ir[q], acc[p * 3 + q]);
            }
        }
    }
    const float scale = A.sg * B.sg * (float)kInv4Pi;
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] *= scale;
}

// ---------------------------------------------------------------------------
// Touching pairs: one warp per pair, FP64.
//
// In the canonical vertex orders the shared vertices come first, so
//   identical:  x - y = (x1-y1) e1 + (x2-y2) e2          (both maps equal)
//   edge:       x - y = (x1-y1) e1 + x2 e2a - y2 e2b      (shared edge e1)
//   vertex:     x - y = x1 e1a + x2 e2a - y1 e1b - y2 e2b
// with the differences x1-y1, x2-y2 read from the rule (formed from each
// subdomain map's factors).  The double layer (x-y).n_b is the height of x
// above the trial plane: zero for identical (flat) pairs, x2 (e2a . n_b) for
// common edges.  The piecewise-linear local matrix is accumulated as the
// nine moments of (1, x1, x2) x (1, y1, y2) and mapped to the hat functions
// lambda = (1-s, s-t, t) once per pair.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void moments_to_hats(const T M[9], T out[9])
{
    // hats = A m with A = [[1,-1,0],[0,1,-1],[0,0,1]] on both sides: out = A M A^T
    T R[9];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        R[0 * 3 + b] = M[0 * 3 + b] - M[1 * 3 + b];
        R[1 * 3 + b] = M[1 * 3 + b] - M[2 * 3 + b];
        R[2 * 3 + b] = M[2 * 3 + b];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        out[a * 3 + 0] = R[a * 3 + 0] - R[a * 3 + 1];
        out[a * 3 + 1] = R[a * 3 + 1] - R[a * 3 + 2];
        out[a * 3 + 2] = R[a * 3 + 2];
    }
}

// float-float value (unevaluated hi + lo) for moments_to_hats in the float kernels
struct FF {
    float h, l;
};
__device__ __forceinline__ FF operator-(FF a, FF b)
{
    FF r;
    dd_sub(a.h, a.l, b.h, b.l, r.h, r.l);
    return r;
}

// xi = 1: the rule has xi integrated out (Laplace kernels only, see
// touch_xi_out); the moments take their xi_moment factors at the end.
template <int KIND, int BASIS, int CAS>
__device__ __forceinline__ void touch_pair(const MeshView &m, int idx, const double *__restrict__ rule,
                                           int np, double kappa, int lane, double eta = 0.0,
                                           int xi = 0)
{
    const int a = __ldg(m.nb_src + idx), b = __ldg(m.nb_tri + idx);
    const int pc = __ldg(m.nb_perm + idx);
    const int *pa = c_perm[pc / 6], *pb = c_perm[pc % 6];
    constexpr int NACC = BASIS == BEM_P0 ? 1 : 9;
    constexpr bool CPLX = kind_complex(KIND);
    // a flat identical pair has no double layer (the height vanishes)
    constexpr bool ZERO = (KIND == BEM_LAPLACE_DLP || KIND == BEM_HELMHOLTZ_DLP) && CAS == kIdentical;
    double accr[NACC], acci[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) accr[k] = acci[k] = 0.0;
    const double *g_a = m.geom + (int64_t)a * kGeomStride;
    const double *g_b = m.geom + (int64_t)b * kGeomStride;
    if (!ZERO) {
        double va[3][3], vb[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int ia = pa[k], ib = pb[k];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                va[k][c] = __ldg(g_a + 3 * ia + c);
                vb[k][c] = __ldg(g_b + 3 * ib + c);
            }
        }
        double e1a[3], e2a[3], e1b[3], e2b[3], nb[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            e1a[c] = va[1][c] - va[0][c];
            e2a[c] = va[2][c] - va[1][c];
            e1b[c] = vb[1][c] - vb[0][c];
            e2b[c] = vb[2][c] - vb[1][c];
            nb[c] = __ldg(g_b + 9 + c);
        }
        // edge: height of x above the trial plane is x2 (e2a . n_b)
        const double H = e2a[0] * nb[0] + e2a[1] * nb[1] + e2a[2] * nb[2];
        const double *X1 = rule, *X2 = rule + np, *Y1 = rule + 2 * np, *Y2 = rule + 3 * np,
                     *W = rule + 4 * np, *D1 = rule + 5 * np, *D2 = rule + 6 * np;
        for (int p = lane; p < np; p += 32) {
            const double w = __ldg(W + p);
            double x1 = 0.0, x2 = __ldg(X2 + p), y1 = 0.0, y2 = 0.0;
            double dx, dy, dz;
            if (CAS == kIdentical) {
                const double d1 = __ldg(D1 + p), d2 = __ldg(D2 + p);
                dx = d1 * e1a[0] + d2 * e2a[0];
                dy = d1 * e1a[1] + d2 * e2a[1];
                dz = d1 * e1a[2] + d2 * e2a[2];
            } else if (CAS == kEdge) {
                const double d1 = __ldg(D1 + p);
                y2 = __ldg(Y2 + p);
                dx = d1 * e1a[0] + x2 * e2a[0] - y2 * e2b[0];
                dy = d1 * e1a[1] + x2 * e2a[1] - y2 * e2b[1];
                dz = d1 * e1a[2] + x2 * e2a[2] - y2 * e2b[2];
            } else {
                x1 = __ldg(X1 + p);
                y1 = __ldg(Y1 + p);
                y2 = __ldg(Y2 + p);
                dx = x1 * e1a[0] + x2 * e2a[0] - y1 * e1b[0] - y2 * e2b[0];
                dy = x1 * e1a[1] + x2 * e2a[1] - y1 * e1b[1] - y2 * e2b[1];
                dz = x1 * e1a[2] + x2 * e2a[2] - y1 * e1b[2] - y2 * e2b[2];
            }
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double ri = rsqrt(r2);
            double kr, ki = 0.0;
            if (KIND == BEM_LAPLACE_SLP) {
                kr = ri;
            } else if (KIND == BEM_LAPLACE_DLP) {
                const double dn = CAS == kEdge ? x2 * H : dx * nb[0] + dy * nb[1] + dz * nb[2];
                kr = dn * ri * ri * ri;
            } else if (KIND == BEM_HELMHOLTZ_SLP) {
                double sn, cs;
                sincos(kappa * (r2 * ri), &sn, &cs);
                kr = cs * ri;
                ki = sn * ri;
            } else {
                // Helmholtz double layer (and Brakhage-Werner): the height is
                // zero on an identical flat pair, x2 H on a common edge
                const double dn = CAS == kIdentical ? 0.0
                                  : (CAS == kEdge ? x2 * H : dx * nb[0] + dy * nb[1] + dz * nb[2]);
                const double kd = kappa * (r2 * ri);
                double sn, cs;
                sincos(kd, &sn, &cs);
                const double f = dn * ri * ri * ri;
                kr = f * (cs + kd * sn);
                ki = f * (sn - kd * cs);
                if (KIND == BEM_HELMHOLTZ_BW) {
                    kr += eta * sn * ri;
                    ki -= eta * cs * ri;
                }
            }
            const double wr = w * kr, wi = w * ki;
            if (BASIS == BEM_P0) {
                accr[0] += wr;
                if (CPLX) acci[0] += wi;
            } else {
                if (CAS != kVertex) {
                    x1 = __ldg(X1 + p);
                    y1 = __ldg(Y1 + p);
                    if (CAS == kIdentical) y2 = __ldg(Y2 + p);
                }
                const double mx[3] = {1.0, x1, x2}, my[3] = {1.0, y1, y2};
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const double fr = wr * mx[i];
                    const double fi = wi * mx[i];
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        accr[i * 3 + j] += fr * my[j];
                        if (CPLX) acci[i * 3 + j] += fi * my[j];
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NACC; ++k) {
            accr[k] = warp_sum(accr[k]);
            if (CPLX) acci[k] = warp_sum(acci[k]);
        }
    }
    if (lane == 0) {
        if (!CPLX && xi) {
#pragma unroll
            for (int k = 0; k < NACC; ++k) accr[k] *= xi_moment(KIND, k / 3, k % 3);
        }
        const double scale = __ldg(g_a + 12) * __ldg(g_b + 12) * kInv4Pi;
        if (BASIS == BEM_P0) {
            m.table[idx] = make_double2(accr[0] * scale, acci[0] * scale);
        } else {
            double hr[9], hi[9];
            moments_to_hats(accr, hr);
            moments_to_hats(acci, hi);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    m.table[(int64_t)idx * 9 + pa[i] * 3 + pb[j]] =
                        make_double2(hr[i * 3 + j] * scale, hi[i * 3 + j] * scale);
        }
    }
}

// Both Laplace layers of a regular pair (two 3x3 local matrices): each is formed
// exactly as regular_p1_f32 forms it, sharing the points, distances and
// reciprocal square roots.
template <int NP>
__device__ __forceinline__ void regular_p1_f32_fused(const TriF &A, const TriF &B, const Rule2D &R,
                                                     float *acc_s, float *acc_d)
{
    float d0[3], yx[NP], yy[NP], yz[NP];
#pragma unroll
    for (int c = 0; c < 3; ++c) d0[c] = dd_diff(A.vh[0][c], A.vl[0][c], B.vh[0][c], B.vl[0][c]);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        yx[j] = fmaf(R.sf[j], B.e1[0], R.tf[j] * B.e2[0]);
        yy[j] = fmaf(R.sf[j], B.e1[1], R.tf[j] * B.e2[1]);
        yz[j] = fmaf(R.sf[j], B.e1[2], R.tf[j] * B.e2[2]);
    }
    const Height H = make_height(A.vh[0], A.vl[0], A.vh[1], A.vl[1], A.vh[2], A.vl[2], B.vh[0],
                                 B.vl[0], B.nh, B.nl);
#pragma unroll
    for (int k = 0; k < 9; ++k) acc_s[k] = acc_d[k] = 0.0f;
#pragma unroll 1
    for (int i = 0; i < NP; ++i) {
        const float xx = fmaf(R.sf[i], A.e1[0], fmaf(R.tf[i], A.e2[0], d0[0]));
        const float xy = fmaf(R.sf[i], A.e1[1], fmaf(R.tf[i], A.e2[1], d0[1]));
        const float xz = fmaf(R.sf[i], A.e1[2], fmaf(R.tf[i], A.e2[2], d0[2]));
        const float dn = height_at(H, R.sf[i], R.tf[i]);
        float is[3] = {0.0f, 0.0f, 0.0f}, id[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            const float dx = xx - yx[j], dy = xy - yy[j], dz = xz - yz[j];
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float ri = rsqrt_fast(r2);
            const float r3 = ri * ri * ri;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                is[q] = fmaf(R.wl[q][j], ri, is[q]);
                id[q] = fmaf(R.wl[q][j], r3, id[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) id[q] *= dn;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const float f = R.wl[p][i];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                acc_s[p * 3 + q] = fmaf(f, is[q], acc_s[p * 3 + q]);
                acc_d[p * 3 + q] = fmaf(f, id[q], acc_d[p * 3 + q]);
            }
        }
    }
    const float scale = A.sg * B.sg * (float)kInv4Pi;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        acc_s[k] *= scale;
        acc_d[k] *= scale;
    }
}

// Touching pairs in float (mixed form).  The canonical vertex order puts the
// shared vertices first, so x - y is formed from edge vectors and the rule's
// difference columns only and keeps float precision down to the singular set:
//   common vertex: x - y = x1 e1a + x2 e2a - y1 e1b - y2 e2b
//   common edge:   x - y = (x1 - y1) e1 + x2 e2a - y2 e2b   (e1 shared)
//   identical:     x - y = (x1 - y1) e1 + (x2 - y2) e2
// The double-layer numerator (x - y) . n_y is the height of x above the trial
// plane, an affine function on the test triangle whose vertex heights come
// from the FP64 records (neighbours can be nearly coplanar): h(x) for a common
// vertex, x2 h(a2) for a common edge (the shared vertices lie in the plane), 0
// for identical pairs.  Every lane sums its points with Kahan compensation.
// With xi = 1 the rule holds the points at xi = 1 (xi integrated out): the
// Laplace moments take their xi_moment factors at the end, and the Helmholtz
// single layer sums over the Gauss nodes of xi (XR) at each point, sharing the
// distance and its reciprocal square root.
// A pair takes an aligned group of LPP lanes (sub = lane within the group):
// 32 for the q^4 rules, fewer for the shorter xi-integrated ones, so that the
// per-pair set-up and reduction are shared by fewer points.  Every lane of the
// warp calls this (the group reductions shuffle across the warp); a group
// without a pair of its own repeats another and passes store = false.
template <int CAS, int KIND, int BASIS, int LPP = 32>
__device__ __forceinline__ void touch_f32(const MeshView &m, int idx, const float *__restrict__ rule,
                                          int np, int sub, float kappa, int xi, const XiRule &XR,
                                          bool store = true)
{
    static_assert(LPP == 4 || LPP == 8 || LPP == 16 || LPP == 32, "lanes per pair");
    static_assert(BASIS == BEM_P0 || LPP >= 16, "nine hats need nine lanes");
    constexpr bool CPLX = kind_complex(KIND);
    const int a = __ldg(m.nb_src + idx), b = __ldg(m.nb_tri + idx);
    const int pc = __ldg(m.nb_perm + idx);
    const int *pa = c_perm[pc / 6], *pb = c_perm[pc % 6];
    TriF A, B;
    load_trif(m.geomf, a, A);
    load_trif(m.geomf, b, B);
    // canonical vertex order by selects (no dynamically indexed local arrays)
    float ah[3][3], al[3][3], bh[3][3], bl[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int ia = pa[k], ib = pb[k];
            ah[k][c] = ia == 0 ? A.vh[0][c] : (ia == 1 ? A.vh[1][c] : A.vh[2][c]);
            al[k][c] = ia == 0 ? A.vl[0][c] : (ia == 1 ? A.vl[1][c] : A.vl[2][c]);
            bh[k][c] = ib == 0 ? B.vh[0][c] : (ib == 1 ? B.vh[1][c] : B.vh[2][c]);
            bl[k][c] = ib == 0 ? B.vl[0][c] : (ib == 1 ? B.vl[1][c] : B.vl[2][c]);
        }
    float e1a[3], e2a[3], e1b[3], e2b[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        e1a[c] = dd_diff(ah[1][c], al[1][c], ah[0][c], al[0][c]);
        e2a[c] = dd_diff(ah[2][c], al[2][c], ah[1][c], al[1][c]);
        e1b[c] = dd_diff(bh[1][c], bl[1][c], bh[0][c], bl[0][c]);
        e2b[c] = dd_diff(bh[2][c], bl[2][c], bh[1][c], bl[1][c]);
    }
    // Double-layer heights of a's canonical vertices 1, 2 above b's plane (the
    // shared vertex 0 lies in it).  Neighbours can be nearly coplanar, and then
    // the height is a tiny difference of edge-sized terms: the 48-bit hi + lo
    // vertices are too coarse for it, so lane 0 takes it from the FP64 records
    // (the precision of the input) and broadcasts it.
    Height H = {};
    float h2 = 0.0f;
    if (KIND == BEM_LAPLACE_DLP && CAS != kIdentical) {
        double d1 = 0.0, d2 = 0.0;
        if (sub == 0) {
            const double *ga = m.geom + (int64_t)a * kGeomStride;
            const double *gb = m.geom + (int64_t)b * kGeomStride;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double b0 = __ldg(gb + 3 * pb[0] + c), n = __ldg(gb + 9 + c);
                d1 = fma(__ldg(ga + 3 * pa[1] + c) - b0, n, d1);
                d2 = fma(__ldg(ga + 3 * pa[2] + c) - b0, n, d2);
            }
        }
        d1 = __shfl_sync(0xffffffffu, d1, 0, LPP);
        d2 = __shfl_sync(0xffffffffu, d2, 0, LPP);
        if (CAS == kEdge) {
            h2 = (float)d2;
        } else {
            const double d21 = d2 - d1;
            H.h0 = 0.0f;
            H.h0l = 0.0f;
            H.h10 = (float)d1;
            H.h10l = (float)(d1 - (double)H.h10);
            H.h21 = (float)d21;
            H.h21l = (float)(d21 - (double)H.h21);
        }
    }
    constexpr int NACC = BASIS == BEM_P0 ? 1 : 9;
    constexpr int MM = BASIS == BEM_P0 ? 1 : 3;   // moment powers 0, 1, 2
    float acc[NACC], cmp[NACC], acci[NACC], cmpi[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k] = cmp[k] = acci[k] = cmpi[k] = 0.0f;
    // an in-plane double layer vanishes identically on identical pairs
    const bool zero = KIND == BEM_LAPLACE_DLP && CAS == kIdentical;
    const float *X1 = rule, *X2 = rule + np, *Y1 = rule + 2 * np, *Y2 = rule + 3 * np,
                *W = rule + 4 * np, *D1 = rule + 5 * np, *D2 = rule + 6 * np;
    // Each lane takes its points in blocks of KB (stride LPP): the terms of a
    // block are added plainly (error at most KB - 1 ulps of the block's
    // magnitudes) and each block sum enters the lane's sums with Kahan
    // compensation, which keeps the compensated accuracy at a quarter of the
    // additions.
    constexpr int KB = 4;
    // piecewise-constant double layer: the sum of |terms| goes to the unused
    // imaginary part of the table entry (scale of the rounding error, read by
    // the cancellation guard)
    constexpr bool ABS = KIND == BEM_LAPLACE_DLP && BASIS == BEM_P0;
    float asum = 0.0f;
    for (int p0 = sub; p0 < np && !zero; p0 += LPP * KB) {
        float br[NACC], bi[NACC];
#pragma unroll
        for (int k = 0; k < NACC; ++k) br[k] = bi[k] = 0.0f;
#pragma unroll
        for (int u = 0; u < KB; ++u) {
            const int p = p0 + LPP * u;
            if (p >= np) break;
            const float x1 = __ldg(X1 + p), x2 = __ldg(X2 + p), y1 = __ldg(Y1 + p),
                        y2 = __ldg(Y2 + p), w = __ldg(W + p);
            float dx, dy, dz, dn = 0.0f;
            if (CAS == kVertex) {
                dx = fmaf(x1, e1a[0], fmaf(x2, e2a[0], -fmaf(y1, e1b[0], y2 * e2b[0])));
                dy = fmaf(x1, e1a[1], fmaf(x2, e2a[1], -fmaf(y1, e1b[1], y2 * e2b[1])));
                dz = fmaf(x1, e1a[2], fmaf(x2, e2a[2], -fmaf(y1, e1b[2], y2 * e2b[2])));
                if (KIND == BEM_LAPLACE_DLP) dn = height_at(H, x1, x2);
            } else if (CAS == kEdge) {
                const float d1 = __ldg(D1 + p);
                dx = fmaf(d1, e1a[0], fmaf(x2, e2a[0], -y2 * e2b[0]));
                dy = fmaf(d1, e1a[1], fmaf(x2, e2a[1], -y2 * e2b[1]));
                dz = fmaf(d1, e1a[2], fmaf(x2, e2a[2], -y2 * e2b[2]));
                if (KIND == BEM_LAPLACE_DLP) dn = x2 * h2;
            } else {
                const float d1 = __ldg(D1 + p), d2 = __ldg(D2 + p);
                dx = fmaf(d1, e1a[0], d2 * e2a[0]);
                dy = fmaf(d1, e1a[1], d2 * e2a[1]);
                dz = fmaf(d1, e1a[2], d2 * e2a[2]);
            }
            // term of moment power m (the number of coordinate factors x, y):
            // one value for all m unless the Helmholtz xi sum runs here
            float wk[MM], wki[MM];
            if (CPLX) {
                // the pair touches: kappa r stays below kappa times two diameters
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const float ri = rsqrt_fast(r2);
                if (xi) {
                    // (dx, dy, dz) = u(eta) at xi = 1: the Gauss sum over xi of
                    // w_k xi_k^(2+m) exp(i kappa xi_k |u|) / |u| in pairs of
                    // nodes 1/2 -+ t, one sine and cosine per pair (XiRule)
                    const float th = kappa * (r2 * ri);
                    float sr[MM], si[MM];
#pragma unroll
                    for (int q = 0; q < MM; ++q) {
                        sr[q] = XR.cmid[q];
                        si[q] = 0.0f;
                    }
#pragma unroll 1
                    for (int jp = 0; jp < XR.npair; ++jp) {
                        float sn, cs;
                        sincosf(th * XR.t[jp], &sn, &cs);
#pragma unroll
                        for (int q = 0; q < MM; ++q) {
                            sr[q] = fmaf(XR.cp[jp][q], cs, sr[q]);
                            si[q] = fmaf(XR.cm[jp][q], sn, si[q]);
                        }
                    }
                    float s0, c0;
                    sincosf(0.5f * th, &s0, &c0);
                    const float wr = w * ri;
#pragma unroll
                    for (int q = 0; q < MM; ++q) {
                        wk[q] = wr * (sr[q] * c0 - si[q] * s0);
                        wki[q] = wr * (sr[q] * s0 + si[q] * c0);
                    }
                } else {
                    float sn, cs;
                    sincosf(kappa * (r2 * ri), &sn, &cs);
#pragma unroll
                    for (int q = 0; q < MM; ++q) {
                        wk[q] = w * cs * ri;
                        wki[q] = w * sn * ri;
                    }
                }
            } else {
                const float v = w * kvalf<KIND>(dx, dy, dz, dn);
#pragma unroll
                for (int q = 0; q < MM; ++q) {
                    wk[q] = v;
                    wki[q] = 0.0f;
                }
            }
            if (ABS) asum += fabsf(wk[0]);
            const float mx[3] = {1.0f, x1, x2}, my[3] = {1.0f, y1, y2};
#pragma unroll
            for (int i = 0; i < (BASIS == BEM_P0 ? 1 : 3); ++i)
#pragma unroll
                for (int j = 0; j < (BASIS == BEM_P0 ? 1 : 3); ++j) {
                    const int k = BASIS == BEM_P0 ? 0 : i * 3 + j;
                    const int q = BASIS == BEM_P0 ? 0 : (i > 0) + (j > 0);
                    br[k] += BASIS == BEM_P0 ? wk[q] : wk[q] * mx[i] * my[j];
                    if (CPLX) bi[k] += BASIS == BEM_P0 ? wki[q] : wki[q] * mx[i] * my[j];
                }
        }
#pragma unroll
        for (int k = 0; k < NACC; ++k) {
            const float yv = br[k] - cmp[k];
            const float t = acc[k] + yv;
            cmp[k] = (t - acc[k]) - yv;
            acc[k] = t;
            if (CPLX) {
                const float yi = bi[k] - cmpi[k];
                const float ti = acci[k] + yi;
                cmpi[k] = (ti - acci[k]) - yi;
                acci[k] = ti;
            }
        }
    }
    // lane partial sums with their compensations, reduced as float pairs;
    // the hats are formed in float-float as well, and lane q < 9 converts and
    // stores hat q, so the few double operations run once per pair
    FF mr[NACC], mi[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) {
        mr[k] = FF{acc[k], -cmp[k]};
        group_sum2f<LPP>(mr[k].h, mr[k].l);
        mi[k] = FF{0.0f, 0.0f};
        if (CPLX) {
            mi[k] = FF{acci[k], -cmpi[k]};
            group_sum2f<LPP>(mi[k].h, mi[k].l);
        }
    }
    if (ABS) asum = group_sumf<LPP>(asum);
    if (!store) return;
    if (BASIS == BEM_P0) {
        if (sub == 0) {
            // xi integrated out: every term (and so the sum of |terms|) takes one factor
            const double scale = (double)A.sg * (double)B.sg * kInv4Pi *
                                 (!CPLX && xi ? xi_moment(KIND, 0, 0) : 1.0);
            m.table[idx] = make_double2(((double)mr[0].h + (double)mr[0].l) * scale,
                                        ABS ? (double)asum * scale
                                            : ((double)mi[0].h + (double)mi[0].l) * scale);
        }
    } else {
        if (!CPLX && xi) {
#pragma unroll
            for (int k = 0; k < NACC; ++k) {
                const double c = xi_moment(KIND, k / 3, k % 3);
                const float ch = (float)c, cl = (float)(c - (double)ch);
                dd_mul(mr[k].h, mr[k].l, ch, cl, mr[k].h, mr[k].l);
            }
        }
        FF hr[9], hi[9];
        moments_to_hats(mr, hr);
        if (CPLX) moments_to_hats(mi, hi);
        FF vr = hr[0], vi = CPLX ? hi[0] : FF{0.0f, 0.0f};
#pragma unroll
        for (int q = 1; q < 9; ++q)
            if (sub == q) {
                vr = hr[q];
                if (CPLX) vi = hi[q];
            }
        if (sub < 9) {
            const double scale = (double)A.sg * (double)B.sg * kInv4Pi;
            m.table[(int64_t)idx * 9 + pa[sub / 3] * 3 + pb[sub % 3]] =
                make_double2(((double)vr.h + (double)vr.l) * scale,
                             ((double)vi.h + (double)vi.l) * scale);
        }
    }
}

// ---------------------------------------------------------------------------
// Regular pair integrals in one thread (product of a 2D rule with itself).
// ---------------------------------------------------------------------------
template <int KIND, int NP>
__device__ __forceinline__ void regular_p0(const Tri &A, const Tri &B, const Rule2D &R,
                                           double kappa, double &out_re, double &out_im,
                                           double eta = 0.0)
{
    double e1a[3], e2a[3], d0[3], yx[NP], yy[NP], yz[NP];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        e1a[c] = A.v[1][c] - A.v[0][c];
        e2a[c] = A.v[2][c] - A.v[1][c];
        d0[c] = A.v[0][c] - B.v[0][c];
    }
    {
        const double e1b0 = B.v[1][0] - B.v[0][0], e1b1 = B.v[1][1] - B.v[0][1],
                     e1b2 = B.v[1][2] - B.v[0][2];
        const double e2b0 = B.v[2][0] - B.v[1][0], e2b1 = B.v[2][1] - B.v[1][1],
                     e2b2 = B.v[2][2] - B.v[1][2];
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            yx[j] = R.s[j] * e1b0 + R.t[j] * e2b0;
            yy[j] = R.s[j] * e1b1 + R.t[j] * e2b1;
            yz[j] = R.s[j] * e1b2 + R.t[j] * e2b2;
        }
    }
    double sr = 0.0, si = 0.0;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const double xx = d0[0] + R.s[i] * e1a[0] + R.t[i] * e2a[0];
        const double xy = d0[1] + R.s[i] * e1a[1] + R.t[i] * e2a[1];
        const double xz = d0[2] + R.s[i] * e1a[2] + R.t[i] * e2a[2];
        double ir = 0.0, ii = 0.0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            double kr, ki;
            kval<KIND>(xx - yx[j], xy - yy[j], xz - yz[j], B.n, kappa, kr, ki, eta);
            ir += R.w[j] * kr;
            if (kind_complex(KIND)) ii += R.w[j] * ki;
        }
        sr += R.w[i] * ir;
        if (kind_complex(KIND)) si += R.w[i] * ii;
    }
    const double scale = A.sg * B.sg * kInv4Pi;
    out_re = sr * scale;
    out_im = si * scale;
}

template <int KIND, int NP>
__device__ __forceinline__ void regular_p1(const Tri &A, const Tri &B, const Rule2D &R,
                                           double kappa, double *accr, double *acci,
                                           double eta = 0.0)
{
    double e1a[3], e2a[3], d0[3], yx[NP], yy[NP], yz[NP];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        e1a[c] = A.v[1][c] - A.v[0][c];
        e2a[c] = A.v[2][c] - A.v[1][c];
        d0[c] = A.v[0][c] - B.v[0][c];
    }
    {
        const double e1b0 = B.v[1][0] - B.v[0][0], e1b1 = B.v[1][1] - B.v[0][1],
                     e1b2 = B.v[1][2] - B.v[0][2];
        const double e2b0 = B.v[2][0] - B.v[1][0], e2b1 = B.v[2][1] - B.v[1][1],
                     e2b2 = B.v[2][2] - B.v[1][2];
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            yx[j] = R.s[j] * e1b0 + R.t[j] * e2b0;
            yy[j] = R.s[j] * e1b1 + R.t[j] * e2b1;
            yz[j] = R.s[j] * e1b2 + R.t[j] * e2b2;
        }
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) accr[k] = acci[k] = 0.0;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const double xx = d0[0] + R.s[i] * e1a[0] + R.t[i] * e2a[0];
        const double xy = d0[1] + R.s[i] * e1a[1] + R.t[i] * e2a[1];
        const double xz = d0[2] + R.s[i] * e1a[2] + R.t[i] * e2a[2];
        double ir[3] = {0.0, 0.0, 0.0}, ii[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            double kr, ki;
            kval<KIND>(xx - yx[j], xy - yy[j], xz - yz[j], B.n, kappa, kr, ki, eta);
            const double lb[3] = {1.0 - R.s[j], R.s[j] - R.t[j], R.t[j]};
            const double wr = R.w[j] * kr;
            const double wi = R.w[j] * ki;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                ir[q] += wr * lb[q];
                if (kind_complex(KIND)) ii[q] += wi * lb[q];
            }
        }
        const double la[3] = {1.0 - R.s[i], R.s[i] - R.t[i], R.t[i]};
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const double f = R.w[i] * la[p];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                accr[p * 3 + q] += f * ir[q];
                if (kind_complex(KIND)) acci[p * 3 + q] += f * ii[q];
            }
        }
    }
    const double scale = A.sg * B.sg * kInv4Pi;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        accr[k] *= scale;
        acci[k] *= scale;
    }
}

// ---------------------------------------------------------------------------
// Block bookkeeping
// ---------------------------------------------------------------------------
struct BlockInfo {
    int ok;
    int t, s;            // row and column cluster
    int r_lo, nr, c_lo, nc;
    int64_t off;
    int tile_in_blk;
};

__device__ __forceinline__ int64_t find_block(const int64_t *prefix, int64_t nb, int64_t tile)
{
    // first b with prefix[b] > tile (prefix = inclusive sums of tiles per block)
    int64_t lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (prefix[mid] > tile) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ BlockInfo block_info(const BlockLaunch &L, const int64_t *prefix,
                                                int64_t tile, int *status)
{
    BlockInfo bi;
    const int64_t b = find_block(prefix, L.n_blocks, tile);
    const int t = L.blk_row[b], s = L.blk_col[b];
    bi.ok = 0;
    bi.t = t;
    bi.s = s;
    if (t < 0 || t >= L.n_row_clusters || s < 0 || s >= L.n_col_clusters) {
        set_status(status, BEM_ERR_INVALID_ARG);
        return bi;
    }
    bi.r_lo = L.row_ptr[t];
    bi.nr = L.row_ptr[t + 1] - bi.r_lo;
    bi.c_lo = L.col_ptr[s];
    bi.nc = L.col_ptr[s + 1] - bi.c_lo;
    bi.off = L.blk_off[b];
    bi.tile_in_blk = (int)(tile - (b > 0 ? prefix[b - 1] : 0));
    bi.ok = (bi.nr > 0 && bi.nc > 0);
    return bi;
}

// ---------------------------------------------------------------------------
// Block engine, piecewise constant.  The entries of a block list are numbered
// block after block, each block column-major (rows fastest, the order of its
// output); a tile is kP0Tile consecutive entries, one thread each, and may
// span several blocks, so that small blocks (coupling blocks of a few pivots,
// leaves of a few triangles) leave no lane idle.  prefix[b] = entries of
// blocks 0..b (inclusive).
// ---------------------------------------------------------------------------
// Entry threadIdx.x of flat tile `tile` of a block list (prefix = inclusive
// entry counts per block): its triangle pair (a, b) and output position.
// Each warp finds the blocks of its 32 entries by itself (no CTA barrier):
// one search for the block of its first entry, then the inclusive sums of the
// 32 blocks from there, one per lane; an entry's block is the first of them
// whose sum exceeds it (a search over the lanes by shuffles), unless more than
// 32 of the blocks are empty.  Every lane of a warp whose first entry lies
// within the list must call this (shuffles); ok = false past the list's end
// and for invalid blocks or indices (these set the status word).
struct FlatEntry {
    bool ok;
    int a, b;        // test and trial triangle
    int64_t pos;     // output position: block offset + row + column * rows
};

// hint (warp-uniform, in and out): a block index at or before the block of the
// warp's first entry, from the warp's previous tile of the same list (-1:
// none).  Tiles taken in increasing order then find their first block after a
// step or two forward instead of a binary search.
__device__ __forceinline__ FlatEntry flat_entry(const MeshView &m, const BlockLaunch &L,
                                                const int64_t *__restrict__ prefix, int64_t tile,
                                                int *status, int64_t &hint)
{
    static_assert(kP0Tile == 256, "one thread per entry of a tile");
    FlatEntry fe;
    fe.ok = false;
    fe.a = fe.b = 0;
    fe.pos = 0;
    const int lane = threadIdx.x & 31;
    const int64_t ew = tile * kP0Tile + (threadIdx.x & ~31);
    const int64_t total = prefix[L.n_blocks - 1];
    if (ew >= total) return fe;   // the whole warp
    const int64_t e = ew + lane;
    int64_t b0 = -1;
    if (hint >= 0 && hint < L.n_blocks) {
        int64_t h = hint;
        for (int step = 0; step < 8 && h < L.n_blocks - 1 && prefix[h] <= ew; ++step) ++h;
        if (prefix[h] > ew && (h == 0 || prefix[h - 1] <= ew)) b0 = h;
    }
    if (b0 < 0) b0 = find_block(prefix, L.n_blocks, ew);
    hint = b0;
    const int64_t pw = b0 + lane < L.n_blocks ? prefix[b0 + lane] : INT64_MAX;
    const int64_t p_before = b0 > 0 ? prefix[b0 - 1] : 0;
    // k = first window slot with a sum above e (32 if none); six steps
    // narrow [0, 32] to one slot, every lane shuffling in every step
    int lo = 0, hi = 32;
#pragma unroll
    for (int step = 0; step < 6; ++step) {
        const int mid = (lo + hi) >> 1;
        const int64_t v = __shfl_sync(0xffffffffu, pw, mid & 31);
        if (lo < hi) {
            if (v > e) hi = mid;
            else lo = mid + 1;
        }
    }
    const int k = lo;
    const int64_t p_prev = __shfl_sync(0xffffffffu, pw, k > 0 ? k - 1 : 0);
    int64_t b, before;
    if (k < 32) {
        b = b0 + k;
        before = k > 0 ? p_prev : p_before;
    } else {
        b = find_block(prefix, L.n_blocks, e);
        before = b > 0 ? prefix[b - 1] : 0;
    }
    if (e >= total) return fe;
    const int t = L.blk_row[b], s = L.blk_col[b];
    if (t < 0 || t >= L.n_row_clusters || s < 0 || s >= L.n_col_clusters) {
        set_status(status, BEM_ERR_INVALID_ARG);
        return fe;
    }
    const int r_lo = L.row_ptr[t], nr = L.row_ptr[t + 1] - r_lo;
    const int c_lo = L.col_ptr[s], nc = L.col_ptr[s + 1] - c_lo;
    const int64_t le = e - before;
    if (le < 0 || nr <= 0 || le >= (int64_t)nr * nc) {   // the prefix and the blocks disagree
        set_status(status, BEM_ERR_INVALID_ARG);
        return fe;
    }
    const int c = (int)(le / nr), r = (int)(le - (int64_t)c * nr);
    fe.a = L.row_idx[r_lo + r];
    fe.b = L.col_idx[c_lo + c];
    if (fe.a < 0 || fe.a >= m.nt || fe.b < 0 || fe.b >= m.nt) {
        set_status(status, BEM_ERR_INVALID_ARG);
        return fe;
    }
    fe.pos = L.blk_off[b] + le;
    fe.ok = true;
    return fe;
}

// One tile of one block list; `tile` indexes the list's tiles (called by
// every thread of the CTA with the same `tile`; the warps run independently;
// hint as flat_entry's).
template <int KIND, int NP, bool MIXED>
__device__ __forceinline__ void p0_tile(const MeshView &m, const BlockLaunch &L, const Rule2D &R,
                                        const int64_t *__restrict__ prefix, int64_t tile,
                                        int *status, int64_t &hint)
{
    const FlatEntry fe = flat_entry(m, L, prefix, tile, status, hint);
    if (!fe.ok) return;
    const int a = fe.a, bb = fe.b;
    if (L.lower_only && a < bb) return;
    double re, im;
    float absum = 0.0f;   // guarded double layer: sum of |terms|
    const bool guard = MIXED && KIND == BEM_LAPLACE_DLP && L.guard;
    const int4 va = __ldg(m.tvid + a), vb = __ldg(m.tvid + bb);
    if (touching(va, vb)) {
        const int k = L.allow_touching ? find_touching(m, a, bb) : -1;
        if (k < 0) {
            set_status(status, BEM_ERR_INVALID_ARG);
            return;
        }
        const double2 v = m.table[k];
        re = v.x;
        im = v.y;     // the double layer's float touching kernels put A here
        if (guard) absum = (float)v.y;
    } else if (MIXED) {
        TriF A, B;
        load_trif(m.geomf, a, A);
        load_trif(m.geomf, bb, B);
        if (KIND == BEM_HELMHOLTZ_SLP) {
            float fr, fi;
            regular_p0_f32_helm_x2<NP>(A, B, R, L.kappa, fr, fi);
            re = (double)fr;
            im = (double)fi;
        } else if (guard) {
            re = (double)regular_p0_f32<BEM_LAPLACE_DLP, NP, true>(A, B, R, &absum);
            im = 0.0;
        } else {
            re = (double)regular_p0_f32<KIND, NP>(A, B, R);
            im = 0.0;
        }
    } else {
        Tri A, B;
        load_tri(m.geom, a, A);
        load_tri(m.geom, bb, B);
        regular_p0<KIND, NP>(A, B, R, L.kappa, re, im, L.eta);
    }
    const int64_t o = fe.pos;
    if (kind_complex(KIND)) reinterpret_cast<double2 *>(L.out)[o] = make_double2(re, im);
    else if (guard) reinterpret_cast<float2 *>(L.out)[o] = make_float2((float)re, absum);
    else reinterpret_cast<double *>(L.out)[o] = re;
}

// ---------------------------------------------------------------------------
// Block engine, piecewise linear: tile = 32 x 32 vertices.  The triangles
// touching the tile's rows (Ta) and columns (Tb) come to shared memory from the
// per-run support records (plans) or are collected by the tile itself (single
// calls; same function, same result); the 3x3 local matrices of all pairs
// Ta x Tb are computed chunk by chunk (one thread per pair) into shared memory
// and gathered in two fixed-order stages (deterministic sums): per (row
// triangle, column vertex) over the column's support, then by the owner
// thread of each entry over its row's support.
// ---------------------------------------------------------------------------
// pairs per chunk: float results (36 KB per chunk) leave room for four CTAs
// per SM; double results stay at 512 pairs so that complex chunks fit too
__host__ __device__ constexpr int p1_cap(bool mixed, bool fused = false)
{
    return mixed && !fused ? 1024 : 512;   // fused: two float results per pair, same bytes
}
// Row triangles per chunk at most: the gather first sums each (row triangle,
// column vertex) over the column's support into a staging array of this many
// rows x (kTile + 1) columns x 3 local test indices (6.3 KB per result).
__host__ __device__ constexpr int p1_chunk_rows(bool mixed, bool fused = false)
{
    return mixed && !fused ? 16 : 8;
}
constexpr int kP1StageLd = kTile + 1;   // padded column stride of the staging array
constexpr int kP1MaxTri = kTile * kMaxDegP1;

struct P1Smem {
    int rows[kTile], cols[kTile];
    int ta[kP1MaxTri], tb[kP1MaxTri];
    // per-vertex support lists, stored [k][vertex] so that the 32 lanes of a
    // warp (one vertex each) read consecutive words (no bank conflicts)
    int rl[kMaxDegP1][kTile], cl[kMaxDegP1][kTile];
    int rl_n[kTile], cl_n[kTile];
    int cnt_r[kTile], off_r[kTile], cnt_c[kTile], off_c[kTile];
    int nta, ntb;
};

__device__ __forceinline__ int pos_in(const int *set, int n, int v)
{
    for (int k = 0; k < n; ++k)
        if (set[k] == v) return k;
    return -1;
}

__device__ __forceinline__ int owner_pos(const MeshView &m, int T, const int *set, int n)
{
    const int4 tv = __ldg(m.tvid + T);
    int p = pos_in(set, n, tv.x);
    int q = pos_in(set, n, tv.y);
    int r = pos_in(set, n, tv.z);
    int best = 1 << 30;
    if (p >= 0) best = min(best, p);
    if (q >= 0) best = min(best, q);
    if (r >= 0) best = min(best, r);
    return best;
}

// Collect the triangles touching the vertex set `set` (n <= 32): deterministic
// order (by owner position, then adjacency order), and per vertex the list of
// (triangle slot << 2 | local index), sorted by slot so that the gather can
// walk it once across the chunks of triangle rows.
__device__ __forceinline__ void p1_support(const MeshView &m, const int *set, int n, int *tri, int *cnt,
                           int *off, int (*lists)[kTile], int *list_n, int *ntri,
                           int *status)
{
    const int tid = threadIdx.x;
    if (tid < n) {
        const int v = set[tid];
        const int lo = __ldg(m.vt_ptr + v), hi = __ldg(m.vt_ptr + v + 1);
        int c = 0;
        for (int k = lo; k < hi; ++k)
            if (owner_pos(m, __ldg(m.vt_tri + k), set, n) == tid) ++c;
        cnt[tid] = c;
    }
    __syncthreads();
    if (tid == 0) {
        int s = 0;
        for (int k = 0; k < n; ++k) {
            off[k] = s;
            s += cnt[k];
        }
        *ntri = s;
    }
    __syncthreads();
    if (tid < n) {
        const int v = set[tid];
        const int lo = __ldg(m.vt_ptr + v), hi = __ldg(m.vt_ptr + v + 1);
        int c = off[tid];
        for (int k = lo; k < hi; ++k) {
            const int T = __ldg(m.vt_tri + k);
            if (owner_pos(m, T, set, n) == tid) tri[c++] = T;
        }
    }
    __syncthreads();
    if (tid < n) {
        const int v = set[tid];
        const int lo = __ldg(m.vt_ptr + v), hi = __ldg(m.vt_ptr + v + 1);
        for (int k = lo; k < hi; ++k) {
            const int T = __ldg(m.vt_tri + k);
            const int q = owner_pos(m, T, set, n);
            int slot = -1;
            for (int u = off[q]; u < off[q] + cnt[q]; ++u)
                if (tri[u] == T) slot = u;
            const int4 tv = __ldg(m.tvid + T);
            const int loc = tv.x == v ? 0 : (tv.y == v ? 1 : 2);
            // insertion into the slot-sorted list (slots are distinct)
            int u = k - lo;
            const int key = (slot << 2) | loc;
            while (u > 0 && lists[u - 1][tid] > key) {
                lists[u][tid] = lists[u - 1][tid];
                --u;
            }
            lists[u][tid] = key;
        }
        list_n[tid] = hi - lo;
    }
    __syncthreads();
}

static_assert(kSupCount + 1 <= kSupInts && kSupLists % 4 == 0 && kSupTris % 4 == 0 &&
                  kSupInts % 4 == 0,
              "support records must be int4-aligned");

// Copies one support record (built by k_build_supports) into shared memory;
// returns the triangle count, or -1 for a record marked invalid.
__device__ __forceinline__ int p1_load_support(const int32_t *__restrict__ rec, int *tri,
                                               int (*lists)[kTile], int *list_n)
{
    const int nt = __ldg(rec + kSupCount);
    const int4 *src = reinterpret_cast<const int4 *>(rec);
    for (int k = threadIdx.x; k < kSupCount / 4; k += blockDim.x) {
        const int w = 4 * k;
        if (w < kSupLists) {
            *reinterpret_cast<int4 *>(list_n + w) = __ldg(src + k);
        } else if (w < kSupTris) {
            *reinterpret_cast<int4 *>(&lists[0][0] + (w - kSupLists)) = __ldg(src + k);
        } else if (w - kSupTris < nt) {
            *reinterpret_cast<int4 *>(tri + (w - kSupTris)) = __ldg(src + k);
        }
    }
    return nt;
}

// Threads per CTA of the P1 block engine: the FP64 form saturates the FP64
// pipe with one 256-thread CTA per SM; the float form runs 128-thread CTAs,
// several per SM, so that one CTA's barrier waits overlap another's math.
__host__ __device__ constexpr int p1_threads(bool mixed) { return mixed ? 128 : 256; }
__host__ __device__ constexpr int p1_min_blocks(bool mixed) { return mixed ? 4 : 1; }

// One 32 x 32 tile of one block list (called by every thread of the CTA).
template <int KIND, int NP, bool MIXED>
__device__ __forceinline__ void p1_tile(const MeshView &m, const BlockLaunch &L, const Rule2D &R,
                                        const int64_t *__restrict__ prefix, int64_t tile,
                                        int *status, unsigned char *smem_raw)
{
    constexpr bool CPLX = kind_complex(KIND);
    // fused: single layer in the real slots, double layer in the second ones
    constexpr bool FUSED = KIND == kFusedLaplace;
    constexpr bool TWO = CPLX || FUSED;
    constexpr int NT = p1_threads(MIXED);
    constexpr int NE = kTile * kTile / NT;     // entries owned per thread
    constexpr int EW = NT / 32;                // column stride of owned entries
    constexpr int CAP = p1_cap(MIXED, FUSED);
    constexpr int CR = p1_chunk_rows(MIXED, FUSED);
    constexpr int TN = CR * kP1StageLd * 3;    // staging values per result
    // pair results: double in the FP64 form, float in the mixed form
    using Val = typename std::conditional<MIXED, float, double>::type;
    P1Smem &S = *reinterpret_cast<P1Smem *>(smem_raw);
    Val *buf_r = reinterpret_cast<Val *>(smem_raw + ((sizeof(P1Smem) + 15) & ~size_t(15)));
    Val *buf_i = buf_r + CAP * 9;
    Val *stg_r = buf_r + CAP * 9 * (TWO ? 2 : 1);
    Val *stg_i = stg_r + TN;
    const int tid = threadIdx.x;
    {
        const BlockInfo bi = block_info(L, prefix, tile, status);
        if (!bi.ok) return;   // uniform across the CTA
        const int ntr = (bi.nr + kTile - 1) / kTile;
        const int r0 = (bi.tile_in_blk % ntr) * kTile, c0 = (bi.tile_in_blk / ntr) * kTile;
        const int tr = min(kTile, bi.nr - r0), tc = min(kTile, bi.nc - c0);
        __shared__ int bad;
        if (tid == 0) bad = 0;
        __syncthreads();
        if (tid < tr) {
            const int v = L.row_idx[bi.r_lo + r0 + tid];
            if (v < 0 || v >= m.nv) bad = 1;
            S.rows[tid] = v;
        }
        if (tid >= 64 && tid - 64 < tc) {
            const int v = L.col_idx[bi.c_lo + c0 + tid - 64];
            if (v < 0 || v >= m.nv) bad = 1;
            S.cols[tid - 64] = v;
        }
        __syncthreads();
        if (bad) {
            if (tid == 0) set_status(status, BEM_ERR_INVALID_ARG);
            __syncthreads();
            return;
        }
        int nta, ntb;
        if (L.sup_r) {
            // supports built once per run for every cluster slice
            const int64_t sr = (int64_t)__ldg(L.slice_r + bi.t) + r0 / kTile;
            const int64_t sc = (int64_t)__ldg(L.slice_c + bi.s) + c0 / kTile;
            if (sr >= L.cap_r || sc >= L.cap_c) {
                if (tid == 0) set_status(status, BEM_ERR_INVALID_ARG);
                return;   // uniform across the CTA
            }
            nta = p1_load_support(L.sup_r + sr * kSupInts, S.ta, S.rl, S.rl_n);
            ntb = p1_load_support(L.sup_c + sc * kSupInts, S.tb, S.cl, S.cl_n);
            __syncthreads();
            if (nta < 0 || ntb < 0) {
                if (tid == 0) set_status(status, BEM_ERR_INVALID_ARG);
                __syncthreads();
                return;
            }
        } else {
            p1_support(m, S.rows, tr, S.ta, S.cnt_r, S.off_r, S.rl, S.rl_n, &S.nta, status);
            p1_support(m, S.cols, tc, S.tb, S.cnt_c, S.off_c, S.cl, S.cl_n, &S.ntb, status);
            nta = S.nta;
            ntb = S.ntb;
        }
        const int ia_step = max(1, min(CR, CAP / max(ntb, 1)));
        // cmpr, cmpi: Kahan compensations (mixed form)
        Val accr[NE], acci[NE], cmpr[NE], cmpi[NE];
#pragma unroll
        for (int e = 0; e < NE; ++e) accr[e] = acci[e] = cmpr[e] = cmpi[e] = 0;
        const int er = tid & 31;
        // this thread's row vertex: its support list is sorted by triangle
        // slot, so the rows of each chunk are the next run of the list
        const int nrl = er < tr ? S.rl_n[er] : 0;
        int u_end = 0;
        for (int ia0 = 0; ia0 < nta; ia0 += ia_step) {
            const int ia1 = min(nta, ia0 + ia_step);
            const int npairs = (ia1 - ia0) * ntb;
            for (int p = tid; p < npairs; p += blockDim.x) {
                const int a = S.ta[ia0 + p / ntb], b = S.tb[p % ntb];
                const int4 va = __ldg(m.tvid + a), vb = __ldg(m.tvid + b);
                Val vr[9], vi[9];
                if (touching(va, vb)) {
                    const int k = L.allow_touching ? find_touching(m, a, b) : -1;
                    if (k < 0) {
                        set_status(status, BEM_ERR_INVALID_ARG);
#pragma unroll
                        for (int q = 0; q < 9; ++q) vr[q] = vi[q] = 0;
                    } else {
#pragma unroll
                        for (int q = 0; q < 9; ++q) {
                            const double2 t = m.table[(int64_t)k * 9 + q];
                            vr[q] = (Val)t.x;
                            vi[q] = FUSED ? (Val)L.table2[(int64_t)k * 9 + q].x : (Val)t.y;
                        }
                    }
                } else if (FUSED) {
                    TriF A, B;
                    load_trif(m.geomf, a, A);
                    load_trif(m.geomf, b, B);
                    float fs[9], fd[9];
                    regular_p1_f32_fused<NP>(A, B, R, fs, fd);
#pragma unroll
                    for (int q = 0; q < 9; ++q) {
                        vr[q] = (Val)fs[q];
                        vi[q] = (Val)fd[q];
                    }
                } else if (MIXED) {
                    TriF A, B;
                    load_trif(m.geomf, a, A);
                    load_trif(m.geomf, b, B);
                    float f[9];
                    regular_p1_f32<KIND, NP>(A, B, R, f);
#pragma unroll
                    for (int q = 0; q < 9; ++q) {
                        vr[q] = (Val)f[q];
                        vi[q] = 0;
                    }
                } else {
                    Tri A, B;
                    load_tri(m.geom, a, A);
                    load_tri(m.geom, b, B);
                    double dr[9], di[9];
                    regular_p1<KIND, NP>(A, B, R, L.kappa, dr, di, L.eta);
#pragma unroll
                    for (int q = 0; q < 9; ++q) {
                        vr[q] = (Val)dr[q];
                        vi[q] = (Val)di[q];
                    }
                }
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    buf_r[p * 9 + q] = vr[q];
                    if (TWO) buf_i[p * 9 + q] = vi[q];
                }
            }
            __syncthreads();
            // gather, stage 1: per (row triangle a of the chunk, column vertex
            // j) the sums over the triangles b of j's support, for the three
            // local indices of a (consecutive threads take the row triangles
            // of one column, so they walk the same support list)
            const int na = ia1 - ia0;
            for (int it = tid; it < na * tc; it += NT) {
                const int al = it % na, jc = it / na;
                Val sr[3] = {0, 0, 0}, si[3] = {0, 0, 0};
                const int rowbase = al * ntb;
                const int nv = S.cl_n[jc];
                for (int v = 0; v < nv; ++v) {
                    const int key = S.cl[v][jc];
                    const int q = (rowbase + (key >> 2)) * 9 + (key & 3);
#pragma unroll
                    for (int la = 0; la < 3; ++la) {
                        sr[la] += buf_r[q + la * 3];
                        if (TWO) si[la] += buf_i[q + la * 3];
                    }
                }
                const int o = (al * kP1StageLd + jc) * 3;
#pragma unroll
                for (int la = 0; la < 3; ++la) {
                    stg_r[o + la] = sr[la];
                    if (TWO) stg_i[o + la] = si[la];
                }
            }
            __syncthreads();
            // stage 2: each entry's owner adds the staged sums of its row
            // vertex's support triangles in this chunk (the next run of its
            // slot-sorted list), compensated in the float forms
            const int u_beg = u_end;
            while (u_end < nrl && (S.rl[u_end][er] >> 2) < ia1) ++u_end;
#pragma unroll
            for (int e = 0; e < NE; ++e) {
                const int ec = (tid >> 5) + EW * e;
                if (er < tr && ec < tc) {
                    for (int u = u_beg; u < u_end; ++u) {
                        const int key = S.rl[u][er];
                        const int q = (((key >> 2) - ia0) * kP1StageLd + ec) * 3 + (key & 3);
                        if (MIXED) {
                            const Val y = stg_r[q] - cmpr[e];
                            const Val t = accr[e] + y;
                            cmpr[e] = (t - accr[e]) - y;
                            accr[e] = t;
                            if (FUSED) {
                                const Val y2 = stg_i[q] - cmpi[e];
                                const Val t2 = acci[e] + y2;
                                cmpi[e] = (t2 - acci[e]) - y2;
                                acci[e] = t2;
                            }
                        } else {
                            accr[e] += stg_r[q];
                        }
                        if (CPLX) acci[e] += stg_i[q];
                    }
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            const int ec = (tid >> 5) + EW * e;
            if (er < tr && ec < tc) {
                if (L.lower_only && S.rows[er] < S.cols[ec]) continue;
                const int64_t o = bi.off + (int64_t)(r0 + er) + (int64_t)(c0 + ec) * bi.nr;
                if (CPLX) {
                    reinterpret_cast<double2 *>(L.out)[o] = make_double2((double)accr[e], (double)acci[e]);
                } else {
                    reinterpret_cast<double *>(L.out)[o] = (double)accr[e];
                    if (FUSED) reinterpret_cast<double *>(L.out2)[o] = (double)acci[e];
                }
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int find_job(const int64_t *job_end, int n_jobs, int64_t tile)
{
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (job_end[mid] > tile) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

struct RuleSet {
    const double *d[4];
    int n[4];
};

}  // namespace bem
