// Green quadrature matrices of the GCA (Section 2.3) on the device.
//
// For a cluster t, Green's representation formula on an auxiliary domain
// omega_t that encloses the supports of the cluster's basis functions,
// discretised by a quadrature rule (z_nu, w_nu) on the boundary of omega_t,
// turns the far field of every basis function phi_i of t into the rows of
//   A_t+[i, nu] = sp_nu int phi_i(x) g(x, z_nu) dx
//   A_t-[i, nu] = sm_nu int phi_i(x) d/dn(z_nu) g(x, z_nu) dx
// (the GCA takes sp = sqrt(w_nu) and sm = sqrt(w_nu) delta_t).  Cross
// approximation on these matrices picks the pivots of the H^2 coupling
// blocks.  The paper assembles them on the CPU, where they cost about as much
// as its whole GPU phase; here they are one launch for a list of clusters.
//
// g(x, z) = exp(i kappa r) / (4 pi r), r = |x - z| (kappa = 0 for the Laplace
// kernels), and the normal derivative is taken in z along the unit normal n:
//   n . grad_z g = (x - z).n (1 - i kappa r) exp(i kappa r) / (4 pi r^3).
// Every support triangle is integrated by a 2D rule on the reference triangle
// D = {0 <= t <= s <= 1} with the affine map Phi(s,t) = v0 + s (v1 - v0) +
// t (v2 - v1) and Gram factor sqrt(g) (Section 2.2), in FP64.
//
// Work split: one CTA per cluster, one warp per row (basis function) and the
// cluster's points across the lanes, 32 at a time.  The lanes of a warp walk
// the same support triangles and rule points, so geometry loads are warp-
// uniform broadcasts and the support loop of the piecewise-linear basis does
// not diverge; the lanes differ only in z_nu.  The plus and minus entries
// share the distance and its reciprocal square root.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "bem_device.cuh"

namespace bem {
namespace {

constexpr int kGreenThreads = 256;

struct GreenArgs {
    const int32_t *row_ptr, *row_idx, *pt_ptr;
    const double *z, *nz, *sp, *sm;
    const int64_t *out_off;
    void *out;
    int64_t n_row_idx, n_points, out_len;
    double kappa;
};

// Sums over one support triangle T of the rule points' contributions for the
// point z with normal n (Section 2.3), without sqrt(g) and 1/(4 pi):
//   plus  += w_q phi(s_q, t_q) exp(i kappa r) / r
//   minus += w_q phi(s_q, t_q) (x - z).n (1 - i kappa r) exp(i kappa r) / r^3
// with x = Phi_T(s_q, t_q), r = |x - z|.  loc < 0: constant basis; otherwise
// the local vertex (original order) whose hat function phi is.
template <bool HELM, int NP>
__device__ __forceinline__ void green_triangle(const Tri &T, int loc, const double *z,
                                               const double *n, const Rule2D &R, double kappa,
                                               double &pr, double &pi, double &mr, double &mi)
{
    double e1[3], e2[3], d0[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        e1[c] = T.v[1][c] - T.v[0][c];
        e2[c] = T.v[2][c] - T.v[1][c];
        d0[c] = T.v[0][c] - z[c];
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const double s = R.s[q], t = R.t[q];
        const double phi = loc < 0 ? 1.0 : (loc == 0 ? 1.0 - s : (loc == 1 ? s - t : t));
        const double wq = R.w[q] * phi;
        const double dx = d0[0] + s * e1[0] + t * e2[0];
        const double dy = d0[1] + s * e1[1] + t * e2[1];
        const double dz = d0[2] + s * e1[2] + t * e2[2];
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double ri = rsqrt(r2);
        const double dn = dx * n[0] + dy * n[1] + dz * n[2];
        const double h = wq * dn * (ri * ri * ri);
        if (!HELM) {
            pr += wq * ri;
            mr += h;
        } else {
            const double kr = kappa * (r2 * ri);
            double sn, cs;
            sincos(kr, &sn, &cs);
            pr += wq * cs * ri;
            pi += wq * sn * ri;
            mr += h * (cs + kr * sn);
            mi += h * (sn - kr * cs);
        }
    }
}

template <bool HELM, int NP>
__global__ void __launch_bounds__(kGreenThreads) k_green(MeshView m, GreenArgs a, Rule2D R,
                                                         int *status)
{
    __shared__ int s_ok;
    __shared__ int s_rb, s_nr, s_pb, s_mp;
    __shared__ long long s_off;
    const int c = blockIdx.x;
    if (threadIdx.x == 0) {
        const int32_t rb = a.row_ptr[c], re = a.row_ptr[c + 1];
        const int32_t pb = a.pt_ptr[c], pe = a.pt_ptr[c + 1];
        const int64_t off = a.out_off[c];
        // the row and point loops step in int: a cluster holds fewer than 2^30 of each
        bool ok = rb >= 0 && re >= rb && re <= a.n_row_idx && pb >= 0 && pe >= pb &&
                  pe <= a.n_points && re - rb < (1 << 30) && pe - pb < (1 << 30);
        if (ok && re > rb && pe > pb) {
            // both factors are below 2^31, so the block size fits in int64
            const int64_t need = 2 * (int64_t)(re - rb) * (int64_t)(pe - pb);
            ok = off >= 0 && off <= a.out_len - need;
        }
        if (!ok) set_status(status, BEM_ERR_INVALID_ARG);
        s_ok = ok && re > rb && pe > pb;
        s_rb = rb;
        s_nr = re - rb;
        s_pb = pb;
        s_mp = pe - pb;
        s_off = off;
    }
    __syncthreads();
    if (!s_ok) return;
    const int rb = s_rb, nr = s_nr, pb = s_pb, mp = s_mp;
    const int64_t off = s_off;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t lim = m.basis == BEM_P0 ? m.nt : m.nv;
    for (int r = warp; r < nr; r += nwarps) {
        const int i = __ldg(a.row_idx + rb + r);
        if (i < 0 || i >= lim) {
            if (lane == 0) set_status(status, BEM_ERR_INVALID_ARG);
            continue;
        }
        const int klo = m.basis == BEM_P0 ? 0 : __ldg(m.vt_ptr + i);
        const int khi = m.basis == BEM_P0 ? 1 : __ldg(m.vt_ptr + i + 1);
        for (int base = 0; base < mp; base += 32) {
            const int nu = base + lane;
            const bool act = nu < mp;
            // idle lanes of the last chunk repeat the cluster's last point and write nothing
            const int64_t p = pb + (act ? nu : mp - 1);
            double z[3], n[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                z[d] = __ldg(a.z + 3 * p + d);
                n[d] = __ldg(a.nz + 3 * p + d);
            }
            double pr = 0.0, pi = 0.0, mr = 0.0, mi = 0.0;
            for (int k = klo; k < khi; ++k) {
                const int tr = m.basis == BEM_P0 ? i : __ldg(m.vt_tri + k);
                Tri T;
                load_tri(m.geom, tr, T);
                int loc = -1;
                if (m.basis == BEM_P1) {
                    const int4 tv = __ldg(m.tvid + tr);
                    loc = tv.x == i ? 0 : (tv.y == i ? 1 : 2);
                }
                double tpr = 0.0, tpi = 0.0, tmr = 0.0, tmi = 0.0;
                green_triangle<HELM, NP>(T, loc, z, n, R, a.kappa, tpr, tpi, tmr, tmi);
                pr += T.sg * tpr;
                mr += T.sg * tmr;
                if (HELM) {
                    pi += T.sg * tpi;
                    mi += T.sg * tmi;
                }
            }
            if (act) {
                const double fp = (a.sp ? __ldg(a.sp + p) : 1.0) * kInv4Pi;
                const double fm = (a.sm ? __ldg(a.sm + p) : 1.0) * kInv4Pi;
                const int64_t ep = off + r + (int64_t)nu * nr;          // A+ column nu
                const int64_t em = off + r + (int64_t)(mp + nu) * nr;   // A- column nu
                if (HELM) {
                    double2 *o = reinterpret_cast<double2 *>(a.out);
                    o[ep] = make_double2(fp * pr, fp * pi);
                    o[em] = make_double2(fm * mr, fm * mi);
                } else {
                    double *o = reinterpret_cast<double *>(a.out);
                    o[ep] = fp * pr;
                    o[em] = fm * mr;
                }
            }
        }
    }
}

template <bool HELM>
cudaError_t launch_green(const MeshView &m, const GreenArgs &a, int n_clusters, const Rule2D &R,
                         int *status, cudaStream_t st)
{
#define BEM_GREEN(NP) k_green<HELM, NP><<<n_clusters, kGreenThreads, 0, st>>>(m, a, R, status)
    switch (R.np) {
    case 1: BEM_GREEN(1); break;
    case 4: BEM_GREEN(4); break;
    case 7: BEM_GREEN(7); break;
    case 9: BEM_GREEN(9); break;
    case 16: BEM_GREEN(16); break;
    case 25: BEM_GREEN(25); break;
    default: return cudaErrorInvalidValue;
    }
#undef BEM_GREEN
    return cudaGetLastError();
}

}  // namespace
}  // namespace bem

extern "C" int bem_green_matrices(bem_ctx *ctx, const bem_green_job *job)
{
    using namespace bem;
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (!job) return api_fail(ctx, BEM_ERR_INVALID_ARG, "null job");
    const bem_green_job &J = *job;
    auto it = ctx->meshes.find(J.mesh_id);
    if (it == ctx->meshes.end()) return api_fail(ctx, BEM_ERR_INVALID_ARG, "unknown mesh id");
    const Mesh *mesh = it->second;
    if (J.kernel.kind < BEM_LAPLACE_SLP || J.kernel.kind > BEM_HELMHOLTZ_SLP ||
        !std::isfinite(J.kernel.kappa))
        return api_fail(ctx, BEM_ERR_INVALID_ARG, "bad kernel descriptor");
    Rule2D R;
    std::memset(&R, 0, sizeof R);
    if (!(J.rule == BEM_RULE_TRI7 || (J.rule == BEM_RULE_DUFFY && J.q >= 1 && J.q <= 5)) ||
        !make_rule2d(J.rule, J.q, R))
        return api_fail(ctx, BEM_ERR_INVALID_ARG,
                        "bem_green_matrices: rule must be TRI7 or DUFFY with q in [1, 5]");
    if (J.n_clusters < 0 || J.n_row_idx < 0 || J.n_points < 0 || J.out_len < 0)
        return api_fail(ctx, BEM_ERR_INVALID_ARG, "negative count");
    if (J.n_clusters == 0) return BEM_OK;
    if (!J.row_ptr || !J.pt_ptr || !J.out_off || (J.n_row_idx > 0 && !J.row_idx) ||
        (J.n_points > 0 && (!J.z || !J.nz)) || (J.out_len > 0 && !J.out))
        return api_fail(ctx, BEM_ERR_INVALID_ARG, "null pointer");
    const bool helm = J.kernel.kind == BEM_HELMHOLTZ_SLP;
    if (helm && (reinterpret_cast<uintptr_t>(J.out) & 15))
        return api_fail(ctx, BEM_ERR_INVALID_ARG, "complex output must be 16-byte aligned");
    GreenArgs a;
    a.row_ptr = J.row_ptr;
    a.row_idx = J.row_idx;
    a.pt_ptr = J.pt_ptr;
    a.z = J.z;
    a.nz = J.nz;
    a.sp = J.sp;
    a.sm = J.sm;
    a.out_off = J.out_off;
    a.out = J.out;
    a.n_row_idx = J.n_row_idx;
    a.n_points = J.n_points;
    a.out_len = J.out_len;
    a.kappa = helm ? J.kernel.kappa : 0.0;
    cudaError_t e;
    {
        ProfScope ps(ctx, "green");
        e = helm ? launch_green<true>(mesh->v, a, J.n_clusters, R, ctx->status, ctx->stream)
                 : launch_green<false>(mesh->v, a, J.n_clusters, R, ctx->status, ctx->stream);
    }
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "green kernel");
    return BEM_OK;
}

extern "C" int bem_gca_pivots_device(bem_ctx *ctx, int32_t mesh_id, const double *verts,
                                     int64_t nv, const int32_t *tris, int64_t nt, int32_t basis,
                                     double kappa, const int32_t *cl_ptr, const int32_t *cl_idx,
                                     const int32_t *cl_son, int32_t n_clusters,
                                     int32_t gauss_per_face, double eps, int32_t max_rank,
                                     int32_t n_threads, int32_t *piv_ptr, int32_t *piv_idx,
                                     int64_t cap)
{
    using namespace bem;
    if (!ctx) return BEM_ERR_INVALID_ARG;
    auto it = ctx->meshes.find(mesh_id);
    if (it == ctx->meshes.end()) return api_fail(ctx, BEM_ERR_INVALID_ARG, "unknown mesh id");
    const Mesh *mesh = it->second;
    if (mesh->v.nv != nv || mesh->v.nt != nt || mesh->v.basis != basis || !verts || !tris ||
        mesh_hash(verts, nv, tris, nt) != mesh->host_hash)
        return api_fail(ctx, BEM_ERR_INVALID_ARG,
                        "bem_gca_pivots_device: the host mesh is not the uploaded one "
                        "(coordinates, connectivity or basis)");
    Rule2D R;
    std::memset(&R, 0, sizeof R);
    make_rule2d(BEM_RULE_TRI7, 0, R);
    // one device buffer for a level's inputs and blocks, grown for the largest level
    struct Scratch {
        char *p = nullptr;
        size_t bytes = 0;
        ~Scratch()
        {
            if (p) cudaFree(p);
        }
    } S;
    auto produce = [&](const GreenLevel &L, bool cplx_out, std::vector<double> &out) -> int {
        auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
        const size_t n_cl = L.off.size();
        const size_t parts[9] = {L.row_ptr.size() * 4, L.pt_ptr.size() * 4, L.rows.size() * 4,
                                 L.z.size() * 8,       L.nz.size() * 8,     L.sp.size() * 8,
                                 L.sm.size() * 8,      n_cl * 8,            out.size() * 8};
        const void *src[8] = {L.row_ptr.data(), L.pt_ptr.data(), L.rows.data(), L.z.data(),
                              L.nz.data(),      L.sp.data(),     L.sm.data(),   L.off.data()};
        size_t at[9], need = 0;
        for (int k = 0; k < 9; ++k) {
            at[k] = need;
            need += al(std::max<size_t>(parts[k], 1));
        }
        cudaError_t e = cudaSuccess;
        if (need > S.bytes) {
            if (S.p) cudaFree(S.p);
            S.p = nullptr;
            S.bytes = 0;
            e = cudaMalloc((void **)&S.p, need);
            if (e != cudaSuccess) return api_cuda_fail(ctx, e, "cudaMalloc(GCA level)");
            S.bytes = need;
        }
        for (int k = 0; k < 8 && e == cudaSuccess; ++k)
            if (parts[k] > 0)
                e = cudaMemcpyAsync(S.p + at[k], src[k], parts[k], cudaMemcpyHostToDevice,
                                    ctx->stream);
        if (e != cudaSuccess) return api_cuda_fail(ctx, e, "GCA level upload");
        GreenArgs a;
        a.row_ptr = reinterpret_cast<const int32_t *>(S.p + at[0]);
        a.pt_ptr = reinterpret_cast<const int32_t *>(S.p + at[1]);
        a.row_idx = reinterpret_cast<const int32_t *>(S.p + at[2]);
        a.z = reinterpret_cast<const double *>(S.p + at[3]);
        a.nz = reinterpret_cast<const double *>(S.p + at[4]);
        a.sp = reinterpret_cast<const double *>(S.p + at[5]);
        a.sm = reinterpret_cast<const double *>(S.p + at[6]);
        a.out_off = reinterpret_cast<const int64_t *>(S.p + at[7]);
        a.out = S.p + at[8];
        a.n_row_idx = (int64_t)L.rows.size();
        a.n_points = (int64_t)L.sp.size();
        a.out_len = L.total;
        a.kappa = cplx_out ? kappa : 0.0;
        {
            ProfScope ps(ctx, "green");
            e = cplx_out ? launch_green<true>(mesh->v, a, (int)n_cl, R, ctx->status, ctx->stream)
                         : launch_green<false>(mesh->v, a, (int)n_cl, R, ctx->status, ctx->stream);
        }
        if (e != cudaSuccess) return api_cuda_fail(ctx, e, "green kernel");
        e = cudaMemcpyAsync(out.data(), S.p + at[8], parts[8], cudaMemcpyDeviceToHost, ctx->stream);
        if (e != cudaSuccess) return api_cuda_fail(ctx, e, "GCA level download");
        return bem_sync(ctx);
    };
    return gca_pivots_levels(verts, nv, tris, nt, basis, kappa, cl_ptr, cl_idx, cl_son, n_clusters,
                             gauss_per_face, eps, max_rank, n_threads, produce, piv_ptr, piv_idx,
                             cap);
}
