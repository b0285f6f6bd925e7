// Potentials and a dense complex GMRES solve: the exterior Helmholtz problem
// of Section 4 (Brakhage-Werner formulation) end to end on the device.
//
//   bem_potentials     u(z_k) = sum_j w_j int_{T_j} k(z_k, y) dy for points z_k
//                      off the surface (piecewise-constant density w), with the
//                      library's kernels; one warp per point, the lanes over the
//                      triangles, a Duffy q x q rule per triangle (FP64).
//   bem_dense_gmres    restarted GMRES (Saad and Schultz) for a dense complex
//                      system (A + diag(d)) x = b: Arnoldi with classical
//                      Gram-Schmidt applied twice, Givens rotations on the host.
//                      The matrix-vector product (memory-bound, one thread per
//                      row, column-major A) and the Gram-Schmidt projections
//                      run in kernels; each Arnoldi step reads its projection
//                      coefficients back (a few hundred bytes).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "bem_device.cuh"

namespace bem {

namespace {

struct PotRule {
    int np;
    double s[kMaxNp], t[kMaxNp], w[kMaxNp];
};

template <int KIND>
__global__ void __launch_bounds__(256) k_potentials(MeshView m, const double *__restrict__ z,
                                                    int64_t n_pts, const double2 *__restrict__ w,
                                                    PotRule R, double kappa, double eta,
                                                    double2 *out)
{
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= n_pts) return;
    const double zx = z[3 * p], zy = z[3 * p + 1], zz = z[3 * p + 2];
    double ar = 0.0, ai = 0.0;
    for (int64_t j = lane; j < m.nt; j += 32) {
        Tri B;
        load_tri(m.geom, j, B);
        double e1[3], e2[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            e1[c] = B.v[1][c] - B.v[0][c];
            e2[c] = B.v[2][c] - B.v[1][c];
        }
        double sr = 0.0, si = 0.0;
        for (int k = 0; k < R.np; ++k) {
            const double dx = zx - (B.v[0][0] + R.s[k] * e1[0] + R.t[k] * e2[0]);
            const double dy = zy - (B.v[0][1] + R.s[k] * e1[1] + R.t[k] * e2[1]);
            const double dz = zz - (B.v[0][2] + R.s[k] * e1[2] + R.t[k] * e2[2]);
            double kr, ki;
            kval<KIND>(dx, dy, dz, B.n, kappa, kr, ki, eta);
            sr += R.w[k] * kr;
            si += R.w[k] * ki;
        }
        const double2 wj = w[j];
        const double sc = B.sg * kInv4Pi;
        sr *= sc;
        si *= sc;
        ar += wj.x * sr - wj.y * si;
        ai += wj.x * si + wj.y * sr;
    }
    ar = warp_sum(ar);
    ai = warp_sum(ai);
    if (lane == 0) out[p] = make_double2(ar, ai);
}

// y = (A + diag(d)) x, A column-major n x n complex; one thread per row
__global__ void __launch_bounds__(256) k_zgemv(int64_t n, const double2 *__restrict__ A,
                                               const double2 *__restrict__ d,
                                               const double2 *__restrict__ x, double2 *y)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double ar = 0.0, ai = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        const double2 a = A[i + j * n], v = x[j];
        ar = fma(a.x, v.x, fma(-a.y, v.y, ar));
        ai = fma(a.x, v.y, fma(a.y, v.x, ai));
    }
    if (d) {
        const double2 a = d[i], v = x[i];
        ar += a.x * v.x - a.y * v.y;
        ai += a.x * v.y + a.y * v.x;
    }
    y[i] = make_double2(ar, ai);
}

// h_k = <V_k, w> = sum_i conj(V[i, k]) w_i for k < kk (V column-major n x ld):
// one block per k, fixed reduction order
__global__ void __launch_bounds__(256) k_project(int64_t n, const double2 *__restrict__ V,
                                                 const double2 *__restrict__ w, double2 *h)
{
    __shared__ double sr[256], si[256];
    const int k = blockIdx.x;
    const double2 *v = V + (int64_t)k * n;
    double ar = 0.0, ai = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double2 a = v[i], b = w[i];
        ar = fma(a.x, b.x, fma(a.y, b.y, ar));
        ai = fma(a.x, b.y, fma(-a.y, b.x, ai));
    }
    sr[threadIdx.x] = ar;
    si[threadIdx.x] = ai;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sr[threadIdx.x] += sr[threadIdx.x + o];
            si[threadIdx.x] += si[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) h[k] = make_double2(sr[0], si[0]);
}

// w -= V h (the first kk columns)
__global__ void __launch_bounds__(256) k_subtract(int64_t n, int kk, const double2 *__restrict__ V,
                                                  const double2 *__restrict__ h, double2 *w)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double ar = w[i].x, ai = w[i].y;
    for (int k = 0; k < kk; ++k) {
        const double2 a = V[i + (int64_t)k * n], b = h[k];
        ar -= a.x * b.x - a.y * b.y;
        ai -= a.x * b.y + a.y * b.x;
    }
    w[i] = make_double2(ar, ai);
}

// w = b - w
__global__ void __launch_bounds__(256) k_residual(int64_t n, const double2 *__restrict__ b, double2 *w)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    w[i] = make_double2(b[i].x - w[i].x, b[i].y - w[i].y);
}

// v = s w (complex scale), and x += V y (the first kk columns)
__global__ void __launch_bounds__(256) k_scale(int64_t n, double sr, double si,
                                               const double2 *__restrict__ w, double2 *v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 a = w[i];
    v[i] = make_double2(sr * a.x - si * a.y, sr * a.y + si * a.x);
}

__global__ void __launch_bounds__(256) k_update(int64_t n, int kk, const double2 *__restrict__ V,
                                                const double2 *__restrict__ y, double2 *x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double ar = x[i].x, ai = x[i].y;
    for (int k = 0; k < kk; ++k) {
        const double2 a = V[i + (int64_t)k * n], b = y[k];
        ar += a.x * b.x - a.y * b.y;
        ai += a.x * b.y + a.y * b.x;
    }
    x[i] = make_double2(ar, ai);
}

unsigned grid_of(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

}  // namespace bem

extern "C" {

int bem_potentials(bem_ctx *ctx, int32_t mesh_id, const bem_kernel_desc *kernel, int32_t q,
                   const double *points, int64_t n_points, const double *density, double *out)
{
    using namespace bem;
    if (!ctx) return BEM_ERR_INVALID_ARG;
    auto it = ctx->meshes.find(mesh_id);
    if (it == ctx->meshes.end()) return api_fail(ctx, BEM_ERR_INVALID_ARG, "unknown mesh id");
    const MeshView &m = it->second->v;
    if (m.basis != BEM_P0)
        return api_fail(ctx, BEM_ERR_UNSUPPORTED, "bem_potentials: piecewise-constant densities");
    if (!kernel || kernel->kind < BEM_LAPLACE_SLP || kernel->kind > BEM_HELMHOLTZ_BW ||
        !std::isfinite(kernel->kappa) || !std::isfinite(kernel->eta) || q < 1 || q > 5 ||
        n_points < 0)
        return api_fail(ctx, BEM_ERR_INVALID_ARG, "bem_potentials: bad arguments");
    if (n_points == 0) return BEM_OK;
    if (!points || !density || !out ||
        (reinterpret_cast<uintptr_t>(density) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
        return api_fail(ctx, BEM_ERR_INVALID_ARG,
                        "bem_potentials: null or misaligned pointer (complex arrays: 16 bytes)");
    Rule2D r2;
    if (!make_rule2d(BEM_RULE_DUFFY, q, r2)) return api_fail(ctx, BEM_ERR_INVALID_ARG, "bad order");
    PotRule R;
    R.np = r2.np;
    for (int k = 0; k < r2.np; ++k) {
        R.s[k] = r2.s[k];
        R.t[k] = r2.t[k];
        R.w[k] = r2.w[k];
    }
    const unsigned grid = (unsigned)((n_points * 32 + 255) / 256);
    const double2 *w = reinterpret_cast<const double2 *>(density);
    double2 *o = reinterpret_cast<double2 *>(out);
    const double ka = kernel->kappa, et = kernel->eta;
    cudaStream_t st = ctx->stream;
    switch (kernel->kind) {
    case BEM_LAPLACE_SLP: k_potentials<BEM_LAPLACE_SLP><<<grid, 256, 0, st>>>(m, points, n_points, w, R, ka, et, o); break;
    case BEM_LAPLACE_DLP: k_potentials<BEM_LAPLACE_DLP><<<grid, 256, 0, st>>>(m, points, n_points, w, R, ka, et, o); break;
    case BEM_HELMHOLTZ_SLP: k_potentials<BEM_HELMHOLTZ_SLP><<<grid, 256, 0, st>>>(m, points, n_points, w, R, ka, et, o); break;
    case BEM_HELMHOLTZ_DLP: k_potentials<BEM_HELMHOLTZ_DLP><<<grid, 256, 0, st>>>(m, points, n_points, w, R, ka, et, o); break;
    default: k_potentials<BEM_HELMHOLTZ_BW><<<grid, 256, 0, st>>>(m, points, n_points, w, R, ka, et, o); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "bem_potentials");
    return BEM_OK;
}

int bem_dense_gmres(bem_ctx *ctx, int64_t n, const double *A, const double *diag,
                    const double *b, double *x, double tol, int32_t restart, int32_t maxit,
                    int32_t *iters, double *rel_res)
{
    using namespace bem;
    using cplx = std::complex<double>;
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (n < 1 || !A || !b || !x || b == x || !(tol > 0.0) || restart < 1 || restart > 500 ||
        maxit < 0 || !iters || !rel_res)
        return api_fail(ctx, BEM_ERR_INVALID_ARG, "bem_dense_gmres: bad arguments");
    for (const double *p : {A, diag, b, (const double *)x})
        if (p && (reinterpret_cast<uintptr_t>(p) & 15))
            return api_fail(ctx, BEM_ERR_INVALID_ARG, "bem_dense_gmres: complex arrays must be 16-byte aligned");
    cudaStream_t st = ctx->stream;
    const double2 *dA = reinterpret_cast<const double2 *>(A);
    const double2 *dd = reinterpret_cast<const double2 *>(diag);
    const double2 *db = reinterpret_cast<const double2 *>(b);
    double2 *dx = reinterpret_cast<double2 *>(x);
    const int m = restart;
    double2 *V = nullptr, *w = nullptr, *h = nullptr;
    cudaError_t e = cudaMalloc((void **)&V, sizeof(double2) * (size_t)n * (m + 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&w, sizeof(double2) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h, sizeof(double2) * (size_t)(m + 2));
    auto done = [&](int rc) {
        cudaStreamSynchronize(st);
        cudaFree(V);
        cudaFree(w);
        cudaFree(h);
        return rc;
    };
    if (e != cudaSuccess) return done(api_cuda_fail(ctx, e, "cudaMalloc(gmres)"));
    const unsigned g = grid_of(n);
    // |b|
    auto norm = [&](const double2 *v, double &out) -> cudaError_t {
        k_project<<<1, 256, 0, st>>>(n, v, v, h + m + 1);
        double2 r;
        cudaError_t ee = cudaMemcpyAsync(&r, h + m + 1, sizeof(r), cudaMemcpyDeviceToHost, st);
        if (ee == cudaSuccess) ee = cudaStreamSynchronize(st);
        out = std::sqrt(std::max(r.x, 0.0));
        return ee;
    };
    double bn = 0.0;
    e = cudaMemsetAsync(dx, 0, sizeof(double2) * (size_t)n, st);
    if (e == cudaSuccess) e = norm(db, bn);
    if (e != cudaSuccess) return done(api_cuda_fail(ctx, e, "bem_dense_gmres"));
    int it = 0;
    double res = bn > 0.0 ? 1.0 : 0.0;
    std::vector<cplx> H((size_t)(m + 1) * m), cs(m), sn(m), gvec(m + 1), hk(m + 1);
    while (it < maxit && res > tol && bn > 0.0) {
        // r = b - (A + D) x (into w), beta = |r|, V_0 = r / beta
        k_zgemv<<<g, 256, 0, st>>>(n, dA, dd, dx, w);
        k_residual<<<g, 256, 0, st>>>(n, db, w);
        double beta = 0.0;
        e = norm(w, beta);
        if (e != cudaSuccess) return done(api_cuda_fail(ctx, e, "bem_dense_gmres"));
        res = beta / bn;
        if (res <= tol) break;
        k_scale<<<g, 256, 0, st>>>(n, 1.0 / beta, 0.0, w, V);
        std::fill(gvec.begin(), gvec.end(), cplx(0.0));
        gvec[0] = beta;
        int k = 0;
        for (; k < m && it < maxit; ++k, ++it) {
            k_zgemv<<<g, 256, 0, st>>>(n, dA, dd, V + (size_t)k * n, w);
            // classical Gram-Schmidt, twice
            std::fill(hk.begin(), hk.end(), cplx(0.0));
            for (int pass = 0; pass < 2; ++pass) {
                k_project<<<k + 1, 256, 0, st>>>(n, V, w, h);
                k_subtract<<<g, 256, 0, st>>>(n, k + 1, V, h, w);
                std::vector<double2> hh(k + 1);
                e = cudaMemcpyAsync(hh.data(), h, sizeof(double2) * (size_t)(k + 1),
                                    cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) return done(api_cuda_fail(ctx, e, "bem_dense_gmres"));
                for (int i = 0; i <= k; ++i) hk[i] += cplx(hh[i].x, hh[i].y);
            }
            double hn = 0.0;
            if ((e = norm(w, hn)) != cudaSuccess) return done(api_cuda_fail(ctx, e, "bem_dense_gmres"));
            hk[k + 1] = hn;
            if (hn > 0.0) k_scale<<<g, 256, 0, st>>>(n, 1.0 / hn, 0.0, w, V + (size_t)(k + 1) * n);
            // apply the previous rotations, then a new one that zeroes hk[k + 1]
            for (int i = 0; i < k; ++i) {
                const cplx t = std::conj(cs[i]) * hk[i] + std::conj(sn[i]) * hk[i + 1];
                hk[i + 1] = -sn[i] * hk[i] + cs[i] * hk[i + 1];
                hk[i] = t;
            }
            const double a = std::abs(hk[k]), bb = std::abs(hk[k + 1]);
            const double r = std::hypot(a, bb);
            if (r == 0.0) {
                cs[k] = 1.0;
                sn[k] = 0.0;
            } else {
                cs[k] = hk[k] / r;
                sn[k] = hk[k + 1] / r;
            }
            hk[k] = r;
            hk[k + 1] = 0.0;
            gvec[k + 1] = -sn[k] * gvec[k];
            gvec[k] = std::conj(cs[k]) * gvec[k];
            for (int i = 0; i <= k; ++i) H[(size_t)i * m + k] = hk[i];
            res = std::abs(gvec[k + 1]) / bn;
            if (res <= tol || hn == 0.0) {
                ++k;
                ++it;
                break;
            }
        }
        // y = H^-1 g (upper triangular k x k), x += V y
        std::vector<cplx> y(k);
        for (int i = k - 1; i >= 0; --i) {
            cplx s = gvec[i];
            for (int j = i + 1; j < k; ++j) s -= H[(size_t)i * m + j] * y[j];
            y[i] = s / H[(size_t)i * m + i];
        }
        std::vector<double2> yd(k);
        for (int i = 0; i < k; ++i) yd[i] = make_double2(y[i].real(), y[i].imag());
        e = cudaMemcpyAsync(h, yd.data(), sizeof(double2) * (size_t)k, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            k_update<<<g, 256, 0, st>>>(n, k, V, h, dx);
            e = cudaStreamSynchronize(st);   // h is reused by the next cycle
        }
        if (e != cudaSuccess) return done(api_cuda_fail(ctx, e, "bem_dense_gmres"));
    }
    *iters = it;
    *rel_res = res;
    return done(BEM_OK);
}

}  // extern "C"
