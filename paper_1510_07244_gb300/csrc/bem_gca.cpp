// Green cross approximation (GCA) pivots on the host (Sections 2.3-2.4).
//
// The coupling matrices of the H^2 form are the Galerkin entries at pivot rows
// t~ x pivot columns s~ of every admissible block.  The pivots come from the
// cluster's own geometry alone:
//   * B_t = bounding box of the supports of the cluster's basis functions,
//     delta_t = diam(B_t), and omega_t = B_t grown by delta_t / 2 on every
//     side, so dist(B_t, boundary of omega_t) = delta_t / 2;
//   * a tensor Gauss rule (points z_nu, weights w_nu) on the six faces of
//     omega_t discretises Green's representation formula, which gives
//     A_t = (A_t+, A_t-) with, for i in t,
//         a_{t+, i nu} = sqrt(w_nu)         int phi_i(x) g(x, z_nu) dx
//         a_{t-, i nu} = sqrt(w_nu) delta_t int phi_i(x) d/dn(z_nu) g(x, z_nu) dx
//     (outward face normals; the integrands are smooth because z_nu stays
//     delta_t / 2 away from the supports, so Radon's 7-point rule on each
//     support triangle evaluates them);
//   * cross approximation with complete pivoting on A_t picks the pivot rows
//     t~ (at most max_rank, stopping when the largest remaining entry falls
//     below eps times the first pivot);
//   * nested bases: a cluster with sons runs the same cross approximation on
//     the rows t^ = t~_1 u t~_2 of A_t only, so its pivots are a subset of
//     its sons' pivots.
// g is the kernel's Green function: 1/(4 pi r) (Laplace, kappa = 0) or
// exp(i kappa r)/(4 pi r) (Helmholtz).  Every cluster of one tree level is
// independent, so the levels run bottom-up with the clusters of a level
// spread over host threads; the result does not depend on the thread count.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <functional>
#include <thread>
#include <vector>

#include "bem_internal.h"

namespace {

using cplx = std::complex<double>;
constexpr double kPi = 3.14159265358979323846;

struct HostMesh {
    const double *v;
    const int32_t *t;
    int64_t nv, nt;
    int basis;
    double kappa;
    std::vector<int64_t> vt_ptr;   // triangles around each vertex (P1)
    std::vector<int32_t> vt_tri;
    double S[7], T[7], W[7];       // Radon's 7-point rule on the reference triangle
};

void radon7(HostMesh &M)
{
    const double r = std::sqrt(15.0);
    const double p1 = (6.0 - r) / 21.0, p2 = (6.0 + r) / 21.0;
    const double L[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3},
                            {1 - 2 * p1, p1, p1}, {p1, 1 - 2 * p1, p1}, {p1, p1, 1 - 2 * p1},
                            {1 - 2 * p2, p2, p2}, {p2, 1 - 2 * p2, p2}, {p2, p2, 1 - 2 * p2}};
    const double w1 = (155.0 - r) / 2400.0, w2 = (155.0 + r) / 2400.0;
    const double W[7] = {9.0 / 80.0, w1, w1, w1, w2, w2, w2};
    for (int k = 0; k < 7; ++k) {
        M.S[k] = L[k][1] + L[k][2];
        M.T[k] = L[k][2];
        M.W[k] = W[k];
    }
}

// Points z_nu (with unit normals) of a cluster's box, one array per coordinate.
struct BoxPoints {
    int m = 0;
    std::vector<double> x, y, z, nx, ny, nz;
};

// For one basis function and all m points of a box at once:
//   gp[nu] = int phi_i(x) g(x, z_nu) dx,  gm[nu] = int phi_i(x) d/dn(z_nu) g(x, z_nu) dx.
// The support triangles' rule points and weights are formed once per basis
// function and the innermost loop runs over the points.  Every entry is the
// sum over support triangles, then rule points, with the same operations as
// evaluating one entry at a time.
void basis_integrals(const HostMesh &M, int index, const BoxPoints &Z, cplx *gp, cplx *gm)
{
    const int m = Z.m;
    std::fill(gp, gp + m, cplx(0.0));
    std::fill(gm, gm + m, cplx(0.0));
    std::vector<double> pr, mr;
    if (M.kappa == 0.0) {
        pr.assign(m, 0.0);
        mr.assign(m, 0.0);
    }
    auto tri = [&](int64_t tr, int local) {
        const int32_t *tv = M.t + 3 * tr;
        const double *v0 = M.v + 3 * (int64_t)tv[0], *v1 = M.v + 3 * (int64_t)tv[1],
                     *v2 = M.v + 3 * (int64_t)tv[2];
        double e1[3], e2[3];
        for (int c = 0; c < 3; ++c) {
            e1[c] = v1[c] - v0[c];
            e2[c] = v2[c] - v1[c];
        }
        const double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
                     cz = e1[0] * e2[1] - e1[1] * e2[0];
        const double sg = std::sqrt(cx * cx + cy * cy + cz * cz);
        for (int k = 0; k < 7; ++k) {
            double x[3];
            for (int c = 0; c < 3; ++c) x[c] = v0[c] + M.S[k] * e1[c] + M.T[k] * e2[c];
            const double lam = local < 0 ? 1.0
                                         : (local == 0 ? 1.0 - M.S[k]
                                                       : (local == 1 ? M.S[k] - M.T[k] : M.T[k]));
            const double wk = M.W[k] * sg * lam;
            const double *zx = Z.x.data(), *zy = Z.y.data(), *zz = Z.z.data();
            const double *nx = Z.nx.data(), *ny = Z.ny.data(), *nz = Z.nz.data();
            if (M.kappa == 0.0) {
                double *p = pr.data(), *q = mr.data();
                for (int nu = 0; nu < m; ++nu) {
                    const double d0 = x[0] - zx[nu], d1 = x[1] - zy[nu], d2 = x[2] - zz[nu];
                    const double r = std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                    const double f = wk / (4.0 * kPi * r);
                    // n(z) . grad_z of 1/r with r = |x - z|: (x - z).n / r^2 / r
                    const double dn = (d0 * nx[nu] + d1 * ny[nu] + d2 * nz[nu]) / (r * r);
                    p[nu] += f;
                    q[nu] += f * dn;
                }
            } else {
                for (int nu = 0; nu < m; ++nu) {
                    const double d0 = x[0] - zx[nu], d1 = x[1] - zy[nu], d2 = x[2] - zz[nu];
                    const double r = std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                    const double f = wk / (4.0 * kPi * r);
                    // n(z) . grad_z of exp(i kappa r)/r with r = |x - z|:
                    //   (x - z).n / r^2 * (1 - i kappa r) exp(i kappa r) / r
                    const double dn = (d0 * nx[nu] + d1 * ny[nu] + d2 * nz[nu]) / (r * r);
                    const cplx e = std::polar(1.0, M.kappa * r);
                    gp[nu] += f * e;
                    gm[nu] += f * dn * cplx(1.0, -M.kappa * r) * e;
                }
            }
        }
    };
    if (M.basis == BEM_P0) {
        tri(index, -1);
    } else {
        for (int64_t k = M.vt_ptr[index]; k < M.vt_ptr[index + 1]; ++k) {
            const int64_t tr = M.vt_tri[k];
            const int32_t *tv = M.t + 3 * tr;
            tri(tr, tv[0] == index ? 0 : (tv[1] == index ? 1 : 2));
        }
    }
    if (M.kappa == 0.0)
        for (int nu = 0; nu < m; ++nu) {
            gp[nu] += pr[nu];
            gm[nu] += mr[nu];
        }
}

void grow_box(const HostMesh &M, int index, double *lo, double *hi)
{
    auto add_tri = [&](int64_t tr) {
        for (int k = 0; k < 3; ++k)
            for (int c = 0; c < 3; ++c) {
                const double x = M.v[3 * (int64_t)M.t[3 * tr + k] + c];
                lo[c] = std::min(lo[c], x);
                hi[c] = std::max(hi[c], x);
            }
    };
    if (M.basis == BEM_P0) add_tri(index);
    else
        for (int64_t k = M.vt_ptr[index]; k < M.vt_ptr[index + 1]; ++k) add_tri(M.vt_tri[k]);
}

// Position of the entry of largest magnitude, the first in row-major order
// among equals (bi = -1 if every entry is zero).  Real entries compare by
// fabs.  Complex entries compare by std::abs (hypot); a first pass over the
// squared magnitudes finds the largest, and only entries within a relative
// 1e-12 of it (the hypot maximum is among them: hypot and the square root of
// the squared magnitude differ by a few ulps) are compared by std::abs, in
// the same order, so the choice is the one of a full std::abs scan.
void largest(const std::vector<double> &A, int rows, int cols, int &bi, int &bj, double &best)
{
    bi = bj = -1;
    best = 0.0;
    for (int i = 0; i < rows; ++i)
        for (int j = 0; j < cols; ++j) {
            const double a = std::fabs(A[(size_t)i * cols + j]);
            if (a > best) {
                best = a;
                bi = i;
                bj = j;
            }
        }
}

void largest(const std::vector<cplx> &A, int rows, int cols, int &bi, int &bj, double &best)
{
    const size_t n = (size_t)rows * cols;
    double top = 0.0;
    for (size_t k = 0; k < n; ++k) top = std::max(top, std::norm(A[k]));
    // squared magnitudes that underflow: compare every entry by std::abs
    const double floor = top > 1e-280 ? top * (1.0 - 1e-12) : 0.0;
    bi = bj = -1;
    best = 0.0;
    for (int i = 0; i < rows; ++i)
        for (int j = 0; j < cols; ++j) {
            const cplx &x = A[(size_t)i * cols + j];
            if (std::norm(x) < floor) continue;
            const double a = std::abs(x);
            if (a > best) {
                best = a;
                bi = i;
                bj = j;
            }
        }
}

// Cross approximation with complete pivoting of the rows x cols matrix A
// (row-major, overwritten by its residual); returns the pivot rows in the
// order they were chosen.  T = double for real matrices (kappa = 0), whose
// arithmetic is that of the complex form with zero imaginary parts.
template <class T>
std::vector<int> aca_complete(std::vector<T> &A, int rows, int cols, double eps, int max_rank,
                              std::vector<int> *piv_cols = nullptr)
{
    std::vector<int> piv;
    double first = 0.0;
    std::vector<T> colv(rows), rowv(cols);
    for (int k = 0; k < std::min(max_rank, std::min(rows, cols)); ++k) {
        int bi, bj;
        double best;
        largest(A, rows, cols, bi, bj, best);
        if (bi < 0) break;
        if (k == 0) first = best;
        else if (best <= eps * first) break;
        piv.push_back(bi);
        if (piv_cols) piv_cols->push_back(bj);
        const T p = A[(size_t)bi * cols + bj];
        for (int i = 0; i < rows; ++i) colv[i] = A[(size_t)i * cols + bj] / p;
        for (int j = 0; j < cols; ++j) rowv[j] = A[(size_t)bi * cols + j];
        for (int i = 0; i < rows; ++i) {
            if (colv[i] == 0.0) continue;
            for (int j = 0; j < cols; ++j) A[(size_t)i * cols + j] -= colv[i] * rowv[j];
        }
    }
    return piv;
}

struct Tree {
    const int32_t *ptr, *idx, *son;
};

// The Green problem of cluster c (Section 2.3): its rows (all indices of a
// leaf; otherwise its sons' pivots, first son first), the points z_nu of the
// boundary of omega_t with outward normals and weights w_nu, and delta_t.
// A cluster without rows gets no points.
struct ClusterGreen {
    std::vector<int32_t> rows;
    BoxPoints Z;
    std::vector<double> Wq;
    double delta = 0.0;
};

ClusterGreen cluster_green(const HostMesh &M, const Tree &T, int c,
                           const std::vector<std::vector<int32_t>> &piv,
                           const std::vector<double> &g, const std::vector<double> &gw)
{
    ClusterGreen G;
    std::vector<int32_t> &rows = G.rows;
    const int s0 = T.son[2 * c], s1 = T.son[2 * c + 1];
    if (s0 < 0 && s1 < 0) rows.assign(T.idx + T.ptr[c], T.idx + T.ptr[c + 1]);
    else
        for (int s : {s0, s1})
            if (s >= 0) rows.insert(rows.end(), piv[s].begin(), piv[s].end());
    if (rows.empty()) return G;

    double lo[3] = {HUGE_VAL, HUGE_VAL, HUGE_VAL}, hi[3] = {-HUGE_VAL, -HUGE_VAL, -HUGE_VAL};
    for (int32_t k = T.ptr[c]; k < T.ptr[c + 1]; ++k) grow_box(M, T.idx[k], lo, hi);
    const double delta = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) +
                                   (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                   (hi[2] - lo[2]) * (hi[2] - lo[2]));
    G.delta = delta;
    double wlo[3], whi[3];
    for (int d = 0; d < 3; ++d) {
        wlo[d] = lo[d] - 0.5 * delta;
        whi[d] = hi[d] + 0.5 * delta;
    }
    const int q = (int)g.size();
    BoxPoints &Z = G.Z;
    for (int ax = 0; ax < 3; ++ax)
        for (int side = 0; side < 2; ++side) {
            const int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
            const double len1 = whi[a1] - wlo[a1], len2 = whi[a2] - wlo[a2];
            for (int i = 0; i < q; ++i)
                for (int j = 0; j < q; ++j) {
                    double z[3], n[3] = {0.0, 0.0, 0.0};
                    z[ax] = side ? whi[ax] : wlo[ax];
                    z[a1] = wlo[a1] + g[i] * len1;
                    z[a2] = wlo[a2] + g[j] * len2;
                    n[ax] = side ? 1.0 : -1.0;
                    Z.x.push_back(z[0]);
                    Z.y.push_back(z[1]);
                    Z.z.push_back(z[2]);
                    Z.nx.push_back(n[0]);
                    Z.ny.push_back(n[1]);
                    Z.nz.push_back(n[2]);
                    G.Wq.push_back(gw[i] * gw[j] * len1 * len2);
                }
        }
    Z.m = (int)G.Wq.size();
    return G;
}

// A_t = (A_t+, A_t-) on the host, row-major rows x 2m: sqrt(w_nu) int phi_i g,
// then sqrt(w_nu) delta_t int phi_i dg/dn(z_nu).
void host_green_matrix(const HostMesh &M, const ClusterGreen &G, std::vector<cplx> &A)
{
    const int m = G.Z.m, rn = (int)G.rows.size();
    A.assign((size_t)rn * 2 * m, cplx(0.0));
    std::vector<cplx> gp(m), gm(m);
    for (int i = 0; i < rn; ++i) {
        basis_integrals(M, G.rows[i], G.Z, gp.data(), gm.data());
        for (int nu = 0; nu < m; ++nu) {
            const double sw = std::sqrt(G.Wq[nu]);
            A[(size_t)i * 2 * m + nu] = sw * gp[nu];
            A[(size_t)i * 2 * m + m + nu] = sw * G.delta * gm[nu];
        }
    }
}

// The cluster's pivots (ascending indices) by cross approximation on A_t.
std::vector<int32_t> pivots_of(const HostMesh &M, const ClusterGreen &G, std::vector<cplx> &A,
                               double eps, int max_rank)
{
    const int m = G.Z.m, rn = (int)G.rows.size();
    std::vector<int> chosen;
    if (M.kappa == 0.0) {
        // real matrix: the same values as the real parts of the complex form
        std::vector<double> Ar(A.size());
        for (size_t k = 0; k < A.size(); ++k) Ar[k] = A[k].real();
        chosen = aca_complete(Ar, rn, 2 * m, eps, max_rank);
    } else {
        chosen = aca_complete(A, rn, 2 * m, eps, max_rank);
    }
    std::vector<int32_t> out;
    for (int r : chosen) out.push_back(G.rows[r]);
    std::sort(out.begin(), out.end());
    return out;
}

// The cluster's interpolation matrix (Section 2.3): with the pivot rows t~
// (ascending) and the pivot columns tau that the cross approximation chose,
//     V = (A_t)|rows x tau  ((A_t)|t~ x tau)^-1,
// rows x K row-major (K = |t~|, columns in the order of t~), so that
// A_t ~ V (A_t)|t~ x all and the rows of V at t~ form the identity.  Solved by
// Gaussian elimination with partial pivoting on the K x K system.
struct ClusterBasis {
    std::vector<int32_t> piv;    // ascending
    std::vector<cplx> V;         // rows x K
};

ClusterBasis basis_of(const HostMesh &M, const ClusterGreen &G, std::vector<cplx> &A, double eps,
                      int max_rank)
{
    const int m = G.Z.m, rn = (int)G.rows.size(), cols = 2 * m;
    const std::vector<cplx> A0 = A;
    std::vector<int> chosen, tau;
    if (M.kappa == 0.0) {
        std::vector<double> Ar(A.size());
        for (size_t k = 0; k < A.size(); ++k) Ar[k] = A[k].real();
        chosen = aca_complete(Ar, rn, cols, eps, max_rank, &tau);
    } else {
        chosen = aca_complete(A, rn, cols, eps, max_rank, &tau);
    }
    const int K = (int)chosen.size();
    // pivot rows in ascending index order
    std::vector<int> order(K);
    for (int k = 0; k < K; ++k) order[k] = k;
    std::sort(order.begin(), order.end(),
              [&](int x, int y) { return G.rows[chosen[x]] < G.rows[chosen[y]]; });
    ClusterBasis B;
    for (int k = 0; k < K; ++k) B.piv.push_back(G.rows[chosen[order[k]]]);
    if (K == 0) return B;
    // P[k][l] = A0[row chosen[order[k]], col tau[l]]; V P = C with C = A0[:, tau]
    // <=> P^T V^T = C^T: factor Q = P^T (K x K) once, solve for every row of C
    std::vector<cplx> Q((size_t)K * K);
    for (int k = 0; k < K; ++k)
        for (int l = 0; l < K; ++l) Q[(size_t)l * K + k] = A0[(size_t)chosen[order[k]] * cols + tau[l]];
    std::vector<int> pr(K);
    for (int k = 0; k < K; ++k) pr[k] = k;
    for (int k = 0; k < K; ++k) {
        int best = k;
        for (int i = k + 1; i < K; ++i)
            if (std::abs(Q[(size_t)i * K + k]) > std::abs(Q[(size_t)best * K + k])) best = i;
        if (best != k) {
            for (int j = 0; j < K; ++j) std::swap(Q[(size_t)k * K + j], Q[(size_t)best * K + j]);
            std::swap(pr[k], pr[best]);
        }
        for (int i = k + 1; i < K; ++i) {
            const cplx f = Q[(size_t)i * K + k] / Q[(size_t)k * K + k];
            Q[(size_t)i * K + k] = f;
            for (int j = k + 1; j < K; ++j) Q[(size_t)i * K + j] -= f * Q[(size_t)k * K + j];
        }
    }
    B.V.assign((size_t)rn * K, cplx(0.0));
    std::vector<cplx> b(K);
    for (int r = 0; r < rn; ++r) {
        // right-hand side: row r of C, i.e. A0[r, tau[l]] for l < K, permuted
        for (int k = 0; k < K; ++k) b[k] = A0[(size_t)r * cols + tau[pr[k]]];
        for (int i = 1; i < K; ++i)
            for (int j = 0; j < i; ++j) b[i] -= Q[(size_t)i * K + j] * b[j];
        for (int i = K - 1; i >= 0; --i) {
            for (int j = i + 1; j < K; ++j) b[i] -= Q[(size_t)i * K + j] * b[j];
            b[i] /= Q[(size_t)i * K + i];
        }
        for (int k = 0; k < K; ++k) B.V[(size_t)r * K + k] = b[k];
    }
    return B;
}

// Pivots of cluster c, given its sons' pivots.
std::vector<int32_t> cluster_pivots(const HostMesh &M, const Tree &T, int c,
                                    const std::vector<std::vector<int32_t>> &piv,
                                    const std::vector<double> &g, const std::vector<double> &gw,
                                    double eps, int max_rank)
{
    const ClusterGreen G = cluster_green(M, T, c, piv, g, gw);
    if (G.rows.empty()) return {};
    std::vector<cplx> A;
    host_green_matrix(M, G, A);
    return pivots_of(M, G, A, eps, max_rank);
}

// Runs body(k) for k = 0 .. n-1 on up to nthr threads (the calling one included).
template <class F>
void parallel_for(size_t n, int nthr, F &&body)
{
    std::atomic<size_t> next(0);
    auto work = [&]() {
        for (size_t k; (k = next.fetch_add(1)) < n;) body(k);
    };
    const int t = (int)std::min<size_t>((size_t)std::max(1, nthr), n);
    std::vector<std::thread> pool;
    for (int k = 1; k < t; ++k) pool.emplace_back(work);
    work();
    for (auto &th : pool) th.join();
}

// Checked inputs of a GCA run: the mesh, the tree, every cluster's depth.
struct GcaRun {
    HostMesh M;
    Tree T{nullptr, nullptr, nullptr};
    std::vector<int> depth;
    int max_depth = 0;
    std::vector<double> g, gw;
    int nthr = 1;
};

int gca_setup(const double *verts, int64_t nv, const int32_t *tris, int64_t nt, int32_t basis,
              double kappa, const int32_t *cl_ptr, const int32_t *cl_idx, const int32_t *cl_son,
              int32_t n_clusters, int32_t gauss_per_face, double eps, int32_t max_rank,
              int32_t n_threads, const int32_t *piv_ptr, const int32_t *piv_idx, int64_t cap,
              GcaRun &R)
{
    if (!verts || !tris || nv < 1 || nt < 1 || (basis != BEM_P0 && basis != BEM_P1) ||
        !std::isfinite(kappa) || kappa < 0.0 || !cl_ptr || !cl_idx || !cl_son || n_clusters < 1 ||
        gauss_per_face < 1 || gauss_per_face > 16 || !(eps > 0.0) || max_rank < 1 ||
        n_threads < 0 || !piv_ptr || !piv_idx || cap < 0)
        return BEM_ERR_INVALID_ARG;
    for (int64_t k = 0; k < 3 * nt; ++k)
        if (tris[k] < 0 || tris[k] >= nv) return BEM_ERR_INVALID_ARG;
    for (int64_t k = 0; k < 3 * nv; ++k)
        if (!std::isfinite(verts[k])) return BEM_ERR_INVALID_ARG;
    const int64_t nidx = basis == BEM_P0 ? nt : nv;
    if (cl_ptr[0] != 0) return BEM_ERR_INVALID_ARG;
    for (int c = 0; c < n_clusters; ++c) {
        if (cl_ptr[c + 1] < cl_ptr[c]) return BEM_ERR_INVALID_ARG;
        for (int s = 0; s < 2; ++s)
            if (cl_son[2 * c + s] >= n_clusters || cl_son[2 * c + s] == c ||
                cl_son[2 * c + s] < -1)
                return BEM_ERR_INVALID_ARG;
    }
    for (int64_t k = 0; k < cl_ptr[n_clusters]; ++k)
        if (cl_idx[k] < 0 || cl_idx[k] >= nidx) return BEM_ERR_INVALID_ARG;

    // depth of every cluster; a cluster with two parents or a cycle is an error
    R.depth.assign(n_clusters, -1);
    std::vector<int> parent(n_clusters, -1);
    for (int c = 0; c < n_clusters; ++c)
        for (int s = 0; s < 2; ++s) {
            const int x = cl_son[2 * c + s];
            if (x < 0) continue;
            if (parent[x] >= 0) return BEM_ERR_INVALID_ARG;
            parent[x] = c;
        }
    R.max_depth = 0;
    for (int c = 0; c < n_clusters; ++c) {
        int d = 0, x = c;
        while (parent[x] >= 0) {
            x = parent[x];
            if (++d > n_clusters) return BEM_ERR_INVALID_ARG;
        }
        R.depth[c] = d;
        R.max_depth = std::max(R.max_depth, d);
    }

    HostMesh &M = R.M;
    M.v = verts;
    M.t = tris;
    M.nv = nv;
    M.nt = nt;
    M.basis = basis;
    M.kappa = kappa;
    radon7(M);
    if (basis == BEM_P1) {
        M.vt_ptr.assign(nv + 1, 0);
        M.vt_tri.resize(3 * nt);
        for (int64_t k = 0; k < 3 * nt; ++k) M.vt_ptr[tris[k] + 1]++;
        for (int64_t v = 0; v < nv; ++v) M.vt_ptr[v + 1] += M.vt_ptr[v];
        std::vector<int64_t> fill(M.vt_ptr.begin(), M.vt_ptr.end() - 1);
        for (int64_t t = 0; t < nt; ++t)
            for (int k = 0; k < 3; ++k) M.vt_tri[fill[tris[3 * t + k]]++] = (int32_t)t;
    }
    bem::gauss_legendre_unit(gauss_per_face, R.g, R.gw);
    R.T = Tree{cl_ptr, cl_idx, cl_son};
    R.nthr = n_threads > 0 ? n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
    return BEM_OK;
}

std::vector<int> level_clusters(const GcaRun &R, int d)
{
    std::vector<int> level;
    for (int c = 0; c < (int)R.depth.size(); ++c)
        if (R.depth[c] == d) level.push_back(c);
    return level;
}

int gca_write(const std::vector<std::vector<int32_t>> &piv, int32_t *piv_ptr, int32_t *piv_idx,
              int64_t cap)
{
    int64_t at = 0;
    piv_ptr[0] = 0;
    for (size_t c = 0; c < piv.size(); ++c) {
        if (at + (int64_t)piv[c].size() > cap) return BEM_ERR_INVALID_ARG;
        for (int32_t v : piv[c]) piv_idx[at++] = v;
        piv_ptr[c + 1] = (int32_t)at;
    }
    return BEM_OK;
}

}  // namespace

extern "C" int bem_gca_pivots(const double *verts, int64_t nv, const int32_t *tris, int64_t nt,
                              int32_t basis, double kappa, const int32_t *cl_ptr,
                              const int32_t *cl_idx, const int32_t *cl_son, int32_t n_clusters,
                              int32_t gauss_per_face, double eps, int32_t max_rank,
                              int32_t n_threads, int32_t *piv_ptr, int32_t *piv_idx, int64_t cap)
{
    GcaRun R;
    const int rc = gca_setup(verts, nv, tris, nt, basis, kappa, cl_ptr, cl_idx, cl_son, n_clusters,
                             gauss_per_face, eps, max_rank, n_threads, piv_ptr, piv_idx, cap, R);
    if (rc != BEM_OK) return rc;
    std::vector<std::vector<int32_t>> piv(n_clusters);
    for (int d = R.max_depth; d >= 0; --d) {
        const std::vector<int> level = level_clusters(R, d);
        parallel_for(level.size(), R.nthr, [&](size_t k) {
            piv[level[k]] = cluster_pivots(R.M, R.T, level[k], piv, R.g, R.gw, eps, max_rank);
        });
    }
    return gca_write(piv, piv_ptr, piv_idx, cap);
}

extern "C" int bem_gca_bases(const double *verts, int64_t nv, const int32_t *tris, int64_t nt,
                             int32_t basis, double kappa, const int32_t *cl_ptr,
                             const int32_t *cl_idx, const int32_t *cl_son, int32_t n_clusters,
                             int32_t gauss_per_face, double eps, int32_t max_rank,
                             int32_t n_threads, int32_t *piv_ptr, int32_t *piv_idx, int64_t cap,
                             int64_t *v_off, double *V, int64_t v_cap)
{
    if (!v_off || !V || v_cap < 0) return BEM_ERR_INVALID_ARG;
    GcaRun R;
    const int rc = gca_setup(verts, nv, tris, nt, basis, kappa, cl_ptr, cl_idx, cl_son, n_clusters,
                             gauss_per_face, eps, max_rank, n_threads, piv_ptr, piv_idx, cap, R);
    if (rc != BEM_OK) return rc;
    std::vector<std::vector<int32_t>> piv(n_clusters);
    std::vector<std::vector<cplx>> mats(n_clusters);
    for (int d = R.max_depth; d >= 0; --d) {
        const std::vector<int> level = level_clusters(R, d);
        parallel_for(level.size(), R.nthr, [&](size_t k) {
            const int c = level[k];
            const ClusterGreen G = cluster_green(R.M, R.T, c, piv, R.g, R.gw);
            if (G.rows.empty()) {
                piv[c].clear();
                mats[c].clear();
                return;
            }
            std::vector<cplx> A;
            host_green_matrix(R.M, G, A);
            ClusterBasis B = basis_of(R.M, G, A, eps, max_rank);
            piv[c] = std::move(B.piv);
            mats[c] = std::move(B.V);
        });
    }
    const int w = kappa != 0.0 ? 2 : 1;   // doubles per element
    int64_t at = 0;
    v_off[0] = 0;
    for (int c = 0; c < n_clusters; ++c) {
        if (at + (int64_t)mats[c].size() > v_cap) return BEM_ERR_INVALID_ARG;
        for (size_t k = 0; k < mats[c].size(); ++k) {
            V[w * (at + (int64_t)k)] = mats[c][k].real();
            if (w == 2) V[2 * (at + (int64_t)k) + 1] = mats[c][k].imag();
        }
        at += (int64_t)mats[c].size();
        v_off[c + 1] = at;
    }
    return gca_write(piv, piv_ptr, piv_idx, cap);
}

namespace bem {

int gca_pivots_levels(const double *verts, int64_t nv, const int32_t *tris, int64_t nt,
                      int32_t basis, double kappa, const int32_t *cl_ptr, const int32_t *cl_idx,
                      const int32_t *cl_son, int32_t n_clusters, int32_t gauss_per_face,
                      double eps, int32_t max_rank, int32_t n_threads,
                      const GreenLevelProducer &produce, int32_t *piv_ptr, int32_t *piv_idx,
                      int64_t cap)
{
    GcaRun R;
    int rc = gca_setup(verts, nv, tris, nt, basis, kappa, cl_ptr, cl_idx, cl_son, n_clusters,
                       gauss_per_face, eps, max_rank, n_threads, piv_ptr, piv_idx, cap, R);
    if (rc != BEM_OK) return rc;
    const bool cplx_out = kappa != 0.0;
    std::vector<std::vector<int32_t>> piv(n_clusters);
    for (int d = R.max_depth; d >= 0; --d) {
        const std::vector<int> level = level_clusters(R, d);
        std::vector<ClusterGreen> G(level.size());
        parallel_for(level.size(), R.nthr, [&](size_t k) {
            G[k] = cluster_green(R.M, R.T, level[k], piv, R.g, R.gw);
        });
        // the level in the layout of bem_green_matrices: rows and points per
        // cluster, factors sqrt(w) and sqrt(w) delta_t, one block per cluster
        GreenLevel L;
        L.row_ptr.push_back(0);
        L.pt_ptr.push_back(0);
        for (const ClusterGreen &C : G) {
            L.rows.insert(L.rows.end(), C.rows.begin(), C.rows.end());
            L.row_ptr.push_back((int32_t)L.rows.size());
            for (int nu = 0; nu < C.Z.m; ++nu) {
                L.z.insert(L.z.end(), {C.Z.x[nu], C.Z.y[nu], C.Z.z[nu]});
                L.nz.insert(L.nz.end(), {C.Z.nx[nu], C.Z.ny[nu], C.Z.nz[nu]});
                const double sw = std::sqrt(C.Wq[nu]);
                L.sp.push_back(sw);
                L.sm.push_back(sw * C.delta);
            }
            L.pt_ptr.push_back((int32_t)(L.z.size() / 3));
            L.off.push_back(L.total);
            L.total += 2 * (int64_t)C.rows.size() * C.Z.m;
        }
        std::vector<double> out;
        if (L.total > 0) {
            out.assign((size_t)L.total * (cplx_out ? 2 : 1), 0.0);
            if ((rc = produce(L, cplx_out, out)) != BEM_OK) return rc;
        }
        parallel_for(level.size(), R.nthr, [&](size_t k) {
            const ClusterGreen &C = G[k];
            const int rn = (int)C.rows.size(), m = C.Z.m;
            if (rn == 0) {
                piv[level[k]].clear();
                return;
            }
            // block k: column-major rn x 2m at off[k] -> row-major A_t
            std::vector<cplx> A((size_t)rn * 2 * m);
            for (int col = 0; col < 2 * m; ++col)
                for (int i = 0; i < rn; ++i) {
                    const size_t e = (size_t)L.off[k] + (size_t)i + (size_t)col * rn;
                    A[(size_t)i * 2 * m + col] =
                        cplx_out ? cplx(out[2 * e], out[2 * e + 1]) : cplx(out[e], 0.0);
                }
            piv[level[k]] = pivots_of(R.M, C, A, eps, max_rank);
        });
    }
    return gca_write(piv, piv_ptr, piv_idx, cap);
}

}  // namespace bem
