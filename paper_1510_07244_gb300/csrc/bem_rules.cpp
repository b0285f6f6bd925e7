// Quadrature rules of the library (host side; uploaded once per context).
//
//  * Gauss-Legendre on [0,1]: Newton iteration in long double on P_q with a
//    Tricomi-type initial guess for each root.
//  * Regular (disjoint) pairs (Section 2.2): the Duffy map T(s,t) = (s, s t)
//    on each triangle turns D into [0,1]^2 with Jacobian s, so the 4D rule
//    is the product of two copies of a 2D triangle rule (q^2 points); the
//    alternative 2D rule is Radon's 7-point degree-5 formula.
//  * Touching pairs (Section 2.2, Sauter-Schwab): [0,1]^4 rules obtained by
//    splitting D x D into subdomains on which a Duffy-type map collapses the
//    singular set.  Our own derivation, with R+ = {y1 <= x1} and the
//    scaling x1 = xi (x = xi (1, a), y = xi (b, c), Jacobian xi^3):
//      common vertex (shared vertex = local vertex 0 of both triangles):
//        b = eta2, c = eta2 eta3                      J = xi^3 eta2
//      common edge (shared edge = local edge v0 -> v1 of both), u = 1 - b:
//        cone over {a = 1}:    (a,u,c) = eta1 (1, eta2 (1-eta3), eta2 eta3),
//                                                    J = xi^3 eta1^2 eta2
//        cone over {u + c = 1}: (a,u,c) = eta1 (eta2, eta3, 1-eta3),
//                                                    J = xi^3 eta1^2
//      identical (u = 1 - b, w = a - c; three Duffy triangles of the (u,w)
//        quadrilateral around the singular line u = w = 0):
//        (u, w) = eta1 (eta2, 1),         a = eta1 + (1-eta1) eta3
//        (u, w) = eta1 (1, eta2),         a = eta1 eta2 + (1-eta1) eta3
//        (u, w) = eta1 (1-eta2, -eta2),   a = (1-eta1) eta3
//                                                    J = xi^3 eta1 (1-eta1)
//    Every piece is used as is and with x and y exchanged (R- = swap of R+):
//    2, 4 and 6 subdomains with q^4 points each.
//  * In every piece x1, x2, y1, y2 and the differences are xi times a function
//    of (eta1, eta2, eta3), and the weight is xi^3 times one.  For the Laplace
//    kernels on flat triangles the integrand is then a monomial in xi times a
//    function of eta (r = xi |u(eta)|, heights xi h(eta), the hats' arguments
//    xi times ...), so a Gauss rule in xi that is exact for that degree sums
//    to the monomial's integral 1 / (n + 1): the same rule with xi integrated
//    out has q^3 points per subdomain, taken at xi = 1 with weight
//    J(eta) w(eta) (xi_moment gives the factor of each moment).
#include <cmath>
#include <functional>
#include <vector>

#include "bem_internal.h"

namespace bem {

const int kPerm[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {1, 0, 2}, {2, 1, 0}};

bool gauss_legendre_unit(int q, std::vector<double> &x, std::vector<double> &w)
{
    if (q < 1 || q > 64) return false;
    x.assign(q, 0.0);
    w.assign(q, 0.0);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int i = 1; i <= q; ++i) {
        // Tricomi: theta = pi (4i - 1) / (4q + 2), z ~ (1 - (q-1)/(8 q^3)) cos theta
        long double th = pi * (4.0L * i - 1.0L) / (4.0L * q + 2.0L);
        long double z = (1.0L - (q - 1.0L) / (8.0L * q * q * q)) * std::cos(th);
        long double pq = 0, pqm1 = 0;
        for (int it = 0; it < 60; ++it) {
            long double a = 1.0L, b = z;      // P_0, P_1
            if (q == 1) { pq = z; pqm1 = 1.0L; }
            else {
                for (int k = 2; k <= q; ++k) {
                    long double c = ((2.0L * k - 1.0L) * z * b - (k - 1.0L) * a) / k;
                    a = b;
                    b = c;
                }
                pq = b;
                pqm1 = a;
            }
            long double dp = q * (pqm1 - z * pq) / (1.0L - z * z);
            long double step = pq / dp;
            z -= step;
            if (std::fabs((double)step) < 1e-19) break;
        }
        long double a = 1.0L, b = z;
        if (q == 1) { pq = z; pqm1 = 1.0L; }
        else {
            for (int k = 2; k <= q; ++k) {
                long double c = ((2.0L * k - 1.0L) * z * b - (k - 1.0L) * a) / k;
                a = b;
                b = c;
            }
            pq = b;
            pqm1 = a;
        }
        long double dp = q * (pqm1 - z * pq) / (1.0L - z * z);
        // roots come out in descending z; store ascending on [0,1]
        x[i - 1] = (double)((1.0L - z) / 2.0L);
        w[i - 1] = (double)(1.0L / ((1.0L - z * z) * dp * dp));
    }
    return true;
}

static void round_rule(Rule2D &r)
{
    for (int k = 0; k < r.np; ++k) {
        r.sf[k] = (float)r.s[k];
        r.tf[k] = (float)r.t[k];
        r.wf[k] = (float)r.w[k];
        r.wl[0][k] = (float)(r.w[k] * (1.0 - r.s[k]));
        r.wl[1][k] = (float)(r.w[k] * (r.s[k] - r.t[k]));
        r.wl[2][k] = (float)(r.w[k] * r.t[k]);
    }
}

bool make_rule2d(int regular_rule, int q, Rule2D &out)
{
    if (regular_rule == BEM_RULE_TRI7) {
        const double r = std::sqrt(15.0);
        const double p1 = (6.0 - r) / 21.0, p2 = (6.0 + r) / 21.0;
        const double w0 = 9.0 / 80.0;                 // 9/40 * |D|
        const double w1 = (155.0 - r) / 2400.0, w2 = (155.0 + r) / 2400.0;
        // barycentric (l0, l1, l2) -> (s, t) = (l1 + l2, l2)
        const double L[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3},
                                {1 - 2 * p1, p1, p1}, {p1, 1 - 2 * p1, p1}, {p1, p1, 1 - 2 * p1},
                                {1 - 2 * p2, p2, p2}, {p2, 1 - 2 * p2, p2}, {p2, p2, 1 - 2 * p2}};
        const double W[7] = {w0, w1, w1, w1, w2, w2, w2};
        out.np = 7;
        for (int k = 0; k < 7; ++k) {
            out.s[k] = L[k][1] + L[k][2];
            out.t[k] = L[k][2];
            out.w[k] = W[k];
        }
        round_rule(out);
        return true;
    }
    if (regular_rule != BEM_RULE_DUFFY || q < 1 || q * q > kMaxNp) return false;
    std::vector<double> g, gw;
    gauss_legendre_unit(q, g, gw);
    out.np = q * q;
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) {
            out.s[i * q + j] = g[i];
            out.t[i * q + j] = g[i] * g[j];
            out.w[i * q + j] = gw[i] * gw[j] * g[i];
        }
    round_rule(out);
    return true;
}

bool make_xi_rule(int q, XiRule &out)
{
    std::vector<double> g, gw;
    if (q < 1 || q > 2 * kMaxXiPairs || !gauss_legendre_unit(q, g, gw)) return false;
    out = XiRule();
    // nodes ascend: g[k] = 1/2 - t, g[q-1-k] = 1/2 + t with equal weights
    for (int k = 0; k < q / 2; ++k) {
        const double a = g[q - 1 - k], b = g[k];
        const double w = 0.5 * (gw[k] + gw[q - 1 - k]);
        out.t[k] = (float)(a - 0.5);
        for (int m = 0; m < 3; ++m) {
            const double pa = std::pow(a, 2 + m), pb = std::pow(b, 2 + m);
            out.cp[k][m] = (float)(w * (pa + pb));
            out.cm[k][m] = (float)(w * (pa - pb));
        }
    }
    out.npair = q / 2;
    if (q % 2)
        for (int m = 0; m < 3; ++m) out.cmid[m] = (float)(gw[q / 2] * std::pow(0.5, 2 + m));
    return true;
}

namespace {

struct Pt {
    double x1, x2, y1, y2, w;
    double d1, d2;   // x1 - y1, x2 - y2 formed from the map's own factors
};

// One piece of R+: maps (xi, e1, e2, e3) to (x, y) and its Jacobian.
using Piece = std::function<Pt(double, double, double, double)>;

std::vector<Piece> pieces(int cas)
{
    std::vector<Piece> P;
    if (cas == kVertex) {
        P.push_back([](double xi, double e1, double e2, double e3) {
            return Pt{xi, xi * e1, xi * e2, xi * e2 * e3, xi * xi * xi * e2,
                      xi * (1.0 - e2), xi * (e1 - e2 * e3)};
        });
    } else if (cas == kEdge) {
        P.push_back([](double xi, double e1, double e2, double e3) {
            double a = e1, u = e1 * e2 * (1.0 - e3), c = e1 * e2 * e3;
            return Pt{xi, xi * a, xi * (1.0 - u), xi * c, xi * xi * xi * e1 * e1 * e2,
                      xi * u, xi * (a - c)};
        });
        P.push_back([](double xi, double e1, double e2, double e3) {
            double a = e1 * e2, u = e1 * e3, c = e1 * (1.0 - e3);
            return Pt{xi, xi * a, xi * (1.0 - u), xi * c, xi * xi * xi * e1 * e1,
                      xi * u, xi * (a - c)};
        });
    } else if (cas == kIdentical) {
        auto mk = [](double u, double w, double a, double xi, double e1) {
            return Pt{xi, xi * a, xi * (1.0 - u), xi * (a - w), xi * xi * xi * e1 * (1.0 - e1),
                      xi * u, xi * w};
        };
        P.push_back([mk](double xi, double e1, double e2, double e3) {
            return mk(e1 * e2, e1, e1 + (1.0 - e1) * e3, xi, e1);
        });
        P.push_back([mk](double xi, double e1, double e2, double e3) {
            return mk(e1, e1 * e2, e1 * e2 + (1.0 - e1) * e3, xi, e1);
        });
        P.push_back([mk](double xi, double e1, double e2, double e3) {
            return mk(e1 * (1.0 - e2), -e1 * e2, (1.0 - e1) * e3, xi, e1);
        });
    }
    return P;
}

}  // namespace

bool make_rule4d_host(int cas, int regular_rule, int q, std::vector<double> &soa, bool xi_out)
{
    if (xi_out && cas == kRegular) return false;
    std::vector<Pt> pts;
    if (cas == kRegular) {
        // 2D rule on D (any Duffy order here; the block engine's Rule2D holds <= 25 points)
        std::vector<double> S, T, W;
        if (regular_rule == BEM_RULE_TRI7) {
            Rule2D r;
            make_rule2d(BEM_RULE_TRI7, 1, r);
            S.assign(r.s, r.s + r.np);
            T.assign(r.t, r.t + r.np);
            W.assign(r.w, r.w + r.np);
        } else {
            std::vector<double> g, gw;
            if (regular_rule != BEM_RULE_DUFFY || !gauss_legendre_unit(q, g, gw)) return false;
            for (int i = 0; i < q; ++i)
                for (int j = 0; j < q; ++j) {
                    S.push_back(g[i]);
                    T.push_back(g[i] * g[j]);
                    W.push_back(gw[i] * gw[j] * g[i]);
                }
        }
        for (size_t i = 0; i < S.size(); ++i)
            for (size_t j = 0; j < S.size(); ++j)
                pts.push_back(Pt{S[i], T[i], S[j], T[j], W[i] * W[j], S[i] - S[j], T[i] - T[j]});
    } else {
        std::vector<double> g, gw;
        if (!gauss_legendre_unit(q, g, gw)) return false;
        // xi integrated out: one node xi = 1 with weight 1
        const int nxi = xi_out ? 1 : q;
        for (const Piece &f : pieces(cas))
            for (int swap = 0; swap < 2; ++swap)
                for (int i = 0; i < nxi; ++i)
                    for (int j = 0; j < q; ++j)
                        for (int k = 0; k < q; ++k)
                            for (int l = 0; l < q; ++l) {
                                Pt p = f(xi_out ? 1.0 : g[i], g[j], g[k], g[l]);
                                p.w *= (xi_out ? 1.0 : gw[i]) * gw[j] * gw[k] * gw[l];
                                if (swap) {
                                    std::swap(p.x1, p.y1);
                                    std::swap(p.x2, p.y2);
                                    p.d1 = -p.d1;
                                    p.d2 = -p.d2;
                                }
                                pts.push_back(p);
                            }
    }
    const size_t n = pts.size();
    soa.assign(kRuleCols * n, 0.0);
    for (size_t k = 0; k < n; ++k) {
        soa[k] = pts[k].x1;
        soa[n + k] = pts[k].x2;
        soa[2 * n + k] = pts[k].y1;
        soa[3 * n + k] = pts[k].y2;
        soa[4 * n + k] = pts[k].w;
        soa[5 * n + k] = pts[k].d1;
        soa[6 * n + k] = pts[k].d2;
    }
    return true;
}

}  // namespace bem
