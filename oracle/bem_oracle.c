/*
 * bem_oracle.c -- plain FP64 CPU oracle for Galerkin BEM matrix entries.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library calls this file; only the
 * tests, the small smoke check and the benchmark's CPU-baseline leg load it.
 * It shares no source with the CUDA path: its own Gauss-Legendre generator,
 * its own Radon rule, its own Sauter-Schwab subdomain maps, its own pair
 * classification.
 *
 * What it computes (Section 2.1, Eq. 1): for test basis phi_i and trial basis
 * psi_j on a flat-triangle mesh,
 *     g_ij = sum over triangle pairs (T_a in supp phi_i, T_b in supp psi_j) of
 *            sqrt(g_a g_b) * int_D int_D  phi_i(Phi_a(x)) k(Phi_a(x), Phi_b(y))
 *                                         psi_j(Phi_b(y)) dy dx
 * on the reference triangle D = {0 <= t <= s <= 1} with the affine map
 * Phi(s,t) = v0 + s (v1 - v0) + t (v2 - v1) and sqrt(g) = |(v1-v0) x (v2-v1)|
 * (Section 2.2).  Each pair integral is a quadrature approximation:
 *   - disjoint pairs: Duffy map T(s,t) = (s, s t) on both triangles and a
 *     tensor Gauss rule on [0,1]^4 with weight xi1*xi3 (Section 2.2), or the
 *     Radon 7-point degree-5 triangle rule on each triangle;
 *   - identical / common-edge / common-vertex pairs: the Sauter-Schwab idea
 *     (Section 2.2): split D x D into subdomains, map each onto [0,1]^4 so
 *     that the Jacobian cancels the kernel singularity, and apply tensor Gauss.
 *     The paper cites the maps without printing them; the maps below are our
 *     own derivation (6, 4 and 2 subdomains), explained at each function.
 * Kernels (Eq. 2 and Section 4): Laplace single layer 1/(4 pi r), Laplace
 * double layer (x-y).n_y/(4 pi r^3), Helmholtz single layer
 * exp(i kappa r)/(4 pi r), and the Helmholtz double layer of the
 * Brakhage-Werner formulation (Section 4), the normal derivative in y of the
 * Helmholtz kernel: (x-y).n_y (1 - i kappa r) exp(i kappa r)/(4 pi r^3).
 *
 * Everything is evaluated in double precision with plain sums in the nested
 * point order (subdomain, xi, eta1, eta2, eta3).
 *
 * It also computes the entries of the Green quadrature matrices A_t of
 * Section 2.3 (orc_green_entries): integrals of one basis function against
 * the Green function and its normal derivative at a point off the surface,
 * with a triangle rule on each support triangle.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#if defined(_OPENMP)
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

enum { ORC_LAPLACE_SLP = 0, ORC_LAPLACE_DLP = 1, ORC_HELMHOLTZ_SLP = 2, ORC_HELMHOLTZ_DLP = 3 };
enum { ORC_P0 = 0, ORC_P1 = 1 };
enum { ORC_RULE_DUFFY = 0, ORC_RULE_TRI7 = 1 };
enum { ORC_CASE_REGULAR = 0, ORC_CASE_VERTEX = 1, ORC_CASE_EDGE = 2, ORC_CASE_IDENTICAL = 3 };

#define ORC_MAXQ 40

/* ------------------------------------------------------------------------ */
/* 1D Gauss-Legendre on [0,1]: Newton's method on the Legendre polynomial    */
/* P_q evaluated by the three-term recurrence                                */
/*   (n+1) P_{n+1}(x) = (2n+1) x P_n(x) - n P_{n-1}(x).                      */
/* ------------------------------------------------------------------------ */
int orc_gauss_legendre01(int q, double *x, double *w)
{
    if (q < 1 || q > ORC_MAXQ) return -1;
    for (int k = 0; k < q; ++k) {
        double z = cos(ORC_PI * (k + 0.75) / (q + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int n = 1; n < q; ++n) {
                double p2 = ((2.0 * n + 1.0) * z * p1 - n * p0) / (n + 1.0);
                p0 = p1;
                p1 = p2;
            }
            if (q == 1) { p1 = z; p0 = 1.0; }
            /* derivative: P_q'(z) = q (z P_q - P_{q-1}) / (z^2 - 1) */
            dp = q * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int n = 1; n < q; ++n) {
                double p2 = ((2.0 * n + 1.0) * z * p1 - n * p0) / (n + 1.0);
                p0 = p1;
                p1 = p2;
            }
            if (q == 1) { p1 = z; p0 = 1.0; }
            dp = q * (z * p1 - p0) / (z * z - 1.0);
        }
        /* weight on [-1,1]: 2 / ((1 - z^2) P_q'(z)^2); map to [0,1] */
        x[k] = 0.5 * (1.0 - z);
        w[k] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* Radon's 7-point rule of degree 5 on D = {0 <= t <= s <= 1}.  Barycentric
 * points: the centroid and two 3-point orbits (a, a, 1-2a) with
 * a = (6 -+ sqrt 15)/21; normalised weights 9/40 and (155 -+ sqrt 15)/1200.
 * A point with barycentric coordinates (l0, l1, l2) w.r.t. the vertices
 * (0,0), (1,0), (1,1) of D is (s, t) = (l1 + l2, l2).  Weights are scaled by
 * |D| = 1/2. */
int orc_radon7(double *s, double *t, double *w)
{
    const double r15 = sqrt(15.0);
    const double a = (6.0 - r15) / 21.0, b = (6.0 + r15) / 21.0;
    const double wa = (155.0 - r15) / 1200.0, wb = (155.0 + r15) / 1200.0;
    double bary[7][3] = {
        {1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0},
        {a, a, 1.0 - 2.0 * a}, {a, 1.0 - 2.0 * a, a}, {1.0 - 2.0 * a, a, a},
        {b, b, 1.0 - 2.0 * b}, {b, 1.0 - 2.0 * b, b}, {1.0 - 2.0 * b, b, b}};
    double ww[7] = {9.0 / 40.0, wa, wa, wa, wb, wb, wb};
    for (int k = 0; k < 7; ++k) {
        s[k] = bary[k][1] + bary[k][2];
        t[k] = bary[k][2];
        w[k] = 0.5 * ww[k];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 4D rules on D x D.  A rule is a list of points (x1, x2, y1, y2, weight):   */
/* x = (x1, x2) in the test triangle's reference domain, y in the trial's.   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n;
    double *x1, *x2, *y1, *y2, *w;
} orc_rule;

static void rule_alloc(orc_rule *r, int n)
{
    r->n = 0;
    r->x1 = (double *)malloc(sizeof(double) * n);
    r->x2 = (double *)malloc(sizeof(double) * n);
    r->y1 = (double *)malloc(sizeof(double) * n);
    r->y2 = (double *)malloc(sizeof(double) * n);
    r->w = (double *)malloc(sizeof(double) * n);
}

static void rule_free(orc_rule *r)
{
    free(r->x1); free(r->x2); free(r->y1); free(r->y2); free(r->w);
}

static void rule_push(orc_rule *r, double x1, double x2, double y1, double y2, double w)
{
    int k = r->n++;
    r->x1[k] = x1; r->x2[k] = x2; r->y1[k] = y1; r->y2[k] = y2; r->w[k] = w;
}

/* Disjoint pairs, Duffy form (Section 2.2): x = T(xi1, xi2) = (xi1, xi1 xi2),
 * y = T(xi3, xi4), Jacobian xi1 * xi3, tensor Gauss with q points per axis. */
static void rule_duffy(orc_rule *r, int q)
{
    double g[ORC_MAXQ], gw[ORC_MAXQ];
    orc_gauss_legendre01(q, g, gw);
    rule_alloc(r, q * q * q * q);
    for (int a = 0; a < q; ++a)
        for (int b = 0; b < q; ++b)
            for (int c = 0; c < q; ++c)
                for (int d = 0; d < q; ++d) {
                    double xi1 = g[a], xi2 = g[b], xi3 = g[c], xi4 = g[d];
                    rule_push(r, xi1, xi1 * xi2, xi3, xi3 * xi4,
                              gw[a] * gw[b] * gw[c] * gw[d] * xi1 * xi3);
                }
}

/* Disjoint pairs, Radon 7-point rule on each triangle (49 points). */
static void rule_tri7(orc_rule *r)
{
    double s[7], t[7], w[7];
    orc_radon7(s, t, w);
    rule_alloc(r, 49);
    for (int i = 0; i < 7; ++i)
        for (int j = 0; j < 7; ++j)
            rule_push(r, s[i], t[i], s[j], t[j], w[i] * w[j]);
}

/*
 * Singular cases.  Common derivation: by the symmetry of D x D under the swap
 * x <-> y, integrate over the half R+ = {y1 <= x1} and add the same rule with
 * the roles of x and y exchanged.  On R+ scale by x1 = xi:
 *     x = xi (1, a),   y = xi (b, c),   a in [0,1],  0 <= c <= b <= 1,
 * Jacobian xi^3.  Since |x - y| = xi |(1-b, a-c)| (mapped), the factor xi^3
 * removes the singularity at the common corner; what remains is a 3D
 * integral over (a, b, c) whose singular set depends on the case.  Each case
 * splits that 3D domain into pieces whose Duffy-type parametrisation puts the
 * singular set at eta1 = 0 and contributes a factor eta1 (or eta1^2) to the
 * Jacobian.
 */

/* Common vertex at local vertex 0 of both triangles (x = y = 0).  In R+ the
 * singular set is only xi = 0, so (b, c) is parametrised by the Duffy map
 * b = eta2, c = eta2 eta3 (Jacobian eta2):
 *     x = xi (1, eta1),  y = xi eta2 (1, eta3),  J = xi^3 eta2.
 * Two subdomains (R+ and its swap). */
static void rule_vertex(orc_rule *r, int q)
{
    double g[ORC_MAXQ], gw[ORC_MAXQ];
    orc_gauss_legendre01(q, g, gw);
    rule_alloc(r, 2 * q * q * q * q);
    for (int sub = 0; sub < 2; ++sub)
        for (int i0 = 0; i0 < q; ++i0)
            for (int i1 = 0; i1 < q; ++i1)
                for (int i2 = 0; i2 < q; ++i2)
                    for (int i3 = 0; i3 < q; ++i3) {
                        double xi = g[i0], e1 = g[i1], e2 = g[i2], e3 = g[i3];
                        double wt = gw[i0] * gw[i1] * gw[i2] * gw[i3] * xi * xi * xi * e2;
                        double px1 = xi, px2 = xi * e1, py1 = xi * e2, py2 = xi * e2 * e3;
                        if (sub == 0) rule_push(r, px1, px2, py1, py2, wt);
                        else          rule_push(r, py1, py2, px1, px2, wt);
                    }
}

/* Common edge = local edge (v0, v1) of both triangles, traversed in the same
 * direction (x = (s, 0) and y = (s, 0) are the same physical point).  In R+
 * with u = 1 - b the singular set is the single point (a, u, c) = 0 of the
 * prism P = {a in [0,1]} x {u, c >= 0, u + c <= 1}.  P is the union of the
 * two cones from the origin over its faces not containing the origin:
 *   (i)  face a = 1 (a triangle):  (a, u, c) = eta1 (1, eta2 (1-eta3), eta2 eta3),
 *        Jacobian eta1^2 eta2;
 *   (ii) face u + c = 1 (a unit square): (a, u, c) = eta1 (eta2, eta3, 1-eta3),
 *        Jacobian eta1^2.
 * With x = xi (1, a), y = xi (1 - u, c) and J = xi^3 * (cone Jacobian).
 * Four subdomains (two cones, each with its swap). */
static void rule_edge(orc_rule *r, int q)
{
    double g[ORC_MAXQ], gw[ORC_MAXQ];
    orc_gauss_legendre01(q, g, gw);
    rule_alloc(r, 4 * q * q * q * q);
    for (int sub = 0; sub < 4; ++sub)
        for (int i0 = 0; i0 < q; ++i0)
            for (int i1 = 0; i1 < q; ++i1)
                for (int i2 = 0; i2 < q; ++i2)
                    for (int i3 = 0; i3 < q; ++i3) {
                        double xi = g[i0], e1 = g[i1], e2 = g[i2], e3 = g[i3];
                        double w4 = gw[i0] * gw[i1] * gw[i2] * gw[i3];
                        double a, u, c, jac;
                        if (sub / 2 == 0) {
                            a = e1; u = e1 * e2 * (1.0 - e3); c = e1 * e2 * e3;
                            jac = e1 * e1 * e2;
                        } else {
                            a = e1 * e2; u = e1 * e3; c = e1 * (1.0 - e3);
                            jac = e1 * e1;
                        }
                        double wt = w4 * xi * xi * xi * jac;
                        double px1 = xi, px2 = xi * a, py1 = xi * (1.0 - u), py2 = xi * c;
                        if (sub % 2 == 0) rule_push(r, px1, px2, py1, py2, wt);
                        else              rule_push(r, py1, py2, px1, px2, wt);
                    }
}

/* Identical triangles.  In R+ with u = 1 - b and w = a - c the singular set
 * is the line u = w = 0 (a free).  For fixed (u, w) the line coordinate a
 * runs over an interval; the (u, w) domain is the quadrilateral with corners
 * (0,-1), (0,1), (1,1), (1,0), split into three triangles with a vertex at
 * the origin and Duffy-mapped, (u, w) = eta1 (P + eta2 (Q - P)), Jacobian eta1:
 *   A: P = (0,1), Q = (1,1):   u = eta1 eta2,      w = eta1,
 *      a in [w, 1]:            a = eta1 + (1 - eta1) eta3
 *   B: P = (1,1), Q = (1,0):   u = eta1,           w = eta1 eta2,
 *      a in [w, 1 - u + w]:    a = eta1 eta2 + (1 - eta1) eta3
 *   C: P = (1,0), Q = (0,-1):  u = eta1 (1-eta2),  w = -eta1 eta2,
 *      a in [0, 1 - u + w]:    a = (1 - eta1) eta3
 * Every interval has length 1 - eta1, so J = xi^3 eta1 (1 - eta1), and
 * x = xi (1, a), y = xi (1 - u, a - w).  Six subdomains (three pieces, each
 * with its swap). */
static void rule_identical(orc_rule *r, int q)
{
    double g[ORC_MAXQ], gw[ORC_MAXQ];
    orc_gauss_legendre01(q, g, gw);
    rule_alloc(r, 6 * q * q * q * q);
    for (int sub = 0; sub < 6; ++sub)
        for (int i0 = 0; i0 < q; ++i0)
            for (int i1 = 0; i1 < q; ++i1)
                for (int i2 = 0; i2 < q; ++i2)
                    for (int i3 = 0; i3 < q; ++i3) {
                        double xi = g[i0], e1 = g[i1], e2 = g[i2], e3 = g[i3];
                        double w4 = gw[i0] * gw[i1] * gw[i2] * gw[i3];
                        double u, w, a;
                        int piece = sub / 2;
                        if (piece == 0) {
                            u = e1 * e2; w = e1; a = e1 + (1.0 - e1) * e3;
                        } else if (piece == 1) {
                            u = e1; w = e1 * e2; a = e1 * e2 + (1.0 - e1) * e3;
                        } else {
                            u = e1 * (1.0 - e2); w = -e1 * e2; a = (1.0 - e1) * e3;
                        }
                        double wt = w4 * xi * xi * xi * e1 * (1.0 - e1);
                        double px1 = xi, px2 = xi * a, py1 = xi * (1.0 - u), py2 = xi * (a - w);
                        if (sub % 2 == 0) rule_push(r, px1, px2, py1, py2, wt);
                        else              rule_push(r, py1, py2, px1, px2, wt);
                    }
}

/* Build the 4D rule for a case.  Returns the number of points or -1. */
static int make_rule(orc_rule *r, int cas, int regular_rule, int q)
{
    if (q < 1 || q > ORC_MAXQ) return -1;
    switch (cas) {
    case ORC_CASE_REGULAR:
        if (regular_rule == ORC_RULE_TRI7) rule_tri7(r);
        else rule_duffy(r, q);
        break;
    case ORC_CASE_VERTEX: rule_vertex(r, q); break;
    case ORC_CASE_EDGE: rule_edge(r, q); break;
    case ORC_CASE_IDENTICAL: rule_identical(r, q); break;
    default: return -1;
    }
    return r->n;
}

/* Export a rule's points for the rule-exactness tests. */
int orc_rule_points(int cas, int regular_rule, int q, double *x1, double *x2,
                    double *y1, double *y2, double *w, int cap)
{
    orc_rule r;
    int n = make_rule(&r, cas, regular_rule, q);
    if (n < 0) return -1;
    if (n <= cap && x1) {
        memcpy(x1, r.x1, sizeof(double) * n);
        memcpy(x2, r.x2, sizeof(double) * n);
        memcpy(y1, r.y1, sizeof(double) * n);
        memcpy(y2, r.y2, sizeof(double) * n);
        memcpy(w, r.w, sizeof(double) * n);
    }
    rule_free(&r);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Geometry and kernels                                                      */
/* ------------------------------------------------------------------------ */
static void sub3(const double *a, const double *b, double *c)
{
    c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2];
}

static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double norm3(const double *a) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

/* Phi(s,t) = v0 + s (v1 - v0) + t (v2 - v1) */
static void affine_map(const double v[3][3], double s, double t, double *p)
{
    for (int k = 0; k < 3; ++k)
        p[k] = v[0][k] + s * (v[1][k] - v[0][k]) + t * (v[2][k] - v[1][k]);
}

/* Piecewise-linear nodal basis on D: lambda0 = 1 - s, lambda1 = s - t,
 * lambda2 = t (lambda_k = 1 at local vertex k). */
static double lambda_ref(int k, double s, double t)
{
    if (k == 0) return 1.0 - s;
    if (k == 1) return s - t;
    return t;
}

/* Kernel value k(x, y) (real and imaginary part).  ny = unit normal of the
 * trial triangle (used only by the double layer). */
static void kernel_eval(int kind, double kappa, const double *x, const double *y,
                        const double *ny, double *re, double *im)
{
    double d[3];
    sub3(x, y, d);
    double r = norm3(d);
    if (kind == ORC_LAPLACE_SLP) {
        *re = 1.0 / (4.0 * ORC_PI * r);
        *im = 0.0;
    } else if (kind == ORC_LAPLACE_DLP) {
        double dn = d[0] * ny[0] + d[1] * ny[1] + d[2] * ny[2];
        *re = dn / (4.0 * ORC_PI * r * r * r);
        *im = 0.0;
    } else if (kind == ORC_HELMHOLTZ_SLP) {
        *re = cos(kappa * r) / (4.0 * ORC_PI * r);
        *im = sin(kappa * r) / (4.0 * ORC_PI * r);
    } else {
        /* d/dn_y exp(i kappa r)/(4 pi r): dr/dn_y = -(x-y).n_y / r and
         * d/dr [exp(i kappa r)/r] = (i kappa r - 1) exp(i kappa r)/r^2, so the
         * value is (x-y).n_y (1 - i kappa r) exp(i kappa r)/(4 pi r^3) */
        double dn = d[0] * ny[0] + d[1] * ny[1] + d[2] * ny[2];
        double kr = kappa * r, c = cos(kr), sn = sin(kr);
        double f = dn / (4.0 * ORC_PI * r * r * r);
        *re = f * (c + kr * sn);
        *im = f * (sn - kr * c);
    }
}

/* ------------------------------------------------------------------------ */
/* Pair classification (Section 2.2: identical, common edge, common vertex,  */
/* disjoint), by the number of shared vertex indices, and the local vertex   */
/* orders that put the shared vertices where the case's maps expect them.    */
/* ord_a[k] = original local index of a's vertex placed at position k.       */
/* ------------------------------------------------------------------------ */
static int classify(const int32_t *ta, const int32_t *tb, int ord_a[3], int ord_b[3])
{
    int shared = 0, ia[3], ib[3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (ta[i] == tb[j]) { ia[shared] = i; ib[shared] = j; ++shared; }
    for (int k = 0; k < 3; ++k) { ord_a[k] = k; ord_b[k] = k; }
    if (shared == 0) return ORC_CASE_REGULAR;
    if (shared == 3) {
        /* identical: same vertex sequence on both sides (b follows a's order) */
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j)
                if (tb[j] == ta[k]) ord_b[k] = j;
        return ORC_CASE_IDENTICAL;
    }
    if (shared == 2) {
        /* common edge: the two shared vertices first, in the order they have in
         * a (cyclically: start at the shared vertex whose successor in a is
         * the other shared vertex), the third vertex last; b uses the same two
         * shared vertices in the same order. */
        int s0 = ia[0], s1 = ia[1];
        int first, second;
        if ((s0 + 1) % 3 == s1) { first = s0; second = s1; }
        else { first = s1; second = s0; }
        ord_a[0] = first; ord_a[1] = second; ord_a[2] = 3 - first - second;
        int jf = -1, js = -1;
        for (int j = 0; j < 3; ++j) {
            if (tb[j] == ta[first]) jf = j;
            if (tb[j] == ta[second]) js = j;
        }
        ord_b[0] = jf; ord_b[1] = js; ord_b[2] = 3 - jf - js;
        return ORC_CASE_EDGE;
    }
    /* common vertex: the shared vertex first, then the other two in cyclic order */
    ord_a[0] = ia[0]; ord_a[1] = (ia[0] + 1) % 3; ord_a[2] = (ia[0] + 2) % 3;
    ord_b[0] = ib[0]; ord_b[1] = (ib[0] + 1) % 3; ord_b[2] = (ib[0] + 2) % 3;
    return ORC_CASE_VERTEX;
}

/* Case of a triangle pair (exported for tests). */
int orc_classify(const int32_t *ta, const int32_t *tb)
{
    int oa[3], ob[3];
    return classify(ta, tb, oa, ob);
}

/* Case and the local vertex orders of a triangle pair (exported for tests):
 * ord[0..2] = a's order, ord[3..5] = b's. */
int orc_classify_orders(const int32_t *ta, const int32_t *tb, int32_t *ord)
{
    int oa[3], ob[3];
    const int c = classify(ta, tb, oa, ob);
    for (int k = 0; k < 3; ++k) {
        ord[k] = oa[k];
        ord[3 + k] = ob[k];
    }
    return c;
}

/* ------------------------------------------------------------------------ */
/* Mesh with vertex -> triangle adjacency                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    const double *verts;
    int64_t nv;
    const int32_t *tris;
    int64_t nt;
    int64_t *vt_ptr;   /* nv + 1 */
    int32_t *vt_tri;   /* 3 nt   */
} orc_mesh;

static void mesh_init(orc_mesh *m, const double *verts, int64_t nv, const int32_t *tris, int64_t nt)
{
    m->verts = verts; m->nv = nv; m->tris = tris; m->nt = nt;
    m->vt_ptr = (int64_t *)calloc((size_t)nv + 1, sizeof(int64_t));
    m->vt_tri = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * nt + 1));
    for (int64_t t = 0; t < nt; ++t)
        for (int k = 0; k < 3; ++k) m->vt_ptr[tris[3 * t + k] + 1]++;
    for (int64_t v = 0; v < nv; ++v) m->vt_ptr[v + 1] += m->vt_ptr[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nv + 1));
    memcpy(fill, m->vt_ptr, sizeof(int64_t) * (size_t)(nv + 1));
    for (int64_t t = 0; t < nt; ++t)           /* ascending triangle order */
        for (int k = 0; k < 3; ++k) m->vt_tri[fill[tris[3 * t + k]]++] = (int32_t)t;
    free(fill);
}

static void mesh_free(orc_mesh *m) { free(m->vt_ptr); free(m->vt_tri); }

/* ------------------------------------------------------------------------ */
/* One pair integral: sqrt(g_a g_b) * sum_p w_p lamA(x_p) k(Phi_a x_p,      */
/* Phi_b y_p) lamB(y_p), for the given local basis functions.  la / lb are   */
/* the ORIGINAL local vertex indices of the test / trial basis function, or  */
/* -1 for the constant function 1.                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int kernel;
    double kappa;
    int regular_rule;
    int q_regular, q_vertex, q_edge, q_identical;
    orc_rule rules[4];
} orc_setup;

static void pair_integral(const orc_mesh *m, const orc_setup *S, int64_t a, int64_t b,
                          int la, int lb, double *out_re, double *out_im, int64_t *npts,
                          int absolute)
{
    const int32_t *ta = m->tris + 3 * a, *tb = m->tris + 3 * b;
    int oa[3], ob[3];
    int cas = classify(ta, tb, oa, ob);
    const orc_rule *R = &S->rules[cas];

    double va[3][3], vb[3][3];
    for (int k = 0; k < 3; ++k)
        for (int c = 0; c < 3; ++c) {
            va[k][c] = m->verts[3 * (int64_t)ta[oa[k]] + c];
            vb[k][c] = m->verts[3 * (int64_t)tb[ob[k]] + c];
        }
    /* Gram factors sqrt(g) = |(v1 - v0) x (v2 - v1)| (invariant under the
     * reordering) */
    double e1[3], e2[3], cr[3];
    sub3(va[1], va[0], e1); sub3(va[2], va[1], e2); cross3(e1, e2, cr);
    double ga = norm3(cr);
    sub3(vb[1], vb[0], e1); sub3(vb[2], vb[1], e2); cross3(e1, e2, cr);
    double gb = norm3(cr);
    /* outward unit normal of the trial triangle from its ORIGINAL vertex order */
    double nb[3];
    {
        double w0[3], w1[3], w2[3];
        for (int c = 0; c < 3; ++c) {
            w0[c] = m->verts[3 * (int64_t)tb[0] + c];
            w1[c] = m->verts[3 * (int64_t)tb[1] + c];
            w2[c] = m->verts[3 * (int64_t)tb[2] + c];
        }
        sub3(w1, w0, e1); sub3(w2, w1, e2); cross3(e1, e2, nb);
        double nn = norm3(nb);
        nb[0] /= nn; nb[1] /= nn; nb[2] /= nn;
    }
    /* position of the basis functions' vertices in the reordered triangles */
    int pa = -1, pb = -1;
    for (int k = 0; k < 3; ++k) {
        if (oa[k] == la) pa = k;
        if (ob[k] == lb) pb = k;
    }

    double sre = 0.0, sim = 0.0;
    for (int p = 0; p < R->n; ++p) {
        double x[3], y[3], kre, kim;
        affine_map(va, R->x1[p], R->x2[p], x);
        affine_map(vb, R->y1[p], R->y2[p], y);
        kernel_eval(S->kernel, S->kappa, x, y, nb, &kre, &kim);
        double fa = (la < 0) ? 1.0 : lambda_ref(pa, R->x1[p], R->x2[p]);
        double fb = (lb < 0) ? 1.0 : lambda_ref(pb, R->y1[p], R->y2[p]);
        double wf = R->w[p] * fa * fb;
        if (absolute) {
            /* magnitude of the term: the scale of the rounding error of a
             * floating-point evaluation of this sum */
            sre += fabs(wf) * sqrt(kre * kre + kim * kim);
        } else {
            sre += wf * kre;
            sim += wf * kim;
        }
    }
    *out_re = ga * gb * sre;
    *out_im = ga * gb * sim;
    if (npts) *npts += R->n;
}

static int setup_init(orc_setup *S, int kernel, double kappa, int regular_rule, int q_regular,
                      int q_identical, int q_edge, int q_vertex)
{
    memset(S, 0, sizeof(*S));
    if (kernel < ORC_LAPLACE_SLP || kernel > ORC_HELMHOLTZ_DLP) return -1;
    S->kernel = kernel; S->kappa = kappa; S->regular_rule = regular_rule;
    S->q_regular = q_regular; S->q_identical = q_identical;
    S->q_edge = q_edge; S->q_vertex = q_vertex;
    if (make_rule(&S->rules[ORC_CASE_REGULAR], ORC_CASE_REGULAR, regular_rule, q_regular) < 0) return -1;
    if (make_rule(&S->rules[ORC_CASE_VERTEX], ORC_CASE_VERTEX, 0, q_vertex) < 0) return -1;
    if (make_rule(&S->rules[ORC_CASE_EDGE], ORC_CASE_EDGE, 0, q_edge) < 0) return -1;
    if (make_rule(&S->rules[ORC_CASE_IDENTICAL], ORC_CASE_IDENTICAL, 0, q_identical) < 0) return -1;
    return 0;
}

static void setup_free(orc_setup *S)
{
    for (int k = 0; k < 4; ++k) rule_free(&S->rules[k]);
}

/* ------------------------------------------------------------------------ */
/* Matrix entries g_ij (Eq. 1), one at a time.                               */
/*   test_basis / trial_basis: 0 = piecewise constant (index = triangle),    */
/*                             1 = piecewise linear (index = vertex).        */
/*   rows[k], cols[k]: the k-th requested entry.                             */
/*   out[2k], out[2k+1]: real and imaginary part.                            */
/*   npoints (optional): total quadrature points used.                       */
/* Returns 0, or -1 on invalid arguments (index out of range, bad order,     */
/* degenerate triangle).                                                     */
/* ------------------------------------------------------------------------ */
static int entries_impl(const double *verts, int64_t nv, const int32_t *tris, int64_t nt,
                        int test_basis, int trial_basis, int kernel, double kappa,
                        int regular_rule, int q_regular, int q_identical, int q_edge,
                        int q_vertex, const int64_t *rows, const int64_t *cols, int64_t n,
                        double *out, int64_t *npoints, int nthreads, int absolute)
{
    if (nv <= 0 || nt <= 0 || n < 0) return -1;
    if (kernel < 0 || kernel > 3) return -1;
    for (int64_t t = 0; t < 3 * nt; ++t)
        if (tris[t] < 0 || tris[t] >= nv) return -1;
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t *tt = tris + 3 * t;
        double a[3], b[3], c[3], e1[3], e2[3], cr[3];
        for (int k = 0; k < 3; ++k) {
            a[k] = verts[3 * (int64_t)tt[0] + k];
            b[k] = verts[3 * (int64_t)tt[1] + k];
            c[k] = verts[3 * (int64_t)tt[2] + k];
        }
        sub3(b, a, e1); sub3(c, b, e2); cross3(e1, e2, cr);
        if (!(norm3(cr) > 0.0)) return -1;
    }
    int64_t nrow = test_basis == ORC_P0 ? nt : nv, ncol = trial_basis == ORC_P0 ? nt : nv;
    for (int64_t k = 0; k < n; ++k)
        if (rows[k] < 0 || rows[k] >= nrow || cols[k] < 0 || cols[k] >= ncol) return -1;

    orc_setup S;
    if (setup_init(&S, kernel, kappa, regular_rule, q_regular, q_identical, q_edge, q_vertex) < 0) {
        setup_free(&S);
        return -1;
    }
    orc_mesh M;
    mesh_init(&M, verts, nv, tris, nt);
    int64_t total_pts = 0;

#if defined(_OPENMP)
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total_pts)
#endif
    for (int64_t k = 0; k < n; ++k) {
        int64_t i = rows[k], j = cols[k];
        /* supports: P0 -> the triangle itself; P1 -> all triangles at vertex */
        int64_t a_lo, a_hi, b_lo, b_hi;
        int64_t one_a = i, one_b = j;
        const int32_t *alist, *blist;
        int32_t sa = (int32_t)i, sb = (int32_t)j;
        if (test_basis == ORC_P0) { alist = &sa; a_lo = 0; a_hi = 1; }
        else { alist = M.vt_tri; a_lo = M.vt_ptr[i]; a_hi = M.vt_ptr[i + 1]; }
        if (trial_basis == ORC_P0) { blist = &sb; b_lo = 0; b_hi = 1; }
        else { blist = M.vt_tri; b_lo = M.vt_ptr[j]; b_hi = M.vt_ptr[j + 1]; }
        (void)one_a; (void)one_b;
        double sre = 0.0, sim = 0.0;
        int64_t pts = 0;
        for (int64_t ia = a_lo; ia < a_hi; ++ia) {
            int64_t a = alist[ia];
            int la = -1;
            if (test_basis == ORC_P1)
                for (int c = 0; c < 3; ++c) if (M.tris[3 * a + c] == i) la = c;
            for (int64_t ib = b_lo; ib < b_hi; ++ib) {
                int64_t b = blist[ib];
                int lb = -1;
                if (trial_basis == ORC_P1)
                    for (int c = 0; c < 3; ++c) if (M.tris[3 * b + c] == j) lb = c;
                double re, im;
                pair_integral(&M, &S, a, b, la, lb, &re, &im, &pts, absolute);
                sre += re;
                sim += im;
            }
        }
        out[2 * k] = sre;
        out[2 * k + 1] = sim;
        total_pts += pts;
    }
    if (npoints) *npoints = total_pts;
    mesh_free(&M);
    setup_free(&S);
    return 0;
}

int orc_entries(const double *verts, int64_t nv, const int32_t *tris, int64_t nt,
                int test_basis, int trial_basis, int kernel, double kappa,
                int regular_rule, int q_regular, int q_identical, int q_edge, int q_vertex,
                const int64_t *rows, const int64_t *cols, int64_t n, double *out,
                int64_t *npoints, int nthreads)
{
    return entries_impl(verts, nv, tris, nt, test_basis, trial_basis, kernel, kappa,
                        regular_rule, q_regular, q_identical, q_edge, q_vertex, rows, cols, n,
                        out, npoints, nthreads, 0);
}

/* The same sums with every quadrature term replaced by its magnitude:
 * A_ij = sum over pairs sqrt(g_a g_b) sum_p |w_p phi psi k|, the scale of the
 * rounding error of any floating-point evaluation of g_ij with this rule
 * (out[2k] = A, out[2k+1] = 0). */
int orc_entries_absolute(const double *verts, int64_t nv, const int32_t *tris, int64_t nt,
                         int test_basis, int trial_basis, int kernel, double kappa,
                         int regular_rule, int q_regular, int q_identical, int q_edge,
                         int q_vertex, const int64_t *rows, const int64_t *cols, int64_t n,
                         double *out, int nthreads)
{
    return entries_impl(verts, nv, tris, nt, test_basis, trial_basis, kernel, kappa,
                        regular_rule, q_regular, q_identical, q_edge, q_vertex, rows, cols, n,
                        out, NULL, nthreads, 1);
}

/* Triangle-pair integral with explicit local basis functions (for tests):
 * la, lb in {-1, 0, 1, 2} (original local vertex index, -1 = constant 1). */
int orc_pair(const double *verts, int64_t nv, const int32_t *tris, int64_t nt, int64_t a,
             int64_t b, int la, int lb, int kernel, double kappa, int regular_rule,
             int q_regular, int q_identical, int q_edge, int q_vertex, double *out)
{
    if (a < 0 || a >= nt || b < 0 || b >= nt) return -1;
    orc_setup S;
    if (setup_init(&S, kernel, kappa, regular_rule, q_regular, q_identical, q_edge, q_vertex) < 0) {
        setup_free(&S);
        return -1;
    }
    orc_mesh M;
    mesh_init(&M, verts, nv, tris, nt);
    pair_integral(&M, &S, a, b, la, lb, &out[0], &out[1], NULL, 0);
    mesh_free(&M);
    setup_free(&S);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Green quadrature entries (Section 2.3: the matrices A_t of Green's        */
/* representation formula).  For basis function i (P0: triangle i; P1: the  */
/* hat function of vertex i) and a point z with unit normal nz off the      */
/* surface:                                                                  */
/*   plus  = int phi_i(x) g(x, z) dx,                                        */
/*   minus = int phi_i(x) d/dn(z) g(x, z) dx                                 */
/* with g(x, z) = exp(i kappa r)/(4 pi r), r = |x - z| (kappa = 0: Laplace). */
/* The normal derivative is taken in z: grad_z r = (z - x)/r and            */
/* dg/dr = (i kappa r - 1) exp(i kappa r)/(4 pi r^2), so                     */
/*   nz . grad_z g = (x - z).nz (1 - i kappa r) exp(i kappa r)/(4 pi r^3).   */
/* Each support triangle is integrated with a triangle rule on D: Radon's   */
/* 7 points (rule 1) or the Duffy square (s, t) = (xi1, xi1 xi2) with q     */
/* Gauss points per axis and weight xi1 (rule 0), times sqrt(g).  The       */
/* sqrt(w_nu) and delta_t scalings of A_t are left to the caller.  plus and  */
/* minus are complex, interleaved (re, im), one per entry.                   */
/* ------------------------------------------------------------------------ */
int orc_green_entries(const double *verts, int64_t nv, const int32_t *tris, int64_t nt,
                      int basis, double kappa, int rule, int q, const int64_t *idx,
                      const double *z, const double *nz, int64_t n, double *plus, double *minus)
{
    double s[ORC_MAXQ * ORC_MAXQ], t[ORC_MAXQ * ORC_MAXQ], w[ORC_MAXQ * ORC_MAXQ];
    int np = 0;
    if (rule == 1) {
        orc_radon7(s, t, w);
        np = 7;
    } else {
        if (q < 1 || q > ORC_MAXQ) return -1;
        double g[ORC_MAXQ], gw[ORC_MAXQ];
        orc_gauss_legendre01(q, g, gw);
        for (int a = 0; a < q; ++a)
            for (int b = 0; b < q; ++b) {
                s[np] = g[a];
                t[np] = g[a] * g[b];
                w[np] = gw[a] * gw[b] * g[a];
                ++np;
            }
    }
    orc_mesh m;
    mesh_init(&m, verts, nv, tris, nt);
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t e = 0; e < n; ++e) {
        const int64_t i = idx[e];
        double pr = 0.0, pi = 0.0, mr = 0.0, mi = 0.0;
        if ((basis == 0 && (i < 0 || i >= nt)) || (basis == 1 && (i < 0 || i >= nv))) {
            bad = 1;
        } else {
            const int64_t lo = basis == 0 ? i : m.vt_ptr[i];
            const int64_t hi = basis == 0 ? i + 1 : m.vt_ptr[i + 1];
            for (int64_t k = lo; k < hi; ++k) {
                const int64_t T = basis == 0 ? i : m.vt_tri[k];
                double v[3][3], e1[3], e2[3], c[3];
                int loc = -1;
                for (int a = 0; a < 3; ++a) {
                    const int32_t vi = tris[3 * T + a];
                    if (basis == 1 && vi == i) loc = a;
                    for (int d = 0; d < 3; ++d) v[a][d] = verts[3 * (int64_t)vi + d];
                }
                sub3(v[1], v[0], e1);
                sub3(v[2], v[1], e2);
                cross3(e1, e2, c);
                const double sg = norm3(c);
                for (int p = 0; p < np; ++p) {
                    double x[3], d[3];
                    affine_map(v, s[p], t[p], x);
                    sub3(x, &z[3 * e], d);
                    const double r = norm3(d);
                    const double phi = basis == 0 ? 1.0 : lambda_ref(loc, s[p], t[p]);
                    const double f = w[p] * sg * phi / (4.0 * ORC_PI * r);
                    const double dn = (d[0] * nz[3 * e] + d[1] * nz[3 * e + 1] +
                                       d[2] * nz[3 * e + 2]) / (r * r);
                    const double cr = cos(kappa * r), ci = sin(kappa * r);
                    /* plus: f exp(i kappa r); minus: f dn (1 - i kappa r) exp(i kappa r) */
                    pr += f * cr;
                    pi += f * ci;
                    mr += f * dn * (cr + kappa * r * ci);
                    mi += f * dn * (ci - kappa * r * cr);
                }
            }
        }
        plus[2 * e] = pr;
        plus[2 * e + 1] = pi;
        minus[2 * e] = mr;
        minus[2 * e + 1] = mi;
    }
    mesh_free(&m);
    return bad ? -1 : 0;
}
