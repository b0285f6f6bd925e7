"""Closed-form flat-triangle potentials and a graded outer rule (test helpers).

Independent of the oracle: these formulas come from the divergence theorem on
a flat triangle, not from any quadrature of the singular kernel.  For a point
x and a triangle T with unit normal n, let rho be the projection of x onto
T's plane and w = (x - y).n (y in T).  Per edge e (endpoints P-, P+, unit
direction l_e, outward in-plane normal u_e = l_e x n):
    t0 = (P- - rho).u_e,  l+- = (P+- - rho).l_e,  R0^2 = t0^2 + w^2,
    R+- = |x - P+-|,  L_e = ln((R+ + l+) / (R- + l-)).
Then
    int_T 1/r dA         = sum_e t0 L_e - |w| sum_e [atan(t0 l+/(R0^2+|w|R+))
                                                    - atan(t0 l-/(R0^2+|w|R-))]
    int_T (y-rho)/r dA   = sum_e u_e (1/2)[l+ R+ - l- R- + R0^2 L_e]
    int_T (y-rho)/r^3 dA = -sum_e u_e L_e
    w int_T 1/r^3 dA     = solid angle of T seen from x (signed with w),
                           by the Van Oosterom-Strackee formula.
An affine density lambda(y) = lambda(rho) + grad(lambda).(y - rho) then gives
the piecewise-linear potentials.  The outer integral over the test triangle
uses a Duffy square (s, t) = (sigma, sigma tau) with a sigmoidal grading of
both sigma and tau, so every edge and vertex of the test triangle (where the
potential of a touching triangle is not smooth) sits at a graded end point.
"""
import numpy as np

FOUR_PI = 4.0 * np.pi


def _geom(tri):
    v0, v1, v2 = tri
    n = np.cross(v1 - v0, v2 - v1)
    area2 = np.linalg.norm(n)
    return n / area2, area2


def _log_ratio(Rp, lp, Rm, lm, R02):
    """ln((R+ + l+)/(R- + l-)) without cancellation: since (R + l)(R - l) = R0^2,
    R + l is replaced by R0^2 / (R - l) wherever l < 0."""
    with np.errstate(divide="ignore", invalid="ignore"):
        lnum = np.where(lp >= 0, np.log(Rp + np.abs(lp)), np.log(R02) - np.log(Rp + np.abs(lp)))
        lden = np.where(lm >= 0, np.log(Rm + np.abs(lm)), np.log(R02) - np.log(Rm + np.abs(lm)))
    return lnum - lden


def _edges(tri, n):
    for k in range(3):
        Pm, Pp = tri[k], tri[(k + 1) % 3]
        le = (Pp - Pm) / np.linalg.norm(Pp - Pm)
        ue = np.cross(le, n)
        yield Pm, Pp, le, ue


def potentials(x, tri):
    """For points x (m,3): (S, Gvec, D, Dvec, w, rho) with
    S = int_T 1/r, Gvec = int_T (y-rho)/r, D = w int_T 1/r^3 (solid angle),
    Dvec = int_T (y-rho)/r^3."""
    tri = np.asarray(tri, float)
    n, _ = _geom(tri)
    w = (x - tri[0]) @ n
    rho = x - w[:, None] * n[None, :]
    aw = np.abs(w)
    S = np.zeros(len(x))
    G = np.zeros((len(x), 3))
    Dv = np.zeros((len(x), 3))
    for Pm, Pp, le, ue in _edges(tri, n):
        t0 = (Pm - rho) @ ue
        lp = (Pp - rho) @ le
        lm = (Pm - rho) @ le
        R02 = t0 * t0 + w * w
        Rp = np.linalg.norm(x - Pp, axis=1)
        Rm = np.linalg.norm(x - Pm, axis=1)
        L = _log_ratio(Rp, lp, Rm, lm, R02)
        L = np.where(np.abs(t0) + aw > 0, L, 0.0)
        S += np.where(np.abs(t0) > 0, t0 * L, 0.0)
        with np.errstate(divide="ignore", invalid="ignore"):
            at = np.arctan(t0 * lp / (R02 + aw * Rp)) - np.arctan(t0 * lm / (R02 + aw * Rm))
        S -= aw * np.where(R02 > 0, at, 0.0)
        G += (0.5 * (lp * Rp - lm * Rm + R02 * L))[:, None] * ue[None, :]
        Dv -= L[:, None] * ue[None, :]
    # Van Oosterom-Strackee solid angle, oriented so that it has the sign of w
    R1, R2, R3 = (tri[0] - x), (tri[1] - x), (tri[2] - x)
    r1, r2, r3 = (np.linalg.norm(R, axis=1) for R in (R1, R2, R3))
    num = np.einsum("ij,ij->i", R1, np.cross(R2, R3))
    den = (r1 * r2 * r3 + np.einsum("ij,ij->i", R1, R2) * r3
           + np.einsum("ij,ij->i", R1, R3) * r2 + np.einsum("ij,ij->i", R2, R3) * r1)
    D = -2.0 * np.arctan2(num, den)
    # points in T's own plane: the double-layer integrand (x-y).n / r^3 vanishes
    # identically there (the one-sided solid-angle limit does not apply)
    scale = np.linalg.norm(tri[1] - tri[0])
    inplane = np.abs(w) <= 1e-13 * scale
    D = np.where(inplane, 0.0, D)
    w = np.where(inplane, 0.0, w)
    return S, G, D, Dv, w, rho


def affine_basis(tri, k):
    """(alpha, beta) with lambda_k(y) = alpha + beta.y on T's plane, beta in plane."""
    tri = np.asarray(tri, float)
    n, _ = _geom(tri)
    A = np.zeros((4, 4))
    rhs = np.zeros(4)
    for m in range(3):
        A[m, 0] = 1.0
        A[m, 1:] = tri[m]
        rhs[m] = 1.0 if m == k else 0.0
    A[3, 1:] = n
    sol = np.linalg.solve(A, rhs)
    return sol[0], sol[1:]


def inner(x, tri, kernel, lb=-1):
    """Inner potential int_T k(x, y) psi(y) dy at points x for the Laplace kernels;
    psi = 1 (lb = -1) or the nodal hat function of local vertex lb."""
    S, G, D, Dv, w, rho = potentials(x, tri)
    if lb < 0:
        val_s, val_d = S, D
    else:
        alpha, beta = affine_basis(tri, lb)
        lam_rho = alpha + rho @ beta
        val_s = lam_rho * S + G @ beta
        val_d = lam_rho * D + w * (Dv @ beta)
    if kernel == "laplace_slp":
        return val_s / FOUR_PI
    if kernel == "laplace_dlp":
        # k = (x - y).n_y / (4 pi r^3) = w / (4 pi r^3)
        return val_d / FOUR_PI
    raise ValueError(kernel)


def _sigmoid(z, p):
    a = z ** p
    b = (1.0 - z) ** p
    s = a / (a + b)
    ds = p * (z ** (p - 1) * b + a * (1.0 - z) ** (p - 1)) / (a + b) ** 2
    return s, ds


def outer_rule(tri, n=64, p=5):
    """Points x (m,3) and weights (m,) for int_T f(x) dx, graded to T's boundary."""
    tri = np.asarray(tri, float)
    z, wz = np.polynomial.legendre.leggauss(n)
    z = 0.5 * (z + 1.0)
    wz = 0.5 * wz
    s, ds = _sigmoid(z, p)
    SIG, TAU = np.meshgrid(s, s, indexing="ij")
    W = np.outer(wz * ds, wz * ds) * SIG           # Duffy Jacobian sigma
    S_ref = SIG
    T_ref = SIG * TAU
    v0, v1, v2 = tri
    X = (v0[None, None, :] + S_ref[..., None] * (v1 - v0)[None, None, :]
         + T_ref[..., None] * (v2 - v1)[None, None, :])
    _, area2 = _geom(tri)
    return X.reshape(-1, 3), (W * area2).ravel(), S_ref.ravel(), T_ref.ravel()


def pair_reference(tri_a, tri_b, kernel, la=-1, lb=-1, n=64, p=5):
    """int_{T_a} phi(x) int_{T_b} k(x,y) psi(y) dy dx from the closed forms."""
    X, W, s, t = outer_rule(tri_a, n, p)
    if la < 0:
        fa = 1.0
    else:
        fa = [1.0 - s, s - t, t][la]
    with np.errstate(all="ignore"):
        val = inner(X, tri_b, kernel, lb)
    bad = ~np.isfinite(val)
    # the sigmoidal grading puts a few points within ~1e-17 of a vertex, where the
    # closed forms lose all digits; their weights are far below double precision
    assert np.sum(W[bad]) < 1e-30, "non-finite potential at a point with weight"
    val = np.where(bad, 0.0, val)
    return float(np.sum(W * fa * val))


# ---------------------------------------------------------------------------
# Odd powers of the distance, for the real part of the Helmholtz kernel.
#
# cos(kappa r)/r - 1/r = sum_{k>=1} (-1)^k kappa^(2k) r^(2k-1) / (2k)!, so the
# real part of a Helmholtz single-layer integral minus the Laplace one is a
# series of potentials P_n = int_T r^n dA with odd n >= 1.  With rho' = y - rho
# in T's plane and r^2 = |rho'|^2 + w^2 the divergence theorem gives
#     div(rho' r^n) = (n + 2) r^n - n w^2 r^(n-2)
#  => (n + 2) P_n = n w^2 P_(n-2) + sum_e t0_e E_n(e),
# and grad(r^(n+2)) = (n + 2) r^n rho' gives the first moment
#     int_T rho' r^n dA = sum_e u_e E_(n+2)(e) / (n + 2),
# where the edge integrals E_n = int_e r^n dl (r^2 = R0^2 + l^2 along the edge)
# follow from d/dl (l r^n) = (n + 1) r^n - n R0^2 r^(n-2):
#     E_n = ([l r^n] + n R0^2 E_(n-2)) / (n + 1),  E_(-1) = L_e.
# The recursion starts from the closed forms above (n = -1).
# ---------------------------------------------------------------------------
def odd_power_potentials(x, tri, kmax):
    """For points x (m,3): lists P, V with P[k] = int_T r^(2k-1) dA (m,) and
    V[k] = int_T (y - rho) r^(2k-1) dA (m,3), k = 0..kmax."""
    tri = np.asarray(tri, float)
    n, _ = _geom(tri)
    S, G, _, _, w, rho = potentials(x, tri)
    w2 = w * w
    edges = []
    for Pm, Pp, le, ue in _edges(tri, n):
        t0 = (Pm - rho) @ ue
        lp = (Pp - rho) @ le
        lm = (Pm - rho) @ le
        R02 = t0 * t0 + w2
        Rp = np.linalg.norm(x - Pp, axis=1)
        Rm = np.linalg.norm(x - Pm, axis=1)
        L = np.where(np.abs(t0) + np.abs(w) > 0, _log_ratio(Rp, lp, Rm, lm, R02), 0.0)
        # E[j] = int_e r^(2j-1) dl for j = 0..kmax+1
        E = [L]
        for j in range(1, kmax + 2):
            m_ = 2 * j - 1
            E.append((lp * Rp ** m_ - lm * Rm ** m_ + m_ * R02 * E[-1]) / (m_ + 1))
        edges.append((t0, ue, E))
    P = [S]
    V = [G]
    for k in range(1, kmax + 1):
        m_ = 2 * k - 1
        acc = m_ * w2 * P[-1]
        vec = np.zeros((len(x), 3))
        for t0, ue, E in edges:
            acc = acc + t0 * E[k]
            vec += (E[k + 1] / (m_ + 2))[:, None] * ue[None, :]
        P.append(acc / (m_ + 2))
        V.append(vec)
    return P, V


def helmholtz_real_excess(x, tri, kappa, lb=-1, kmax=24):
    """int_T (cos(kappa r) - 1)/(4 pi r) psi(y) dy at points x, psi = 1 (lb = -1)
    or the hat function of local vertex lb, summed from the odd-power series."""
    P, V = odd_power_potentials(x, tri, kmax)
    if lb < 0:
        lam = np.ones(len(x))
        beta = np.zeros(3)
    else:
        alpha, beta = affine_basis(tri, lb)
        _, _, _, _, _, rho = potentials(x, tri)
        lam = alpha + rho @ beta
    out = np.zeros(len(x))
    coef = 1.0
    for k in range(1, kmax + 1):
        coef *= -kappa * kappa / ((2 * k - 1) * (2 * k))
        out += coef * (lam * P[k] + V[k] @ beta)
    return out / FOUR_PI


def helmholtz_real_excess_pair(tri_a, tri_b, kappa, la=-1, lb=-1, n=64, p=5, kmax=24):
    """int_{T_a} phi(x) int_{T_b} (cos(kappa r) - 1)/(4 pi r) psi(y) dy dx."""
    X, W, s, t = outer_rule(tri_a, n, p)
    fa = 1.0 if la < 0 else [1.0 - s, s - t, t][la]
    with np.errstate(all="ignore"):
        val = helmholtz_real_excess(X, tri_b, kappa, lb, kmax)
    bad = ~np.isfinite(val)
    assert np.sum(W[bad]) < 1e-30, "non-finite potential at a point with weight"
    val = np.where(bad, 0.0, val)
    return float(np.sum(W * fa * val))


def helmholtz_dlp_real_excess(x, tri, kappa, lb=-1, kmax=24):
    """int_T [Re dg_kappa/dn_y - dg_0/dn_y] psi(y) dy at points x.

    The Helmholtz double layer is w (1 - i kappa r) exp(i kappa r)/(4 pi r^3)
    with w = (x - y).n_y, the height of x above T's plane (constant over T).
    Its real part minus the Laplace one is w (cos z + z sin z - 1)/(4 pi r^3),
    z = kappa r, and cos z + z sin z - 1 = sum_{k>=1} (-1)^(k+1) (2k-1)
    z^(2k)/(2k)!, so the excess is w/(4 pi) sum_k c_k kappa^(2k) P_(2k-3)."""
    P, V = odd_power_potentials(x, tri, kmax)
    _, _, _, _, w, rho = potentials(x, tri)
    if lb < 0:
        lam = np.ones(len(x))
        beta = np.zeros(3)
    else:
        alpha, beta = affine_basis(tri, lb)
        lam = alpha + rho @ beta
    out = np.zeros(len(x))
    fact = 1.0                        # (2k)!
    for k in range(1, kmax + 1):
        fact *= (2 * k - 1) * (2 * k)
        c = (-1) ** (k + 1) * (2 * k - 1) * kappa ** (2 * k) / fact
        out += c * (lam * P[k - 1] + V[k - 1] @ beta)
    return w * out / FOUR_PI


def helmholtz_dlp_real_excess_pair(tri_a, tri_b, kappa, la=-1, lb=-1, n=64, p=5, kmax=24):
    X, W, s, t = outer_rule(tri_a, n, p)
    fa = 1.0 if la < 0 else [1.0 - s, s - t, t][la]
    with np.errstate(all="ignore"):
        val = helmholtz_dlp_real_excess(X, tri_b, kappa, lb, kmax)
    bad = ~np.isfinite(val)
    assert np.sum(W[bad]) < 1e-30, "non-finite potential at a point with weight"
    val = np.where(bad, 0.0, val)
    return float(np.sum(W * fa * val))
