"""H2-matrix products and the conjugate gradient method, written out from their
definitions (Sections 2.3-2.4 and 4) -- TEST INFRASTRUCTURE ONLY.

Only the tests and the benchmark's CPU legs use this module; the library
shares no code with it.

An H2 matrix (Section 2.4) over a cluster tree is
    G ~ sum over near blocks (t, s)      of  N_ts              on t x s
      + sum over admissible blocks (t, s) of  V_t S_ts V_s^T   on t x s
with the coupling matrix S_ts = G|t~ x s~ (Galerkin entries at the pivots)
and the cluster bases V_t (|t| x |t~|): for a leaf the interpolation matrix
of the cross approximation, for a cluster with sons the nested product
V_t = diag(V_t1, V_t2) V^_t of the sons' bases and the transfer matrix V^_t
whose rows are the sons' pivots.  The functions below form V_t as that
product and add every block's contribution to y = G x directly, with no
forward or backward transformation: the plain definition.
"""
import numpy as np


def full_bases(cl_ptr, cl_idx, cl_son, piv_ptr, mats):
    """{cluster: (indices, V_t)} with V_t = |t| x K_t as the nested product.

    mats[c] is the matrix bem_gca_bases returns for cluster c: rows = the
    cluster's indices (leaf) or its sons' pivots, first son first (else)."""
    nc = len(cl_ptr) - 1
    out = {}

    def build(c):
        if c in out:
            return out[c]
        sons = [s for s in cl_son[c] if s >= 0]
        if not sons:
            out[c] = (np.asarray(cl_idx[cl_ptr[c]:cl_ptr[c + 1]]), np.asarray(mats[c]))
            return out[c]
        # diag(V_s1, V_s2): rows = the sons' indices, columns = the sons' pivots
        parts = [build(s) for s in sons]
        rows = np.concatenate([p[0] for p in parts])
        k_tot = sum(p[1].shape[1] for p in parts)
        D = np.zeros((len(rows), k_tot), dtype=np.result_type(*[p[1] for p in parts], mats[c]))
        r0 = c0 = 0
        for idx_s, V_s in parts:
            D[r0:r0 + V_s.shape[0], c0:c0 + V_s.shape[1]] = V_s
            r0 += V_s.shape[0]
            c0 += V_s.shape[1]
        out[c] = (rows, D @ np.asarray(mats[c]) if k_tot else np.zeros((len(rows), 0)))
        return out[c]

    for c in range(nc):
        build(c)
    return out


def h2_matvec(n, x, near, far, bases, piv_ptr):
    """y = G x for the H2 matrix: near = [(rows, cols, N)] dense blocks; far =
    [(t, s, S)] coupling matrices |t~| x |s~|; bases from full_bases."""
    y = np.zeros(n, dtype=np.result_type(x, *[b[2] for b in near], *[f[2] for f in far]))
    for rows, cols, N in near:
        y[rows] += N @ x[cols]
    for t, s, S in far:
        it, Vt = bases[t]
        is_, Vs = bases[s]
        if Vt.shape[1] == 0 or Vs.shape[1] == 0:
            continue
        y[it] += Vt @ (S @ (Vs.T @ x[is_]))
    return y


def cg(apply, b, tol=1e-10, maxit=1000):
    """The conjugate gradient method (Hestenes-Stiefel) for a symmetric
    positive definite operator: returns (x, iterations, relative residual)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    nb = np.sqrt(float(b @ b))
    it = 0
    while it < maxit and np.sqrt(rr) > tol * nb:
        q = apply(p)
        alpha = rr / float(p @ q)
        x += alpha * p
        r -= alpha * q
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it, np.sqrt(rr) / nb
