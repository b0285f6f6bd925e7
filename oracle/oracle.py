"""ctypes wrapper around bem_oracle.c (plain FP64 C, OpenMP over entries).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Parity status of each
function is listed in the C file's header; every public function here is
pinned by the oracle tests (rule exactness, closed-form potentials, Gauss's
identity, symmetry, invariances, convergence).
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bem_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libbem_oracle.so")
_lock = threading.Lock()
_lib = None

CASES = {"regular": 0, "vertex": 1, "edge": 2, "identical": 3}
KERNELS = {"laplace_slp": 0, "laplace_dlp": 1, "helmholtz_slp": 2, "helmholtz_dlp": 3}
BASES = {"p0": 0, "p1": 1}
RULES = {"duffy": 0, "tri7": 1}

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_gauss_legendre01.argtypes = [ctypes.c_int, _d, _d]
            lib.orc_radon7.argtypes = [_d, _d, _d]
            lib.orc_rule_points.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            _d, _d, _d, _d, _d, ctypes.c_int]
            lib.orc_classify.argtypes = [_i32, _i32]
            lib.orc_classify_orders.argtypes = [_i32, _i32, _i32]
            lib.orc_green_entries.argtypes = [_d, ctypes.c_int64, _i32, ctypes.c_int64,
                                              ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                              ctypes.c_int, _i64, _d, _d, ctypes.c_int64,
                                              _d, _d]
            lib.orc_entries.argtypes = [_d, ctypes.c_int64, _i32, ctypes.c_int64,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        _i64, _i64, ctypes.c_int64, _d, _i64, ctypes.c_int]
            lib.orc_entries_absolute.argtypes = [_d, ctypes.c_int64, _i32, ctypes.c_int64,
                                                 ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 _i64, _i64, ctypes.c_int64, _d, ctypes.c_int]
            lib.orc_pair.argtypes = [_d, ctypes.c_int64, _i32, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, _d]
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def gauss_legendre01(q: int):
    x = np.zeros(q)
    w = np.zeros(q)
    if _get().orc_gauss_legendre01(q, _p(x, _d), _p(w, _d)) != 0:
        raise ValueError("bad order")
    return x, w


def radon7():
    s, t, w = np.zeros(7), np.zeros(7), np.zeros(7)
    _get().orc_radon7(_p(s, _d), _p(t, _d), _p(w, _d))
    return s, t, w


def rule_points(case: str, q: int, regular_rule: str = "duffy"):
    """(x1, x2, y1, y2, w) arrays of the 4D rule on D x D for a case."""
    lib = _get()
    n = lib.orc_rule_points(CASES[case], RULES[regular_rule], q, None, None, None, None, None, 0)
    if n < 0:
        raise ValueError("bad rule")
    arrs = [np.zeros(n) for _ in range(5)]
    lib.orc_rule_points(CASES[case], RULES[regular_rule], q, *[_p(a, _d) for a in arrs], n)
    return tuple(arrs)


def classify(ta, tb) -> str:
    a = np.ascontiguousarray(ta, np.int32)
    b = np.ascontiguousarray(tb, np.int32)
    c = _get().orc_classify(_p(a, _i32), _p(b, _i32))
    return {v: k for k, v in CASES.items()}[c]


def classify_orders(ta, tb):
    """(case, a's vertex order, b's vertex order) of a triangle pair."""
    a = np.ascontiguousarray(ta, np.int32)
    b = np.ascontiguousarray(tb, np.int32)
    o = np.zeros(6, np.int32)
    c = _get().orc_classify_orders(_p(a, _i32), _p(b, _i32), _p(o, _i32))
    return {v: k for k, v in CASES.items()}[c], o[:3].copy(), o[3:].copy()


def green_entries(verts, tris, basis, idx, z, nz, kappa=0.0, rule="tri7", q=0):
    """Green quadrature entries (plus, minus), complex arrays: for each k,
    int phi_idx[k] g(x, z_k) dx and int phi_idx[k] d/dn(z_k) g(x, z_k) dx
    (nz_k the unit normal at z_k), with Radon's 7-point rule ("tri7") or a
    Duffy square of q Gauss points per axis ("duffy") on every support
    triangle."""
    v, t = _mesh(verts, tris)
    i = np.ascontiguousarray(idx, np.int64)
    zz = np.ascontiguousarray(z, np.float64).reshape(-1, 3)
    nn = np.ascontiguousarray(nz, np.float64).reshape(-1, 3)
    n = len(i)
    assert zz.shape[0] == n and nn.shape[0] == n
    plus = np.zeros(2 * n)
    minus = np.zeros(2 * n)
    rc = _get().orc_green_entries(_p(v, _d), len(v), _p(t, _i32), len(t), BASES[basis],
                                  float(kappa), RULES[rule], int(q), _p(i, _i64), _p(zz, _d),
                                  _p(nn, _d), n, _p(plus, _d), _p(minus, _d))
    if rc != 0:
        raise ValueError("green_entries: bad index or order")
    return plus[0::2] + 1j * plus[1::2], minus[0::2] + 1j * minus[1::2]


def _mesh(verts, tris):
    v = np.ascontiguousarray(verts, np.float64)
    t = np.ascontiguousarray(tris, np.int32)
    return v, t


def entries(verts, tris, rows, cols, *, kernel="laplace_slp", kappa=0.0, basis="p0",
            trial_basis=None, regular_rule="duffy", q_regular=3, q_identical=5, q_edge=5,
            q_vertex=5, nthreads=0, return_points=False):
    """Complex array of g_ij for the requested (row, col) pairs (Eq. 1)."""
    v, t = _mesh(verts, tris)
    r = np.ascontiguousarray(rows, np.int64).ravel()
    c = np.ascontiguousarray(cols, np.int64).ravel()
    if r.shape != c.shape:
        raise ValueError("rows/cols shape mismatch")
    out = np.zeros(2 * max(len(r), 1))
    npts = np.zeros(1, np.int64)
    tb = basis if trial_basis is None else trial_basis
    rc = _get().orc_entries(_p(v, _d), v.shape[0], _p(t, _i32), t.shape[0], BASES[basis],
                            BASES[tb], KERNELS[kernel], float(kappa), RULES[regular_rule],
                            q_regular, q_identical, q_edge, q_vertex, _p(r, _i64), _p(c, _i64),
                            len(r), _p(out, _d), _p(npts, _i64), int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    z = out[0:2 * len(r):2] + 1j * out[1:2 * len(r):2]
    return (z, int(npts[0])) if return_points else z


def entries_absolute(verts, tris, rows, cols, *, kernel="laplace_slp", kappa=0.0, basis="p0",
                     trial_basis=None, regular_rule="duffy", q_regular=3, q_identical=5, q_edge=5,
                     q_vertex=5, nthreads=0):
    """A_ij: the entries' quadrature sums with every term replaced by its magnitude."""
    v, t = _mesh(verts, tris)
    r = np.ascontiguousarray(rows, np.int64).ravel()
    c = np.ascontiguousarray(cols, np.int64).ravel()
    out = np.zeros(2 * max(len(r), 1))
    tb = basis if trial_basis is None else trial_basis
    rc = _get().orc_entries_absolute(_p(v, _d), v.shape[0], _p(t, _i32), t.shape[0], BASES[basis],
                                     BASES[tb], KERNELS[kernel], float(kappa), RULES[regular_rule],
                                     q_regular, q_identical, q_edge, q_vertex, _p(r, _i64),
                                     _p(c, _i64), len(r), _p(out, _d), int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return out[0:2 * len(r):2].copy()


def pair(verts, tris, a, b, la=-1, lb=-1, *, kernel="laplace_slp", kappa=0.0,
         regular_rule="duffy", q_regular=3, q_identical=5, q_edge=5, q_vertex=5):
    """One triangle-pair integral with local basis functions la, lb (-1 = constant)."""
    v, t = _mesh(verts, tris)
    out = np.zeros(2)
    rc = _get().orc_pair(_p(v, _d), v.shape[0], _p(t, _i32), t.shape[0], a, b, la, lb,
                         KERNELS[kernel], float(kappa), RULES[regular_rule], q_regular,
                         q_identical, q_edge, q_vertex, _p(out, _d))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return complex(out[0], out[1])
