"""ctypes binding of libbem_gb300.so (the C ABI in include/bem.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device buffers are torch CUDA tensors (int32 index lists, float64
or complex128 outputs); the stream is torch's current stream unless given.
If the shared library is missing this module raises instead of computing
anything another way.
"""
import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libbem_gb300.so")

BEM_OK = 0
ERRORS = {-1: "BEM_ERR_INVALID_ARG", -2: "BEM_ERR_CUDA", -3: "BEM_ERR_OOM",
          -4: "BEM_ERR_TIMEOUT", -5: "BEM_ERR_DEGENERATE", -6: "BEM_ERR_UNSUPPORTED"}
KERNELS = {"laplace_slp": 0, "laplace_dlp": 1, "helmholtz_slp": 2, "helmholtz_dlp": 3,
           "helmholtz_bw": 4}
COMPLEX_KERNELS = ("helmholtz_slp", "helmholtz_dlp", "helmholtz_bw")
_COMPLEX_IDS = tuple(KERNELS[k] for k in COMPLEX_KERNELS)
BASES = {"p0": 0, "p1": 1}
RULES = {"duffy": 0, "tri7": 1}
PRECISIONS = {"fp64": 0, "mixed": 1, "mixed_full": 2}
ORDER_MODES = {"fixed": 0, "learned": 1}
EXPORTS = ["bem_create", "bem_destroy", "bem_last_error", "bem_sync", "bem_mesh_upload",
           "bem_mesh_free", "bem_mesh_info", "bem_near_field", "bem_coupling_blocks",
           "bem_pivot_entries", "bem_assemble_dense", "bem_profile_enable",
           "bem_profile_reset", "bem_profile_read", "bem_near_field_noalloc", "bem_rule_points",
           "bem_plan_create", "bem_plan_run", "bem_plan_destroy", "bem_plan_info",
           "bem_pivot_entries_absolute", "bem_mlp_create", "bem_mlp_destroy", "bem_mlp_num_params",
           "bem_mlp_set_params", "bem_mlp_get_params", "bem_mlp_gradients", "bem_mlp_train_step",
           "bem_mlp_infer", "bem_pair_features", "bem_set_order_model", "bem_learned_counts",
           "bem_shard_blocks", "bem_gca_pivots", "bem_touching_pairs", "bem_green_matrices",
           "bem_gca_pivots_device", "bem_plan_guard_stats", "bem_peak_probe", "bem_gca_bases", "bem_h2_create", "bem_h2_matvec",
           "bem_h2_cg", "bem_h2_destroy", "bem_plan_learned_counts", "bem_mlp_fit_norm",
           "bem_mlp_train_epoch", "bem_order_labels", "bem_potentials", "bem_dense_gmres",
           "bem_rule_points_xi"]
ORDER_CLASSES = [("duffy", 2), ("tri7", 1), ("duffy", 4), ("duffy", 5), ("duffy", 6), ("duffy", 8)]
ORDER_CLASS_POINTS = [16, 49, 256, 625, 1296, 4096]
PLAN_GRAPH, PLAN_AUTOTUNE, PLAN_PROFILE, PLAN_STATIC_LISTS = 1, 2, 4, 8


class BemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class bem_kernel_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("kappa", ctypes.c_double), ("eta", ctypes.c_double)]


class bem_quad_desc(ctypes.Structure):
    _fields_ = [("q_regular", ctypes.c_int32), ("regular_rule", ctypes.c_int32),
                ("q_identical", ctypes.c_int32), ("q_edge", ctypes.c_int32),
                ("q_vertex", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("order_mode", ctypes.c_int32)]


_vp = ctypes.c_void_p


class bem_block_job(ctypes.Structure):
    _fields_ = [("mesh_id", ctypes.c_int32), ("kernel", bem_kernel_desc),
                ("quad", bem_quad_desc),
                ("row_ptr", _vp), ("row_idx", _vp), ("n_row_clusters", ctypes.c_int32),
                ("col_ptr", _vp), ("col_idx", _vp), ("n_col_clusters", ctypes.c_int32),
                ("blk_row", _vp), ("blk_col", _vp), ("blk_off", _vp),
                ("n_blocks", ctypes.c_int64), ("out", _vp)]


class bem_green_job(ctypes.Structure):
    _fields_ = [("mesh_id", ctypes.c_int32), ("kernel", bem_kernel_desc),
                ("rule", ctypes.c_int32), ("q", ctypes.c_int32), ("n_clusters", ctypes.c_int32),
                ("row_ptr", _vp), ("row_idx", _vp), ("n_row_idx", ctypes.c_int64),
                ("pt_ptr", _vp), ("z", _vp), ("nz", _vp), ("sp", _vp), ("sm", _vp),
                ("n_points", ctypes.c_int64), ("out_off", _vp), ("out", _vp),
                ("out_len", ctypes.c_int64)]


class bem_mesh_stats(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_triangles", ctypes.c_int64),
                ("n_identical", ctypes.c_int64), ("n_edge", ctypes.c_int64),
                ("n_vertex", ctypes.c_int64), ("max_vertex_degree", ctypes.c_int32),
                ("basis", ctypes.c_int32)]


class bem_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


_lib = None


def load():
    """Loads the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_1510_07244_gb300.build` (nvcc, sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    lib.bem_create.argtypes = [P(_vp), ctypes.c_int, _vp]
    lib.bem_destroy.argtypes = [_vp]
    lib.bem_last_error.argtypes = [_vp]
    lib.bem_last_error.restype = ctypes.c_char_p
    lib.bem_sync.argtypes = [_vp]
    lib.bem_mesh_upload.argtypes = [_vp, _vp, ctypes.c_int64, _vp, ctypes.c_int64,
                                    ctypes.c_int32, P(ctypes.c_int32)]
    lib.bem_mesh_free.argtypes = [_vp, ctypes.c_int32]
    lib.bem_mesh_info.argtypes = [_vp, ctypes.c_int32, P(bem_mesh_stats)]
    lib.bem_near_field.argtypes = [_vp, P(bem_block_job), ctypes.c_int32]
    lib.bem_coupling_blocks.argtypes = [_vp, P(bem_block_job), ctypes.c_int32]
    lib.bem_pivot_entries.argtypes = [_vp, ctypes.c_int32, P(bem_kernel_desc),
                                      P(bem_quad_desc), _vp, _vp, ctypes.c_int64, _vp]
    lib.bem_assemble_dense.argtypes = [_vp, ctypes.c_int32, P(bem_kernel_desc),
                                       P(bem_quad_desc), ctypes.c_int32, _vp]
    lib.bem_near_field_noalloc.argtypes = [_vp, P(bem_block_job)]
    lib.bem_green_matrices.argtypes = [_vp, P(bem_green_job)]
    lib.bem_pivot_entries_absolute.argtypes = [_vp, ctypes.c_int32, P(bem_kernel_desc),
                                               P(bem_quad_desc), _vp, _vp, ctypes.c_int64, _vp]
    lib.bem_mlp_create.argtypes = [_vp, ctypes.c_uint64, P(_vp)]
    lib.bem_mlp_destroy.argtypes = [_vp, _vp]
    lib.bem_mlp_num_params.argtypes = []
    lib.bem_mlp_set_params.argtypes = [_vp, _vp, _vp, _vp]
    lib.bem_mlp_get_params.argtypes = [_vp, _vp, _vp, _vp]
    lib.bem_mlp_gradients.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int32, _vp, P(ctypes.c_float)]
    lib.bem_mlp_train_step.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int32, ctypes.c_float,
                                       P(ctypes.c_float)]
    lib.bem_mlp_infer.argtypes = [_vp, _vp, _vp, ctypes.c_int64, _vp]
    lib.bem_pair_features.argtypes = [_vp, ctypes.c_int32, P(bem_kernel_desc), _vp, _vp, _vp,
                                      ctypes.c_int64, _vp]
    lib.bem_set_order_model.argtypes = [_vp, _vp, ctypes.c_float]
    lib.bem_shard_blocks.argtypes = [_vp, ctypes.c_int64, ctypes.c_int32, _vp]
    lib.bem_touching_pairs.argtypes = [_vp, ctypes.c_int64, ctypes.c_int64, _vp, _vp, _vp, _vp,
                                       ctypes.c_int64, P(ctypes.c_int64)]
    lib.bem_gca_pivots.argtypes = [_vp, ctypes.c_int64, _vp, ctypes.c_int64, ctypes.c_int32,
                                   ctypes.c_double, _vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_double, ctypes.c_int32, ctypes.c_int32, _vp, _vp,
                                   ctypes.c_int64]
    lib.bem_gca_pivots_device.argtypes = [_vp, ctypes.c_int32] + lib.bem_gca_pivots.argtypes
    lib.bem_gca_bases.argtypes = lib.bem_gca_pivots.argtypes + [_vp, _vp, ctypes.c_int64]
    lib.bem_h2_create.argtypes = [_vp, ctypes.c_int64, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp,
                                  _vp, _vp, ctypes.c_int64, _vp, _vp, _vp, _vp, ctypes.c_int64,
                                  _vp, _vp, _vp, _vp, _vp, P(_vp)]
    lib.bem_h2_matvec.argtypes = [_vp, _vp, _vp, _vp]
    lib.bem_h2_cg.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_int32,
                              P(ctypes.c_int32), P(ctypes.c_double)]
    lib.bem_h2_destroy.argtypes = [_vp, _vp]
    lib.bem_learned_counts.argtypes = [_vp, P(ctypes.c_int64)]
    lib.bem_plan_create.argtypes = [_vp, P(bem_block_job), ctypes.c_int32, P(bem_block_job),
                                    ctypes.c_int32, ctypes.c_int32, P(_vp)]
    lib.bem_plan_run.argtypes = [_vp, _vp]
    lib.bem_plan_destroy.argtypes = [_vp, _vp]
    lib.bem_plan_info.argtypes = [_vp, _vp, P(ctypes.c_int32), P(ctypes.c_int32),
                                  P(ctypes.c_int32), P(ctypes.c_int32), ctypes.c_int32]
    lib.bem_plan_guard_stats.argtypes = [_vp, _vp, P(ctypes.c_int64), P(ctypes.c_int64)]
    lib.bem_peak_probe.argtypes = [_vp, ctypes.c_int32, ctypes.c_int64, P(ctypes.c_double)]
    lib.bem_plan_learned_counts.argtypes = [_vp, _vp, P(ctypes.c_int64)]
    lib.bem_potentials.argtypes = [_vp, ctypes.c_int32, P(bem_kernel_desc), ctypes.c_int32, _vp,
                                   ctypes.c_int64, _vp, _vp]
    lib.bem_dense_gmres.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp, ctypes.c_double,
                                    ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int32),
                                    P(ctypes.c_double)]
    lib.bem_mlp_fit_norm.argtypes = [_vp, _vp, _vp, ctypes.c_int64]
    lib.bem_mlp_train_epoch.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int64, _vp, ctypes.c_int32,
                                        ctypes.c_float, P(ctypes.c_float)]
    lib.bem_order_labels.argtypes = [_vp, ctypes.c_int32, P(bem_kernel_desc), _vp, _vp,
                                     ctypes.c_int64, ctypes.c_float, ctypes.c_int32, _vp, _vp]
    lib.bem_rule_points.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp,
                                    ctypes.c_int64]
    lib.bem_rule_points_xi.argtypes = [ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_int64]
    lib.bem_profile_enable.argtypes = [_vp, ctypes.c_int32]
    lib.bem_profile_reset.argtypes = [_vp]
    lib.bem_profile_read.argtypes = [_vp, P(bem_kernel_time), ctypes.c_int32,
                                     P(ctypes.c_int32)]
    for name in EXPORTS:
        if name not in ("bem_last_error", "bem_rule_points", "bem_rule_points_xi"):
            getattr(lib, name).restype = ctypes.c_int
    lib.bem_rule_points.restype = ctypes.c_int64
    lib.bem_rule_points_xi.restype = ctypes.c_int64
    _lib = lib
    return lib


CASES = {"regular": 0, "vertex": 1, "edge": 2, "identical": 3}


def bem_rule_points(case: str, q: int, regular_rule: str = "duffy"):
    """The library's 4D rule for a case: dict of numpy columns x1, x2, y1, y2, w, d1, d2."""
    lib = load()
    n = lib.bem_rule_points(CASES[case], RULES[regular_rule], q, None, 0)
    if n < 0:
        raise BemError(int(n), "bad rule")
    out = np.zeros(7 * n)
    lib.bem_rule_points(CASES[case], RULES[regular_rule], q, out.ctypes.data_as(_vp), out.size)
    cols = out.reshape(7, n)
    return dict(zip(("x1", "x2", "y1", "y2", "w", "d1", "d2"), cols))


def bem_rule_points_xi(case: str, q: int):
    """A touching case's rule with xi integrated out (q^3 points per subdomain
    at xi = 1): dict of numpy columns x1, x2, y1, y2, w, d1, d2."""
    lib = load()
    n = lib.bem_rule_points_xi(CASES[case], q, None, 0)
    if n < 0:
        raise BemError(int(n), "bad rule")
    out = np.zeros(7 * n)
    lib.bem_rule_points_xi(CASES[case], q, out.ctypes.data_as(_vp), out.size)
    cols = out.reshape(7, n)
    return dict(zip(("x1", "x2", "y1", "y2", "w", "d1", "d2"), cols))


def bem_shard_blocks(cost, n_shards: int) -> np.ndarray:
    """Contiguous block ranges of nearly equal cost (host only): bounds (n_shards + 1)."""
    c = np.ascontiguousarray(cost, np.int64)
    bounds = np.zeros(n_shards + 1, np.int64)
    rc = load().bem_shard_blocks(c.ctypes.data_as(_vp), len(c), int(n_shards),
                                 bounds.ctypes.data_as(_vp))
    if rc != BEM_OK:
        raise BemError(rc, "bad shard arguments")
    return bounds


def bem_touching_pairs(tris, nv: int):
    """Touching triangle pairs of a mesh (host only), ascending in (a, b):
    dict of src, dst (int32), case (1 vertex, 2 edge, 3 identical) and ord
    (n x 6: a's canonical vertex order, then b's)."""
    t = np.ascontiguousarray(tris, np.int32)
    nt = t.shape[0]
    n = ctypes.c_int64(0)
    lib = load()
    rc = lib.bem_touching_pairs(t.ctypes.data_as(_vp), nt, int(nv), None, None, None, None, 0,
                                ctypes.byref(n))
    if rc != BEM_OK:
        raise BemError(rc, "bem_touching_pairs: bad mesh")
    src, dst, cas = (np.zeros(n.value, np.int32) for _ in range(3))
    ord_ = np.zeros((n.value, 6), np.int32)
    rc = lib.bem_touching_pairs(t.ctypes.data_as(_vp), nt, int(nv), src.ctypes.data_as(_vp),
                                dst.ctypes.data_as(_vp), cas.ctypes.data_as(_vp),
                                ord_.ctypes.data_as(_vp), n.value, ctypes.byref(n))
    if rc != BEM_OK:
        raise BemError(rc, "bem_touching_pairs: bad mesh")
    return {"src": src, "dst": dst, "case": cas, "ord": ord_}


def bem_gca_pivots(verts, tris, basis: str, cl_ptr, cl_idx, cl_son, kappa: float = 0.0,
                   gauss_per_face: int = 4, eps: float = 1e-6, max_rank: int = 16,
                   n_threads: int = 0, _device_gca=None):
    """GCA pivots of every cluster (host only): cluster CSR (piv_ptr, piv_idx) int32.
    (Context.bem_gca_pivots_device passes _device_gca: the same call with the
    Green matrices on the device.)"""
    v = np.ascontiguousarray(verts, np.float64)
    t = np.ascontiguousarray(tris, np.int32)
    ptr = np.ascontiguousarray(cl_ptr, np.int32)
    idx = np.ascontiguousarray(cl_idx, np.int32)
    son = np.ascontiguousarray(cl_son, np.int32)
    nc = len(ptr) - 1
    if son.shape != (nc, 2):
        raise BemError(-1, "cl_son must be (n_clusters, 2)")
    piv_ptr = np.zeros(nc + 1, np.int32)
    piv_idx = np.zeros(max(1, nc * max_rank), np.int32)
    args = (v.ctypes.data_as(_vp), len(v), t.ctypes.data_as(_vp), len(t), BASES[basis],
            float(kappa), ptr.ctypes.data_as(_vp), idx.ctypes.data_as(_vp),
            son.ctypes.data_as(_vp), nc, int(gauss_per_face), float(eps), int(max_rank),
            int(n_threads), piv_ptr.ctypes.data_as(_vp), piv_idx.ctypes.data_as(_vp),
            piv_idx.size)
    rc = _device_gca(*args) if _device_gca is not None else load().bem_gca_pivots(*args)
    if rc != BEM_OK:
        raise BemError(rc, "bad GCA arguments")
    return piv_ptr, piv_idx[: piv_ptr[-1]].copy()


def bem_gca_bases(verts, tris, basis: str, cl_ptr, cl_idx, cl_son, kappa: float = 0.0,
                  gauss_per_face: int = 4, eps: float = 1e-6, max_rank: int = 16,
                  n_threads: int = 0):
    """GCA pivots and interpolation matrices (host only): (piv_ptr, piv_idx,
    mats) with mats[c] the rows x K_c matrix of cluster c (float64, complex128
    for kappa > 0): V_t of a leaf (rows = its indices), the transfer matrix of
    a cluster with sons (rows = the sons' pivots, first son first)."""
    v = np.ascontiguousarray(verts, np.float64)
    t = np.ascontiguousarray(tris, np.int32)
    ptr = np.ascontiguousarray(cl_ptr, np.int32)
    idx = np.ascontiguousarray(cl_idx, np.int32)
    son = np.ascontiguousarray(cl_son, np.int32)
    nc = len(ptr) - 1
    if son.shape != (nc, 2):
        raise BemError(-1, "cl_son must be (n_clusters, 2)")
    piv_ptr = np.zeros(nc + 1, np.int32)
    piv_idx = np.zeros(max(1, nc * max_rank), np.int32)
    cplx = kappa != 0.0
    v_cap = (int(ptr[-1]) + 2 * max_rank * nc) * max_rank
    v_off = np.zeros(nc + 1, np.int64)
    V = np.zeros(max(1, v_cap * (2 if cplx else 1)), np.float64)
    rc = load().bem_gca_bases(v.ctypes.data_as(_vp), len(v), t.ctypes.data_as(_vp), len(t),
                              BASES[basis], float(kappa), ptr.ctypes.data_as(_vp),
                              idx.ctypes.data_as(_vp), son.ctypes.data_as(_vp), nc,
                              int(gauss_per_face), float(eps), int(max_rank), int(n_threads),
                              piv_ptr.ctypes.data_as(_vp), piv_idx.ctypes.data_as(_vp),
                              piv_idx.size, v_off.ctypes.data_as(_vp), V.ctypes.data_as(_vp),
                              v_cap)
    if rc != BEM_OK:
        raise BemError(rc, "bad GCA arguments")
    vals = V.view(np.complex128) if cplx else V
    mats = []
    for c in range(nc):
        k = int(piv_ptr[c + 1] - piv_ptr[c])
        blk = vals[v_off[c]:v_off[c + 1]]
        mats.append(blk.reshape(-1, k).copy() if k > 0 else np.zeros((0, 0), vals.dtype))
    return piv_ptr, piv_idx[: piv_ptr[-1]].copy(), mats


def kernel_desc(kind="laplace_slp", kappa=0.0, eta=0.0) -> bem_kernel_desc:
    return bem_kernel_desc(KERNELS[kind], float(kappa), float(eta))


def quad_desc(q_regular=3, regular_rule="duffy", q_identical=5, q_edge=5, q_vertex=5,
              precision="fp64", order_mode="fixed") -> bem_quad_desc:
    return bem_quad_desc(int(q_regular), RULES[regular_rule], int(q_identical), int(q_edge),
                         int(q_vertex), PRECISIONS[precision], ORDER_MODES[order_mode])


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_dev(t, dtype, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA tensor of {dtype}")


@dataclass
class BlockJob:
    """Blocks of one mesh in cluster-CSR form (all CUDA tensors)."""
    mesh_id: int
    row_ptr: object
    row_idx: object
    col_ptr: object
    col_idx: object
    blk_row: object
    blk_col: object
    blk_off: object
    out: object
    kernel: bem_kernel_desc = field(default_factory=kernel_desc)
    quad: bem_quad_desc = field(default_factory=quad_desc)

    def to_c(self) -> bem_block_job:
        import torch
        for n in ("row_ptr", "row_idx", "col_ptr", "col_idx", "blk_row", "blk_col"):
            _check_dev(getattr(self, n), torch.int32, n)
        _check_dev(self.blk_off, torch.int64, "blk_off")
        cplx = self.kernel.kind in _COMPLEX_IDS
        _check_dev(self.out, torch.complex128 if cplx else torch.float64, "out")
        return bem_block_job(self.mesh_id, self.kernel, self.quad,
                             _ptr(self.row_ptr), _ptr(self.row_idx), self.row_ptr.numel() - 1,
                             _ptr(self.col_ptr), _ptr(self.col_idx), self.col_ptr.numel() - 1,
                             _ptr(self.blk_row), _ptr(self.blk_col), _ptr(self.blk_off),
                             self.blk_row.numel(), _ptr(self.out))


@dataclass
class GreenJob:
    """Green quadrature matrices A_t = (A_t+, A_t-) of a list of clusters
    (CUDA tensors): rows row_idx[row_ptr[c]:row_ptr[c+1]], points z / normals nz
    [pt_ptr[c]:pt_ptr[c+1]] (float64, shape (n, 3)), optional per-point factors
    sp / sm, block c written column-major (n_c x 2 m_c) at out_off[c] of out."""
    mesh_id: int
    row_ptr: object
    row_idx: object
    pt_ptr: object
    z: object
    nz: object
    out_off: object
    out: object
    sp: object = None
    sm: object = None
    kernel: bem_kernel_desc = field(default_factory=kernel_desc)
    rule: str = "tri7"
    q: int = 0

    def to_c(self) -> bem_green_job:
        import torch
        for n in ("row_ptr", "row_idx", "pt_ptr"):
            _check_dev(getattr(self, n), torch.int32, n)
        for n in ("z", "nz"):
            _check_dev(getattr(self, n), torch.float64, n)
        for n in ("sp", "sm"):
            if getattr(self, n) is not None:
                _check_dev(getattr(self, n), torch.float64, n)
        _check_dev(self.out_off, torch.int64, "out_off")
        cplx = self.kernel.kind in _COMPLEX_IDS
        _check_dev(self.out, torch.complex128 if cplx else torch.float64, "out")
        n_clusters = self.row_ptr.numel() - 1
        n_points = self.z.numel() // 3
        if (self.pt_ptr.numel() != n_clusters + 1 or self.out_off.numel() != n_clusters
                or self.nz.numel() != self.z.numel()
                or any(t is not None and t.numel() != n_points for t in (self.sp, self.sm))):
            raise ValueError("GreenJob: inconsistent array sizes")
        return bem_green_job(self.mesh_id, self.kernel, RULES[self.rule], int(self.q), n_clusters,
                             _ptr(self.row_ptr), _ptr(self.row_idx), self.row_idx.numel(),
                             _ptr(self.pt_ptr), _ptr(self.z), _ptr(self.nz), _ptr(self.sp),
                             _ptr(self.sm), n_points, _ptr(self.out_off), _ptr(self.out),
                             self.out.numel())


class Context:
    """Owns a bem_ctx.  Methods mirror the C entry points."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.lib = load()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = ctypes.c_void_p()
        rc = self.lib.bem_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream))
        if rc != BEM_OK:
            raise BemError(rc, "bem_create failed")
        self.h = h

    def _check(self, rc):
        if rc != BEM_OK:
            raise BemError(rc, self.lib.bem_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.bem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bem_last_error(self) -> str:
        return self.lib.bem_last_error(self.h).decode()

    def bem_sync(self):
        self._check(self.lib.bem_sync(self.h))

    def bem_mesh_upload(self, verts, tris, basis="p0") -> int:
        v = np.ascontiguousarray(verts, np.float64)
        t = np.ascontiguousarray(tris, np.int32)
        mid = ctypes.c_int32(0)
        self._check(self.lib.bem_mesh_upload(self.h, v.ctypes.data_as(_vp), v.shape[0],
                                             t.ctypes.data_as(_vp), t.shape[0], BASES[basis],
                                             ctypes.byref(mid)))
        return mid.value

    def bem_mesh_free(self, mesh_id: int):
        self._check(self.lib.bem_mesh_free(self.h, mesh_id))

    def bem_mesh_info(self, mesh_id: int) -> dict:
        s = bem_mesh_stats()
        self._check(self.lib.bem_mesh_info(self.h, mesh_id, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def bem_near_field(self, jobs):
        arr = (bem_block_job * len(jobs))(*[j.to_c() for j in jobs])
        self._check(self.lib.bem_near_field(self.h, arr, len(jobs)))

    def bem_near_field_noalloc(self, job):
        """Near field of one job without any device allocation (static scratch)."""
        c = job.to_c()
        self._check(self.lib.bem_near_field_noalloc(self.h, ctypes.byref(c)))

    def bem_green_matrices(self, job):
        c = job.to_c()
        self._check(self.lib.bem_green_matrices(self.h, ctypes.byref(c)))

    def bem_gca_pivots_device(self, mesh_id, verts, tris, basis: str, cl_ptr, cl_idx, cl_son,
                              kappa: float = 0.0, gauss_per_face: int = 4, eps: float = 1e-6,
                              max_rank: int = 16, n_threads: int = 0):
        """bem_gca_pivots with every Green matrix A_t assembled on the device
        (mesh_id: the same mesh, uploaded); cluster CSR (piv_ptr, piv_idx)."""
        def call(*args):
            return self.lib.bem_gca_pivots_device(self.h, int(mesh_id), *args)
        try:
            return bem_gca_pivots(verts, tris, basis, cl_ptr, cl_idx, cl_son, kappa=kappa,
                                  gauss_per_face=gauss_per_face, eps=eps, max_rank=max_rank,
                                  n_threads=n_threads, _device_gca=call)
        except BemError as e:
            raise BemError(e.code, self.lib.bem_last_error(self.h).decode() or str(e)) from None

    def bem_coupling_blocks(self, jobs):
        arr = (bem_block_job * len(jobs))(*[j.to_c() for j in jobs])
        self._check(self.lib.bem_coupling_blocks(self.h, arr, len(jobs)))

    def bem_pivot_entries(self, mesh_id, kernel, quad, rows, cols, out):
        import torch
        _check_dev(rows, torch.int32, "rows")
        _check_dev(cols, torch.int32, "cols")
        cplx = kernel.kind in _COMPLEX_IDS
        _check_dev(out, torch.complex128 if cplx else torch.float64, "out")
        if rows.numel() != cols.numel() or out.numel() < rows.numel():
            raise ValueError("rows/cols/out size mismatch")
        self._check(self.lib.bem_pivot_entries(self.h, mesh_id, ctypes.byref(kernel),
                                               ctypes.byref(quad), _ptr(rows), _ptr(cols),
                                               rows.numel(), _ptr(out)))

    def bem_assemble_dense(self, mesh_id, kernel, quad, lower_only, out):
        import torch
        cplx = kernel.kind in _COMPLEX_IDS
        _check_dev(out, torch.complex128 if cplx else torch.float64, "out")
        info = self.bem_mesh_info(mesh_id)
        n = info["n_triangles"] if info["basis"] == 0 else info["n_vertices"]
        if out.numel() < n * n:
            raise ValueError(f"out must hold {n} x {n} entries")
        self._check(self.lib.bem_assemble_dense(self.h, mesh_id, ctypes.byref(kernel),
                                                ctypes.byref(quad), int(lower_only), _ptr(out)))

    def bem_profile_enable(self, on: bool = True):
        self._check(self.lib.bem_profile_enable(self.h, 1 if on else 0))

    def bem_profile_reset(self):
        self._check(self.lib.bem_profile_reset(self.h))

    def bem_profile_read(self) -> dict:
        """{kernel class: (launches, total_ms)} of all finished profiled launches."""
        cap = 32
        arr = (bem_kernel_time * cap)()
        n = ctypes.c_int32(0)
        self._check(self.lib.bem_profile_read(self.h, arr, cap, ctypes.byref(n)))
        return {arr[k].name.decode(): (arr[k].launches, arr[k].total_ms)
                for k in range(min(cap, n.value))}

    def bem_plan_create(self, near_jobs, coupling_jobs, flags=PLAN_GRAPH):
        """Plan over near-field and coupling jobs; returns an opaque handle.  The
        jobs' tensors must stay alive until bem_plan_destroy."""
        nj = (bem_block_job * max(1, len(near_jobs)))(*[j.to_c() for j in near_jobs])
        cj = (bem_block_job * max(1, len(coupling_jobs)))(*[j.to_c() for j in coupling_jobs])
        h = ctypes.c_void_p()
        self._check(self.lib.bem_plan_create(self.h, nj, len(near_jobs), cj, len(coupling_jobs),
                                             int(flags), ctypes.byref(h)))
        self._plans = getattr(self, "_plans", {})
        self._plans[h.value] = (near_jobs, coupling_jobs)   # keep the tensors alive
        return h

    def bem_plan_run(self, plan):
        self._check(self.lib.bem_plan_run(self.h, plan))

    def bem_plan_destroy(self, plan):
        self._check(self.lib.bem_plan_destroy(self.h, plan))
        getattr(self, "_plans", {}).pop(plan.value, None)

    def bem_plan_info(self, plan):
        nt, nb, na = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        g = (ctypes.c_int32 * 64)()
        self._check(self.lib.bem_plan_info(self.h, plan, ctypes.byref(nt), ctypes.byref(nb),
                                           ctypes.byref(na), g, 64))
        return {"touch_launches": nt.value, "block_launches": nb.value, "aux_launches": na.value,
                "grid_mult": [g[k] for k in range(min(64, nb.value))]}

    # ---- H2 matrix-vector product and conjugate gradients -------------------
    def bem_h2_create(self, n, cl_ptr, cl_idx, cl_son, piv_ptr, piv_idx, mats, near, near_vals,
                      far, far_vals, diag=None):
        """H2 matrix from the tree (host), the bases of bem_gca_bases (host:
        piv_ptr, piv_idx and the list of matrices) and the near / coupling
        blocks: near, far = (blk_row, blk_col, blk_off) host arrays with their
        device values (float64 tensors that must outlive the handle); diag:
        optional host array added to the diagonal."""
        import torch
        _check_dev(near_vals, torch.float64, "near_vals")
        _check_dev(far_vals, torch.float64, "far_vals")
        ptr = np.ascontiguousarray(cl_ptr, np.int32)
        idx = np.ascontiguousarray(cl_idx, np.int32)
        son = np.ascontiguousarray(cl_son, np.int32)
        pp = np.ascontiguousarray(piv_ptr, np.int32)
        pi = np.ascontiguousarray(piv_idx, np.int32)
        sizes = [np.asarray(m).size for m in mats]
        v_off = np.zeros(len(mats) + 1, np.int64)
        v_off[1:] = np.cumsum(sizes)
        V = np.ascontiguousarray(np.concatenate([np.asarray(m, np.float64).ravel() for m in mats])
                                 if sizes else np.zeros(1), np.float64)
        nr, nc_, no = (np.ascontiguousarray(a, t) for a, t in zip(near, (np.int32, np.int32, np.int64)))
        fr, fc, fo = (np.ascontiguousarray(a, t) for a, t in zip(far, (np.int32, np.int32, np.int64)))
        h = _vp()
        dg = None if diag is None else np.ascontiguousarray(diag, np.float64)
        if dg is not None and dg.shape != (int(n),):
            raise BemError(-1, "diag must have n entries")
        keep = (ptr, idx, son, pp, pi, v_off, V, nr, nc_, no, fr, fc, fo, dg)
        self._check(self.lib.bem_h2_create(
            self.h, int(n), len(ptr) - 1, *[a.ctypes.data_as(_vp) for a in keep[:7]],
            len(nr), nr.ctypes.data_as(_vp), nc_.ctypes.data_as(_vp), no.ctypes.data_as(_vp),
            _ptr(near_vals), len(fr), fr.ctypes.data_as(_vp), fc.ctypes.data_as(_vp),
            fo.ctypes.data_as(_vp), _ptr(far_vals),
            None if dg is None else dg.ctypes.data_as(_vp), ctypes.byref(h)))
        return h

    def bem_h2_matvec(self, h2, x, y):
        import torch
        _check_dev(x, torch.float64, "x")
        _check_dev(y, torch.float64, "y")
        self._check(self.lib.bem_h2_matvec(self.h, h2, _ptr(x), _ptr(y)))

    def bem_h2_cg(self, h2, b, x, tol=1e-8, maxit=1000):
        import torch
        _check_dev(b, torch.float64, "b")
        _check_dev(x, torch.float64, "x")
        it, res = ctypes.c_int32(0), ctypes.c_double(0.0)
        self._check(self.lib.bem_h2_cg(self.h, h2, _ptr(b), _ptr(x), float(tol), int(maxit),
                                       ctypes.byref(it), ctypes.byref(res)))
        return it.value, res.value

    def bem_h2_destroy(self, h2):
        self._check(self.lib.bem_h2_destroy(self.h, h2))

    def bem_peak_probe(self, kind: int, trips: int) -> float:
        """Launches one arithmetic-pipe probe on the context's stream; returns
        the number of operations the launch performs."""
        ops = ctypes.c_double(0.0)
        self._check(self.lib.bem_peak_probe(self.h, int(kind), int(trips), ctypes.byref(ops)))
        return ops.value

    def bem_potentials(self, mesh_id, kernel, points, density, out, q=4):
        """Potentials of a piecewise-constant complex density at points off the
        surface (device tensors: points (m, 3) float64, density (nt,) and out (m,)
        complex128)."""
        import torch
        _check_dev(points, torch.float64, "points")
        _check_dev(density, torch.complex128, "density")
        _check_dev(out, torch.complex128, "out")
        self._check(self.lib.bem_potentials(self.h, mesh_id, ctypes.byref(kernel), int(q),
                                            _ptr(points), points.shape[0], _ptr(density),
                                            _ptr(out)))

    def bem_dense_gmres(self, A, b, x, diag=None, tol=1e-8, restart=100, maxit=1000):
        """GMRES for (A + diag(diag)) x = b; A column-major complex (n*n,) device
        tensor, b, x, diag complex (n,).  Returns (iterations, relative residual)."""
        import torch
        for t, nm in ((A, "A"), (b, "b"), (x, "x")):
            _check_dev(t, torch.complex128, nm)
        if diag is not None:
            _check_dev(diag, torch.complex128, "diag")
        it, res = ctypes.c_int32(0), ctypes.c_double(0.0)
        self._check(self.lib.bem_dense_gmres(self.h, b.numel(), _ptr(A), _ptr(diag), _ptr(b),
                                             _ptr(x), float(tol), int(restart), int(maxit),
                                             ctypes.byref(it), ctypes.byref(res)))
        return it.value, res.value

    def bem_plan_learned_counts(self, plan):
        c = (ctypes.c_int64 * 6)()
        self._check(self.lib.bem_plan_learned_counts(self.h, plan, c))
        return [c[k] for k in range(6)]

    def bem_plan_guard_stats(self, plan):
        n, r = ctypes.c_int64(0), ctypes.c_int64(0)
        self._check(self.lib.bem_plan_guard_stats(self.h, plan, ctypes.byref(n), ctypes.byref(r)))
        return {"entries": n.value, "recomputed": r.value}

    # ---- pivots (absolute sums) and the order model --------------------------
    def bem_pivot_entries_absolute(self, mesh_id, kernel, quad, rows, cols, out):
        import torch
        _check_dev(rows, torch.int32, "rows")
        _check_dev(cols, torch.int32, "cols")
        _check_dev(out, torch.float64, "out")
        self._check(self.lib.bem_pivot_entries_absolute(self.h, mesh_id, ctypes.byref(kernel),
                                                        ctypes.byref(quad), _ptr(rows), _ptr(cols),
                                                        rows.numel(), _ptr(out)))

    def bem_mlp_create(self, seed=0):
        h = ctypes.c_void_p()
        self._check(self.lib.bem_mlp_create(self.h, ctypes.c_uint64(seed), ctypes.byref(h)))
        return h

    def bem_mlp_destroy(self, mlp):
        self._check(self.lib.bem_mlp_destroy(self.h, mlp))

    def bem_mlp_num_params(self):
        return int(self.lib.bem_mlp_num_params())

    def bem_mlp_set_params(self, mlp, params=None, norm=None):
        p = None if params is None else np.ascontiguousarray(params, np.float32)
        q = None if norm is None else np.ascontiguousarray(norm, np.float32)
        self._check(self.lib.bem_mlp_set_params(self.h, mlp, None if p is None else p.ctypes.data_as(_vp),
                                                None if q is None else q.ctypes.data_as(_vp)))

    def bem_mlp_get_params(self, mlp):
        p = np.zeros(self.bem_mlp_num_params(), np.float32)
        q = np.zeros(16, np.float32)
        self._check(self.lib.bem_mlp_get_params(self.h, mlp, p.ctypes.data_as(_vp), q.ctypes.data_as(_vp)))
        return p, q

    def bem_mlp_gradients(self, mlp, X, y, grads=None):
        import torch
        _check_dev(X, torch.float32, "X")
        _check_dev(y, torch.int32, "y")
        loss = ctypes.c_float(0.0)
        self._check(self.lib.bem_mlp_gradients(self.h, mlp, _ptr(X), _ptr(y), y.numel(), _ptr(grads),
                                               ctypes.byref(loss)))
        return loss.value

    def bem_mlp_train_step(self, mlp, X, y, lr):
        import torch
        _check_dev(X, torch.float32, "X")
        _check_dev(y, torch.int32, "y")
        loss = ctypes.c_float(0.0)
        self._check(self.lib.bem_mlp_train_step(self.h, mlp, _ptr(X), _ptr(y), y.numel(),
                                                ctypes.c_float(lr), ctypes.byref(loss)))
        return loss.value

    def bem_mlp_fit_norm(self, mlp, X):
        import torch
        _check_dev(X, torch.float32, "X")
        self._check(self.lib.bem_mlp_fit_norm(self.h, mlp, _ptr(X), X.shape[0]))

    def bem_mlp_train_epoch(self, mlp, X, y, perm, batch, lr):
        import torch
        _check_dev(X, torch.float32, "X")
        _check_dev(y, torch.int32, "y")
        _check_dev(perm, torch.int64, "perm")
        loss = ctypes.c_float(0.0)
        self._check(self.lib.bem_mlp_train_epoch(self.h, mlp, _ptr(X), _ptr(y), X.shape[0],
                                                 _ptr(perm), int(batch), ctypes.c_float(lr),
                                                 ctypes.byref(loss)))
        return loss.value

    def bem_order_labels(self, mesh_id, kernel, a, b, labels, errors=None, tol=1e-7, q_ref=12):
        import torch
        _check_dev(a, torch.int32, "a")
        _check_dev(b, torch.int32, "b")
        _check_dev(labels, torch.int32, "labels")
        if errors is not None:
            _check_dev(errors, torch.float32, "errors")
        self._check(self.lib.bem_order_labels(self.h, mesh_id, ctypes.byref(kernel), _ptr(a),
                                              _ptr(b), a.numel(), ctypes.c_float(tol), int(q_ref),
                                              _ptr(labels), _ptr(errors)))

    def bem_mlp_infer(self, mlp, X, logits):
        import torch
        _check_dev(X, torch.float32, "X")
        _check_dev(logits, torch.float32, "logits")
        self._check(self.lib.bem_mlp_infer(self.h, mlp, _ptr(X), X.shape[0], _ptr(logits)))

    def bem_pair_features(self, mesh_id, kernel, mlp, a, b, X):
        import torch
        _check_dev(a, torch.int32, "a")
        _check_dev(b, torch.int32, "b")
        _check_dev(X, torch.float32, "X")
        self._check(self.lib.bem_pair_features(self.h, mesh_id, ctypes.byref(kernel), mlp, _ptr(a),
                                               _ptr(b), a.numel(), _ptr(X)))

    def bem_set_order_model(self, mlp, confidence=0.9):
        self._check(self.lib.bem_set_order_model(self.h, mlp, ctypes.c_float(confidence)))

    def bem_learned_counts(self):
        c = (ctypes.c_int64 * 6)()
        self._check(self.lib.bem_learned_counts(self.h, c))
        return [int(v) for v in c]
