"""Host-side accounting of the benchmark: the algorithmic operation counts
per kernel (fused launches count the work both layers share once) and the
committed DRAM-traffic figures it reports."""
import pytest

import bench
import synth


@pytest.fixture(scope="module")
def small_c2():
    w = synth.workloads.config2(levels=3)
    counts = bench.pair_counts(w)
    assert counts["near_regular_pairs"] > 0 and counts["far_entry_pairs"] > 0
    return w, counts


STATS = {"n_vertex": 0, "n_edge": 0, "n_identical": 0}


def test_fused_launches_count_shared_work_once(small_c2):
    w, counts = small_c2
    npts, npa = 81, 9
    slp = bench.flops_per_point("laplace_slp", "p1", npa)
    dlp = bench.flops_per_point("laplace_dlp", "p1", npa)
    f64 = bench.kernel_flops(w, counts, STATS, "fp64")
    mix = bench.kernel_flops(w, counts, STATS, "mixed_full")
    reg_all = counts["near_regular_pairs"] + counts["far_regular_pairs"]
    # FP64 form: one tile engine for near and coupling blocks, layers separate
    assert set(f64) >= {"block_p1"} and "coupling_p1" not in f64
    assert f64["block_p1"][0] == pytest.approx(reg_all * npts * (slp + dlp))
    assert f64["block_p1"][1] == "fp64"
    # float forms: near field in the fused tile engine, coupling blocks in the
    # fused coupling engine; the difference, r^2 and rsqrt (9) count once
    assert mix["block_p1"][0] == pytest.approx(
        counts["near_regular_pairs"] * npts * (slp + dlp - 9.0))
    p0s = bench.flops_per_point("laplace_slp", "p0", npa)
    p0d = bench.flops_per_point("laplace_dlp", "p0", npa)
    want = counts["far_entry_pairs"] * npts * (p0s + p0d + 20.0 / npa - 9.0 - 6.0 / npa)
    assert mix["coupling_p1"][0] == pytest.approx(want)
    assert mix["coupling_p1"][1] == mix["block_p1"][1] == "fp32"
    assert mix["block_p1"][2] == pytest.approx(bench.PEAK_FP32)


def test_single_operator_is_not_fused(small_c2):
    w, counts = small_c2
    w1 = synth.workloads.Workload(**{**w.__dict__,
                                     "operators": [o for o in w.operators
                                                   if o.kernel == "laplace_dlp"]})
    mix = bench.kernel_flops(w1, counts, STATS, "mixed_full")
    dlp = bench.flops_per_point("laplace_dlp", "p1", 9)
    assert mix["block_p1"][0] == pytest.approx(counts["near_regular_pairs"] * 81 * dlp)


def test_empty_block_set_counts_nothing():
    w = synth.workloads.config2(levels=2)    # 320 triangles: no admissible blocks
    assert len(w.far.blk_row) == 0
    counts = bench.pair_counts(w)
    assert counts["far_regular_pairs"] == counts["far_entry_pairs"] == 0


def test_committed_traffic_figures():
    t = bench.profiled_traffic("coupling_p1")
    assert isinstance(t, int) and 1_000_000 < t < 100_000_000
    assert bench.profiled_traffic("no_such_kernel") is None


def test_green_workload_is_the_gcas_row_sets(small_c2):
    """The Green-matrix workload holds, per cluster, the rows the host GCA
    forms A_t on (leaves: all indices; other clusters: the union of their sons'
    pivots, nested), 96 box points each, and non-overlapping blocks."""
    import numpy as np
    import paper_1510_07244_gb300 as pkg
    w, _ = small_c2
    G = bench.green_workload(pkg, w)
    tree = w.partition.tree
    ptr, idx = w.partition.cluster_csr()
    pp, pi = pkg.bem_gca_pivots(w.mesh.verts, w.mesh.tris, w.basis, ptr, idx,
                                w.partition.son_array(), kappa=0.0, gauss_per_face=4, eps=1e-6,
                                max_rank=w.meta["rank"])
    rp, rows = G["row_ptr"], G["rows"]
    assert len(rp) == tree.n_clusters + 1 and rp[0] == 0 and rp[-1] == len(rows)
    for c in range(tree.n_clusters):
        r = rows[rp[c]:rp[c + 1]]
        if tree.is_leaf(c):
            assert np.array_equal(np.sort(r), np.sort(tree.indices(c)))
        else:
            sons = np.concatenate([pi[pp[s]:pp[s + 1]] for s in tree.sons[c]])
            assert np.array_equal(r, np.unique(sons))
            # nested bases: a cluster's pivots are rows of its A_t
            assert np.isin(pi[pp[c]:pp[c + 1]], r).all()
    m = np.diff(G["pt_ptr"])
    assert (m == 96).all() and len(G["z"]) == m.sum() == len(G["sp"]) == len(G["sm"])
    sizes = 2 * np.diff(rp).astype(np.int64) * m
    assert np.array_equal(G["off"], np.concatenate([[0], np.cumsum(sizes)[:-1]]))
    assert G["total"] == sizes.sum()
    # operation count: a rule point costs more with the Helmholtz phase
    assert bench.green_flops(True, 7) > bench.green_flops(False, 7) > 7 * 30


def test_step_rates_count_pairs_and_points(small_c2):
    """Pair integrals and quadrature points per step: per operator, the regular
    pairs as the form's kernels evaluate them plus every touching pair, each
    with its rule's points; rates divide by the step time."""
    w, counts = small_c2
    stats = {"n_vertex": 30, "n_edge": 12, "n_identical": 5}
    q = w.quad
    touch = 30 + 12 + 5
    tpts = 30 * 2 * q.q_vertex ** 4 + 12 * 4 * q.q_edge ** 4 + 5 * 6 * q.q_identical ** 4
    npts = (q.q_regular ** 2) ** 2 if q.regular_rule == "duffy" else 49
    n_ops = len(w.operators)
    r64 = bench.step_rates(w, counts, stats, "fp64", 2.0)
    reg64 = counts["near_regular_pairs"] + counts["far_regular_pairs"]
    assert r64["pair_integrals_per_step"] == n_ops * (reg64 + touch)
    assert r64["quadrature_points_per_step"] == n_ops * (reg64 * npts + tpts)
    assert r64["pair_integrals_per_s"] == pytest.approx(r64["pair_integrals_per_step"] / 2e-3)
    # the float forms evaluate P1 coupling entries pair by pair
    rmx = bench.step_rates(w, counts, stats, "mixed_full", 2.0)
    regmx = counts["near_regular_pairs"] + counts["far_entry_pairs"]
    assert rmx["pair_integrals_per_step"] == n_ops * (regmx + touch)
    assert counts["far_entry_pairs"] >= counts["far_regular_pairs"]


def test_p0_pair_integrals_equal_entries():
    """Piecewise-constant bases: every entry is one triangle pair, so the
    regular pairs of the block sets plus the mesh's touching pairs (each one
    lies in exactly one near-field block) are the entries; the touching
    pairs' points are the rules' points as the float kernels run them."""
    import numpy as np
    import paper_1510_07244_gb300 as pkg
    w = synth.workloads.config3(n=8)          # 768 triangles, P0
    counts = bench.pair_counts(w)
    tp = pkg.bem_touching_pairs(w.mesh.tris, w.mesh.nv)
    stats = {f"n_{c}": int(np.sum(tp["case"] == k))
             for k, c in ((1, "vertex"), (2, "edge"), (3, "identical"))}
    assert stats["n_identical"] == w.mesh.nt
    pairs = (counts["near_regular_pairs"] + counts["far_regular_pairs"] + stats["n_vertex"] +
             stats["n_edge"] + stats["n_identical"])
    assert pairs == w.near.n_entries + w.far.n_entries
    for op in w.operators:
        pts = bench.kernel_points(w, counts, stats, op.kernel, "mixed_full")
        reg = counts["near_regular_pairs"] + counts["far_regular_pairs"]
        assert pts["block_p0"] == reg * 81
        for cas, q in (("vertex", w.quad.q_vertex), ("edge", w.quad.q_edge),
                       ("identical", w.quad.q_identical)):
            nsub = {"vertex": 2, "edge": 4, "identical": 6}[cas]
            # the float Helmholtz kernels sum xi in node pairs: q^3 points per subdomain
            assert pts[f"touching_{cas}"] == stats[f"n_{cas}"] * nsub * q ** 3
