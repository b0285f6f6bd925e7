#!/usr/bin/env python
"""Benchmark: Galerkin entries/s of near-field + coupling (pivot) blocks.

Default line (--workload all): the largest configuration, C4 -- 48 closed
meshes (16 spheres, 16 cubes, 16 tori; 500 to 30000 triangles each, 389804
in all), piecewise-constant basis, the Laplace double layer and the
Helmholtz single layer (kappa ~ U[1, 10]) of every mesh, H2 blocks (leaf 32,
eta 2, at most 16 host-GCA pivots per cluster), Sauter-Schwab order 5 and
Duffy order 3: 576 M entries per step, all of them in one persistent plan
(one CUDA graph replay per step).  The plain FP64 form and the float forms
are timed; every entry of each float form is compared with the FP64 form on
both error measures, and the headline is the fastest form within 1e-6 on
both.  Inputs are resident on the device before the timed region; L2 is
flushed (256 MiB write) between timed steps.  `e2e` repeats the step through
the per-call entry points from pinned host buffers (mesh upload and host
planning, block lists in, all outputs out).  The roofline divides by peaks
measured in the same run (bem_peak_probe).  C1, C2, C3 and C5 are measured
in the same run under `configs`, the GCA's Green matrices of C2's tree under
`green_matrices`.

--impl reference runs the plain FP64 CPU oracle on bounded samples of the
same workload's entries (the slow baseline arm).
"""
import argparse
import copy
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Galerkin entries/s (near SS + far pivots) at ≤1e-6 rel err vs plain FP64 form"
UNIT = "entries/s"

# FP64 operations per quadrature point (FMA = 2, rsqrt = 1, sincos = 2), as the
# block kernels evaluate them: difference vector 3, r^2 5, rsqrt 1, weight and
# accumulation 2; double layer + (x-y).n 5, r^-3 2, product 1; Helmholtz +
# kappa r 1, sincos 2, two products and a second accumulation 5; piecewise
# linear + three basis-weighted accumulations 6 and the x-side 3x3 update
# 18 / (points per axis pair).
def profiled_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` on the default workload, from the ncu
    summary committed under profiles/ (None if there is none)."""
    import glob
    import re
    key = f"traffic_bytes_per_launch[{kernel}]:"
    for path in sorted(glob.glob(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                              "profiles", "*.md"))):
        for line in open(path):
            if line.startswith(key):
                m = re.search(r"(\d+)", line[len(key):])
                if m:
                    return int(m.group(1))
    return None


def flops_per_point(kernel: str, basis: str, np_axis: int) -> float:
    f = 11.0
    if kernel == "laplace_dlp":
        f += 8.0
    elif kernel == "helmholtz_slp":
        f += 8.0
    if basis == "p1":
        f += 6.0 + 18.0 / np_axis
    return f


def flops_per_point_ss(case: str, kernel: str, basis: str) -> float:
    """Per point of a singular rule, as the touching kernels evaluate it: the
    difference vector from 2 / 3 / 4 scaled edge vectors (identical / edge /
    vertex: 9 / 15 / 21), r^2 5, rsqrt 1, weight 1 and accumulation 1; the
    double layer's height costs 1 for a common edge (x2 H) and 5 for a common
    vertex, plus r^-3 2 and a product 1, and vanishes for identical (flat)
    pairs; Helmholtz adds kappa r 1, sincos 2, products 3; P1 replaces the
    accumulation by three products and nine FMAs on the moments (+20)."""
    if kernel == "laplace_dlp" and case == "identical":
        return 0.0
    f = {"identical": 9.0, "edge": 15.0, "vertex": 21.0}[case] + 8.0
    if kernel == "laplace_dlp":
        f += (1.0 if case == "edge" else 5.0) + 3.0
    elif kernel == "helmholtz_slp":
        f += 6.0 + 2.0
    if basis == "p1":
        f += 20.0
    return f


def touch_rule_xi(kernel: str, basis: str, q: int, f32: bool) -> bool:
    """Whether the library evaluates a touching case with xi integrated out
    (bem_rule_points_xi): the Laplace kernels where the q-point Gauss rule in
    xi is exact for the integrand's degree in xi, the float Helmholtz single
    layer with its xi sums."""
    if kernel == "helmholtz_slp":
        return f32 and q <= 20
    if kernel not in ("laplace_slp", "laplace_dlp"):
        return False
    deg = (2 if kernel == "laplace_slp" else 1) + (2 if basis == "p1" else 0)
    return 2 * q - 1 >= deg


def touch_cost(case: str, kernel: str, basis: str, q: int, f32: bool):
    """(evaluation points per touching pair, algorithmic flops per point).
    With xi integrated out the points are the q^3 per subdomain at xi = 1;
    the float Helmholtz single layer then costs, per point, the distance part
    once (difference, r^2 5, rsqrt 1, kappa |u| 2, weight 1, accumulation 2),
    per node pair a sine/cosine (2) and two FMAs per moment power, and the
    middle node and the rotation by exp(i th / 2) (sincos 2, 8 per power)."""
    nsub = {"vertex": 2, "edge": 4, "identical": 6}[case]
    xi = touch_rule_xi(kernel, basis, q, f32)
    pts = nsub * q ** (3 if xi else 4)
    f = flops_per_point_ss(case, kernel, basis)
    if xi and kernel == "helmholtz_slp":
        mm = 3 if basis == "p1" else 1
        geo = {"identical": 9.0, "edge": 15.0, "vertex": 21.0}[case]
        f = (geo + 11.0 + (q // 2) * (2.0 + 4.0 * mm) + 2.0 + 8.0 * mm +
             (20.0 if basis == "p1" else 0.0))
    return pts, f


PEAK_FP64 = 152 * 2.07e9 * 4.0 / 1e12     # TFLOP/s: 152 SM x 2 FMA/clk x 2.07 GHz
PEAK_FP32 = 152 * 2.07e9 * 256.0 / 1e12   # TFLOP/s: 152 SM x 128 FMA/clk x 2.07 GHz
# the denominators of the rooflines: the measured rates once measure_peaks has
# run (its FP32 and FP64 FMA probes), the unit-count products before
def _measured_hbm():
    """The HBM copy rate measured on this machine (MEASURED_PEAKS.json), else the
    pool's fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


MEASURED_HBM_GBS = _measured_hbm()
PEAKS = {"fp32": PEAK_FP32, "fp64": PEAK_FP64,
         "source": "derived: 152 SM x (2 FP64 | 128 FP32) FMA/clk x 2.07 GHz"}


def measure_peaks(torch, ctx, stream):
    """Measured arithmetic peaks of this GPU (bem_peak_probe): FP32 and FP64 FMA
    rates and the special-function unit's reciprocal square root and sine/cosine
    rates, each the best of three launches of about 20 ms timed with CUDA events
    on the library's stream (after one warm-up launch)."""
    trips = {0: 20000, 1: 300, 2: 2500, 3: 1250, 4: 20000}
    names = {0: "fp32_fma_tflops", 1: "fp64_fma_tflops", 2: "mufu_rsqrt_tops",
             3: "mufu_sincos_tops", 4: "fp32x2_fma_tflops"}
    out = {}
    for kind, n in trips.items():
        ctx.bem_peak_probe(kind, n)
        best = 0.0
        for _ in range(3):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ops = ctx.bem_peak_probe(kind, n)
            b.record(stream)
            b.synchronize()
            best = max(best, ops / (a.elapsed_time(b) / 1e3) / 1e12)
        out[names[kind]] = round(best, 3)
    ctx.bem_sync()
    # the FP32 denominator is the faster of the scalar and the packed-pair FMA
    PEAKS.update({"fp32": max(out["fp32_fma_tflops"], out["fp32x2_fma_tflops"]),
                  "fp64": out["fp64_fma_tflops"],
                  "mufu_rsqrt_tops": out["mufu_rsqrt_tops"],
                  "source": "measured on this GPU (bem_peak_probe), see peaks"})
    out["how"] = ("bem_peak_probe: 8 CTAs x 256 threads per SM, 8 independent chains per "
                  "thread; FMA = 2 operations (fma.rn.f32x2 = 4), sine and cosine = 2; best "
                  "of 3 launches; the FP32 rooflines divide by the larger FP32 rate")
    return out


def kernel_flops(w, counts, stats, precision):
    """{kernel class: (algorithmic flops per step, pipe, peak TFLOP/s)}."""
    q = w.quad
    npts_reg = (q.q_regular ** 2) ** 2 if q.regular_rule == "duffy" else 49
    np_axis = q.q_regular ** 2 if q.regular_rule == "duffy" else 7
    reg = counts["near_regular_pairs"] + counts["far_regular_pairs"]
    mixed = precision in ("mixed", "mixed_full")
    out = {}
    laplace_ops = [o for o in w.operators if o.kernel != "helmholtz_slp"]
    # the float forms cover the Laplace kernels, and Helmholtz on the P0 basis
    pipe = "fp32" if mixed and (w.basis == "p0" or len(laplace_ops) == len(w.operators)) else "fp64"
    coupling = mixed and w.basis == "p1" and pipe == "fp32"
    # plans fuse the single and double layer of the same P1 blocks in the float
    # forms: one launch evaluates both, so the work they share per point (the
    # difference 3, r^2 5, rsqrt 1) and, in the coupling engine, per test point
    # (x 6) counts once
    kinds = sorted(o.kernel for o in w.operators)
    fused = mixed and w.basis == "p1" and kinds == ["laplace_dlp", "laplace_slp"]
    if coupling:
        # coupling blocks run one entry per lane: deg(i) deg(j) pairs per entry,
        # per point the piecewise-constant count (the trial basis value is
        # folded into the trial weight), per test point 10 more (x 6, basis
        # value and weight 2, accumulation 2)
        reg = counts["near_regular_pairs"]
        f_cpl = sum(counts["far_entry_pairs"] * npts_reg *
                    (flops_per_point(o.kernel, "p0", np_axis) + 10.0 / np_axis)
                    for o in w.operators)
        if fused:
            f_cpl -= counts["far_entry_pairs"] * npts_reg * (9.0 + 6.0 / np_axis)
        out["coupling_p1"] = (f_cpl, "fp32")
    f_blk = sum(reg * npts_reg * flops_per_point(o.kernel, w.basis, np_axis) for o in w.operators)
    if fused:
        f_blk -= reg * npts_reg * 9.0
    out["block_p1" if w.basis == "p1" else "block_p0"] = (f_blk, pipe)
    for cas, qq, key in (("touching_vertex", q.q_vertex, "n_vertex"),
                         ("touching_edge", q.q_edge, "n_edge"),
                         ("touching_identical", q.q_identical, "n_identical")):
        f32 = precision == "mixed_full" or (mixed and cas == "touching_vertex")
        f = 0.0
        for o in w.operators:
            pts, fpp = touch_cost(cas.split("_")[1], o.kernel, w.basis, qq, f32)
            f += stats[key] * pts * fpp
        out[cas] = (f, "fp32" if f32 else "fp64")
    return {k: (f, p, PEAKS[p]) for k, (f, p) in out.items()}


def step_rates(w, counts, stats, precision, ms_per_step):
    """Triangle-pair integrals and quadrature points one step evaluates, and
    their rates: regular pairs as the chosen form's kernels evaluate them (once
    per block pair in the tile engines; once per entry and pair in the coupling
    engine of the float forms on the piecewise-linear basis), touching pairs
    once per mesh pair and case, for every operator."""
    q = w.quad
    npts_reg = (q.q_regular ** 2) ** 2 if q.regular_rule == "duffy" else 49
    mixed = precision in ("mixed", "mixed_full")
    laplace = all(o.kernel != "helmholtz_slp" for o in w.operators)
    coupling = mixed and w.basis == "p1" and laplace
    far = counts["far_entry_pairs"] if coupling else counts["far_regular_pairs"]
    regular = counts["near_regular_pairs"] + far
    touch_pairs = stats["n_vertex"] + stats["n_edge"] + stats["n_identical"]
    touch_points = (stats["n_vertex"] * 2 * q.q_vertex ** 4 + stats["n_edge"] * 4 * q.q_edge ** 4 +
                    stats["n_identical"] * 6 * q.q_identical ** 4)
    n_ops = len(w.operators)
    pairs = n_ops * (regular + touch_pairs)
    points = n_ops * (regular * npts_reg + touch_points)
    sec = ms_per_step / 1e3
    return {"pair_integrals_per_step": pairs, "quadrature_points_per_step": points,
            "pair_integrals_per_s": pairs / sec, "quadrature_points_per_s": points / sec}


def block_costs(bs):
    """Cost of each block of a block set: its number of entries."""
    rs = np.diff(bs.row_ptr)[bs.blk_row]
    cs = np.diff(bs.col_ptr)[bs.blk_col]
    return (rs * cs).astype(np.int64)


def shard_range(bs, rank, ws):
    """This rank's contiguous block range (lo, hi) of a block set (strong scaling)."""
    import paper_1510_07244_gb300 as pkg
    b = pkg.bem_shard_blocks(block_costs(bs), ws)
    return int(b[rank]), int(b[rank + 1])


def reduce_over_ranks(x, op, device=None):
    """x reduced over all ranks (MAX or SUM); x itself when not distributed."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()):
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX if op == "max" else tdist.ReduceOp.SUM)
    return float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def pair_counts(w):
    """Host-side accounting of the work one step performs (for the roofline):
    regular triangle pairs evaluated by the block kernel per block set, and the
    touching pairs per case."""
    import scipy.sparse as sp
    mesh = w.mesh
    nt, nv = mesh.nt, mesh.nv
    tri = mesh.tris
    # vertex -> triangle incidence
    VT = sp.csr_matrix((np.ones(3 * nt), (tri.ravel(), np.repeat(np.arange(nt), 3))),
                       shape=(nv, nt))
    # touching incidence: triangles sharing a vertex
    TT = (VT.T @ VT).tocsr()
    TT.data[:] = 1.0

    def block_pairs(bs):
        ncl = len(bs.row_ptr) - 1
        rows = np.repeat(np.arange(ncl), np.diff(bs.row_ptr))
        if w.basis == "p0":       # indices are triangles
            CT = sp.csr_matrix((np.ones(len(bs.row_idx)), (rows, bs.row_idx)), shape=(ncl, nt))
        else:
            CV = sp.csr_matrix((np.ones(len(bs.row_idx)), (rows, bs.row_idx)), shape=(ncl, nv))
            CT = (CV @ VT).tocsr()
        CT.data[:] = 1.0          # Ta(c): triangles touching cluster c
        size = np.asarray(CT.sum(axis=1)).ravel()
        touch = (CT @ TT @ CT.T).tocsr()
        t, s = bs.blk_row, bs.blk_col
        if len(t) == 0:
            return 0.0, 0.0
        total = float(np.sum(size[t] * size[s]))
        tp = float(np.asarray(touch[t, s]).ravel().sum())
        return total - tp, tp

    def entry_pairs(bs):
        # pairs summed entry by entry: sum over blocks of (sum deg i)(sum deg j)
        deg = np.bincount(w.mesh.tris.ravel(), minlength=nv).astype(np.float64)
        sdeg = np.add.reduceat(deg[bs.row_idx], bs.row_ptr[:-1]) if len(bs.row_idx) else np.zeros(0)
        sdeg[np.diff(bs.row_ptr) == 0] = 0.0
        return float(np.sum(sdeg[bs.blk_row] * sdeg[bs.blk_col]))

    near_reg, near_touch = block_pairs(w.near)
    far_reg, far_touch = block_pairs(w.far)
    out = {"near_regular_pairs": near_reg, "near_touching_lookups": near_touch,
           "far_regular_pairs": far_reg, "far_touching_lookups": far_touch}
    if w.basis == "p1":
        out["far_entry_pairs"] = entry_pairs(w.far)
    return out


def build_device_inputs(torch, pkg, w, dev, ranges=None):
    """Device copies of the block sets; with ranges = {"near": (lo, hi), ...} only
    those blocks (outputs keep the full layout, so shards write disjoint parts)."""
    def t32(a):
        return torch.as_tensor(np.ascontiguousarray(a, np.int32)).to(dev)

    def t64(a):
        return torch.as_tensor(np.ascontiguousarray(a, np.int64)).to(dev)

    sets = {}
    for name, bs in (("near", w.near), ("far", w.far)):
        lo, hi = ranges[name] if ranges else (0, len(bs.blk_row))
        costs = block_costs(bs)[lo:hi]
        # rows and columns from the same arrays share one device copy (and one
        # support table in the plan)
        rp, ri = t32(bs.row_ptr), t32(bs.row_idx)
        cp = rp if bs.col_ptr is bs.row_ptr else t32(bs.col_ptr)
        ci = ri if bs.col_idx is bs.row_idx else t32(bs.col_idx)
        sets[name] = dict(row_ptr=rp, row_idx=ri, col_ptr=cp,
                          col_idx=ci, blk_row=t32(bs.blk_row[lo:hi]),
                          blk_col=t32(bs.blk_col[lo:hi]), blk_off=t64(bs.blk_off[lo:hi]),
                          n=bs.n_entries, mine=int(costs.sum()))
    return sets


def make_jobs(torch, pkg, mid, w, sets, outs, precision="fp64"):
    quad = pkg.quad_desc(**w.quad.kw(), precision=precision)
    jobs = {"near": [], "far": []}
    for op in w.operators:
        kd = pkg.kernel_desc(op.kernel, op.kappa)
        for name in ("near", "far"):
            s = sets[name]
            jobs[name].append(pkg.BlockJob(mid, s["row_ptr"], s["row_idx"], s["col_ptr"], s["col_idx"],
                                           s["blk_row"], s["blk_col"], s["blk_off"],
                                           outs[(op.kernel, name)], kd, quad))
    return jobs


def use_gca_pivots(pkg, w, gauss_per_face=4, eps=1e-6):
    """Replaces the workload's coupling blocks by those over the host GCA's
    pivots (Sections 2.3-2.4); returns the GCA's wall time in seconds."""
    from synth import structure, workloads
    part = w.partition
    ptr, idx = part.cluster_csr()
    t0 = time.perf_counter()
    pp, pi = pkg.bem_gca_pivots(w.mesh.verts, w.mesh.tris, w.basis, ptr, idx, part.son_array(),
                                kappa=w.operators[0].kappa, gauss_per_face=gauss_per_face,
                                eps=eps, max_rank=w.meta["rank"])
    dt = time.perf_counter() - t0
    fr, fc, foff, ftot = structure.coupling_blocks(part, pp)
    w.far = workloads.BlockSet(pp, pi, pp, pi, fr, fc, foff, ftot)
    return dt


def error_scales(torch, pkg, ctx, dev, mid, v, quad_kw, outs64):
    """Per entry of one mesh's block sets and operators: max(A_ij, 1e-3 max_row A)
    with A_ij the sum of the magnitudes of its quadrature terms
    (bem_pivot_entries_absolute, FP64; the forward-error scale of the sum, by
    which the float forms are judged, as in the parity tests), and the row
    scale max(|g64|, 1e-3 max_row |g64|)."""
    scales = {}
    for nm in ("near", "far"):
        bs = getattr(v, nm)
        if bs.n_entries == 0:
            continue
        r, c = bs.entry_indices()
        rows = torch.as_tensor(np.ascontiguousarray(r, np.int32)).to(dev)
        cols = torch.as_tensor(np.ascontiguousarray(c, np.int32)).to(dev)
        rl = rows.long()
        for op in v.operators:
            A = torch.empty(bs.n_entries, dtype=torch.float64, device=dev)
            ctx.bem_pivot_entries_absolute(mid, pkg.kernel_desc(op.kernel, op.kappa),
                                           pkg.quad_desc(**quad_kw), rows, cols, A)
            a64 = outs64[(op.kernel, nm)][: bs.n_entries].abs()
            nrow = int(rl.max().item()) + 1
            rowmax = torch.zeros(nrow, dtype=a64.dtype, device=dev).scatter_reduce(
                0, rl, a64, reduce="amax")
            row = torch.maximum(a64, 1e-3 * rowmax[rl])
            amax = torch.zeros(nrow, dtype=A.dtype, device=dev).scatter_reduce(0, rl, A, reduce="amax")
            A = torch.maximum(A, 1e-3 * amax[rl])
            scales[(op.kernel, nm)] = (torch.where(A > 0, A, torch.ones_like(A)),
                                       torch.where(row > 0, row, torch.ones_like(row)))
        del rows, cols, rl
    ctx.bem_sync()
    return scales


def entry_errors(outs, outs64, scales):
    """(largest |g - g64| / A_ij, largest |g - g64| / row scale) over every entry."""
    e_abs = e_row = 0.0
    for key, (A, row) in scales.items():
        n = A.numel()
        d = (outs[key][:n] - outs64[key][:n]).abs()
        e_abs = max(e_abs, (d / A).max().item())
        e_row = max(e_row, (d / row).max().item())
    return e_abs, e_row


def run_ours(args):
    import torch
    import synth
    import paper_1510_07244_gb300 as pkg

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    w = synth.workloads.config2(args.levels)
    # the oracle's timed sample keeps the seeded pivot lists: no oracle input
    # comes from the library
    w_oracle = copy.copy(w)
    gca_s = use_gca_pivots(pkg, w) if args.pivots == "gca" else None
    stream = torch.cuda.current_stream(dev)
    ctx = pkg.Context(local, stream)
    mid = ctx.bem_mesh_upload(w.mesh.verts, w.mesh.tris, w.basis)
    ranges = None
    if args.split and ws > 1:
        ranges = {"near": shard_range(w.near, rank, ws), "far": shard_range(w.far, rank, ws)}
    sets = build_device_inputs(torch, pkg, w, dev, ranges)
    # entries this rank produces per step, and over all ranks
    entries_per_step = len(w.operators) * (sets["near"]["mine"] + sets["far"]["mine"])
    entries_all = reduce_over_ranks(entries_per_step, "sum", dev) if ws > 1 else entries_per_step
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    counts = pair_counts(w)
    stats = ctx.bem_mesh_info(mid)

    def run_form(precision, outs, steps):
        """Plan (one persistent launch per kernel bucket, CUDA graph, autotuned
        grids), warm-up, then `steps` timed graph replays, L2 flushed (untimed)
        before each."""
        jobs = make_jobs(torch, pkg, mid, w, sets, outs, precision)
        plan = ctx.bem_plan_create(jobs["near"], jobs["far"],
                                   pkg.PLAN_GRAPH | pkg.PLAN_AUTOTUNE | pkg.PLAN_PROFILE)

        def step():
            ctx.bem_plan_run(plan)

        for _ in range(args.warmup):
            step()
        ctx.bem_sync()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        ctx.bem_profile_reset()
        ctx.bem_profile_enable(True)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        for k in range(steps):
            flush.zero_()
            evs[k][0].record(stream)
            step()
            evs[k][1].record(stream)
        torch.cuda.synchronize(dev)
        ctx.bem_sync()
        if ws > 1:
            torch.distributed.barrier()
        prof = ctx.bem_profile_read()
        ctx.bem_profile_enable(False)
        info = ctx.bem_plan_info(plan)
        info["guard"] = ctx.bem_plan_guard_stats(plan)
        ctx.bem_plan_destroy(plan)
        total = reduce_over_ranks(float(sum(a.elapsed_time(b) for a, b in evs)), "max", dev)
        # kernels per replay: touching buckets, block engines, prefix sums and support builds
        info["kernels_per_step"] = (info["touch_launches"] + info["block_launches"] +
                                    info["aux_launches"])
        return total, prof, info

    def roofline(prof, precision, steps):
        model = kernel_flops(w, counts, stats, precision)
        per = {}
        for name, (launches, ms) in prof.items():
            if name in model:
                f, pipe, peak = model[name]
                ach = f * steps / (ms / 1e3) / 1e12
                per[name] = {"achieved": round(ach, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                             "pipe": pipe, "frac": round(ach / peak, 4), "ms": round(ms, 3),
                             "launches": launches, "avg_launch_ms": round(ms / launches, 4)}
        dom = max(prof.items(), key=lambda kv: kv[1][1])[0]
        r = dict(per.get(dom, {}))
        # DRAM bytes per launch from the committed ncu capture of the full-size
        # default workload (null for other sizes)
        traffic = profiled_traffic(dom) if args.levels == 5 and not args.split else None
        r.update({"bound": "alu", "kernel": dom, "traffic": traffic,
                  "peak_source": "derived: 152 SM x (2 FP64 | 128 FP32) FMA/clk x 2.07 GHz"})
        return r, per

    def alloc_outs():
        o = {}
        for op in w.operators:
            dt = torch.complex128 if op.kernel == "helmholtz_slp" else torch.float64
            for name in ("near", "far"):
                o[(op.kernel, name)] = torch.zeros(sets[name]["n"], dtype=dt, device=dev)
        return o

    def max_rel_err(outs, outs64):
        """(forward-error-scaled, row-scaled) largest difference to the FP64 form."""
        ea, er = entry_errors(outs, outs64, scales)
        return reduce_over_ranks(ea, "max", dev), reduce_over_ranks(er, "max", dev)

    # the FP64 form, then the two mixed forms; the headline is the fastest form
    # within 1e-6 of the FP64 form on every entry
    mixed_forms = ["mixed_full", "mixed"] if args.form == "auto" else [args.form]
    outs64 = alloc_outs()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    ms64, prof64, info64 = run_form("fp64", outs64, args.fp64_steps)
    forms = {}
    for f in mixed_forms:
        o = alloc_outs()
        ms, prof, info = run_form(f, o, args.steps)
        forms[f] = {"ms": ms, "prof": prof, "info": info, "outs": o,
                    "value": entries_all * args.steps / (ms / 1e3)}
    clk = clocks.stop()
    # accuracy (after the timed runs): every entry against the FP64 form
    scales = error_scales(torch, pkg, ctx, dev, mid, w, w.quad.kw(), outs64)
    for f in mixed_forms:
        forms[f]["max_rel_err"], forms[f]["max_row_err"] = max_rel_err(forms[f]["outs"], outs64)
    del scales
    ok = [f for f in mixed_forms if forms[f]["max_rel_err"] <= 1e-6]
    chosen = max(ok, key=lambda f: forms[f]["value"]) if ok else "fp64"
    chosen_ok = chosen != "fp64"
    value64 = entries_all * args.fp64_steps / (ms64 / 1e3)
    if chosen_ok:
        F = forms[chosen]
        value, steps_used, total_ms, prof, info = F["value"], args.steps, F["ms"], F["prof"], F["info"]
        outs, maxerr, rowerr = F["outs"], F["max_rel_err"], F["max_row_err"]
    else:
        value, steps_used, total_ms, prof, info = value64, args.fp64_steps, ms64, prof64, info64
        outs, maxerr, rowerr = outs64, 0.0, 0.0
    roof, per_kernel = roofline(prof, chosen, steps_used)
    roof64, per64 = roofline(prof64, "fp64", args.fp64_steps)
    launches = int(info["kernels_per_step"] * steps_used)
    other_forms = {f: {"value": F["value"], "ms_per_step": F["ms"] / args.steps,
                       "max_rel_err_vs_fp64_form": F["max_rel_err"],
                       "max_row_scaled_err": F["max_row_err"],
                       "kernels": roofline(F["prof"], f, args.steps)[1]}
                   for f, F in forms.items() if f != chosen}
    for f in list(forms):
        if f != chosen:
            del forms[f]["outs"]

    # end to end through the C ABI with host buffers
    e2e = None
    if args.e2e_steps > 0:
        pin = {}
        for name in ("near", "far"):
            bs = w.near if name == "near" else w.far
            keys = ["row_ptr", "row_idx", "blk_row", "blk_col", "blk_off"]
            if sets[name]["col_ptr"] is not sets[name]["row_ptr"]:
                keys += ["col_ptr", "col_idx"]      # columns not shared with the rows
            pin[name] = {k: torch.from_numpy(np.ascontiguousarray(getattr(bs, k),
                                                                  np.int64 if k == "blk_off" else np.int32)).pin_memory()
                         for k in keys}
        host_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in outs.items()}
        h2d = sum(t.numel() * t.element_size() for d in pin.values() for t in d.values())
        h2d += w.mesh.verts.nbytes + w.mesh.tris.nbytes
        d2h = sum(t.numel() * t.element_size() for t in host_out.values())
        times = []
        for k in range(args.e2e_steps + 1):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            mid2 = ctx.bem_mesh_upload(w.mesh.verts, w.mesh.tris, w.basis)
            for name in ("near", "far"):
                for key, t in pin[name].items():
                    sets[name][key].copy_(t, non_blocking=True)
            jobs2 = make_jobs(torch, pkg, mid2, w, sets, outs, chosen)
            ctx.bem_near_field(jobs2["near"])
            ctx.bem_coupling_blocks(jobs2["far"])
            for key, t in outs.items():
                host_out[key].copy_(t, non_blocking=True)
            torch.cuda.synchronize(dev)
            ctx.bem_sync()
            t1 = time.perf_counter()
            ctx.bem_mesh_free(mid2)
            if k > 0:
                times.append(t1 - t0)
        e2e = {"value": entries_per_step / statistics.mean(times), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "steps": len(times), "includes": "mesh upload + host planning, block lists H2D, "
                                                "all kernels, outputs D2H"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w_oracle, args.cpu_seconds)

    # the GCA's Green quadrature matrices of this workload's tree, timed after
    # everything above and outside the step: their own launches, their own key
    green = None
    if rank == 0 and ws == 1 and not args.no_green:
        try:
            green, _ = measure_green(torch, pkg, ctx, mid, w, dev, stream, args.steps,
                                     args.warmup)
        except Exception as e:      # recorded beside the headline, which is already measured
            green = {"error": f"{type(e).__name__}: {e}"}

    try:
        rates = step_rates(w, counts, stats, chosen, total_ms / steps_used)
    except Exception as e:       # an added figure never costs the headline line
        rates = {"error": f"{type(e).__name__}: {e}"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / steps_used, "higher_is_better": True,
                "scaling": "strong" if ranges else "weak", "vs_baseline": None,
                "dtype": "f32+f64 (mixed)" if chosen_ok else "f64", "data": "synthetic",
                "config": {"workload": w.name, "triangles": w.mesh.nt, "vertices": w.mesh.nv,
                           "basis": w.basis, "operators": [o.kernel for o in w.operators],
                           "entries_per_step": entries_per_step,
                           "near_entries": w.near.n_entries, "far_entries": w.far.n_entries,
                           "near_blocks": len(w.near.blk_row), "far_blocks": len(w.far.blk_row),
                           "pivots": ("host GCA, 4x4 Gauss points per face of omega_t, "
                                      "eps 1e-6, rank <= 16" if gca_s is not None
                                      else "seeded, rank <= 16"),
                           "gca_setup_s": gca_s,
                           "quadrature": w.quad.kw(), "precision": chosen,
                           "order_mode": "fixed",
                           "l2": "flushed between timed steps (256 MiB write, untimed)",
                           "pairs_per_step_per_operator": counts},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "driver": {"kind": "persistent batched plan, one CUDA graph replay per step",
                           "touch_launches": info["touch_launches"],
                           "block_launches": info["block_launches"],
                           "autotuned_ctas_per_sm": info["grid_mult"]},
                "kernels": per_kernel,
                "accuracy": {"max_rel_err_vs_fp64_form": maxerr, "bound": 1e-6,
                             "measure": "|g - g_fp64| / max(A, 1e-3 row max A), A = sum of "
                                        "|quadrature terms| (forward-error scale), every entry",
                             "max_row_scaled_err": rowerr,
                             "row_scaled": "|g - g_fp64| / max(|g_fp64|, 1e-3 row max)",
                             "entries_compared": entries_per_step},
                "rates": rates,
                "fp64_form": {"value": value64, "ms_per_step": ms64 / args.fp64_steps,
                              "steps": args.fp64_steps, "roofline": roof64, "kernels": per64},
                "other_forms": other_forms,
                "green_matrices": green,
                "clocks": clk}
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def sample_entries(w, n, seed):
    """Seeded uniform sample of (operator, row, col) over the step's entries."""
    import synth
    rng = synth.SplitMix64(seed)
    nr, nf = w.near.n_entries, w.far.n_entries
    tot = nr + nf
    pick = rng.integers(n, tot * len(w.operators))
    op = pick // tot
    k = pick % tot
    rn, cn = w.near.entry_indices()
    rf, cf = w.far.entry_indices()
    R = np.where(k < nr, rn[np.minimum(k, nr - 1)], rf[np.maximum(k - nr, 0)])
    C = np.where(k < nr, cn[np.minimum(k, nr - 1)], cf[np.maximum(k - nr, 0)])
    return op, R, C


def time_oracle(w, n, seed):
    import oracle
    op, R, C = sample_entries(w, n, seed)
    t0 = time.perf_counter()
    for i, o in enumerate(w.operators):
        sel = op == i
        if sel.any():
            oracle.entries(w.mesh.verts, w.mesh.tris, R[sel], C[sel], kernel=o.kernel, kappa=o.kappa,
                           basis=w.basis, **w.quad.kw())
    return time.perf_counter() - t0


def cpu_baseline(w, budget_s):
    import oracle
    oracle.build()
    n0 = 2000
    t0 = time_oracle(w, n0, 1)
    n = int(max(n0, min(5_000_000, n0 * budget_s / max(t0, 1e-3))))
    t = time_oracle(w, n, 2)
    return {"value": n / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} entries drawn uniformly (seeded) from the step's near-field and coupling "
                      f"entries of both operators; {t:.1f} s on {os.cpu_count()} OpenMP threads"}


def run_reference(args):
    """The oracle (plain FP64 C, OpenMP on all host cores) timed as it stands on
    the default line's workload, C4: each step a bounded seeded sample of the
    48 meshes' near-field and coupling entries of both operators (seeded pivot
    sets of the same sizes, so no oracle input comes from the library)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import types
    import synth
    import oracle
    oracle.build()
    bw = synth.workloads.config4()
    views = [types.SimpleNamespace(mesh=it.mesh, basis=bw.basis, quad=bw.quad,
                                   operators=it.operators, near=it.near, far=it.far)
             for it in bw.items]
    entries_per_step = bw.n_entries
    n0, t0 = batch_cpu_baseline(views, 0.0, seed=3)      # calibration sample
    per_step = args.ref_seconds_per_step
    n = int(max(2000, n0 * per_step / max(t0, 1e-3)))
    tot = np.array([len(v.operators) * (v.near.n_entries + v.far.n_entries) for v in views],
                   float)
    frac = tot / tot.sum()
    times, counts = [], []
    for k in range(args.warmup + args.steps):
        t, done = 0.0, 0
        for m, v in enumerate(views):
            c = int(round(n * frac[m]))
            if c > 0:
                t += time_oracle(v, c, 100 + 1000 * k + m)
                done += c
        if k >= args.warmup:
            times.append(t)
            counts.append(done)
    value = sum(counts) / sum(times)
    sample = (f"each step: {counts[0]} of the {entries_per_step} entries of the workload, drawn "
              f"uniformly (seeded) from every mesh's near-field and coupling entries of both "
              f"operators in proportion to its entries")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": bw.name, "entries_per_step": int(entries_per_step),
                       "precision": "fp64",
                       "pivots": "seeded, rank <= 16 (per-cluster counts as the host GCA's)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Further workloads (--workload c3 | c4): the same plan-driven step over one
# or many meshes, the FP64 form and the mixed forms timed and compared entry
# by entry.  These lines are measurements of the other configurations, not the
# default benchmark line.
# ---------------------------------------------------------------------------
def extra_items(name, args):
    """(workload name, basis, Quad, items); an item has mesh, operators, near, far,
    partition (for the host GCA)."""
    import synth
    if name == "c3":
        w = synth.workloads.config3()
        return w.name, w.basis, w.quad, [w]
    bw = synth.workloads.config4(args.c4_meshes)
    return bw.name, bw.basis, bw.quad, bw.items


def run_extra(args):
    import types
    import torch
    import paper_1510_07244_gb300 as pkg
    from synth import structure, workloads

    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    name, basis, quad, items = extra_items(args.workload, args)
    # host GCA pivots per mesh, with the largest wave number of its operators
    gca_s = 0.0
    if args.pivots == "gca":
        for it in items:
            ptr, idx = it.partition.cluster_csr()
            kappa = max(op.kappa for op in it.operators)
            t0 = time.perf_counter()
            pp, pi = pkg.bem_gca_pivots(it.mesh.verts, it.mesh.tris, basis, ptr, idx,
                                        it.partition.son_array(), kappa=kappa, gauss_per_face=4,
                                        eps=1e-6, max_rank=16)
            gca_s += time.perf_counter() - t0
            fr, fc, foff, ftot = structure.coupling_blocks(it.partition, pp)
            it.far = workloads.BlockSet(pp, pi, pp, pi, fr, fc, foff, ftot)
    stream = torch.cuda.current_stream(dev)
    ctx = pkg.Context(0, stream)
    views, mids, sets, counts, stats = [], [], [], [], []
    for it in items:
        v = types.SimpleNamespace(mesh=it.mesh, basis=basis, quad=quad, operators=it.operators,
                                  near=it.near, far=it.far)
        views.append(v)
        mids.append(ctx.bem_mesh_upload(it.mesh.verts, it.mesh.tris, basis))
        sets.append(build_device_inputs(torch, pkg, v, dev))
        counts.append(pair_counts(v))
        stats.append(ctx.bem_mesh_info(mids[-1]))
    entries = sum(len(v.operators) * (v.near.n_entries + v.far.n_entries) for v in views)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def alloc_outs():
        o = []
        for v in views:
            d = {}
            for op in v.operators:
                dt = torch.complex128 if op.kernel == "helmholtz_slp" else torch.float64
                for nm in ("near", "far"):
                    d[(op.kernel, nm)] = torch.zeros(max(1, getattr(v, nm).n_entries), dtype=dt,
                                                     device=dev)
            o.append(d)
        return o

    def run_form(precision, outs, steps, warmup):
        near, far = [], []
        for v, mid, st, o in zip(views, mids, sets, outs):
            j = make_jobs(torch, pkg, mid, v, st, o, precision)
            near += j["near"]
            far += j["far"]
        plan = ctx.bem_plan_create(near, far, pkg.PLAN_GRAPH | pkg.PLAN_AUTOTUNE | pkg.PLAN_PROFILE)
        for _ in range(warmup):
            ctx.bem_plan_run(plan)
        ctx.bem_sync()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        ctx.bem_profile_reset()
        ctx.bem_profile_enable(True)
        torch.cuda.synchronize(dev)
        for k in range(steps):
            flush.zero_()
            evs[k][0].record(stream)
            ctx.bem_plan_run(plan)
            evs[k][1].record(stream)
        torch.cuda.synchronize(dev)
        ctx.bem_sync()
        prof = ctx.bem_profile_read()
        ctx.bem_profile_enable(False)
        info = ctx.bem_plan_info(plan)
        info["guard"] = ctx.bem_plan_guard_stats(plan)
        ctx.bem_plan_destroy(plan)
        ms = float(sum(a.elapsed_time(b) for a, b in evs))
        info["kernels_per_step"] = (info["touch_launches"] + info["block_launches"] +
                                    info["aux_launches"])
        return ms, prof, info

    def roofline(prof, precision, steps):
        model = {}
        for v, c, st in zip(views, counts, stats):
            for k, (f, pipe, peak) in kernel_flops(v, c, st, precision).items():
                f0 = model.get(k, (0.0, pipe, peak))[0]
                model[k] = (f0 + f, pipe, peak)
        per = {}
        for kname, (launches, ms) in prof.items():
            if kname in model:
                f, pipe, peak = model[kname]
                ach = f * steps / (ms / 1e3) / 1e12
                per[kname] = {"achieved": round(ach, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                              "pipe": pipe, "frac": round(ach / peak, 4), "ms": round(ms, 3),
                              "launches": launches, "avg_launch_ms": round(ms / launches, 4)}
            else:
                per[kname] = {"ms": round(ms, 3), "launches": launches}
        return per

    def max_rel_err(outs, outs64):
        """(forward-error-scaled, row-scaled) largest difference over all meshes."""
        ea = er = 0.0
        for v, mid, o, o64 in zip(views, mids, outs, outs64):
            sc = error_scales(torch, pkg, ctx, dev, mid, v, quad.kw(), o64)
            a, r = entry_errors(o, o64, sc)
            ea, er = max(ea, a), max(er, r)
            del sc
        return ea, er

    forms = ["mixed_full", "mixed"] if args.form == "auto" else [args.form]
    clocks = Clocks(0)
    clocks.start()
    time.sleep(0.3)
    outs64 = alloc_outs()
    ms64, prof64, info64 = run_form("fp64", outs64, args.fp64_steps, 1)
    res = {}
    for f in forms:
        o = alloc_outs()
        ms, prof, info = run_form(f, o, args.steps, args.warmup)
        res[f] = {"value": entries * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps,
                  "kernels": roofline(prof, f, args.steps), "launches": info["kernels_per_step"],
                  "guard": info["guard"]}
        # accuracy outside the timed region, against the FP64 form on every entry
        res[f]["max_rel_err_vs_fp64_form"], res[f]["max_row_scaled_err"] = max_rel_err(o, outs64)
        del o
    clk = clocks.stop()
    ok = [f for f in forms if res[f]["max_rel_err_vs_fp64_form"] <= 1e-6]
    chosen = max(ok, key=lambda f: res[f]["value"]) if ok else None
    value64 = entries * args.fp64_steps / (ms64 / 1e3)
    head = res[chosen] if chosen else {"value": value64, "ms_per_step": ms64 / args.fp64_steps,
                                       "kernels": roofline(prof64, "fp64", args.fp64_steps),
                                       "launches": info64["kernels_per_step"]}
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps if chosen else args.fp64_steps, "warmup": args.warmup,
            "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64 (mixed)" if chosen else "f64",
            "data": "synthetic",
            "config": {"workload": name, "meshes": len(items),
                       "triangles": int(sum(v.mesh.nt for v in views)), "basis": basis,
                       "entries_per_step": int(entries), "quadrature": quad.kw(),
                       "precision": chosen or "fp64",
                       "pivots": "host GCA per mesh (4x4 Gauss points per face, eps 1e-6, rank <= 16)"
                                 if args.pivots == "gca" else "seeded, rank <= 16",
                       "gca_setup_s": gca_s if args.pivots == "gca" else None,
                       "l2": "flushed between timed steps (256 MiB write, untimed)"},
            "kernels": head["kernels"], "gpu_launches": int(head["launches"] *
                                                            (args.steps if chosen else args.fp64_steps)),
            "fp64_form": {"value": value64, "ms_per_step": ms64 / args.fp64_steps,
                          "steps": args.fp64_steps, "kernels": roofline(prof64, "fp64", args.fp64_steps)},
            "forms": {f: {k: r[k] for k in ("value", "ms_per_step", "max_rel_err_vs_fp64_form",
                                            "max_row_scaled_err", "guard")}
                      for f, r in res.items()},
            "accuracy": {"measure": "|g - g_fp64| / max(A, 1e-3 row max A), A = sum of |quadrature "
                                    "terms| (forward-error scale), every entry", "bound": 1e-6},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    ctx.close()


# ---------------------------------------------------------------------------
# Plan-driven workloads (C2, C3, C4): the FP64 form and the float forms, each
# one persistent plan (one CUDA graph replay per step) over all meshes of the
# workload, every entry of every float form compared with the FP64 form on
# both error measures; the chosen form is the fastest within 1e-6 on both.
# ---------------------------------------------------------------------------
# special-function operations per quadrature point of the float kernels:
# rsqrt for the Laplace kernels; Helmholtz adds the reciprocal of the phase
# offset and its sine and cosine (__fdividef, __sincosf)
def mufu_per_point(kernel: str, kclass: str, precision: str) -> float:
    if precision == "fp64":
        return 1.0
    # the float Helmholtz pair: reciprocal square root, sine and cosine
    if kernel == "helmholtz_slp" and kclass.startswith("block"):
        return 3.0
    return 1.0


def kernel_points(v, counts, stats, kernel, precision):
    """{kernel class: evaluation points per step} of one view and operator
    (touching cases as touch_cost counts them)."""
    q = v.quad
    npts = (q.q_regular ** 2) ** 2 if q.regular_rule == "duffy" else 49
    mixed = precision in ("mixed", "mixed_full")
    out = {}
    reg = counts["near_regular_pairs"] + counts["far_regular_pairs"]
    out["block_p1" if v.basis == "p1" else "block_p0"] = reg * npts
    for cas, qq, key in (("touching_vertex", q.q_vertex, "n_vertex"),
                         ("touching_edge", q.q_edge, "n_edge"),
                         ("touching_identical", q.q_identical, "n_identical")):
        f32 = precision == "mixed_full" or (mixed and cas == "touching_vertex")
        out[cas] = stats[key] * touch_cost(cas.split("_")[1], kernel, v.basis, qq, f32)[0]
    return out


def plan_workload(torch, pkg, ctx, dev, stream, name, basis, quad, items, forms, steps,
                  fp64_steps, warmup, gca=True, e2e_steps=0, flush=None, barrier=None,
                  reduce_ms=None):
    """Runs one plan-driven workload (items: mesh, operators, near, far,
    partition) in the FP64 form and the given float forms; returns a dict with
    the chosen form's value and per-kernel rooflines, every form's value and
    errors, the guard's statistics, and (e2e_steps > 0) the chosen form end to
    end through the per-call entry points with pinned host buffers."""
    import types
    from synth import structure, workloads
    gca_s = 0.0
    if gca:
        for it in items:
            ptr, idx = it.partition.cluster_csr()
            kappa = max(op.kappa for op in it.operators)
            t0 = time.perf_counter()
            pp, pi = pkg.bem_gca_pivots(it.mesh.verts, it.mesh.tris, basis, ptr, idx,
                                        it.partition.son_array(), kappa=kappa, gauss_per_face=4,
                                        eps=1e-6, max_rank=16)
            gca_s += time.perf_counter() - t0
            fr, fc, foff, ftot = structure.coupling_blocks(it.partition, pp)
            it.far = workloads.BlockSet(pp, pi, pp, pi, fr, fc, foff, ftot)
    views, mids, sets, counts, stats = [], [], [], [], []
    for it in items:
        v = types.SimpleNamespace(mesh=it.mesh, basis=basis, quad=quad, operators=it.operators,
                                  near=it.near, far=it.far)
        views.append(v)
        mids.append(ctx.bem_mesh_upload(it.mesh.verts, it.mesh.tris, basis))
        sets.append(build_device_inputs(torch, pkg, v, dev))
        counts.append(pair_counts(v))
        stats.append(ctx.bem_mesh_info(mids[-1]))
    entries = sum(len(v.operators) * (v.near.n_entries + v.far.n_entries) for v in views)
    if flush is None:
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def alloc_outs():
        o = []
        for v in views:
            d = {}
            for op in v.operators:
                dt = torch.complex128 if op.kernel == "helmholtz_slp" else torch.float64
                for nm in ("near", "far"):
                    d[(op.kernel, nm)] = torch.zeros(max(1, getattr(v, nm).n_entries), dtype=dt,
                                                     device=dev)
            o.append(d)
        return o

    def run_form(precision, outs, n_steps, n_warm):
        near, far = [], []
        for v, mid, st, o in zip(views, mids, sets, outs):
            j = make_jobs(torch, pkg, mid, v, st, o, precision)
            near += j["near"]
            far += j["far"]
        plan = ctx.bem_plan_create(near, far, pkg.PLAN_GRAPH | pkg.PLAN_AUTOTUNE | pkg.PLAN_PROFILE)
        for _ in range(n_warm):
            ctx.bem_plan_run(plan)
        ctx.bem_sync()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(n_steps)]
        ctx.bem_profile_reset()
        ctx.bem_profile_enable(True)
        if barrier:
            barrier()
        torch.cuda.synchronize(dev)
        for k in range(n_steps):
            flush.zero_()
            evs[k][0].record(stream)
            ctx.bem_plan_run(plan)
            evs[k][1].record(stream)
        torch.cuda.synchronize(dev)
        ctx.bem_sync()
        if barrier:
            barrier()
        prof = ctx.bem_profile_read()
        ctx.bem_profile_enable(False)
        info = ctx.bem_plan_info(plan)
        info["guard"] = ctx.bem_plan_guard_stats(plan)
        ctx.bem_plan_destroy(plan)
        ms = float(sum(a.elapsed_time(b) for a, b in evs))
        if reduce_ms:
            ms = reduce_ms(ms)          # the slowest rank's time
        info["kernels_per_step"] = (info["touch_launches"] + info["block_launches"] +
                                    info["aux_launches"])
        return ms, prof, info

    def roofline(prof, precision, n_steps):
        model, mufu = {}, {}
        for v, c, st in zip(views, counts, stats):
            for k, (f, pipe, peak) in kernel_flops(v, c, st, precision).items():
                f0 = model.get(k, (0.0, pipe, peak))[0]
                model[k] = (f0 + f, pipe, peak)
            # plans fuse the two Laplace layers of the same P1 blocks in the float
            # forms: one reciprocal square root per point serves both
            kinds = sorted(o.kernel for o in v.operators)
            fused = (precision in ("mixed", "mixed_full") and v.basis == "p1" and
                     kinds == ["laplace_dlp", "laplace_slp"])
            for i, o in enumerate(v.operators):
                for k, n in kernel_points(v, c, st, o.kernel, precision).items():
                    if fused and k == "block_p1" and i > 0:
                        continue
                    mufu[k] = mufu.get(k, 0.0) + n * mufu_per_point(o.kernel, k, precision)
        per = {}
        for kname, (launches, ms) in prof.items():
            if kname in model:
                f, pipe, peak = model[kname]
                ach = f * n_steps / (ms / 1e3) / 1e12
                per[kname] = {"achieved": round(ach, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                              "pipe": pipe, "frac": round(ach / peak, 4), "ms": round(ms, 3),
                              "launches": launches, "avg_launch_ms": round(ms / launches, 4)}
                if kname in mufu and PEAKS.get("mufu_rsqrt_tops"):
                    mach = mufu[kname] * n_steps / (ms / 1e3) / 1e12
                    per[kname]["mufu"] = {"achieved": round(mach, 4),
                                          "peak": PEAKS["mufu_rsqrt_tops"], "unit": "Tops/s",
                                          "frac": round(mach / PEAKS["mufu_rsqrt_tops"], 4)}
            else:
                per[kname] = {"ms": round(ms, 3), "launches": launches}
        return per

    def errors(outs, outs64):
        ea = er = 0.0
        for v, mid, o, o64 in zip(views, mids, outs, outs64):
            sc = error_scales(torch, pkg, ctx, dev, mid, v, quad.kw(), o64)
            a, r = entry_errors(o, o64, sc)
            ea, er = max(ea, a), max(er, r)
            del sc
        return ea, er

    outs64 = alloc_outs()
    ms64, prof64, info64 = run_form("fp64", outs64, fp64_steps, 1)
    res = {}
    keep = {}
    for f in forms:
        o = alloc_outs()
        ms, prof, info = run_form(f, o, steps, warmup)
        res[f] = {"value": entries * steps / (ms / 1e3), "ms_per_step": ms / steps,
                  "kernels": roofline(prof, f, steps), "launches": info["kernels_per_step"],
                  "guard": info["guard"], "grid_mult": info["grid_mult"]}
        res[f]["max_rel_err_vs_fp64_form"], res[f]["max_row_scaled_err"] = errors(o, outs64)
        keep[f] = o
    ok = [f for f in forms if max(res[f]["max_rel_err_vs_fp64_form"],
                                  res[f]["max_row_scaled_err"]) <= 1e-6]
    chosen = max(ok, key=lambda f: res[f]["value"]) if ok else None
    for f in forms:
        if f != chosen:
            del keep[f]
    value64 = entries * fp64_steps / (ms64 / 1e3)
    out = {"workload": name, "meshes": len(items),
           "triangles": int(sum(v.mesh.nt for v in views)), "basis": basis,
           "operators": sorted({o.kernel for v in views for o in v.operators}),
           "entries_per_step": int(entries), "quadrature": quad.kw(),
           "pivots": ("host GCA per mesh (4x4 Gauss points per face, eps 1e-6, rank <= 16)"
                      if gca else "seeded, rank <= 16"),
           "gca_setup_s": gca_s if gca else None,
           "chosen_form": chosen or "fp64",
           "fp64_form": {"value": value64, "ms_per_step": ms64 / fp64_steps, "steps": fp64_steps,
                         "kernels": roofline(prof64, "fp64", fp64_steps)},
           "forms": {f: {k: r[k] for k in ("value", "ms_per_step", "max_rel_err_vs_fp64_form",
                                           "max_row_scaled_err", "guard")}
                     for f, r in res.items()}}
    head = res[chosen] if chosen else None
    out["value"] = head["value"] if head else value64
    out["ms_per_step"] = head["ms_per_step"] if head else ms64 / fp64_steps
    out["kernels"] = head["kernels"] if head else out["fp64_form"]["kernels"]
    out["kernels_per_step"] = head["launches"] if head else info64["kernels_per_step"]
    out["grid_mult"] = head["grid_mult"] if head else info64["grid_mult"]
    out["steps"] = steps if head else fp64_steps
    out["speedup_vs_fp64_form"] = out["value"] / value64
    out["max_rel_err_vs_fp64_form"] = head["max_rel_err_vs_fp64_form"] if head else 0.0
    out["max_row_scaled_err"] = head["max_row_scaled_err"] if head else 0.0
    # triangle-pair integrals and quadrature points of one step of the reported form
    pairs = points = 0
    for v, c, st in zip(views, counts, stats):
        touch = st["n_vertex"] + st["n_edge"] + st["n_identical"]
        for o in v.operators:
            pairs += c["near_regular_pairs"] + c["far_regular_pairs"] + touch
            points += sum(kernel_points(v, c, st, o.kernel, chosen or "fp64").values())
    sec = out["ms_per_step"] / 1e3
    out["work"] = {"pair_integrals_per_step": int(pairs), "points_per_step": int(points),
                   "pair_integrals_per_s": pairs / sec, "points_per_s": points / sec,
                   "counted": "per operator: the regular pairs of the block kernels and the "
                              "touching pairs of the mesh's table; points of the rules as the "
                              "kernels run them; the guard's recomputations not counted"}

    if e2e_steps > 0:
        # end to end through the per-call entry points, host buffers in and out
        outs = keep[chosen] if chosen else outs64
        prec = chosen or "fp64"
        pin, host_out = [], []
        h2d = d2h = 0
        for v, st, o in zip(views, sets, outs):
            ph = {}
            for nm in ("near", "far"):
                bs = getattr(v, nm)
                keys = ["row_ptr", "row_idx", "blk_row", "blk_col", "blk_off"]
                if st[nm]["col_ptr"] is not st[nm]["row_ptr"]:
                    keys += ["col_ptr", "col_idx"]
                ph[nm] = {k: torch.from_numpy(np.ascontiguousarray(
                    getattr(bs, k), np.int64 if k == "blk_off" else np.int32)).pin_memory()
                    for k in keys}
                h2d += sum(t.numel() * t.element_size() for t in ph[nm].values())
            pin.append(ph)
            ho = {k: torch.empty(t.shape, dtype=t.dtype).pin_memory() for k, t in o.items()}
            d2h += sum(t.numel() * t.element_size() for t in ho.values())
            host_out.append(ho)
            h2d += v.mesh.verts.nbytes + v.mesh.tris.nbytes
        times, uploads = [], []
        for k in range(e2e_steps + 1):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            mids2 = []
            t_up = 0.0
            for v, st, o, ph, ho in zip(views, sets, outs, pin, host_out):
                tu = time.perf_counter()
                mid2 = ctx.bem_mesh_upload(v.mesh.verts, v.mesh.tris, basis)
                t_up += time.perf_counter() - tu
                mids2.append(mid2)
                for nm in ("near", "far"):
                    for key, t in ph[nm].items():
                        st[nm][key].copy_(t, non_blocking=True)
                j2 = make_jobs(torch, pkg, mid2, v, st, o, prec)
                ctx.bem_near_field(j2["near"])
                ctx.bem_coupling_blocks(j2["far"])
                for key, t in o.items():
                    ho[key].copy_(t, non_blocking=True)
            torch.cuda.synchronize(dev)
            ctx.bem_sync()
            t1 = time.perf_counter()
            for m2 in mids2:
                ctx.bem_mesh_free(m2)
            if k > 0:
                times.append(t1 - t0)
                uploads.append(t_up)
        out["e2e"] = {"value": entries / statistics.mean(times), "unit": UNIT,
                      "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                      "steps": len(times), "s_per_step": statistics.mean(times),
                      "mesh_upload_s_per_step": statistics.mean(uploads),
                      "includes": "per mesh: upload + host planning, block lists H2D, "
                                  "bem_near_field + bem_coupling_blocks, all outputs D2H"}
    for mid in mids:
        ctx.bem_mesh_free(mid)
    out["_views"] = views
    return out


def measure_c1(torch, pkg, ctx, dev, stream, steps, warmup, flush):
    """C1: the dense 1280 x 1280 Laplace single-layer matrix (P0, SS q=4, Radon
    7 x 7) through bem_assemble_dense, in the FP64 form and the float forms;
    every entry of each float form against the FP64 form (both measures)."""
    import synth
    w = synth.workloads.config1()
    n = w.mesh.nt
    mid = ctx.bem_mesh_upload(w.mesh.verts, w.mesh.tris, "p0")
    kd = pkg.kernel_desc("laplace_slp")

    def run(prec):
        qd = pkg.quad_desc(**w.quad.kw(), precision=prec)
        out = torch.zeros(n * n, dtype=torch.float64, device=dev)
        for _ in range(warmup):
            ctx.bem_assemble_dense(mid, kd, qd, 0, out)
        ctx.bem_sync()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        torch.cuda.synchronize(dev)
        for k in range(steps):
            flush.zero_()
            evs[k][0].record(stream)
            ctx.bem_assemble_dense(mid, kd, qd, 0, out)
            evs[k][1].record(stream)
        torch.cuda.synchronize(dev)
        ctx.bem_sync()
        return float(sum(a.elapsed_time(b) for a, b in evs)) / steps, out

    ms64, o64 = run("fp64")
    rows = torch.arange(n, dtype=torch.int32, device=dev).repeat_interleave(n)
    cols = torch.arange(n, dtype=torch.int32, device=dev).repeat(n)
    A = torch.empty(n * n, dtype=torch.float64, device=dev)
    ctx.bem_pivot_entries_absolute(mid, kd, pkg.quad_desc(**w.quad.kw()), rows, cols, A)
    ctx.bem_sync()
    # column-major output: entry (i, j) at j n + i; rows/cols above are row-major
    A = A.view(n, n).t().reshape(-1)
    g64 = o64.view(n, n)                      # [j, i]
    rmax = g64.abs().max(dim=0).values        # per row i
    row_scale = torch.maximum(g64.abs(), 1e-3 * rmax[None, :]).reshape(-1)
    Am = A.view(n, n)
    a_scale = torch.maximum(Am, 1e-3 * Am.max(dim=0).values[None, :]).reshape(-1)
    forms = {}
    for f in ("mixed_full", "mixed"):
        ms, o = run(f)
        d = (o - o64).abs()
        forms[f] = {"value": n * n / (ms / 1e3), "ms_per_step": ms,
                    "max_rel_err_vs_fp64_form": (d / a_scale).max().item(),
                    "max_row_scaled_err": (d / row_scale).max().item()}
    ctx.bem_mesh_free(mid)
    ok = [f for f in forms if max(forms[f]["max_rel_err_vs_fp64_form"],
                                  forms[f]["max_row_scaled_err"]) <= 1e-6]
    chosen = max(ok, key=lambda f: forms[f]["value"]) if ok else None
    head = forms[chosen] if chosen else {"value": n * n / (ms64 / 1e3), "ms_per_step": ms64}
    return {"workload": w.name, "triangles": n, "entries_per_step": n * n,
            "quadrature": w.quad.kw(), "call": "bem_assemble_dense (full matrix)",
            "chosen_form": chosen or "fp64", "value": head["value"],
            "ms_per_step": head["ms_per_step"], "steps": steps,
            "fp64_form": {"value": n * n / (ms64 / 1e3), "ms_per_step": ms64},
            "forms": forms}


# ---------------------------------------------------------------------------
# C5 (--workload c5): learned quadrature orders on the 131072-triangle sphere.
# The order model is trained first, on the GPU, from labels the method
# generates on two smaller spheres; then the plain FP64 form (fixed orders),
# the float form (fixed orders) and the chosen form (learned orders for the
# disjoint near-field pairs, float arithmetic) are timed, and their accuracy is
# judged on seeded sampled blocks against FP64 pivot entries at Duffy order 10
# (forward-error scale).
# ---------------------------------------------------------------------------
def run_c5(args, emit=True):
    import types
    import torch
    import synth
    import paper_1510_07244_gb300 as pkg
    from paper_1510_07244_gb300 import order_model as om
    from synth import structure, workloads
    from synth.rng import SplitMix64

    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    w = synth.workloads.config5(args.c5_n)
    stream = torch.cuda.current_stream(dev)
    ctx = pkg.Context(0, stream)

    def dev32(a):
        return torch.as_tensor(np.ascontiguousarray(a, np.int32)).to(dev)

    # ---- training: labels and features from the method on smaller meshes ----
    t0 = time.perf_counter()
    rng = SplitMix64(151007244 + 5000)
    Xs, ys = [], []
    for k, tm in enumerate(synth.workloads.order_training_meshes()):
        _, near, far = synth.workloads.h2_blocks(tm, "p0", 32, 2.0, 16, k + 1)
        mid = ctx.bem_mesh_upload(tm.verts, tm.tris, "p0")
        aa, bb = [], []
        # near-field pairs carry the hard cases: sampled five times as densely
        for bs, n_pick in ((near, 30000), (far, 6000)):
            r, c = bs.entry_indices()
            pick = rng.integers(min(n_pick, len(r)), len(r))
            aa.append(r[pick])
            bb.append(c[pick])
        a, b = np.concatenate(aa), np.concatenate(bb)
        t = tm.tris
        reg = ~np.array([len(set(t[i]) & set(t[j])) > 0 for i, j in zip(a, b)])
        ad, bd = dev32(a[reg]), dev32(b[reg])
        for op in w.operators:
            kd = pkg.kernel_desc(op.kernel, op.kappa)
            Xs.append(om.raw_features(ctx, mid, kd, ad, bd))
            ys.append(om.labels(ctx, mid, kd, ad, bd, tol=1e-7)[0])
        ctx.bem_mesh_free(mid)
    mlp, losses = om.fit(ctx, torch.cat(Xs), torch.cat(ys), epochs=40, batch=2048, lr=3e-3, seed=1)
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    n_train = int(sum(x.shape[0] for x in Xs))

    # ---- workload with GCA pivots ----
    ptr, idx = w.partition.cluster_csr()
    t0 = time.perf_counter()
    pp, pi = pkg.bem_gca_pivots(w.mesh.verts, w.mesh.tris, "p0", ptr, idx,
                                w.partition.son_array(), kappa=16.0, gauss_per_face=4, eps=1e-6,
                                max_rank=16)
    gca_s = time.perf_counter() - t0
    fr, fc, foff, ftot = structure.coupling_blocks(w.partition, pp)
    w.far = workloads.BlockSet(pp, pi, pp, pi, fr, fc, foff, ftot)
    mid = ctx.bem_mesh_upload(w.mesh.verts, w.mesh.tris, "p0")
    sets = build_device_inputs(torch, pkg, w, dev)
    entries = len(w.operators) * (w.near.n_entries + w.far.n_entries)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def alloc_outs():
        o = {}
        for op in w.operators:
            dt = torch.complex128 if op.kernel == "helmholtz_slp" else torch.float64
            for nm in ("near", "far"):
                o[(op.kernel, nm)] = torch.zeros(getattr(w, nm).n_entries, dtype=dt, device=dev)
        return o

    def timed(step, steps):
        for _ in range(args.warmup):
            step()
        ctx.bem_sync()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        torch.cuda.synchronize(dev)
        for k in range(steps):
            flush.zero_()
            evs[k][0].record(stream)
            step()
            evs[k][1].record(stream)
        torch.cuda.synchronize(dev)
        ctx.bem_sync()
        return float(sum(x.elapsed_time(y) for x, y in evs)) / steps

    def plan_form(precision, outs, steps):
        jobs = make_jobs(torch, pkg, mid, w, sets, outs, precision)
        plan = ctx.bem_plan_create(jobs["near"], jobs["far"], pkg.PLAN_GRAPH | pkg.PLAN_AUTOTUNE)
        ms = timed(lambda: ctx.bem_plan_run(plan), steps)
        ctx.bem_plan_destroy(plan)
        return ms

    def learned_form(outs, steps, conf):
        """The chosen form: learned orders + float arithmetic + one persistent
        plan (CUDA graph) over all four jobs."""
        ctx.bem_set_order_model(mlp, conf)
        quad = pkg.quad_desc(**w.quad.kw(), precision="mixed_full", order_mode="learned")
        near, far = [], []
        for op in w.operators:
            kd = pkg.kernel_desc(op.kernel, op.kappa)
            for nm, lst in (("near", near), ("far", far)):
                st = sets[nm]
                lst.append(pkg.BlockJob(mid, st["row_ptr"], st["row_idx"], st["col_ptr"],
                                        st["col_idx"], st["blk_row"], st["blk_col"],
                                        st["blk_off"], outs[(op.kernel, nm)], kd, quad))
        plan = ctx.bem_plan_create(near, far, pkg.PLAN_GRAPH | pkg.PLAN_AUTOTUNE | pkg.PLAN_PROFILE)
        ctx.bem_profile_reset()
        ctx.bem_profile_enable(True)
        ms = timed(lambda: ctx.bem_plan_run(plan), steps)
        prof = ctx.bem_profile_read()
        ctx.bem_profile_enable(False)
        counts = ctx.bem_plan_learned_counts(plan)
        info = ctx.bem_plan_info(plan)
        ctx.bem_plan_destroy(plan)
        runs = args.warmup + steps
        per_step = {k: round(v[1] / runs, 3) for k, v in prof.items()}
        per_step["kernels_per_step"] = info["touch_launches"] + info["block_launches"] + \
            info["aux_launches"]
        return ms, counts, per_step

    clocks = Clocks(0)
    clocks.start()
    time.sleep(0.3)
    o64, ofix = alloc_outs(), alloc_outs()
    ms64 = plan_form("fp64", o64, args.fp64_steps)
    msfix = plan_form("mixed_full", ofix, args.steps)
    confs = (0.95, 0.99, 0.999)
    lrn = {}
    for conf in confs:
        o = alloc_outs()
        ms, cnt, prof = learned_form(o, args.steps, conf)
        lrn[conf] = {"outs": o, "ms": ms, "counts": cnt, "kernels_ms_per_step": prof}
    clk = clocks.stop()

    # ---- accuracy on sampled whole blocks against FP64 Duffy q=10 ----
    srng = SplitMix64(151007244 + 5555)
    acc = {"fp64_fixed": 0.0, "mixed_full_fixed": 0.0}
    acc.update({f"learned_{c}": 0.0 for c in confs})
    n_cmp = 0
    qref = pkg.quad_desc(q_regular=10, regular_rule="duffy", q_identical=5, q_edge=5, q_vertex=5)
    for nm in ("near", "far"):
        bs = getattr(w, nm)
        blocks = srng.integers(min(150, len(bs.blk_row)), len(bs.blk_row))
        r_all, c_all = bs.entry_indices()
        sizes = np.diff(bs.row_ptr)[bs.blk_row] * np.diff(bs.col_ptr)[bs.blk_col]
        pos = np.concatenate([np.arange(bs.blk_off[b], bs.blk_off[b] + sizes[b]) for b in blocks])
        rr, cc = dev32(r_all[pos]), dev32(c_all[pos])
        posd = torch.as_tensor(pos).to(dev)
        n_cmp += len(pos) * len(w.operators)
        for op in w.operators:
            kd = pkg.kernel_desc(op.kernel, op.kappa)
            dt = torch.complex128 if op.kernel == "helmholtz_slp" else torch.float64
            ref = torch.empty(len(pos), dtype=dt, device=dev)
            A = torch.empty(len(pos), dtype=torch.float64, device=dev)
            ctx.bem_pivot_entries(mid, kd, qref, rr, cc, ref)
            ctx.bem_pivot_entries_absolute(mid, kd, qref, rr, cc, A)
            ctx.bem_sync()
            rl = rr.long()
            amax = torch.zeros(int(rl.max().item()) + 1, dtype=A.dtype, device=dev).scatter_reduce(
                0, rl, A, reduce="amax")
            A = torch.maximum(A, 1e-3 * amax[rl])
            A = torch.where(A > 0, A, torch.ones_like(A))
            forms_out = [("fp64_fixed", o64), ("mixed_full_fixed", ofix)] + \
                [(f"learned_{c}", lrn[c]["outs"]) for c in confs]
            for key, o in forms_out:
                e = ((o[(op.kernel, nm)][posd] - ref).abs() / A).max().item()
                acc[key] = max(acc[key], e)
    ctx.bem_set_order_model(None, 0.0)
    ctx.bem_mlp_destroy(mlp)
    sweep = {}
    for c in confs:
        cnt = lrn[c]["counts"]
        sweep[str(c)] = {"value": entries / (lrn[c]["ms"] / 1e3), "ms_per_step": lrn[c]["ms"],
                         "class_counts": cnt, "max_err": acc[f"learned_{c}"],
                         "kernels_ms_per_step": lrn[c]["kernels_ms_per_step"],
                         "points_per_disjoint_pair":
                             float(np.dot(cnt, pkg.ORDER_CLASS_POINTS)) / max(1, sum(cnt))}
    # the headline: the fastest confidence within the bound, else the most accurate
    ok = [c for c in confs if acc[f"learned_{c}"] <= 1e-6]
    conf = max(ok, key=lambda c: sweep[str(c)]["value"]) if ok else \
        min(confs, key=lambda c: acc[f"learned_{c}"])
    mslrn, counts, pts = lrn[conf]["ms"], lrn[conf]["counts"], sweep[str(conf)]["points_per_disjoint_pair"]
    # triangle-pair integrals and quadrature points of one learned step: the
    # disjoint pairs at their classes' rules, the touching pairs of the mesh's
    # table at the fixed singular rules, per operator
    st = ctx.bem_mesh_info(mid)
    tpairs = tpts = 0
    for op in w.operators:
        for cas, qq in (("vertex", w.quad.q_vertex), ("edge", w.quad.q_edge),
                        ("identical", w.quad.q_identical)):
            tpairs += st[f"n_{cas}"]
            tpts += st[f"n_{cas}"] * touch_cost(cas, op.kernel, "p0", qq, True)[0]
    wpairs = int(sum(counts) + tpairs)
    wpoints = int(float(np.dot(counts, pkg.ORDER_CLASS_POINTS)) + tpts)
    line = {"metric": METRIC, "value": entries / (mslrn / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mslrn,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64 (mixed)", "data": "synthetic",
            "config": {"workload": w.name, "triangles": w.mesh.nt, "basis": "p0",
                       "entries_per_step": int(entries), "quadrature": w.quad.kw(),
                       "precision": "mixed_full", "order_mode": "learned for every disjoint "
                       "pair (near field and coupling blocks); touching pairs at the fixed orders",
                       "driver": "one persistent plan (CUDA graph) over the four learned jobs",
                       "pivots": "host GCA (kappa 16)", "gca_setup_s": gca_s,
                       "l2": "flushed between timed steps (256 MiB write, untimed)"},
            "learned": {"class_counts": counts, "class_points": pkg.ORDER_CLASS_POINTS,
                        "points_per_disjoint_pair": pts, "confidence": conf,
                        "within_bound": bool(ok), "confidence_sweep": sweep,
                        "training": {"pairs": n_train, "seconds": train_s,
                                     "loss_first_last": [losses[0], losses[-1]],
                                     "meshes": "jittered octahedral spheres, 2048, 4608 and "
                                               "8192 triangles"}},
            "forms": {"fp64_fixed": {"value": entries / (ms64 / 1e3), "ms_per_step": ms64},
                      "mixed_full_fixed": {"value": entries / (msfix / 1e3), "ms_per_step": msfix},
                      "learned_mixed_full": {"value": entries / (mslrn / 1e3),
                                             "ms_per_step": mslrn, "confidence": conf}},
            "work": {"pair_integrals_per_step": wpairs, "points_per_step": wpoints,
                     "pair_integrals_per_s": wpairs / (mslrn / 1e3),
                     "points_per_s": wpoints / (mslrn / 1e3)},
            "accuracy": {"reference": "FP64 pivot entries at Duffy q=10 (same singular rules)",
                         "measure": "|g - g_ref| / max(A, 1e-3 row max A), A = sum of "
                                    "|quadrature terms of g_ref|",
                         "sampled_entries": n_cmp, "max_err": acc, "bound": 1e-6},
            "clocks": clk}
    ctx.close()
    if emit:
        print(json.dumps(line), flush=True)
    return line


# FP64 operations of the Green-matrix kernel (FMA = 2, rsqrt = 1, sincos = 2):
# per rule point the basis weight 2, the point x - z 12, r^2 5, rsqrt 1,
# (x - z).n 5, r^-3 and its products 4, two accumulations 3 (Laplace: 32);
# Helmholtz adds kappa r 2, sincos 2 and the phase products and two more
# accumulations 11 (47).  Per support triangle and point: edge vectors and
# z offset 9, scaled accumulation 4 (8 for Helmholtz).
def green_flops(helm: bool, np_rule: int) -> float:
    return (47.0 if helm else 32.0) * np_rule + (17.0 if helm else 13.0)


def green_workload(pkg, w, gauss_per_face=4, eps=1e-6):
    """The Green quadrature matrices the host GCA forms (Section 2.3) for the
    workload's cluster tree: leaves with all their indices, every other cluster
    with the rows t^ = pivots of its sons (nested bases), each against its
    6 gauss_per_face^2 box points.  Returns the cluster-CSR arrays of
    bem_green_matrices and the GCA's own wall time."""
    from synth.structure import green_point_sets
    part = w.partition
    tree = part.tree
    ptr, idx = part.cluster_csr()
    t0 = time.perf_counter()
    pp, pi = pkg.bem_gca_pivots(w.mesh.verts, w.mesh.tris, w.basis, ptr, idx, part.son_array(),
                                kappa=0.0, gauss_per_face=gauss_per_face, eps=eps,
                                max_rank=w.meta["rank"])
    gca_s = time.perf_counter() - t0
    clusters = list(range(tree.n_clusters))
    rows = []
    for c in clusters:
        if tree.is_leaf(c):
            rows.append(np.asarray(tree.indices(c), np.int64))
        else:
            rows.append(np.unique(np.concatenate([pi[pp[s]:pp[s + 1]] for s in tree.sons[c]])))
    row_ptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    pt_ptr, z, nz, sp, sm = green_point_sets(tree, clusters, gauss_per_face)
    sizes = 2 * np.diff(row_ptr).astype(np.int64) * np.diff(pt_ptr).astype(np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    return {"row_ptr": row_ptr, "rows": np.concatenate(rows).astype(np.int32), "pt_ptr": pt_ptr,
            "z": z, "nz": nz, "sp": sp, "sm": sm, "off": off, "total": int(sizes.sum()),
            "gca_s": gca_s, "piv_ptr": pp, "piv_idx": pi}


def measure_green(torch, pkg, ctx, mid, w, dev, stream, steps, warmup):
    """Times bem_green_matrices on the A_t the host GCA forms for the
    workload's tree (green_workload), Laplace and Helmholtz kappa = 8: `warmup`
    untimed launches, then `steps` launches, each bracketed by CUDA events on
    the context's stream, L2 flushed (256 MiB write, untimed) before each.
    Then the whole GCA with its A_t from the device (bem_gca_pivots_device,
    wall time, best of 3) beside the host GCA's time, and the number of
    clusters whose pivots differ from the host GCA's."""
    G = green_workload(pkg, w)
    d = {k: torch.as_tensor(G[k], device=dev) for k in ("row_ptr", "rows", "pt_ptr")}
    d.update({k: torch.as_tensor(G[k], dtype=torch.float64, device=dev)
              for k in ("z", "nz", "sp", "sm")})
    d["off"] = torch.as_tensor(G["off"], dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # support triangles per row: 1 (P0) or the vertex degree (P1)
    deg = (np.bincount(w.mesh.tris.ravel(), minlength=w.mesh.nv) if w.basis == "p1"
           else np.ones(w.mesh.nt, np.int64))
    m_c = np.diff(G["pt_ptr"]).astype(np.int64)
    cs = np.concatenate([[0], np.cumsum(deg[G["rows"]])])
    rows_deg = cs[G["row_ptr"][1:]] - cs[G["row_ptr"][:-1]]
    tri_pts = float((rows_deg * m_c).sum())
    res = {}
    for kernel, kappa in (("laplace_slp", 0.0), ("helmholtz_slp", 8.0)):
        helm = kernel == "helmholtz_slp"
        out = torch.empty(G["total"], dtype=torch.complex128 if helm else torch.float64,
                          device=dev)
        job = pkg.GreenJob(mid, d["row_ptr"], d["rows"], d["pt_ptr"], d["z"], d["nz"], d["off"],
                           out, sp=d["sp"], sm=d["sm"], kernel=pkg.kernel_desc(kernel, kappa),
                           rule="tri7")
        for _ in range(warmup):
            ctx.bem_green_matrices(job)
        ctx.bem_sync()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        torch.cuda.synchronize(dev)
        for k in range(steps):
            flush.zero_()
            evs[k][0].record(stream)
            ctx.bem_green_matrices(job)
            evs[k][1].record(stream)
        torch.cuda.synchronize(dev)
        ctx.bem_sync()
        ms = float(sum(a.elapsed_time(b) for a, b in evs))
        flops = tri_pts * green_flops(helm, 7)
        ach = flops * steps / (ms / 1e3) / 1e12
        res[kernel] = {"value": G["total"] * steps / (ms / 1e3), "unit": "entries/s",
                       "ms_per_step": ms / steps, "steps": steps,
                       "roofline": {"bound": "alu", "achieved": round(ach, 4),
                                    "peak": round(PEAKS["fp64"], 4), "unit": "TFLOP/s",
                                    "frac": round(ach / PEAKS["fp64"], 4), "traffic": None,
                                    "kernel": "green", "pipe": "fp64",
                                    "flops_per_step": flops,
                                    "peak_source": PEAKS["source"]}}
        del out
    del flush
    # the GCA with every level's A_t from the device and the cross approximation
    # on the host (bem_gca_pivots_device), beside the host GCA's own time
    part = w.partition
    ptr, idx = part.cluster_csr()
    times = []
    for _ in range(3):
        t0 = time.perf_counter()
        dpp, dpi = ctx.bem_gca_pivots_device(mid, w.mesh.verts, w.mesh.tris, w.basis, ptr, idx,
                                             part.son_array(), kappa=0.0, gauss_per_face=4,
                                             eps=1e-6, max_rank=w.meta["rank"])
        times.append(time.perf_counter() - t0)
    hpp, hpi = G["piv_ptr"], G["piv_idx"]
    differ = sum(1 for c in range(len(hpp) - 1)
                 if not np.array_equal(hpi[hpp[c]:hpp[c + 1]], dpi[dpp[c]:dpp[c + 1]]))
    res["gca_device"] = {"seconds": min(times), "host_gca_seconds": G["gca_s"],
                         "clusters": len(hpp) - 1, "clusters_with_other_pivots": differ}
    n_rows = int(G["row_ptr"][-1])
    res["workload"] = (f"A_t = (A_t+, A_t-) of all {len(m_c)} clusters of the {w.mesh.nt}-triangle "
                       f"{w.basis.upper()} tree (leaves with their indices, other clusters with "
                       f"their sons' GCA pivots): {n_rows} rows x {int(m_c.max())} box points "
                       f"(4 x 4 Gauss per face), Radon 7 per support triangle, FP64")
    res["entries_per_step"] = G["total"]
    res["host_gca_s"] = G["gca_s"]
    return res, G


def run_solves(args):
    """The Section 4 solves alone (the H2 product and CG, the Brakhage-Werner
    exterior problem), as they run under configs in the default line; one JSON
    line with both results."""
    import torch
    import paper_1510_07244_gb300 as pkg

    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = pkg.Context(0, stream)
    out = {"workload": "solves", "H2_solve": measure_h2_solve(torch, pkg, ctx, dev, stream),
           "BW_solve": measure_bw_solve(torch, pkg, ctx, dev, stream)}
    ctx.close()
    print(json.dumps(out))


def run_green(args):
    """Green quadrature matrices A_t of the GCA (Section 2.3) on the device:
    one bem_green_matrices launch per step over every cluster of the
    20480-triangle P1 icosphere's tree (measure_green), an end-to-end figure
    through host buffers, and the oracle on the host cores."""
    import torch
    import synth
    import paper_1510_07244_gb300 as pkg

    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    w = synth.workloads.config2(args.levels)
    stream = torch.cuda.current_stream(dev)
    ctx = pkg.Context(0, stream)
    mid = ctx.bem_mesh_upload(w.mesh.verts, w.mesh.tris, w.basis)
    clocks = Clocks(0)
    clocks.start()
    time.sleep(0.3)
    res, G = measure_green(torch, pkg, ctx, mid, w, dev, stream, args.steps, args.warmup)
    clk = clocks.stop()

    # end to end through the C ABI: host (pinned) inputs in, the matrices out
    host = {k: torch.as_tensor(G[k]).pin_memory() for k in ("row_ptr", "rows", "pt_ptr")}
    host.update({k: torch.as_tensor(G[k], dtype=torch.float64).pin_memory()
                 for k in ("z", "nz", "sp", "sm")})
    host["off"] = torch.as_tensor(G["off"], dtype=torch.int64).pin_memory()
    hout = torch.empty(G["total"], dtype=torch.float64).pin_memory()
    dd = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    dout = torch.empty(G["total"], dtype=torch.float64, device=dev)
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    job = pkg.GreenJob(mid, dd["row_ptr"], dd["rows"], dd["pt_ptr"], dd["z"], dd["nz"],
                       dd["off"], dout, sp=dd["sp"], sm=dd["sm"], rule="tri7")
    e2e_steps = max(1, args.e2e_steps)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for k, v in host.items():
            dd[k].copy_(v, non_blocking=True)
        ctx.bem_green_matrices(job)
        hout.copy_(dout, non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    ctx.bem_sync()

    cpu = None
    if not args.no_cpu_baseline:
        cpu = green_cpu_baseline(w, G, args.cpu_seconds)
    lap = res["laplace_slp"]
    line = {"metric": "Green quadrature matrix entries/s (A_t of the GCA, FP64)",
            "value": lap["value"], "unit": "entries/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": lap["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": res["workload"] + ", Laplace",
                       "entries_per_step": G["total"],
                       "l2": "flushed (256 MiB write) before each step"},
            "roofline": lap["roofline"],
            "helmholtz_kappa8": res["helmholtz_slp"],
            "e2e": {"value": G["total"] / e2e_s, "unit": "entries/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": G["total"] * 8},
            "host_gca_s": G["gca_s"],
            "gpu_launches": args.steps,
            "cpu_baseline": cpu,
            "clocks": clk}
    ctx.bem_mesh_free(mid)
    ctx.close()
    print(json.dumps(line))


def green_cpu_baseline(w, G, budget_s):
    """The oracle's Green entries on a seeded sample of the workload's (row,
    point) pairs, all host cores; entries/s counts plus and minus as two."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(151007244)
    n_cl = len(G["row_ptr"]) - 1
    row_cl = np.repeat(np.arange(n_cl), np.diff(G["row_ptr"]))

    def sample(n):
        r = rng.integers(0, len(G["rows"]), n)
        c = row_cl[r]
        p = G["pt_ptr"][c] + rng.integers(0, np.diff(G["pt_ptr"])[c])
        t0 = time.perf_counter()
        oracle.green_entries(w.mesh.verts, w.mesh.tris, w.basis, G["rows"][r], G["z"][p],
                             G["nz"][p], kappa=0.0, rule="tri7")
        return time.perf_counter() - t0

    n0 = 20000
    t0 = sample(n0)
    n = int(max(n0, min(50_000_000, n0 * budget_s / max(t0, 1e-3))))
    t = sample(n)
    return {"value": 2 * n / t, "unit": "entries/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} seeded (row, point) pairs of the step (two entries each); {t:.1f} s "
                      f"on {os.cpu_count()} OpenMP threads"}


def measure_h2_solve(torch, pkg, ctx, dev, stream, k=64, warmup=3, reps=20):
    """The interior Dirichlet problem of Section 4 on the octahedral sphere with
    8 k^2 triangles (P0; f1 = x1^2 - x3^2, Neumann data 2 f1): GCA bases on
    the host (at most 32 pivots per cluster, tolerance 1e-8), the single- and
    double-layer near-field and coupling blocks assembled on the device (FP64
    form), V in H2 form solved by conjugate gradients for the right-hand side
    (1/2 M + K) f1 (an H2 product).  Reports the H2 product's time and
    bandwidth (it is memory-bound: every stored entry is read once), the
    solve, and the Neumann error."""
    import synth
    from synth import structure, workloads
    mesh = synth.octasphere(k)
    n = mesh.nt
    v = mesh.verts[mesh.tris]
    area = 0.5 * np.linalg.norm(np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 1]), axis=1)
    c = v.mean(axis=1)
    f1 = c[:, 0] ** 2 - c[:, 2] ** 2
    part = structure.build_block_partition(mesh, "p0", 32, 2.0)
    ptr, idx = part.cluster_csr()
    son = part.son_array()
    t0 = time.perf_counter()
    pp, pi, mats = pkg.bem_gca_bases(mesh.verts, mesh.tris, "p0", ptr, idx, son, eps=1e-8,
                                     max_rank=32)
    gca_s = time.perf_counter() - t0
    nr, nc, no, ntot = part.near_blocks()
    fr, fc, fo, ftot = structure.coupling_blocks(part, pp)
    near = workloads.BlockSet(ptr, idx, ptr, idx, nr, nc, no, ntot)
    far = workloads.BlockSet(pp, pi, pp, pi, fr, fc, fo, ftot)
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    quad = pkg.quad_desc(q_regular=3, regular_rule="duffy", q_identical=5, q_edge=5, q_vertex=5)

    def dev_arr(a, dt):
        return torch.as_tensor(np.ascontiguousarray(a)).to(device=dev, dtype=dt)

    rp, ri = dev_arr(ptr, torch.int32), dev_arr(idx, torch.int32)
    pr, pq = dev_arr(pp, torch.int32), dev_arr(pi, torch.int32)
    vals, hs = {}, {}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for kern in ("laplace_slp", "laplace_dlp"):
        kd = pkg.kernel_desc(kern)
        nv_ = torch.zeros(max(1, ntot), dtype=torch.float64, device=dev)
        fv_ = torch.zeros(max(1, ftot), dtype=torch.float64, device=dev)
        ctx.bem_near_field([pkg.BlockJob(mid, rp, ri, rp, ri, dev_arr(nr, torch.int32),
                                         dev_arr(nc, torch.int32), dev_arr(no, torch.int64), nv_,
                                         kd, quad)])
        ctx.bem_coupling_blocks([pkg.BlockJob(mid, pr, pq, pr, pq, dev_arr(fr, torch.int32),
                                              dev_arr(fc, torch.int32), dev_arr(fo, torch.int64),
                                              fv_, kd, quad)])
        vals[kern] = (nv_, fv_)
    ev1.record(stream)
    ctx.bem_sync()
    assembly_ms = ev0.elapsed_time(ev1)
    hs["V"] = ctx.bem_h2_create(n, ptr, idx, son, pp, pi, mats, (nr, nc, no), vals["laplace_slp"][0],
                                (fr, fc, fo), vals["laplace_slp"][1])
    hs["K"] = ctx.bem_h2_create(n, ptr, idx, son, pp, pi, mats, (nr, nc, no), vals["laplace_dlp"][0],
                                (fr, fc, fo), vals["laplace_dlp"][1], diag=0.5 * area)
    x = torch.as_tensor(f1).to(dev)
    y = torch.empty(n, dtype=torch.float64, device=dev)
    for _ in range(warmup):
        ctx.bem_h2_matvec(hs["V"], x, y)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(reps)]
    torch.cuda.synchronize(dev)
    for a, b in evs:
        a.record(stream)
        ctx.bem_h2_matvec(hs["V"], x, y)
        b.record(stream)
    torch.cuda.synchronize(dev)
    mv_ms = min(a.elapsed_time(b) for a, b in evs)
    basis_elems = sum(np.asarray(m).size for m in mats)
    bytes_mv = 8.0 * (ntot + ftot + basis_elems) + 8.0 * 4 * n
    rhs = torch.empty(n, dtype=torch.float64, device=dev)
    ctx.bem_h2_matvec(hs["K"], x, rhs)
    alpha = torch.empty(n, dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    it, res = ctx.bem_h2_cg(hs["V"], rhs, alpha, tol=1e-8, maxit=5000)
    solve_s = time.perf_counter() - t0
    a_h = alpha.cpu().numpy()
    err = float(np.sqrt(np.sum(area * (a_h - 2 * f1) ** 2) / np.sum(area * (2 * f1) ** 2)))
    for h in hs.values():
        ctx.bem_h2_destroy(h)
    ctx.bem_mesh_free(mid)
    bw = bytes_mv / (mv_ms / 1e3) / 1e9
    return {"workload": f"interior Dirichlet problem, octahedral sphere {n} triangles, P0, "
                        f"f1 = x1^2 - x3^2 (Neumann data 2 f1)",
            "gca_bases_s": gca_s, "assembly_ms": assembly_ms,
            "near_entries": int(ntot), "coupling_entries": int(ftot),
            "basis_entries": int(basis_elems), "max_rank": int(np.diff(pp).max()),
            "matvec": {"ms": mv_ms, "bytes": bytes_mv, "achieved_gbs": bw,
                       "peak_gbs": MEASURED_HBM_GBS, "frac": bw / MEASURED_HBM_GBS,
                       "bound": "hbm", "note": "every stored entry read once per product"},
            "cg": {"iterations": it, "rel_residual": res, "seconds": solve_s, "tol": 1e-8},
            "neumann_rel_error_vs_2f1": err}


def measure_bw_solve(torch, pkg, ctx, dev, stream, ks=(16, 32), kappa=3.0, eta=3.0):
    """The exterior Helmholtz problem of Section 4 in the Brakhage-Werner form on
    the octahedral spheres with 8 k^2 triangles: f = g(x, (0, 0, 0.2)), kappa 3,
    eta 3.  The dense matrix K - i eta V (FP64, bem_assemble_dense), F by the
    Green-matrix call, (1/2 M + K - i eta V) w = F by GMRES, and the field at 24
    seeded exterior points against f.  Times the assembly and the solve."""
    import synth
    out = {"problem": "exterior Dirichlet problem, Brakhage-Werner form, f = g(x, (0,0,0.2)), "
                      "kappa 3, eta 3, P0, octahedral spheres", "meshes": []}
    z0 = np.array([0.0, 0.0, 0.2])
    for k in ks:
        mesh = synth.octasphere(k)
        n = mesh.nt
        mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
        quad = pkg.quad_desc(q_regular=3, regular_rule="duffy", q_identical=5, q_edge=5, q_vertex=5)
        A = torch.empty(n * n, dtype=torch.complex128, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ctx.bem_assemble_dense(mid, pkg.kernel_desc("helmholtz_bw", kappa, eta), quad, 0, A)
        ctx.bem_sync()
        e0.record(stream)
        ctx.bem_assemble_dense(mid, pkg.kernel_desc("helmholtz_bw", kappa, eta), quad, 0, A)
        e1.record(stream)
        ctx.bem_sync()
        asm_ms = e0.elapsed_time(e1)
        v = mesh.verts[mesh.tris]
        area = 0.5 * np.linalg.norm(np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 1]), axis=1)

        def d(a, dt):
            return torch.as_tensor(np.ascontiguousarray(a)).to(device=dev, dtype=dt)

        F = torch.empty(2 * n, dtype=torch.complex128, device=dev)
        job = pkg.GreenJob(mid, d([0, n], torch.int32), torch.arange(n, dtype=torch.int32,
                                                                       device=dev),
                           d([0, 1], torch.int32), d(z0[None, :], torch.float64),
                           d([[0.0, 0.0, 1.0]], torch.float64), d([0], torch.int64), F,
                           kernel=pkg.kernel_desc("helmholtz_slp", kappa), rule="duffy", q=5)
        ctx.bem_green_matrices(job)
        w = torch.empty(n, dtype=torch.complex128, device=dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        it, res = ctx.bem_dense_gmres(A, F[:n].contiguous(), w, diag=d(0.5 * area + 0j,
                                                                        torch.complex128),
                                      tol=1e-10, restart=100)
        solve_s = time.perf_counter() - t0
        rng = np.random.default_rng(3)
        dz = rng.standard_normal((24, 3))
        z = dz / np.linalg.norm(dz, axis=1)[:, None] * rng.uniform(1.5, 3.0, 24)[:, None]
        u = torch.empty(24, dtype=torch.complex128, device=dev)
        ctx.bem_potentials(mid, pkg.kernel_desc("helmholtz_bw", kappa, eta), d(z, torch.float64),
                           w, u, q=5)
        ctx.bem_sync()
        r = np.linalg.norm(z - z0, axis=1)
        f = np.exp(1j * kappa * r) / (4 * np.pi * r)
        err = float(np.abs(u.cpu().numpy() - f).max() / np.abs(f).max())
        ctx.bem_mesh_free(mid)
        out["meshes"].append({"triangles": n, "assembly_ms": asm_ms,
                              "entries_per_s": n * n / (asm_ms / 1e3),
                              "gmres_iterations": it, "gmres_rel_residual": res,
                              "solve_s": solve_s, "max_rel_field_error": err})
        del A
        torch.cuda.empty_cache()
    return out


def batch_cpu_baseline(views, budget_s, seed=1):
    """The oracle on a seeded sample of a batch's entries (all meshes, operators,
    near field and coupling blocks), sampled in proportion to each mesh's
    entries, on all host cores; entries/s."""
    import oracle
    oracle.build()
    tot = np.array([len(v.operators) * (v.near.n_entries + v.far.n_entries) for v in views],
                   float)
    frac = tot / tot.sum()

    def run(n, sd):
        t = 0.0
        done = 0
        for k, v in enumerate(views):
            m = int(round(n * frac[k]))
            if m <= 0:
                continue
            t += time_oracle(v, m, sd + k)
            done += m
        return done, t

    n0, t0 = run(4000, seed)
    if budget_s <= 0:
        return n0, t0
    # grow the sample until it takes about the budget (the first samples are
    # dominated by the per-mesh set-up of the oracle's calls)
    n, t, k = n0, t0, 0
    while t < 0.5 * budget_s and n < 50_000_000 and k < 4:
        n = int(min(50_000_000, max(2 * n, n * budget_s / max(t, 1e-3))))
        n, t = run(n, seed + 1000 * (k + 1))
        k += 1
    return n, t


def shard_items(items, rank, ws):
    """Contiguous cost-balanced ranges of a batch's meshes, one per rank (cost:
    entries x operators), from the library's shard planner (bem_shard_blocks)."""
    import paper_1510_07244_gb300 as pkg
    cost = np.array([len(it.operators) * (it.near.n_entries + it.far.n_entries) for it in items],
                    np.int64)
    b = pkg.bem_shard_blocks(cost, ws)
    return items[int(b[rank]):int(b[rank + 1])]


def run_all(args):
    """The default line: the largest configuration, C4 (48 meshes, 576 M entries
    per step, one plan), as the headline, with its roofline against measured
    peaks, the oracle on the host cores and the end-to-end figure; C1, C2, C3
    and C5 measured in the same run under `configs`; the Green matrices of
    C2's tree under `green_matrices`."""
    import torch
    import synth
    import paper_1510_07244_gb300 as pkg

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = pkg.Context(local, stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peaks = measure_peaks(torch, ctx, stream)
    bw = synth.workloads.config4(args.c4_meshes)
    items = shard_items(bw.items, rank, ws) if ws > 1 else bw.items
    barrier = (lambda: torch.distributed.barrier()) if ws > 1 else None
    reduce_ms = (lambda ms: reduce_over_ranks(ms, "max", dev)) if ws > 1 else None
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    forms = ["mixed_full", "mixed"] if args.form == "auto" else [args.form]
    r4 = plan_workload(torch, pkg, ctx, dev, stream, bw.name, bw.basis, bw.quad, items, forms,
                       args.steps, args.fp64_steps, args.warmup, gca=args.pivots == "gca",
                       e2e_steps=args.e2e_steps if ws == 1 else 0, flush=flush,
                       barrier=barrier, reduce_ms=reduce_ms)
    clk = clocks.stop()
    views = r4.pop("_views")
    entries_all = reduce_over_ranks(r4["entries_per_step"], "sum", dev) if ws > 1 else \
        r4["entries_per_step"]
    value = entries_all / (r4["ms_per_step"] / 1e3)
    if ws > 1:   # every rank's pairs and points over the slowest rank's time
        w4 = r4["work"]
        for k in ("pair_integrals", "points"):
            w4[f"{k}_per_step"] = int(reduce_over_ranks(w4[f"{k}_per_step"], "sum", dev))
            w4[f"{k}_per_s"] = w4[f"{k}_per_step"] / (r4["ms_per_step"] / 1e3)

    # roofline of the dominant kernel of the chosen form
    kern = r4["kernels"]
    dom = max((k for k in kern if "ms" in kern[k]), key=lambda k: kern[k]["ms"])
    roof = dict(kern[dom])
    # DRAM bytes per launch from the committed ncu summary (taken on 6 meshes,
    # scaled to the 48 by the entries; see its file), for the full workload only
    traffic = profiled_traffic(dom) if args.c4_meshes == 48 and ws == 1 else None
    roof.update({"bound": "alu", "kernel": dom, "traffic": traffic,
                 "peak_source": PEAKS["source"] + " (FP32 FMA probe; 'mufu': the reciprocal "
                                                  "square root probe)"})

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        n, t = batch_cpu_baseline(views, args.cpu_seconds)
        cpu = {"value": n / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n} entries drawn uniformly (seeded) from the 48 meshes' near-field "
                         f"and coupling entries of both operators, in proportion to each mesh's "
                         f"entries; {t:.1f} s on {os.cpu_count()} OpenMP threads"}

    configs = {}
    if ws == 1 and not args.headline_only:
        steps_x = max(3, args.steps // 2)
        for key, fn in (("C1", lambda: measure_c1(torch, pkg, ctx, dev, stream, steps_x,
                                                  args.warmup, flush)),
                        ("C2", lambda: _config_plan(torch, pkg, ctx, dev, stream, flush, args,
                                                    synth.workloads.config2(args.levels),
                                                    steps_x)),
                        ("C3", lambda: _config_plan(torch, pkg, ctx, dev, stream, flush, args,
                                                    synth.workloads.config3(), steps_x)),
                        ("C5", lambda: _config_c5(args, steps_x)),
                        ("H2_solve", lambda: measure_h2_solve(torch, pkg, ctx, dev, stream)),
                        ("BW_solve", lambda: measure_bw_solve(torch, pkg, ctx, dev, stream))):
            try:
                configs[key] = fn()
            except Exception as e:      # recorded beside the headline, already measured
                configs[key] = {"error": f"{type(e).__name__}: {e}"}
            torch.cuda.empty_cache()

    green = None
    if rank == 0 and ws == 1 and not args.no_green and not args.headline_only:
        try:
            w2 = synth.workloads.config2(args.levels)
            use_gca_pivots(pkg, w2)
            mid = ctx.bem_mesh_upload(w2.mesh.verts, w2.mesh.tris, w2.basis)
            green, _ = measure_green(torch, pkg, ctx, mid, w2, dev, stream, args.steps,
                                     args.warmup)
            ctx.bem_mesh_free(mid)
        except Exception as e:
            green = {"error": f"{type(e).__name__}: {e}"}

    if rank == 0:
        chosen = r4["chosen_form"]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": r4["steps"], "warmup": args.warmup, "ms_per_step": r4["ms_per_step"],
                "higher_is_better": True, "scaling": "strong" if ws > 1 else "weak",
                "vs_baseline": None,
                "dtype": "f32+f64 (mixed)" if chosen != "fp64" else "f64", "data": "synthetic",
                "config": {"workload": r4["workload"], "meshes": len(bw.items),
                           "triangles": int(sum(it.mesh.nt for it in bw.items)),
                           "basis": bw.basis, "operators": r4["operators"],
                           "entries_per_step": int(entries_all), "quadrature": r4["quadrature"],
                           "precision": chosen, "order_mode": "fixed",
                           "pivots": r4["pivots"], "gca_setup_s": r4["gca_setup_s"],
                           "sharding": (f"{ws} ranks, contiguous cost-balanced mesh ranges"
                                        if ws > 1 else None),
                           "l2": "flushed between timed steps (256 MiB write, untimed)"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": r4.get("e2e"),
                "gpu_launches": int(r4["kernels_per_step"] * r4["steps"]),
                "peaks": peaks,
                "accuracy": {"max_rel_err_vs_fp64_form": r4["max_rel_err_vs_fp64_form"],
                             "max_row_scaled_err": r4["max_row_scaled_err"], "bound": 1e-6,
                             "forward_error_scale": "|g - g_fp64| / max(A, 1e-3 row max A), "
                                                    "A = sum of |quadrature terms|",
                             "row_scaled": "|g - g_fp64| / max(|g_fp64|, 1e-3 row max |g_fp64|)"
                                           ", rows per mesh, operator and block set",
                             "entries_compared": int(r4["entries_per_step"])},
                "kernels": kern, "fp64_form": r4["fp64_form"], "forms": r4["forms"],
                "speedup_vs_fp64_form": r4["speedup_vs_fp64_form"], "work": r4.get("work"),
                "driver": {"kind": "persistent batched plan, one CUDA graph replay per step",
                           "autotuned_ctas_per_sm": r4["grid_mult"]},
                "configs": configs, "green_matrices": green, "clocks": clk}
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def _config_plan(torch, pkg, ctx, dev, stream, flush, args, w, steps):
    """One single-mesh workload (C2, C3) as a plan, with the oracle's rate."""
    from synth import workloads
    it = workloads.BatchItem(w.mesh, w.operators, w.near, w.far, w.partition)
    r = plan_workload(torch, pkg, ctx, dev, stream, w.name, w.basis, w.quad, [it],
                      ["mixed_full", "mixed"], steps, max(1, args.fp64_steps - 1), args.warmup,
                      gca=args.pivots == "gca", flush=flush)
    views = r.pop("_views")
    if not args.no_cpu_baseline:
        n, t = batch_cpu_baseline(views, 4.0)
        r["cpu_baseline"] = {"value": n / t, "unit": UNIT, "cores": os.cpu_count(),
                             "sample": f"{n} seeded entries, {t:.1f} s"}
    return r


def _config_c5(args, steps):
    """C5 (learned orders) through run_c5 with fewer timed steps."""
    a = copy.copy(args)
    a.steps = steps
    a.fp64_steps = 1
    line = run_c5(a, emit=False)
    for k in ("metric", "unit", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "data",
              "clocks"):
        line.pop(k, None)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="timed steps of the plain FP64 form (reported beside the chosen form)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-green", action="store_true",
                    help="skip the Green quadrature matrices reported beside the default line")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds-per-step", type=float, default=4.0)
    ap.add_argument("--split", action="store_true",
                    help="under torchrun: shard one workload's blocks across the ranks (strong "
                         "scaling) instead of one workload per rank (weak scaling)")
    ap.add_argument("--form", default="auto", choices=["auto", "mixed_full", "mixed"],
                    help="mixed form(s) timed beside the FP64 form; auto times both and "
                         "reports the fastest within 1e-6 of the FP64 form")
    ap.add_argument("--pivots", default="gca", choices=["gca", "seeded"],
                    help="coupling pivots from the host GCA (default) or seeded per cluster")
    ap.add_argument("--workload", default="all",
                    choices=["all", "c2", "c3", "c4", "c5", "green", "solves"],
                    help="all (default): the C4 headline (48 meshes) with C1, C2, C3 and C5 "
                         "under 'configs'; c2: the 20480-triangle P1 line alone; c3 / c4: the "
                         "49152-triangle Helmholtz cube / the 48-mesh batch alone; c5: learned "
                         "orders; green: the GCA's Green quadrature matrices A_t of the c2 tree")
    ap.add_argument("--headline-only", action="store_true",
                    help="with --workload all: only the C4 headline (no configs, no green)")
    ap.add_argument("--c5-n", type=int, default=128,
                    help="C5 sphere subdivision (8 n^2 triangles; 128 = the 131072-triangle "
                         "workload, smaller values only for profiling captures)")
    ap.add_argument("--c4-meshes", type=int, default=48,
                    help="meshes of the C4 batch (48 = the workload; fewer only for profiling "
                         "captures)")
    ap.add_argument("--levels", type=int, default=5,
                    help="icosphere refinement levels (5 = the 20480-triangle workload; "
                         "smaller values only for profiling captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be at least 3")
    ws_env = os.environ.get("WORLD_SIZE")
    if ws_env is None and args.gpus > 1:
        # start one rank per GPU on this node and hand back the launcher's status
        import socket
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
               f"--nproc-per-node={args.gpus}", "--master-addr=127.0.0.1",
               f"--master-port={port}", os.path.abspath(__file__)] + sys.argv[1:]
        raise SystemExit(subprocess.call(cmd))
    if ws_env is not None and int(ws_env) != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE={ws_env}: launch one rank per GPU")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "all":
        run_all(args)
    elif args.workload == "c5":
        run_c5(args)
    elif args.workload == "green":
        run_green(args)
    elif args.workload == "solves":
        run_solves(args)
    elif args.workload != "c2":
        run_extra(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
