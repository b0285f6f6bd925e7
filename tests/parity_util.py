"""Helpers of the GPU parity tests: device upload of block sets, the relative
error measure, and oracle evaluation of sampled entries."""
import numpy as np

import oracle


def rel_err(got, ref, row_ids):
    """|got - ref| / max(|ref|, 1e-3 * max |ref| over the same row), elementwise.

    Entries can be exactly zero (coplanar double layer), so each entry is
    measured against the largest entry of its row among the compared ones."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    row_ids = np.asarray(row_ids)
    scale = np.zeros(row_ids.max() + 1 if len(row_ids) else 1)
    np.maximum.at(scale, row_ids, np.abs(ref))
    den = np.maximum(np.abs(ref), 1e-3 * scale[row_ids])
    den = np.where(den > 0, den, 1.0)
    return np.abs(got - ref) / den


def rel_err_abs(got, ref, absint, row_ids):
    """|got - ref| / max(A, 1e-3 * max A over the same row), A = the oracle's sum
    of term magnitudes (oracle.entries_absolute).

    A floating-point evaluation of a quadrature sum has a forward error bounded
    by a multiple of the unit roundoff times the sum of the magnitudes of its
    terms; where the integrand changes sign (a double-layer pair whose test
    triangle straddles the trial triangle's plane) A exceeds |ref| and this is
    the measure that a fixed-precision evaluation can meet.  For integrands of
    one sign (single layer) A = |ref| and this equals rel_err."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    absint = np.asarray(absint)
    row_ids = np.asarray(row_ids)
    scale = np.zeros(row_ids.max() + 1 if len(row_ids) else 1)
    np.maximum.at(scale, row_ids, absint)
    den = np.maximum(absint, 1e-3 * scale[row_ids])
    den = np.where(den > 0, den, 1.0)
    return np.abs(got - ref) / den


def oracle_absolute(mesh, basis, rows, cols, kernel, kappa, quad):
    return oracle.entries_absolute(mesh.verts, mesh.tris, rows, cols, kernel=kernel, kappa=kappa,
                                   basis=basis, **quad)


def sample_block_entries(bs, n_blocks, rng):
    """Output positions of every entry of n_blocks seeded random blocks of a
    block set (whole blocks, so each row's scale is that of its block row)."""
    nb = len(bs.blk_row)
    picks = np.unique(rng.integers(min(n_blocks, nb), nb))
    pos = []
    for b in picks:
        t, s = bs.blk_row[b], bs.blk_col[b]
        n = (bs.row_ptr[t + 1] - bs.row_ptr[t]) * (bs.col_ptr[s + 1] - bs.col_ptr[s])
        pos.append(bs.blk_off[b] + np.arange(n))
    return np.concatenate(pos) if pos else np.zeros(0, np.int64)


def to_dev(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def block_job(pkg, mesh_id, bs, kernel, kappa, quad, out):
    """A job over a block set; row and column clusters given by the same host
    arrays share one device copy (and so one support table in a plan)."""
    import torch
    rp, ri = to_dev(bs.row_ptr, torch.int32), to_dev(bs.row_idx, torch.int32)
    cp = rp if bs.col_ptr is bs.row_ptr else to_dev(bs.col_ptr, torch.int32)
    ci = ri if bs.col_idx is bs.row_idx else to_dev(bs.col_idx, torch.int32)
    return pkg.BlockJob(mesh_id, rp, ri, cp, ci,
                        to_dev(bs.blk_row, torch.int32), to_dev(bs.blk_col, torch.int32),
                        to_dev(bs.blk_off, torch.int64), out,
                        pkg.kernel_desc(kernel, kappa), pkg.quad_desc(**quad))


def oracle_entries(mesh, basis, rows, cols, kernel, kappa, quad):
    z = oracle.entries(mesh.verts, mesh.tris, rows, cols, kernel=kernel, kappa=kappa,
                       basis=basis, **quad)
    return z if kernel.startswith("helmholtz") else z.real
