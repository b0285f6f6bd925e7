"""Order model: labels, training and persistence for BEM_ORDER_LEARNED.

Orchestration only: features, rule evaluations, training steps and inference
all run in the library's kernels (bem_pair_features, bem_pivot_entries,
bem_pivot_entries_absolute, bem_mlp_*); torch holds device buffers and does
the minibatch gathers.

Labels come from the method itself: for every training pair the six rule
classes (paper Section 2.2 Duffy rules of orders 2, 4, 5, 6, 8 and the
7-point Radon rule) are evaluated and compared with the same pair at a high
Duffy order (12);
the label is the cheapest class whose error is within `tol` times the sum of
the magnitudes of the pair's quadrature terms (the forward-error scale).
"""
import numpy as np

from ._binding import ORDER_CLASSES, kernel_desc, quad_desc


def _dev(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def pair_values(ctx, mesh_id, kernel, a, b, rule, q):
    """Pair integrals (P0 entries g_ab) of device pairs with one regular rule."""
    import torch
    cplx = kernel.kind == 2
    out = torch.empty(a.numel(), dtype=torch.complex128 if cplx else torch.float64, device="cuda")
    ctx.bem_pivot_entries(mesh_id, kernel, quad_desc(q_regular=q, regular_rule=rule), a, b, out)
    return out


def labels(ctx, mesh_id, kernel, a, b, tol=1e-7, q_ref=12):
    """(labels int32 device, errors n x 6 numpy) of disjoint pairs (a, b)."""
    import torch
    ref = pair_values(ctx, mesh_id, kernel, a, b, "duffy", q_ref)
    A = torch.empty(a.numel(), dtype=torch.float64, device="cuda")
    ctx.bem_pivot_entries_absolute(mesh_id, kernel, quad_desc(q_regular=q_ref), a, b, A)
    errs = []
    for rule, q in ORDER_CLASSES:
        v = pair_values(ctx, mesh_id, kernel, a, b, rule, q)
        errs.append(((v - ref).abs() / A.clamp_min(1e-300)).cpu().numpy())
    errs = np.stack(errs, axis=1)
    ok = errs <= tol
    lab = np.where(ok.any(axis=1), np.argmax(ok, axis=1), len(ORDER_CLASSES) - 1)
    return _dev(lab, torch.int32), errs


def raw_features(ctx, mesh_id, kernel, a, b):
    import torch
    X = torch.empty((a.numel(), 8), dtype=torch.float32, device="cuda")
    ctx.bem_pair_features(mesh_id, kernel, None, a, b, X)
    return X


def fit(ctx, X_raw, y, *, epochs=30, batch=2048, lr=3e-3, seed=0):
    """Trains a new model on raw features X_raw (n x 8, device) and labels y."""
    import torch
    Xh = X_raw.cpu().numpy().astype(np.float64)
    mean = Xh.mean(axis=0)
    std = Xh.std(axis=0)
    std = np.where(std > 1e-6, std, 1.0)
    norm = np.concatenate([mean, 1.0 / std]).astype(np.float32)
    mlp = ctx.bem_mlp_create(seed)
    ctx.bem_mlp_set_params(mlp, None, norm)
    Xn = ((X_raw - _dev(mean, torch.float32)) * _dev(1.0 / std, torch.float32)).contiguous()
    n = Xn.shape[0]
    rng = np.random.default_rng(seed)
    losses = []
    for _ in range(epochs):
        perm = _dev(rng.permutation(n), torch.int64)
        tot = 0.0
        for s in range(0, n, batch):
            idx = perm[s:s + batch]
            tot += ctx.bem_mlp_train_step(mlp, Xn[idx].contiguous(), y[idx].contiguous(), lr) * idx.numel()
        losses.append(tot / n)
    return mlp, losses


def predict(ctx, mlp, X_norm):
    import torch
    logits = torch.empty((X_norm.shape[0], 6), dtype=torch.float32, device="cuda")
    ctx.bem_mlp_infer(mlp, X_norm, logits)
    return logits


def save(ctx, mlp, path):
    p, q = ctx.bem_mlp_get_params(mlp)
    np.savez(path, params=p, norm=q)


def load(ctx, path):
    d = np.load(path)
    mlp = ctx.bem_mlp_create(0)
    ctx.bem_mlp_set_params(mlp, d["params"], d["norm"])
    return mlp
