"""Order model: labels, training and persistence for BEM_ORDER_LEARNED.

Orchestration only: features, rule evaluations, labels, the features'
normalisation, training steps and inference all run in the library's
kernels (bem_pair_features, bem_order_labels, bem_mlp_fit_norm,
bem_mlp_train_epoch, bem_mlp_infer); this module allocates device buffers,
draws the seeded minibatch permutations and keeps the loss history.

Labels come from the method itself (bem_order_labels): every training pair
is integrated with the six rule classes (Section 2.2 Duffy rules of orders
2, 4, 5, 6, 8 and the 7-point Radon rule) and with a high Duffy order (12);
the label is the cheapest class whose error is within `tol` times the sum of
the magnitudes of the pair's quadrature terms (the forward-error scale).
"""
import numpy as np

from ._binding import ORDER_CLASSES


def _dev(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def labels(ctx, mesh_id, kernel, a, b, tol=1e-7, q_ref=12):
    """(labels int32 device, errors n x 6 float32 device) of disjoint pairs (a, b)."""
    import torch
    lab = torch.empty(a.numel(), dtype=torch.int32, device="cuda")
    err = torch.empty((a.numel(), len(ORDER_CLASSES)), dtype=torch.float32, device="cuda")
    ctx.bem_order_labels(mesh_id, kernel, a, b, lab, err, tol=tol, q_ref=q_ref)
    return lab, err


def raw_features(ctx, mesh_id, kernel, a, b):
    import torch
    X = torch.empty((a.numel(), 8), dtype=torch.float32, device="cuda")
    ctx.bem_pair_features(mesh_id, kernel, None, a, b, X)
    return X


def fit(ctx, X_raw, y, *, epochs=30, batch=2048, lr=3e-3, seed=0):
    """Trains a new model on raw features X_raw (n x 8, device) and labels y:
    the normalisation from the features' statistics, then `epochs` epochs of
    seeded minibatch permutations."""
    import torch
    mlp = ctx.bem_mlp_create(seed)
    X = X_raw.contiguous()
    ctx.bem_mlp_fit_norm(mlp, X)
    n = X.shape[0]
    rng = np.random.default_rng(seed)
    losses = []
    for _ in range(epochs):
        perm = _dev(rng.permutation(n), torch.int64)
        losses.append(ctx.bem_mlp_train_epoch(mlp, X, y.contiguous(), perm, batch, lr))
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
