"""FP64 CPU reference of the order model (8 -> 64 -> 64 -> 6, ReLU, softmax
cross entropy), with the library's parameter layout: W1[64][8] b1[64]
W2[64][64] b2[64] W3[6][64] b3[6]."""
import numpy as np

SHAPES = [("W1", (64, 8)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (6, 64)),
          ("b3", (6,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p):
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[k:k + n], np.float64).reshape(shape)
        k += n
    return out


def forward(p, X, bf16=False):
    P = unpack(p)
    rnd = bf16_round if bf16 else (lambda a: a)
    h0 = rnd(np.asarray(X, np.float64))
    z1 = h0 @ rnd(P["W1"]).T + P["b1"]
    h1 = rnd(np.maximum(z1, 0))
    z2 = h1 @ rnd(P["W2"]).T + P["b2"]
    h2 = rnd(np.maximum(z2, 0))
    z3 = h2 @ rnd(P["W3"]).T + P["b3"]
    return z1, h1, z2, h2, z3


def loss_and_grad(p, X, y):
    P = unpack(p)
    X = np.asarray(X, np.float64)
    n = X.shape[0]
    z1, h1, z2, h2, z3 = forward(p, X)
    z = z3 - z3.max(axis=1, keepdims=True)
    e = np.exp(z)
    prob = e / e.sum(axis=1, keepdims=True)
    loss = -np.mean(np.log(prob[np.arange(n), y]))
    dz3 = prob.copy()
    dz3[np.arange(n), y] -= 1.0
    dz3 /= n
    g = {"W3": dz3.T @ h2, "b3": dz3.sum(0)}
    dz2 = (dz3 @ P["W3"]) * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ P["W2"]) * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return loss, np.concatenate([g[name].ravel() for name, _ in SHAPES])


def bf16_round(a):
    """Round float64 values to bfloat16 (round to nearest even) and back."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
