"""fp64 CPU oracle of the surrogate network (3 -> 64 -> 64 -> 64 -> 4, tanh).

TEST INFRASTRUCTURE ONLY (loaded by tests/ and nothing else); shares no code
with the CUDA kernels in paper_1208_2080_gb300/csrc/sw_mlp.cu.

The network is not part of the paper: it is the learned temperature-placement
aid.  Its arithmetic, written out plainly:
  parameters flat, in the order W1[64][3], b1[64], W2[64][64], b2[64],
  W3[64][64], b3[64], W4[4][64], b4[4] (8836 values);
  every parameter and every layer input is rounded to bfloat16 (round to
  nearest, ties to even) before use; sums are exact (fp64 here);
  z1 = W1 r(x) + b1, a1 = tanh(z1), z2 = W2 r(a1) + b2, a2 = tanh(z2),
  z3 = W3 r(a2) + b3, a3 = tanh(z3), y = W4 r(a3) + b4;
  loss = sum(mask * (y - t)^2) / (4B);
  gradients treat the rounding r() as the identity (straight-through), so
  they are the exact gradients of the same network without rounding,
  evaluated at the rounded values.
Adam (Kingma & Ba 2015) with bias correction updates fp32 master weights.
"""
import numpy as np

SHAPES = [("W1", (64, 3)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 64)),
          ("b3", (64,)), ("W4", (4, 64)), ("b4", (4,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(p):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(p[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def flatten(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p, X, rounding=True):
    r = bf16 if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    w = {k: r(v) for k, v in unflatten(p).items()}
    x = r(X)
    a1 = np.tanh(x @ w["W1"].T + w["b1"])
    a2 = np.tanh(r(a1) @ w["W2"].T + w["b2"])
    a3 = np.tanh(r(a2) @ w["W3"].T + w["b3"])
    y = r(a3) @ w["W4"].T + w["b4"]
    return y, (w, x, a1, a2, a3)


def loss_and_grads(p, X, T, mask=None, rounding=True):
    """(loss, flat gradient) of the masked mean-squared error."""
    r = bf16 if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    B = X.shape[0]
    mask = np.ones_like(T) if mask is None else mask
    y, (w, x, a1, a2, a3) = forward(p, X, rounding)
    d = mask * (y - T)
    loss = float((d * (y - T)).sum() / (4 * B))
    dy = 2.0 * d / (4 * B)
    g = {"W4": dy.T @ r(a3), "b4": dy.sum(0)}
    dz3 = (dy @ w["W4"]) * (1 - a3 ** 2)
    g["W3"], g["b3"] = dz3.T @ r(a2), dz3.sum(0)
    dz2 = (dz3 @ w["W3"]) * (1 - a2 ** 2)
    g["W2"], g["b2"] = dz2.T @ r(a1), dz2.sum(0)
    dz1 = (dz2 @ w["W2"]) * (1 - a1 ** 2)
    g["W1"], g["b1"] = dz1.T @ x, dz1.sum(0)
    return loss, flatten(g)


def adam(master, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (in fp64); returns new (master, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return master - lr * mh / (np.sqrt(vh) + eps), m, v
