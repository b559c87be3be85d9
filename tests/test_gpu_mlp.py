"""The surrogate network's GPU kernels against the fp64 oracle (same
bfloat16-rounded weights and layer inputs), and the surrogate's use:
trained on a batched run, it places a temperature grid whose chi-peak
estimate agrees with the plain grid's while resolving the peak far more
finely."""
import numpy as np
import pytest

import paper_1208_2080_gb300 as sw
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def _setup(seed=0, B=300):
    import torch
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.25, omlp.N_PARAMS).astype(np.float32)
    X = rng.normal(size=(B, 3)).astype(np.float32)
    T = rng.normal(size=(B, 4)).astype(np.float32)
    mask = (rng.random((B, 4)) < 0.9).astype(np.float32)
    dev = lambda a: torch.tensor(a, device="cuda")
    return p, X, T, mask, dev


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


# ---- per-element error bounds of the fp32 / bfloat16 kernels against the
# fp64 oracle, derived from the arithmetic (the kernels use the oracle's
# rounded weights and inputs; see oracle/mlp.py):
#  * an fp32 sum of n products (fma chain) is within n * 2^-24 * sum|terms|;
#  * tanhf is within 2^-21 of tanh;
#  * a layer input is rounded to bfloat16 on both sides: if the GPU's fp32
#    activation is within e of the oracle's, the rounded values are equal
#    unless a rounding midpoint lies within e, and then differ by one
#    bfloat16 unit in the last place (2^-7 of the value's binade);
#  * these errors pass through |W| layer by layer, forward and backward.
U = 2.0 ** -24
TANH_ERR = 2.0 ** -21


def _bf16_ulp(a):
    a = np.abs(np.asarray(a, dtype=np.float64))
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -126)))
    return 2.0 ** (e - 7)


def _input_diff(a, e):
    """Bound on |r(a_gpu) - r(a)| when |a_gpu - a| <= e."""
    flip = omlp.bf16(a - e) != omlp.bf16(a + e)
    return np.where(flip, _bf16_ulp(np.abs(a) + e), 0.0)


def _bounds(p, X, T, mask):
    """Per-element bounds on |y|, |dL/dparams| (flat) of the kernels minus
    the oracle's."""
    B = X.shape[0]
    r = omlp.bf16
    w = {k: r(v) for k, v in omlp.unflatten(p).items()}
    x = r(X)
    y, (_, _, a1, a2, a3) = omlp.forward(p, X)
    # forward
    e_z1 = 4 * U * (np.abs(x) @ np.abs(w["W1"]).T + np.abs(w["b1"]))
    e_a1 = e_z1 + TANH_ERR
    d1 = _input_diff(a1, e_a1)
    e_z2 = d1 @ np.abs(w["W2"]).T + 65 * U * (np.abs(r(a1)) @ np.abs(w["W2"]).T + np.abs(w["b2"]))
    e_a2 = e_z2 + TANH_ERR
    d2 = _input_diff(a2, e_a2)
    e_z3 = d2 @ np.abs(w["W3"]).T + 65 * U * (np.abs(r(a2)) @ np.abs(w["W3"]).T + np.abs(w["b3"]))
    e_a3 = e_z3 + TANH_ERR
    d3 = _input_diff(a3, e_a3)
    e_y = d3 @ np.abs(w["W4"]).T + 65 * U * (np.abs(r(a3)) @ np.abs(w["W4"]).T + np.abs(w["b4"]))
    # backward
    scale = 2.0 / (4 * B)
    dy = scale * mask * (y - T)
    e_dy = scale * mask * e_y + 3 * U * np.abs(dy)

    def back(dz_next, e_next, W, a, e_a):
        s = dz_next @ W
        e_s = e_next @ np.abs(W) + (W.shape[0] + 1) * U * (np.abs(dz_next) @ np.abs(W))
        f = 1 - a * a
        e_f = 2 * np.abs(a) * e_a + e_a * e_a + 2 * U
        dz = s * f
        return dz, e_s * np.abs(f) + np.abs(s) * e_f + e_s * e_f + U * np.abs(dz)

    dz3, e_dz3 = back(dy, e_dy, w["W4"], a3, e_a3)
    dz2, e_dz2 = back(dz3, e_dz3, w["W3"], a2, e_a2)
    dz1, e_dz1 = back(dz2, e_dz2, w["W2"], a1, e_a1)

    def wgrad(dz, e_dz, inp, d_inp):
        acc = (B + 1) * U * (np.abs(dz).T @ np.abs(inp))
        return e_dz.T @ np.abs(inp) + np.abs(dz).T @ d_inp + e_dz.T @ d_inp + acc

    def bgrad(dz, e_dz):
        return e_dz.sum(0) + (B + 1) * U * np.abs(dz).sum(0)

    g = {"W4": wgrad(dy, e_dy, r(a3), d3), "b4": bgrad(dy, e_dy),
         "W3": wgrad(dz3, e_dz3, r(a2), d2), "b3": bgrad(dz3, e_dz3),
         "W2": wgrad(dz2, e_dz2, r(a1), d1), "b2": bgrad(dz2, e_dz2),
         "W1": wgrad(dz1, e_dz1, x, np.zeros_like(x)), "b1": bgrad(dz1, e_dz1)}
    return e_y, omlp.flatten(g)


def _adam_move_bound(g, e_g, lr, eps=1e-8):
    """Bound on the difference of the first Adam moves, -lr * g / (|g| + eps)
    (bias-corrected moments of one step), when the gradients differ by at
    most e_g: the mean-value bound of g / (|g| + eps), whose slope is at most
    eps / (|g| - e_g + eps)^2 away from 0 and 1 / eps across it."""
    far = np.abs(g) > e_g
    slope = np.where(far, eps / np.maximum(np.abs(g) - e_g + eps, eps) ** 2, 1.0 / eps)
    return lr * np.minimum(2.0, 2 * e_g * slope)


def test_forward_matches_oracle():
    import torch
    p, X, T, mask, dev = _setup()
    net = sw.Mlp(p)
    Y = torch.empty((X.shape[0], 4), device="cuda")
    net.forward(dev(X), Y)
    torch.cuda.synchronize()
    ref, _ = omlp.forward(p.astype(np.float64), X.astype(np.float64))
    for k in range(4):
        assert _rel(Y.cpu().numpy()[:, k], ref[:, k]) < 1e-2
    # element by element, within the bound derived from the arithmetic
    e_y, _ = _bounds(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64),
                     mask.astype(np.float64))
    err = np.abs(Y.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= 1.01 * e_y + 1e-12), float((err / (e_y + 1e-30)).max())
    # the bfloat16 copy is the rounded master
    m, b16 = net.params()
    assert np.array_equal(m, p)
    assert np.array_equal(((b16.astype(np.uint32) << 16).view(np.float32)).astype(np.float64),
                          omlp.bf16(p))
    net.close()


def test_gradients_match_oracle_per_tensor():
    import torch
    p, X, T, mask, dev = _setup(1)
    net = sw.Mlp(p)
    g = torch.zeros(omlp.N_PARAMS, device="cuda")
    loss = torch.zeros(1, device="cuda")
    net.gradients(dev(X), dev(T), dev(mask), g, loss)
    torch.cuda.synchronize()
    rl, rg = omlp.loss_and_grads(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64),
                                 mask.astype(np.float64))
    assert abs(loss.item() - rl) / rl < 1e-3
    gg = g.cpu().numpy().astype(np.float64)
    _, e_g = _bounds(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64),
                     mask.astype(np.float64))
    o = 0
    for name, shp in omlp.SHAPES:
        n = int(np.prod(shp))
        assert _rel(gg[o:o + n], rg[o:o + n]) < 1e-2, name
        # element by element, within the bound derived from the arithmetic
        err = np.abs(gg[o:o + n] - rg[o:o + n])
        assert np.all(err <= 1.01 * e_g[o:o + n] + 1e-12), (name, float((err / (e_g[o:o + n] + 1e-30)).max()))
        o += n
    net.close()


def test_adam_step_matches_oracle():
    import torch
    p, X, T, mask, dev = _setup(2)
    net = sw.Mlp(p)
    net.train_step(dev(X), dev(T), dev(mask), 1e-2)
    m, _ = net.params()
    _, rg = omlp.loss_and_grads(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64),
                                mask.astype(np.float64))
    w, _, _ = omlp.adam(p.astype(np.float64), rg, 0.0, 0.0, 1, lr=1e-2)
    # the first Adam step moves each weight by ~lr*sign(g): compare the moves
    assert _rel(m.astype(np.float64) - p, w - p) < 2e-2
    # element by element: the gradients differ within their bound, the move
    # by the mean-value bound of the update, plus fp32 rounding of the
    # update and of the new master weight
    _, e_g = _bounds(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64),
                     mask.astype(np.float64))
    bound = _adam_move_bound(rg, 1.01 * e_g + 1e-12, 1e-2) + 8 * U * (np.abs(p) + 1e-2)
    err = np.abs((m.astype(np.float64) - p) - (w - p))
    assert np.all(err <= bound), float((err / bound).max())
    net.close()


def test_training_reduces_loss_on_a_smooth_target():
    import torch
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, size=(512, 3)).astype(np.float32)
    Y = np.stack([np.sin(2 * X[:, 0]), X[:, 1] * X[:, 2], np.exp(-X[:, 0] ** 2), X.sum(1) / 3],
                 axis=1).astype(np.float32)
    from paper_1208_2080_gb300.surrogate import Surrogate
    s = Surrogate(X.astype(np.float64), Y.astype(np.float64), seed=0)
    s.fit(X.astype(np.float64), Y.astype(np.float64), steps=1500, lr=3e-3)
    first, last = s.losses[0][1], s.losses[-1][1]
    assert last < 0.05 * first, (first, last)
    pred = s.predict(X)
    assert np.sqrt(np.mean((pred - Y) ** 2)) < 0.1
    s.close()


def test_surrogate_grid_finds_the_peak_and_resolves_it():
    """Trained on a batched run of 512 mixed replicas, the network places 32
    temperatures for (q=2, L=512); the chi-peak estimated from sweeps at
    those temperatures agrees with the plain uniform grid's within 1%, the
    placed grid samples the peak several times more densely, and -- judged
    against a dense reference grid of 96 temperatures at the same sweeps --
    its peak is at least as close to the reference as the uniform grid's
    (within the reference's own spacing), and within 1%."""
    from paper_1208_2080_gb300 import surrogate as sg
    model, info = sg.train_on_batch(R=512, sweeps=400, steps=2000)
    res = sg.compare_grids(model, qs=(2,), Ls=(512,), sweeps=2000)
    c = res["cells"][0]
    assert not c["placement"]["fallback"]
    assert c["rel_diff"] < 0.01, c
    assert c["grid_spacing_over_Tc"]["surrogate"] * 3 < c["grid_spacing_over_Tc"]["uniform"]
    assert c["points_above_half_max"]["surrogate"] >= 3 * c["points_above_half_max"]["uniform"]
    d = c["dense_reference"]
    assert d["rel_err_surrogate_grid"] < 0.01, d
    assert d["rel_err_surrogate_grid"] <= max(d["rel_err_uniform_grid"], 2 * d["spacing_over_Tc"]), d
    model.close()


def test_predict_is_forward():
    import torch
    rng = np.random.default_rng(5)
    init = rng.uniform(-0.3, 0.3, omlp.N_PARAMS).astype(np.float32)
    X = torch.tensor(rng.uniform(-1, 1, (64, 3)), dtype=torch.float32, device="cuda")
    Y1 = torch.empty((64, 4), dtype=torch.float32, device="cuda")
    Y2 = torch.empty_like(Y1)
    m = sw.Mlp(init)
    m.forward(X, Y1)
    m.predict(X, Y2)
    torch.cuda.synchronize()
    m.close()
    assert torch.equal(Y1, Y2)
