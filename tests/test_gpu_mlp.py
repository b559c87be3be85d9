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
    o = 0
    for name, shp in omlp.SHAPES:
        n = int(np.prod(shp))
        assert _rel(gg[o:o + n], rg[o:o + n]) < 1e-2, name
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
    those temperatures agrees with the plain uniform grid's within 1%, and
    the placed grid samples the peak several times more densely."""
    from paper_1208_2080_gb300 import surrogate as sg
    model, info = sg.train_on_batch(R=512, sweeps=400, steps=2000)
    res = sg.compare_grids(model, qs=(2,), Ls=(512,), sweeps=2000)
    c = res["cells"][0]
    assert not c["placement"]["fallback"]
    assert c["rel_diff"] < 0.01, c
    assert c["grid_spacing_over_Tc"]["surrogate"] * 3 < c["grid_spacing_over_Tc"]["uniform"]
    assert c["points_above_half_max"]["surrogate"] >= 3 * c["points_above_half_max"]["uniform"]
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
