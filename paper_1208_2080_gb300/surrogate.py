"""Learned temperature placement around the susceptibility peak.

A small network (the library's sw_mlp kernels: 3 -> 64 -> 64 -> 64 -> 4,
bfloat16 weights, fp32 accumulation, trained on the GPU) learns, from the
observables of a batch of SW runs, the map (q, log2 L, T/T_c) ->
(u, <|m|>, log chi, U4).  It is used only to decide WHERE to measure: for a
new (q, L) it predicts chi(T) on a fine grid and places the next temperature
grid around the predicted peak.  It never touches the Markov chain; the
measured sweeps at the placed temperatures decide its error, and
the plain uniform grid on [0.9, 1.1] T_c is the fallback and the comparison.

Observables of one run (configurations after a 10% burn-in), with
m = (q max_s n_s - N) / ((q - 1) N) per configuration:
  u = -<E_sat>/N,  <|m|>,  chi = N (<m^2> - <m>^2) / T,
  U4 = 1 - <m^4> / (3 <m^2>^2)   (Binder cumulant).
"""
import json
import math
import time

import numpy as np

import synth

from ._binding import MLP_PARAMS, Batch, Mlp


def run_observables(E, n, L, q, T, burn=0.1):
    """(u, <|m|>, chi, U4) of one run from its E_sat and n[s] series."""
    N = float(L) * float(L)
    k0 = int(len(E) * burn)
    E = np.asarray(E[k0:], dtype=np.float64)
    nn = np.asarray(n[k0:], dtype=np.float64)
    m = (q * nn.max(axis=1) - N) / ((q - 1) * N)
    m1, m2, m4 = m.mean(), (m * m).mean(), (m ** 4).mean()
    chi = N * (m2 - m1 * m1) / T
    u4 = 1.0 - m4 / (3.0 * m2 * m2) if m2 > 0 else 0.0
    return -E.mean() / N, m1, chi, u4


def features(q, L, T):
    q = np.asarray(q, dtype=np.float64)
    tc = np.array([synth.critical_temperature(int(x)) for x in np.atleast_1d(q)])
    return np.stack([q, np.log2(np.asarray(L, dtype=np.float64)), np.asarray(T) / tc], axis=1)


def measure_batch(L, q, T, seed, sweeps, burn=0.1, tile_h=64):
    """Run all replicas `sweeps` sweeps in one batch; returns the (R, 4)
    observables (u, <|m|>, chi, U4) and the device time in seconds."""
    import torch
    R = len(L)
    with Batch(L, q, T, seed, ring=sweeps + 1, tile_h=tile_h) as b:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.sweep(sweeps)
        b.sync()
        dt = time.perf_counter() - t0
        obs = np.zeros((R, 4))
        for r in range(R):
            E, n = b.series(r, 1, sweeps)
            obs[r] = run_observables(E, n, int(L[r]), int(q[r]), float(T[r]), burn)
    return obs, dt


def targets(obs):
    """Network targets: u, <|m|>, log chi, U4."""
    t = obs.copy()
    t[:, 2] = np.log(np.maximum(obs[:, 2], 1e-12))
    return t


class Surrogate:
    """The trained network plus the standardisation of its inputs/outputs."""

    def __init__(self, X, Y, seed=0):
        self.xm, self.xs = X.mean(0), X.std(0) + 1e-12
        self.ym, self.ys = Y.mean(0), Y.std(0) + 1e-12
        rng = np.random.default_rng(seed)
        init = np.zeros(MLP_PARAMS, dtype=np.float32)
        o = 0
        for fan_out, fan_in in [(64, 3), (64, 64), (64, 64), (4, 64)]:
            lim = math.sqrt(6.0 / (fan_in + fan_out))
            init[o:o + fan_out * fan_in] = rng.uniform(-lim, lim, fan_out * fan_in)
            o += fan_out * fan_in + fan_out  # biases start at zero
        self.net = Mlp(init)
        self.losses = []

    def fit(self, X, Y, steps=3000, lr=3e-3, log_every=100):
        import torch
        Xs = torch.tensor((X - self.xm) / self.xs, dtype=torch.float32, device="cuda")
        Ys = torch.tensor((Y - self.ym) / self.ys, dtype=torch.float32, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        for k in range(steps):
            lr_k = lr * 0.5 * (1 + math.cos(math.pi * k / steps)) + 1e-5
            self.net.train_step(Xs, Ys, None, lr_k, loss)
            if k % log_every == 0 or k == steps - 1:
                self.losses.append((k, float(loss.item())))
        return self.losses

    def predict(self, X):
        import torch
        Xs = torch.tensor((np.asarray(X) - self.xm) / self.xs, dtype=torch.float32, device="cuda")
        Y = torch.empty((Xs.shape[0], 4), dtype=torch.float32, device="cuda")
        self.net.forward(Xs, Y)
        torch.cuda.synchronize()
        return Y.cpu().numpy().astype(np.float64) * self.ys + self.ym

    def close(self):
        self.net.close()


def place_grid(model, q, L, n=32, lo=0.9, hi=1.1, fine=2001, min_width=0.04):
    """n temperatures around the predicted chi peak of (q, L): uniform over a
    window centred on the predicted peak, twice as wide as the predicted
    full width at half maximum but at least `min_width` T_c (the network's
    peak position is only as good as its training data), kept inside
    [lo, hi] T_c.  Falls back to the plain uniform grid if the prediction has
    no interior peak."""
    tc = synth.critical_temperature(q)
    t = np.linspace(lo, hi, fine)
    pred = model.predict(features(np.full(fine, q), np.full(fine, L), t * tc))
    lchi = pred[:, 2]
    k = int(np.argmax(lchi))
    if not np.all(np.isfinite(lchi)) or k in (0, fine - 1):
        return synth.temperature_grid(q, n, lo, hi), {"fallback": True}
    half = lchi[k] - math.log(2.0)
    left = k
    while left > 0 and lchi[left] > half:
        left -= 1
    right = k
    while right < fine - 1 and lchi[right] > half:
        right += 1
    fwhm = t[right] - t[left]
    W = min(max(2.0 * fwhm, min_width), hi - lo)
    a = min(max(lo, t[k] - 0.5 * W), hi - W)
    b = a + W
    return np.linspace(a, b, n) * tc, {"fallback": False, "t_peak_pred": float(t[k]),
                                       "fwhm_pred": float(fwhm), "window": [float(a), float(b)]}


def peak_estimate(T, chi):
    """Peak of chi(T) from grid measurements: vertex of the least-squares
    parabola through the maximum and up to two neighbours on each side."""
    T = np.asarray(T, dtype=np.float64)
    chi = np.asarray(chi, dtype=np.float64)
    k = int(np.argmax(chi))
    a, b = max(0, k - 2), min(len(T), k + 3)
    if b - a < 3:
        return float(T[k])
    c2, c1, _ = np.polyfit(T[a:b], chi[a:b], 2)
    if c2 >= 0:
        return float(T[k])
    v = -c1 / (2 * c2)
    return float(v) if T[a] <= v <= T[b - 1] else float(T[k])


def peak_estimate_dense(T, chi, frac=0.7):
    """Peak of chi(T) from a dense grid: vertex of the least-squares parabola
    in T through log chi at every point whose chi is at least `frac` of the
    largest (many points, so the noise of single points averages out)."""
    T = np.asarray(T, dtype=np.float64)
    chi = np.asarray(chi, dtype=np.float64)
    sel = chi >= frac * chi.max()
    if sel.sum() < 3:
        return float(T[int(np.argmax(chi))])
    c2, c1, _ = np.polyfit(T[sel], np.log(chi[sel]), 2)
    v = -c1 / (2 * c2) if c2 < 0 else float(T[int(np.argmax(chi))])
    return float(min(max(v, T[0]), T[-1]))


def train_on_batch(R=512, sweeps=2000, master_seed=6, steps=3000, seed=0):
    """Training set from one batched run (the replica mix of synth.replica_batch)
    and a trained Surrogate."""
    p = synth.replica_batch(R, master_seed=master_seed)
    obs, dt = measure_batch(p["L"], p["q"], p["T"], p["seed"], sweeps)
    X = features(p["q"], p["L"], p["T"])
    Y = targets(obs)
    model = Surrogate(X, Y, seed=seed)
    model.fit(X, Y, steps=steps)
    return model, {"R": R, "sweeps": sweeps, "run_s": dt, "final_loss": model.losses[-1][1]}


def compare_grids(model, qs=(2, 3, 4), Ls=(512, 1024, 2048), n=32, sweeps=5000, master_seed=7,
                  dense=96, dense_halfwidth=0.015):
    """For every (q, L): measure chi on the surrogate-placed grid and on the
    plain uniform grid (one batch each), estimate both peaks, and judge both
    against a dense reference grid (`dense` temperatures over +-`dense_halfwidth`
    around the uniform grid's estimate, the same sweeps; 0 skips it); report
    the surrogate's prediction error at the placed temperatures and at the
    peak."""
    rng = np.random.Generator(np.random.PCG64(master_seed))
    cells = [(q, L) for q in qs for L in Ls]
    grids, info = {}, {}
    for q, L in cells:
        grids[(q, L)], info[(q, L)] = place_grid(model, q, L, n)
    res = {}
    for name in ("surrogate", "uniform"):
        Lb, qb, Tb = [], [], []
        for q, L in cells:
            Ts = grids[(q, L)] if name == "surrogate" else synth.temperature_grid(q, n)
            Lb += [L] * n
            qb += [q] * n
            Tb += list(Ts)
        seeds = rng.integers(0, 2 ** 63, size=len(Lb), dtype=np.uint64)
        obs, dt = measure_batch(np.array(Lb, np.uint64), np.array(qb, np.uint32), np.array(Tb),
                                seeds, sweeps)
        res[name] = (np.array(Tb), obs, dt)
    # the judge: a dense grid around the uniform grid's estimate of every cell
    ref = {}
    if dense:
        Tu_all, ou_all, _ = res["uniform"]
        Lb, qb, Tb = [], [], []
        for c, (q, L) in enumerate(cells):
            sl = slice(c * n, (c + 1) * n)
            pu = peak_estimate(Tu_all[sl], ou_all[sl, 2])
            Lb += [L] * dense
            qb += [q] * dense
            Tb += list(np.linspace(pu * (1 - dense_halfwidth), pu * (1 + dense_halfwidth), dense))
        seeds = rng.integers(0, 2 ** 63, size=len(Lb), dtype=np.uint64)
        obs, dt = measure_batch(np.array(Lb, np.uint64), np.array(qb, np.uint32), np.array(Tb),
                                seeds, sweeps)
        res["dense"] = (np.array(Tb), obs, dt)
        for c, cell in enumerate(cells):
            sl = slice(c * dense, (c + 1) * dense)
            ref[cell] = (res["dense"][0][sl], obs[sl])
    out = {"sweeps": sweeps, "cells": []}
    for c, (q, L) in enumerate(cells):
        sl = slice(c * n, (c + 1) * n)
        tc = synth.critical_temperature(q)
        Ts, os_, _ = res["surrogate"]
        Tu, ou, _ = res["uniform"]
        ps = peak_estimate(Ts[sl], os_[sl, 2])
        pu = peak_estimate(Tu[sl], ou[sl, 2])
        pred = model.predict(features(np.full(n, q), np.full(n, L), Ts[sl]))
        meas = targets(os_[sl])
        width_u = (Tu[sl][1] - Tu[sl][0]) / tc
        width_s = (Ts[sl][1] - Ts[sl][0]) / tc
        half = os_[sl, 2] >= 0.5 * os_[sl, 2].max()
        half_u = ou[sl, 2] >= 0.5 * ou[sl, 2].max()
        out["cells"].append({
            "q": q, "L": L, "peak_T_over_Tc_surrogate_grid": ps / tc,
            "peak_T_over_Tc_uniform_grid": pu / tc, "rel_diff": abs(ps - pu) / pu,
            "grid_spacing_over_Tc": {"surrogate": width_s, "uniform": width_u},
            "points_above_half_max": {"surrogate": int(half.sum()), "uniform": int(half_u.sum())},
            "placement": info[(q, L)],
            "pred_rmse_at_placed_T": {k: float(np.sqrt(np.mean((pred[:, i] - meas[:, i]) ** 2)))
                                      for i, k in enumerate(["u", "m", "log_chi", "U4"])},
        })
        if (q, L) in ref:
            Td, od = ref[(q, L)]
            pd = peak_estimate_dense(Td, od[:, 2])
            cell = out["cells"][-1]
            cell["dense_reference"] = {
                "points": int(len(Td)), "spacing_over_Tc": float((Td[1] - Td[0]) / tc),
                "peak_T_over_Tc": pd / tc,
                # chi-peak errors of the two grids against the dense reference
                "rel_err_surrogate_grid": abs(ps - pd) / pd,
                "rel_err_uniform_grid": abs(pu - pd) / pd,
            }
            # the network against the reference: its predicted peak, next to
            # the infinite-volume T_c as a predictor, and its RMSE within
            # +-0.5% of the peak
            near = np.abs(Td - pd) <= 0.005 * pd
            predd = model.predict(features(np.full(int(near.sum()), q), np.full(int(near.sum()), L), Td[near]))
            measd = targets(od[near])
            t_pred = info[(q, L)].get("t_peak_pred")
            cell["network_at_peak"] = {
                "peak_rel_err_predicted": (abs(t_pred * tc - pd) / pd) if t_pred is not None else None,
                "peak_rel_err_Tc": abs(tc - pd) / pd,
                "rmse_within_0.5pct": {k: float(np.sqrt(np.mean((predd[:, i] - measd[:, i]) ** 2)))
                                       for i, k in enumerate(["u", "m", "log_chi", "U4"])},
                "points": int(near.sum()),
            }
    out["run_s"] = {k: v[2] for k, v in res.items()}
    out["max_rel_diff"] = max(c["rel_diff"] for c in out["cells"])
    if ref:
        out["max_rel_err_surrogate_grid"] = max(c["dense_reference"]["rel_err_surrogate_grid"]
                                                for c in out["cells"])
        out["max_rel_err_uniform_grid"] = max(c["dense_reference"]["rel_err_uniform_grid"]
                                              for c in out["cells"])
    return out


def main():
    import argparse
    ap = argparse.ArgumentParser(description="train the surrogate and compare temperature grids")
    ap.add_argument("--train-sweeps", type=int, default=2000)
    ap.add_argument("--sweeps", type=int, default=5000)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    t0 = time.time()
    model, tinfo = train_on_batch(sweeps=a.train_sweeps, steps=a.steps)
    res = compare_grids(model, sweeps=a.sweeps)
    res["training"] = tinfo
    res["losses"] = model.losses
    res["wall_s"] = time.time() - t0
    s = json.dumps(res, indent=1, default=float)
    if a.out:
        with open(a.out, "w") as f:
            f.write(s)
    print(s)


if __name__ == "__main__":
    main()
