"""Run one workload of the library on the GPU and print a JSON summary.

    python -m paper_1208_2080_gb300.run potts --L 16384 --q 2 --sweeps 5
    python -m paper_1208_2080_gb300.run potts --L 65536 --sweeps 3 --host
    python -m paper_1208_2080_gb300.run xy --L 16384 --M 256 --sweeps 5
    python -m paper_1208_2080_gb300.run wolff --L 4096 --q 2 --steps 10 --mode label
    python -m paper_1208_2080_gb300.run batch --R 128 --sweeps 5 --tile-h 128

Temperatures default to the critical point of each model (T_c of the
q-state Potts model, T_KT of the XY model).  The start is all-zero; the time
is CUDA events around all sweeps / steps.  The batch is the replica mix of
the batched workload (L = 64..2048 log-uniform, q in {2,3,4,5,8}, T in
[0.9, 1.1] T_c(q); master seed 6), its first R replicas, from their seeded
random starts.  Used as the small, fixed cases that profiles are taken on.
"""
import argparse
import json


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("model", choices=["potts", "xy", "wolff", "batch"])
    ap.add_argument("--R", type=int, default=128)
    ap.add_argument("--tile-h", type=int, default=128)
    ap.add_argument("--merge", default="kernel", choices=["kernel", "fused"])
    ap.add_argument("--L", type=int, default=4096)
    ap.add_argument("--q", type=int, default=2)
    ap.add_argument("--M", type=int, default=256)
    ap.add_argument("--T", type=float, default=None)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--sweeps", type=int, default=5)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--label-bits", type=int, default=0)
    ap.add_argument("--mode", default="label", choices=["label", "grow"])
    ap.add_argument("--host", action="store_true")
    a = ap.parse_args()

    import torch

    import paper_1208_2080_gb300 as sw
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    N = a.L * a.L
    if a.model == "potts":
        T = sw.tc(a.q) if a.T is None else a.T
        with sw.Sim(a.L, a.q, T, a.seed, init="zero", label_bits=a.label_bits) as s:
            if a.host:
                host = torch.zeros(N, dtype=torch.uint8).pin_memory().numpy()
                e0.record(stream)
                for _ in range(a.sweeps):
                    E, n, cfg = s.sweep_host(host, 1)
                e1.record(stream)
            else:
                e0.record(stream)
                s.sweep(a.sweeps)
                e1.record(stream)
                E, n, cfg = s.measure()
            s.sync()
        out = {"E_sat": E, "n": [int(x) for x in n], "config": cfg}
        work = N * a.sweeps
    elif a.model == "batch":
        import synth
        p = synth.replica_batch(512, master_seed=6)
        R = a.R
        T = None
        with sw.Batch(p["L"][:R], p["q"][:R], p["T"][:R], p["seed"][:R], tile_h=a.tile_h, graph=False,
                      merge=a.merge) as b:
            e0.record(stream)
            b.sweep(a.sweeps)
            e1.record(stream)
            E, n, cfg = b.measure(0)
            b.sync()
        out = {"E_sat_0": E, "config": cfg, "R": R}
        work = float((p["L"][:R].astype("float64") ** 2).sum()) * a.sweeps
    elif a.model == "xy":
        T = sw.T_KT if a.T is None else a.T
        with sw.XY(a.L, a.M, T, a.seed, init="zero", label_bits=a.label_bits) as x:
            e0.record(stream)
            x.sweep(a.sweeps)
            e1.record(stream)
            D, n, cfg = x.measure()
            x.sync()
        out = {"D_sum": int(D.sum()), "config": cfg}
        work = N * a.sweeps
    else:
        T = sw.tc(a.q) if a.T is None else a.T
        with sw.Wolff(a.L, a.q, T, a.seed, init="zero", mode=a.mode) as w:
            e0.record(stream)
            w.step(a.steps)
            e1.record(stream)
            sizes = w.sizes(0, a.steps)
            w.sync()
        out = {"mean_cluster": float(sizes.mean())}
        work = float(sizes.sum())
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out.update({"model": a.model, "L": a.L, "T": T, "ms": ms, "per_ns": work / (ms * 1e6)})
    print(json.dumps(out))


if __name__ == "__main__":
    main()
