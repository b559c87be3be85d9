"""Writes tests/golden/batch_c4.json: oracle results for every replica of the
512-replica batch (synth.replica_batch(512, master_seed=6)), 2000 sweeps each
from the init stream of the replica's seed.

Calls only the CPU oracle (oracle/) and the input generator (synth/).  Per
replica it stores the integer threshold, the SHA-256 of the final spins, of
the per-sweep E_sat series (configurations 1..2000, little-endian uint64) and
of the per-sweep n[s] series (2000 x q uint64), and the last E_sat / n[s].

Usage: python tests/golden/make_batch_golden.py [--workers 6] [--sweeps 2000]
(about 17 core-hours at 60 ns per site-sweep).
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)


def one(args):
    r, L, q, T, seed, sweeps = args
    import numpy as np
    import oracle
    spins, E, n = oracle.run(L, q, T, seed, sweeps)
    return r, {
        "L": L, "q": q, "T": T, "seed": str(seed), "thr": oracle.threshold(T), "sweeps": sweeps,
        "spins_sha256": hashlib.sha256(np.ascontiguousarray(spins).tobytes()).hexdigest(),
        "E_sha256": hashlib.sha256(E.astype("<u8").tobytes()).hexdigest(),
        "n_sha256": hashlib.sha256(n.astype("<u8").tobytes()).hexdigest(),
        "E_last": int(E[-1]), "n_last": [int(x) for x in n[-1]],
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=6)
    ap.add_argument("--sweeps", type=int, default=2000)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "batch_c4.json"))
    args = ap.parse_args()
    import synth
    b = synth.replica_batch(512, master_seed=6)
    jobs = [(r, int(b["L"][r]), int(b["q"][r]), float(b["T"][r]), int(b["seed"][r]), args.sweeps)
            for r in range(len(b["L"]))]
    jobs.sort(key=lambda j: -j[1])  # largest lattices first
    from oracle import build
    build.build()
    res = {}
    t0 = time.time()
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.workers) as pool:
        for k, (r, d) in enumerate(pool.imap_unordered(one, jobs)):
            res[r] = d
            if k % 16 == 0:
                print(f"{k + 1}/{len(jobs)} done, {time.time() - t0:.0f} s", flush=True)
    out = {"source": "oracle/ (CPU), synth.replica_batch(512, master_seed=6)",
           "sweeps": args.sweeps, "replicas": [res[r] for r in range(len(jobs))]}
    with open(args.out + ".tmp", "w") as f:
        json.dump(out, f, indent=0)
    os.replace(args.out + ".tmp", args.out)
    print("wrote", args.out, f"{time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
