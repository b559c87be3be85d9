"""Writes tests/golden/l8192_q234.json: oracle results for the L=8192
configuration -- q = 2, 3, 4 at T_c = 1/ln(1+sqrt q), random start from the
init stream of seed 2, 3, 4, 200 equilibration + 1000 measured sweeps.

Calls only the CPU oracle (oracle/).  Per q it stores the integer threshold,
the SHA-256 of the spins after sweeps 200 and 1200, of the per-sweep E_sat
series (configurations 1..1200, little-endian uint64) and of the n[s] series
(1200 x q), the measured-part averages of u = -E_sat/N and |M|/N, and the
last E_sat / n[s].

Usage: python tests/golden/make_l8192_golden.py [--workers 3]
(about 1.5 core-hours per q at 70 ns per site-sweep).
"""
import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
L, EQUIL, MEAS = 8192, 200, 1000


def one(q):
    import numpy as np
    import oracle
    T = 1.0 / math.log1p(math.sqrt(q))
    seed = q
    s200, E1, n1 = oracle.run(L, q, T, seed, EQUIL)
    s1200, E2, n2 = oracle.run(L, q, T, seed, MEAS, spins=s200, sweep0=EQUIL)
    E = np.concatenate([E1, E2])
    n = np.concatenate([n1, n2])
    N = L * L
    m = (q * n2.max(1).astype(np.float64) - N) / ((q - 1) * N)
    h = lambda a: hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()
    return q, {"q": q, "T": T, "seed": seed, "thr": oracle.threshold(T), "L": L,
               "equil": EQUIL, "measured": MEAS,
               "spins200_sha256": h(s200), "spins1200_sha256": h(s1200),
               "E_sha256": h(E.astype("<u8")), "n_sha256": h(n.astype("<u8")),
               "u_mean": float(-(E2.astype(np.float64) / N).mean()), "absM_mean": float(m.mean()),
               "E_last": int(E[-1]), "n_last": [int(x) for x in n[-1]]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=3)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "l8192_q234.json"))
    a = ap.parse_args()
    from oracle import build
    build.build()
    t0 = time.time()
    with mp.get_context("spawn").Pool(a.workers) as pool:
        res = dict(pool.map(one, [2, 3, 4]))
    out = {"source": "oracle/ (CPU)", "runs": [res[q] for q in (2, 3, 4)]}
    with open(a.out + ".tmp", "w") as f:
        json.dump(out, f, indent=1)
    os.replace(a.out + ".tmp", a.out)
    print("wrote", a.out, f"{time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
