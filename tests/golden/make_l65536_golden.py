"""Writes tests/golden/l65536_q2_10.json: oracle results for the production
size -- q = 2 at T_c = 1/ln(1 + sqrt 2), L = 65536, all-zero start, seed 5,
sweeps 0..9 (the first tenth of that configuration's 100 sweeps).

Calls only the CPU oracle (oracle/).  Stores the integer threshold, the
per-sweep E_sat and n[s] series (configurations 1..10) and the SHA-256 of
the spins after sweep 10.  Needs about 24 GB of host memory and an hour or
more of one core.

Usage: python tests/golden/make_l65536_golden.py
"""
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
L, Q, SEED, SWEEPS = 65536, 2, 5, 10


def main():
    import numpy as np
    import oracle
    T = oracle.tc(Q)
    t0 = time.time()
    spins = np.zeros((L, L), dtype=np.uint8)
    s, E, n = oracle.run(L, Q, T, SEED, SWEEPS, spins=spins)
    out = {"source": "oracle/ (CPU)", "L": L, "q": Q, "T": T, "seed": SEED, "start": "all-zero",
           "sweeps": SWEEPS, "thr": oracle.threshold(T),
           "E": [int(x) for x in E], "n": [[int(v) for v in row] for row in n],
           "spins_sha256": hashlib.sha256(np.ascontiguousarray(s).tobytes()).hexdigest(),
           "seconds": time.time() - t0}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "l65536_q2_10.json")
    with open(path + ".tmp", "w") as f:
        json.dump(out, f, indent=1)
    os.replace(path + ".tmp", path)
    print("wrote", path, f"{out['seconds']:.0f} s")


if __name__ == "__main__":
    main()
