"""A/B of the two labellers on the same equilibrium bond lattices: the tile
union-find with boundary merge (sw_label_bonds) against the paper's label
equivalence (sw_label_bonds_le; Sec. 2 quotes about 8.6 scan/analysis
iterations at q=2, T_c, 4096^2).  Both give bit-identical roots; this
reports their GPU times and the label-equivalence iteration count.

Usage: python -m paper_1208_2080_gb300.labeller_ab [--L 4096 16384] [--reps 5]
"""
import argparse
import json

from ._binding import Sim, label_bonds, label_bonds_le


def tc(q):
    import math
    return 1.0 / math.log1p(math.sqrt(q))


def ab(L, q=2, seed=11, equil=100, reps=5, samples=5):
    import torch
    out = {"L": L, "q": q, "samples": []}
    with Sim(L, q, tc(q), seed, store_bonds=True) as s:
        s.sweep(equil)
        for k in range(samples):
            s.sweep(1)
            packed = torch.from_numpy(s.bonds().reshape(-1).copy()).cuda()
            ra = torch.empty(L * L, dtype=torch.int32, device="cuda")
            rb = torch.empty_like(ra)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            label_bonds(L, packed, ra)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                label_bonds(L, packed, ra)
            e1.record()
            torch.cuda.synchronize()
            uf = e0.elapsed_time(e1) / reps
            it = label_bonds_le(L, packed, rb)
            e0.record()
            for _ in range(reps):
                it = label_bonds_le(L, packed, rb)
            e1.record()
            torch.cuda.synchronize()
            le = e0.elapsed_time(e1) / reps
            out["samples"].append({"uf_ms": uf, "le_ms": le, "le_iterations": it,
                                   "identical": bool(torch.equal(ra, rb))})
    its = [x["le_iterations"] for x in out["samples"]]
    out["le_iterations_mean"] = sum(its) / len(its)
    out["uf_ms_mean"] = sum(x["uf_ms"] for x in out["samples"]) / samples
    out["le_ms_mean"] = sum(x["le_ms"] for x in out["samples"]) / samples
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, nargs="+", default=[4096, 16384])
    ap.add_argument("--reps", type=int, default=5)
    a = ap.parse_args()
    print(json.dumps([ab(L, reps=a.reps) for L in a.L], indent=1))


if __name__ == "__main__":
    main()
