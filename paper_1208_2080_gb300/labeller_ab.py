"""A/B of the labellers on the same equilibrium bond lattices: the tile
union-find with boundary merge (sw_label_bonds) against the paper's label
equivalence (sw_label_bonds_le; Sec. 2 quotes about 8.6 scan/analysis
iterations at q=2, T_c, 4096^2) and against the paper's two-stage
multi-GPU labelling (sw_label_bonds_2stage, Sec. 3) emulated on one GPU with
sub x sub virtual sub-lattices.  All give bit-identical roots; this reports
their GPU times and iteration counts.

Usage: python -m paper_1208_2080_gb300.labeller_ab [--L 4096 16384] [--sub 1024 2048 4096] [--reps 5]
"""
import argparse
import json

from ._binding import Sim, label_bonds, label_bonds_2stage, label_bonds_le


def tc(q):
    import math
    return 1.0 / math.log1p(math.sqrt(q))


def ab(L, q=2, seed=11, equil=100, reps=5, samples=5, subs=(1024, 2048, 4096)):
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
            rec = {"uf_ms": uf, "le_ms": le, "le_iterations": it, "identical": bool(torch.equal(ra, rb)),
                   "two_stage": []}
            for sub in subs:
                if sub > L or L % sub:
                    continue
                rb.fill_(-1)
                its = label_bonds_2stage(L, sub, packed, rb)
                same = bool(torch.equal(ra, rb))
                stage = [0.0, 0.0, 0.0]
                e0.record()
                for _ in range(reps):
                    i1, i2, ms = label_bonds_2stage(L, sub, packed, rb, timings=True)
                    stage = [a + b / reps for a, b in zip(stage, ms)]
                e1.record()
                torch.cuda.synchronize()
                rec["two_stage"].append({"sub": sub, "sub_lattices": (L // sub) ** 2,
                                         "ms": e0.elapsed_time(e1) / reps, "stage1_ms": stage[0],
                                         "stage2_ms": stage[1], "final_ms": stage[2],
                                         "stage1_iterations": its[0], "stage2_iterations": its[1],
                                         "identical": same})
            out["samples"].append(rec)
    its = [x["le_iterations"] for x in out["samples"]]
    out["le_iterations_mean"] = sum(its) / len(its)
    out["uf_ms_mean"] = sum(x["uf_ms"] for x in out["samples"]) / samples
    out["le_ms_mean"] = sum(x["le_ms"] for x in out["samples"]) / samples
    per_sub = {}
    for x in out["samples"]:
        for t in x["two_stage"]:
            per_sub.setdefault(t["sub"], []).append(t)
    out["two_stage_mean"] = [{"sub": k, "sub_lattices": v[0]["sub_lattices"],
                              "ms": sum(t["ms"] for t in v) / len(v),
                              "stage1_ms": sum(t["stage1_ms"] for t in v) / len(v),
                              "stage2_ms": sum(t["stage2_ms"] for t in v) / len(v),
                              "final_ms": sum(t["final_ms"] for t in v) / len(v),
                              "stage1_iterations": sum(t["stage1_iterations"] for t in v) / len(v),
                              "stage2_iterations": sum(t["stage2_iterations"] for t in v) / len(v),
                              "identical": all(t["identical"] for t in v)} for k, v in sorted(per_sub.items())]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, nargs="+", default=[4096, 16384])
    ap.add_argument("--sub", type=int, nargs="+", default=[1024, 2048, 4096])
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--samples", type=int, default=5)
    a = ap.parse_args()
    print(json.dumps([ab(L, reps=a.reps, samples=a.samples, subs=a.sub) for L in a.L], indent=1))


if __name__ == "__main__":
    main()
