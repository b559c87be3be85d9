#!/usr/bin/env python
"""Benchmark of the Swendsen-Wang sweep on one GB300 (one JSON line).

Workload (default): q = 2 (Ising), L = 65536 (4.29e9 sites), T = T_c =
1/ln(1+sqrt 2), all-zero start, uint64 cluster labels -- the production-size
configuration of Table 1 / the abstract (37.3 spin flips/ns on 256 M2050).
A step is one full SW sweep (bonds, labelling, recolouring, fused E/M
measurement).  W warm-up sweeps, then K timed sweeps; with the defaults
(W=20, K=80) the run covers exactly the 100 sweeps of that configuration.

Metric: spin updates per ns = N * K / device time.  The timed region holds
only the library's kernels (inputs resident in HBM, every buffer far larger
than the 126 MB L2, so no flush is needed).  `e2e` repeats the metric through
the public API with host buffers: each step is one sw_sweep_host call, which
uploads the configuration from pinned host memory (in bands, overlapped with
the sweep's labelling), sweeps once and reads the observables back.
`roofline` reports the dominant kernel's achieved HBM bandwidth from the
library's per-launch CUDA events (and its instruction issue rate);
`cpu_baseline` times the CPU oracle on a bounded sample, and
`cpu_baseline_all_cores` the same oracle on every host core.  The line also
carries the replica batch (`batched`), the XY model (`xy`) and the Wolff
comparison (`wolff`).

--impl reference times the CPU oracle (the only reference implementation of
this paper's method) as the reference arm, on rank 0.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SW spin updates/ns at q=2, T_c, L=65536 (update + measurement)"
UNIT = "spin updates/ns"
PAPER_UPDATE_MEASURE = 33.85  # Table 1, L=65536, 256x Tesla M2050, update + measurement
# Algorithmic HBM bytes per site moved by each kernel of a sweep in this
# design: k_label_rows reads the uint8 spin and writes the 16-bit site code;
# k_recolor reads the code and writes the spin.  O(1/tile) halo and edge
# terms are left out.
ALG_BYTES_PER_SITE = {"k_label_rows": 3.0, "k_merge+k_resolve": 0.0, "k_recolor": 3.0}
PHASES = ["k_label_rows", "k_merge+k_resolve", "k_recolor"]
LAUNCHES_PER_SWEEP = 4  # k_label_rows, k_merge, k_resolve, k_recolor
# XY model (embedded clusters, M angles): the labeller reads the angle and
# writes the code; the reflection reads code and angle and writes the
# angle; the measurement reads the angle (halo rows come from L2).
XY_PHASES = ["k_label_rows<XY>", "k_merge+k_resolve", "k_recolor<XY>", "k_xy_measure"]
XY_ALG_BYTES_PER_SITE = {"k_label_rows<XY>": 3.0, "k_merge+k_resolve": 0.0, "k_recolor<XY>": 4.0,
                         "k_xy_measure": 1.0}
THROTTLE = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=5)

    def summary(self):
        mhz, mx, reasons = [], None, set()
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(THROTTLE, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        mhz.sort()
        return {"sm_mhz": mhz[len(mhz) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


def _kernel_hash():
    h = hashlib.sha256()
    for f in ("sw_kernels.cuh", "sw_label.cuh", "philox.cuh"):
        with open(os.path.join(ROOT, "paper_1208_2080_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profile_figure(kernel, key, L):
    """Per-launch figure (`key` per site x sites) of `kernel` from the
    committed ncu summary, if it was taken on the current kernel source
    (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[kernel]
        if e.get("source_hash") != _kernel_hash():
            return None
        return float(e[key]) * L * L
    except Exception:
        return None


def _traffic(kernel, L):
    """DRAM bytes per launch of `kernel` (ncu), or None."""
    return _profile_figure(kernel, "bytes_per_site", L)


# Instruction issue peak of the GPU: 4 warp instructions per clock per SM
# (four schedulers), 152 SMs, 2070 MHz maximum SM clock.
ISSUE_PEAK = 4 * 152 * 2070e6


def max_over_ranks(ms, dist=None, device="cpu"):
    """The slowest rank's time (every rank gets it); ms itself on one rank."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(sites_per_rank, steps, world, max_ms):
    """Whole-job spin updates per ns: every rank sweeps its own lattice
    (replicas, no exchange), timed by the slowest rank."""
    return sites_per_rank * steps * world / (max_ms * 1e6)


def cpu_baseline(seconds=15.0, L=8192):
    """The oracle, as it stands, single-threaded on a bounded sample: q=2,
    T_c, L x L from the init stream, as many sweeps as fit in ~`seconds`."""
    import numpy as np
    import oracle
    T = oracle.tc(2)
    s = oracle.init_spins(L, 2, 5).reshape(-1).copy()
    t0 = time.perf_counter()
    oracle.run(L, 2, T, 5, 1, spins=s, sweep0=0, series=False)
    one = time.perf_counter() - t0
    n = max(1, int(seconds / max(one, 1e-3)) - 1)
    t0 = time.perf_counter()
    oracle.run(L, 2, T, 5, n, spins=s, sweep0=1, series=False)
    dt = time.perf_counter() - t0
    del np
    return {"value": L * L * n / (dt * 1e9), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"q=2, T_c, L={L} random start, {n} sweeps (after 1 untimed), "
                      f"single-threaded C oracle, {dt:.1f} s"}


def _oracle_sample(job):
    """One process of cpu_baseline_all_cores: seconds for `sweeps` oracle
    sweeps of an L x L q=2 lattice at T_c."""
    L, sweeps, seed = job
    import oracle
    T = oracle.tc(2)
    s = oracle.init_spins(L, 2, seed).reshape(-1).copy()
    t0 = time.perf_counter()
    oracle.run(L, 2, T, seed, sweeps, spins=s, series=False)
    return time.perf_counter() - t0


def cpu_baseline_all_cores(L=4096, sweeps=6):
    """The same oracle on every host core at once, one independent lattice
    per process (replicas are independent, so this is how a CPU would run
    them): aggregate updates over the slowest process's time."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(n) as pool:
        times = pool.map(_oracle_sample, [(L, sweeps, 100 + k) for k in range(n)])
    worst = max(times)
    return {"value": n * L * L * sweeps / (worst * 1e9), "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"{n} processes, each q=2, T_c, L={L} random start, {sweeps} sweeps; "
                      f"slowest {worst:.1f} s"}


def run_reference(args, rank):
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    L = args.ref_L
    T = oracle.tc(2)
    s = np.zeros(L * L, dtype=np.uint8)
    for k in range(args.warmup):
        s, _, _ = oracle.run(L, 2, T, 5, 1, spins=s, sweep0=k, series=False)
    t0 = time.perf_counter()
    for k in range(args.steps):
        s, _, _ = oracle.run(L, 2, T, 5, 1, spins=s, sweep0=args.warmup + k, series=False)
    dt = time.perf_counter() - t0
    value = L * L * args.steps / (dt * 1e9)
    sample = (f"each step one oracle sweep of a q=2, T_c, L={L} lattice (all-zero start), "
              f"single-threaded C oracle")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": f"q=2 Ising, L={args.L}, T=T_c, all-zero start, "
                               f"uint{64 if args.L > 32768 else 32} labels, sweeps {args.warmup}.."
                               f"{args.warmup + args.steps - 1}",
                   "L": args.L, "q": 2, "oracle_sample_L": L},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


def run_ours(args, rank, world):
    import numpy as np
    import torch

    import paper_1208_2080_gb300 as sw

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    L, q = args.L, 2
    N = L * L
    T = sw.tc(q)
    seed = 5 + rank
    sim = sw.Sim(L, q, T, seed, init="zero", label_bits=args.label_bits, tile_h=args.tile_h,
                 merge=args.merge)
    if sim.info()["merge"] == sw._binding.MERGE["fused"]:
        # the labeller does the boundary unions; a one-block filing kernel
        # takes k_merge's place in the launch sequence
        ALG_BYTES_PER_SITE["k_file+k_resolve"] = ALG_BYTES_PER_SITE.pop("k_merge+k_resolve")
        PHASES[1] = "k_file+k_resolve"
    info = sim.info()
    stream = torch.cuda.current_stream()
    evw0, evw1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evw0.record(stream)
    sim.sweep(args.warmup)
    evw1.record(stream)
    torch.cuda.synchronize()
    warm_ms = evw0.elapsed_time(evw1)

    def barrier():
        if dist is not None:
            dist.barrier()

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        sim.profile(True)
        ev0.record(stream)
        tail = min(50, args.steps)  # the steady-state part: the last 50 timed sweeps
        evm = torch.cuda.Event(enable_timing=True)
        sim.sweep(args.steps - tail)
        evm.record(stream)
        sim.sweep(tail)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = ev0.elapsed_time(ev1)
    steady = {"last_sweeps": tail, "value": N * tail / (evm.elapsed_time(ev1) * 1e6),
              "all_sweeps": args.warmup + args.steps,
              "value_all": N * (args.warmup + args.steps) / ((warm_ms + ms) * 1e6), "unit": UNIT}
    phase_ms, phase_n = sim.profile_read()
    sim.profile(False)
    ms = max_over_ranks(ms, dist, device="cuda")
    E, n, cfg = sim.measure()
    assert int(n.sum()) == N and 0 <= E <= 2 * N, "observables out of range"
    value = job_rate(N, args.steps, world, ms)

    # update only (Table 1's other column): same chain with measurement off
    upd = None
    if args.update_only_steps > 0:
        spins_dev = torch.empty(N, dtype=torch.uint8, device="cuda")
        sim.spins(out=spins_dev)
        cur = sim.sweep_count
        sim.close()
        sim = None
        torch.cuda.empty_cache()
        sim2 = sw.Sim(L, q, T, seed, measure=False, label_bits=args.label_bits,
                      tile_h=args.tile_h, merge=args.merge)
        sim2.set_spins(spins_dev)
        sim2.set_sweep(cur)
        del spins_dev
        sim2.sweep(2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim2.sweep(args.update_only_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        upd = N * args.update_only_steps / (e0.elapsed_time(e1) * 1e6)
        sim = sim2

    # end to end through the public API with host buffers
    e2e = None
    if args.e2e_steps > 0:
        host = torch.empty(N, dtype=torch.uint8, pin_memory=True)
        dev_tmp = torch.empty(N, dtype=torch.uint8, device="cuda")
        sim.spins(out=dev_tmp)
        host.copy_(dev_tmp)
        del dev_tmp
        torch.cuda.empty_cache()
        hnp = host.numpy()
        for _ in range(2):
            sim.sweep_host(hnp, 1)
        barrier()
        t0 = time.perf_counter()
        step_ms = []
        for _ in range(args.e2e_steps):
            # one public call per step: upload from page-locked memory (in
            # bands, overlapped with the labelling), one sweep, observables
            # back to the host
            ts = time.perf_counter()
            sim.sweep_host(hnp, 1)
            step_ms.append((time.perf_counter() - ts) * 1e3)
        dt = time.perf_counter() - t0
        e2e = {"value": N * args.e2e_steps * world / (dt * 1e9), "unit": UNIT,
               "h2d_bytes_per_step": N, "d2h_bytes_per_step": 8 * (2 + q),
               "steps": args.e2e_steps, "step_ms_min": min(step_ms),
               "step_ms_median": sorted(step_ms)[len(step_ms) // 2], "step_ms_max": max(step_ms),
               "step_ms": [round(x, 1) for x in step_ms]}

    batched = None
    if args.batch_sweeps > 0:
        sim.close()
        sim = None
        torch.cuda.empty_cache()
        batched = run_batched(args, sw, torch)

    wolff = None
    if args.wolff_steps > 0:
        if sim is not None:
            sim.close()
            sim = None
        torch.cuda.empty_cache()
        wolff = run_wolff(args, sw, torch)

    xy = None
    if args.xy_sweeps > 0:
        if sim is not None:
            sim.close()
            sim = None
        torch.cuda.empty_cache()
        xy = run_xy(args, sw, torch)

    if rank != 0:
        return 0
    peak, peak_kind = _peaks()
    avg = [m / max(c, 1) for m, c in zip(phase_ms, phase_n)]
    dom = max(range(3), key=lambda k: phase_ms[k])
    name = PHASES[dom]
    alg = ALG_BYTES_PER_SITE[name] * N
    achieved = alg / (avg[dom] * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind, "traffic": _traffic(name, L),
            "alg_bytes_per_launch": alg, "avg_launch_ms": avg[dom],
            "phase_ms_per_sweep": {PHASES[k]: avg[k] for k in range(3)}}
    # every phase's algorithmic HBM rate, and the whole sweep's (6 B/site:
    # spin read + code write in the labelling, code read + spin write in the
    # recolour; the merge and resolve touch only sparse tile records)
    phases = {}
    for k, pname in enumerate(PHASES):
        pb = ALG_BYTES_PER_SITE[pname] * N
        rate = pb / (avg[k] * 1e-3) / 1e9 if avg[k] > 0 and pb > 0 else None
        phases[pname] = {"ms": avg[k], "alg_bytes": pb, "GB/s": rate,
                         "frac": rate / peak if rate is not None else None}
    sweep_bytes = sum(ALG_BYTES_PER_SITE.values()) * N
    sweep_ms = sum(avg)
    roof["phases"] = phases
    roof["sweep"] = {"ms": sweep_ms, "alg_bytes": sweep_bytes,
                     "GB/s": sweep_bytes / (sweep_ms * 1e-3) / 1e9 if sweep_ms > 0 else None}
    if roof["sweep"]["GB/s"] is not None:
        roof["sweep"]["frac"] = roof["sweep"]["GB/s"] / peak
    # the tile kernel is bound by instruction issue, not by HBM: its issue
    # rate against the GPU's issue peak (instruction count per site from ncu)
    winst = _profile_figure(name, "warp_inst_per_site", L)
    if winst is not None:
        rate = winst / (avg[dom] * 1e-3)
        roof["issue"] = {"bound": "issue", "achieved": rate, "peak": ISSUE_PEAK,
                         "unit": "warp instructions/s", "frac": rate / ISSUE_PEAK,
                         "warp_inst_per_launch": winst}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": value / PAPER_UPDATE_MEASURE, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": f"q=2 Ising, L={L}, T=T_c, all-zero start, "
                               f"uint{info['label_bits']} labels, sweeps {args.warmup}.."
                               f"{args.warmup + args.steps - 1}",
                   "L": L, "q": q, "tile": f"{info['tile_w']}x{info['tile_h']}",
                   "merge": sw._binding.MERGE_NAMES[info["merge"]],
                   "l2": "inputs larger than L2 (4 GiB spins, 8 GiB codes at L=65536)",
                   "replicas": world},
        "gpu_launches": LAUNCHES_PER_SWEEP * args.steps,
        "roofline": roof,
        "clocks": clk.summary(),
        "e2e": e2e,
        "update_only": {"value": upd, "unit": UNIT, "steps": args.update_only_steps}
        if upd is not None else None,
        "observables_last": {"config": cfg, "E_sat": E, "n": [int(x) for x in n]},
        "steady_state": steady,
        "batched": batched,
        "xy": xy,
        "wolff": wolff,
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline()
        out["cpu_baseline_all_cores"] = cpu_baseline_all_cores()
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_xy(args, sw, torch):
    """The XY model's embedded-cluster sweep (M angles, T = T_KT, all-zero
    start, measurement after every sweep): spin updates/ns over timed sweeps
    and the per-phase roofline of its kernels."""
    import numpy as np
    L, M = args.xy_L, args.xy_M
    N = L * L
    stream = torch.cuda.current_stream()
    peak, peak_kind = _peaks()
    with sw.XY(L, M, sw.T_KT, 9, init="zero") as x:
        x.sweep(args.xy_warmup)
        x.sync()
        x.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x.sweep(args.xy_sweeps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        phase_ms, phase_n = x.profile_read()
        D, n = x.series(x.sweep_count, 1)
        x.sync()
    assert int(D.sum()) == 2 * N and int(n.sum()) == N, "XY observables out of range"
    avg = [m / max(c, 1) for m, c in zip(phase_ms, phase_n)]
    phases = {}
    for k, name in enumerate(XY_PHASES):
        alg = XY_ALG_BYTES_PER_SITE[name] * N
        gbs = alg / (avg[k] * 1e-3) / 1e9 if avg[k] > 0 else None
        phases[name] = {"ms": avg[k], "alg_bytes": alg, "GB/s": gbs,
                        "frac": gbs / peak if gbs else None}
    dom = max(range(4), key=lambda k: avg[k])
    return {"workload": f"XY model, M={M} angles, L={L}, T=T_KT={sw.T_KT:.5f}, all-zero start, "
                        f"sweeps {args.xy_warmup}..{args.xy_warmup + args.xy_sweeps - 1}",
            "metric": "XY embedded-cluster spin updates/ns (update + measurement)",
            "value": N * args.xy_sweeps / (ms * 1e6), "unit": UNIT, "steps": args.xy_sweeps,
            "ms_per_sweep": ms / args.xy_sweeps, "gpu_launches": 6 * args.xy_sweeps,
            "phases": phases, "dominant": XY_PHASES[dom], "peak": peak, "peak_kind": peak_kind,
            "energy_per_site_last": float(-(D[0] * np.cos(2 * np.pi * np.arange(M // 2 + 1) / M)).sum()
                                          / N)}


def run_wolff(args, sw, torch):
    """The Wolff single-cluster comparison workload (q = 2, T_c): spin flips
    per ns over timed steps from a configuration equilibrated by SW sweeps,
    next to the SW sweep on the same lattice."""
    import numpy as np
    L, q = args.wolff_L, 2
    N = L * L
    T = sw.tc(q)
    stream = torch.cuda.current_stream()
    with sw.Sim(L, q, T, 21, init="zero") as s_:
        s_.sweep(200)
        s_.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s_.sweep(20)
        e1.record(stream)
        torch.cuda.synchronize()
        sw_rate = N * 20 / (e0.elapsed_time(e1) * 1e6)
        spins = s_.spins()
    modes = {}
    for mode, steps in (("label", args.wolff_steps), ("grow", max(1, args.wolff_steps // 5))):
        with sw.Wolff(L, q, T, 22, mode=mode) as w:
            w.set_spins(spins)
            w.step(args.wolff_warmup)
            w.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            w.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            sizes = w.sizes(args.wolff_warmup, steps).astype(np.float64)
            w.sync()
        flips = float(sizes.sum())
        modes[mode] = {"value": flips / (ms * 1e6), "unit": "spin flips/ns", "steps": steps,
                       "ms_per_step": ms / steps, "mean_cluster": flips / steps,
                       "mean_cluster_over_N": flips / steps / N,
                       "gpu_launches": (7 if mode == "label" else 3) * steps}
    best = max(modes, key=lambda m: modes[m]["value"])
    return {"workload": f"Wolff single-cluster, q=2, T=T_c, L={L}, from 200 SW sweeps of an all-zero "
                        f"start, {args.wolff_warmup} warm-up steps",
            "metric": "Wolff spin flips/ns", "value": modes[best]["value"], "unit": "spin flips/ns",
            "best_mode": best, "modes": modes,
            "sw_same_lattice": {"value": sw_rate, "unit": UNIT,
                                "note": "SW sweep updates every site each sweep"}}


def single_equivalent(args, sw, torch, p, batch_ms):
    """The batch's work at single-lattice speed: for each q of the mix and
    T/T_c in {0.9, 1.0, 1.1}, one L=16384 lattice (16384 tiles of 128x128,
    which fill the GPU about as the batch's 60,517 tiles do) from its random
    start, timed
    over the same sweeps as the batch (3 untimed, then batch_sweeps); a
    replica's sites cost its q's time per site averaged over T by Simpson's
    rule (T is uniform on [0.9, 1.1] T_c in the mix).  The batch against this
    time is the cost of batching itself; the headline lattice (q = 2 at T_c)
    is the cheapest case of the mix."""
    import numpy as np
    Ls = 16384
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per_site = {}
    classes = {}
    for q in sorted(set(int(x) for x in p["q"])):
        tc = sw.tc(q)
        t = []
        for f in (0.9, 1.0, 1.1):
            with sw.Sim(Ls, q, f * tc, 1000 + q) as s:
                s.sweep(3)
                torch.cuda.synchronize()
                e0.record(stream)
                s.sweep(args.batch_sweeps)
                e1.record(stream)
                torch.cuda.synchronize()
                s.sync()
                t.append(e0.elapsed_time(e1) / args.batch_sweeps / (Ls * Ls))
            torch.cuda.empty_cache()
        per_site[q] = (t[0] + 4 * t[1] + t[2]) / 6
        classes[q] = {"updates_per_ns_at_0.9_1.0_1.1_Tc": [1e-6 / x for x in t]}
    sites = p["L"].astype(np.float64) ** 2
    equiv_ms = float(sum(sites[r] * per_site[int(p["q"][r])] for r in range(len(sites))))
    return {"L": Ls, "sweeps": args.batch_sweeps, "ms_per_batch_sweep": equiv_ms,
            "spin_updates_per_ns": float(sites.sum()) / (equiv_ms * 1e6),
            "batch_over_single": batch_ms / equiv_ms, "per_q": classes}


def run_batched(args, sw, torch):
    """Replica sweeps/s of the 512-replica batch (L = 64..2048 log-uniform,
    q in {2,3,4,5,8}, T in [0.9, 1.1] T_c(q), one Philox key each): all
    replicas in one batch (autotuned tile height / merge schedule / launch
    mode) against the
    same replicas swept one at a time through the single-lattice API."""
    import numpy as np

    import synth
    from paper_1208_2080_gb300 import tune
    p = synth.replica_batch(args.batch_R, master_seed=6)
    R = args.batch_R
    cfg = tune.tune_batch(p["L"], p["q"], p["T"], p["seed"])
    stream = torch.cuda.current_stream()
    out = {"R": R, "sites": int((p["L"].astype(np.float64) ** 2).sum()), "tuned": cfg}
    with sw.Batch(p["L"], p["q"], p["T"], p["seed"], tile_h=cfg["tile_h"], graph=cfg["graph"],
                  merge=cfg.get("merge", "kernel")) as b:
        b.sweep(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.sweep(args.batch_sweeps)
        e1.record(stream)
        torch.cuda.synchronize()
        b.sync()
        ms = e0.elapsed_time(e1)
        # where a batch sweep's time goes: the library's per-launch events
        # over 10 further sweeps (launched directly, not through the graph)
        b.profile(True)
        b.sweep(10)
        pms, pn = b.profile_read()
        b.profile(False)
    out.update({"sweeps": args.batch_sweeps, "ms_per_batch_sweep": ms / args.batch_sweeps,
                "phase_ms_per_sweep": {name: m / max(c, 1) for name, m, c in zip(PHASES, pms, pn)},
                "replica_sweeps_per_s": R * args.batch_sweeps / (ms * 1e-3),
                "spin_updates_per_ns": out["sites"] * args.batch_sweeps / (ms * 1e6)})
    torch.cuda.empty_cache()
    if args.batch_equiv:
        out["single_equiv"] = single_equivalent(args, sw, torch, p, ms / args.batch_sweeps)
    sims = [sw.Sim(int(p["L"][r]), int(p["q"][r]), float(p["T"][r]), int(p["seed"][r]))
            for r in range(R)]
    for s_ in sims:
        s_.sweep(2)
    torch.cuda.synchronize()
    n1 = args.plain_sweeps
    e0.record(stream)
    t0 = time.perf_counter()
    for s_ in sims:  # one replica at a time
        s_.sweep(n1)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms1 = e0.elapsed_time(e1)
    for s_ in sims:
        s_.close()
    out.update({"plain_sweeps": n1, "plain_replica_sweeps_per_s": R * n1 / (ms1 * 1e-3),
                "plain_wall_s": wall})
    out["speedup"] = out["replica_sweeps_per_s"] / out["plain_replica_sweeps_per_s"]
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=80)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=65536, help="lattice size (default: the workload)")
    ap.add_argument("--label-bits", type=int, default=0, help="0 = auto (64 above L=32768)")
    ap.add_argument("--tile-h", type=int, default=0, help="labelling tile height (0 = auto)")
    ap.add_argument("--merge", default="auto", choices=["auto", "kernel", "fused"],
                    help="boundary-union schedule")
    ap.add_argument("--ref-L", type=int, default=4096, help="oracle sample size per reference step")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--update-only-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-R", type=int, default=512, help="replicas in the batched measurement")
    ap.add_argument("--batch-sweeps", type=int, default=40, help="0 skips the batched measurement")
    ap.add_argument("--plain-sweeps", type=int, default=10)
    ap.add_argument("--no-batch-equiv", dest="batch_equiv", action="store_false",
                    help="skip the single-lattice equivalent of the batch")
    ap.add_argument("--wolff-steps", type=int, default=100, help="0 skips the Wolff measurement")
    ap.add_argument("--wolff-warmup", type=int, default=10)
    ap.add_argument("--wolff-L", type=int, default=16384)
    ap.add_argument("--xy-sweeps", type=int, default=20, help="0 skips the XY-model measurement")
    ap.add_argument("--xy-warmup", type=int, default=5)
    ap.add_argument("--xy-L", type=int, default=65536)
    ap.add_argument("--xy-M", type=int, default=256)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank)
    return run_ours(args, rank, world)


if __name__ == "__main__":
    sys.exit(main())
