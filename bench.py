#!/usr/bin/env python
"""Throughput of the implicit EM PIC/MCC step on one GB300.

Metric: particle-pushes/s per nonlinear iteration — every Picard pass and the
commit pass push every particle once; value = pushes of the timed steps /
device time of those whole steps (push+deposit, field solves, MCC, sort).

Workload: the large-electrode VHF reactor, 256(r) x 384(z) cells, R = 0.3 m,
L = 0.03 m, argon 2 Pa, 100 MHz 200 V, 16M macro-particles per species,
FP64 plain method, Picard tolerance 1e-8.  The particle store (~1.9 GB) is
larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (launched with torch.distributed.run) every rank runs an
independent replica discharge (seed + rank): weak scaling, no collective on
the data path.  --impl reference times the FP64 CPU oracle (the only CPU
code path) on a bounded particle sample of the same reactor.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-pushes/s per nonlinear iter"
UNIT = "particle-pushes/s"
# FP64 operations per particle push of the FP64 mover+deposit kernel on this
# workload, from the ncu DADD/DMUL/DFMA instruction counts (profiles/).
FP64_FLOP_PER_PUSH = None
# algorithmic bytes per push of the FP64 kernel: cell (4) + a, b, vr, vt, vz, w (48)
BYTES_PER_PUSH_FP64 = 52
# measured ncu DRAM traffic per push launch of this workload (null until measured)
TRAFFIC_PER_LAUNCH = None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_oracle_rate(n_sample, steps=1, seed=1):
    """FP64 oracle on a bounded sample: the same reactor and grid with n_sample
    particles per species; returns (pushes/s, seconds, pushes)."""
    import oracle as O
    import paper_2212_08836_gb300 as P

    cfg = P.large_reactor()
    g = O.Grid(cfg["nr"], cfg["nz"], cfg["R"], cfg["L"])
    e, i = O.load(g, n_sample, cfg["n0"], cfg["te_ev"], cfg["ti_ev"], seed)
    for sp in (e, i):
        o = np.argsort(sp["cell"], kind="stable")
        for k in sp:
            sp[k] = sp[k][o].copy()
    sim = O.Sim(g, cfg["dt"], freq=cfg["freq"], volt=cfg["volt"], tol=cfg["picard_tol"],
                kmax=cfg["picard_max"], mcc_on=True, ng=cfg["gas_pressure"] / (O.KB * cfg["gas_temp"]),
                tg=cfg["gas_temp"], seed=seed, species=[e, i])
    pushes = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        n_before = sim.sp[0]["n"] + sim.sp[1]["n"]
        rc, st = sim.step()
        if rc not in (0,):
            raise RuntimeError("oracle step failed: %d" % rc)
        pushes += (st.picard_iters + 1) * n_before
    dt = time.perf_counter() - t0
    return pushes / dt, dt, pushes


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    n_sample = args.ref_sample
    rates = []
    # warm-up steps and timed steps, each a fresh bounded sample step
    rate, secs, pushes = cpu_oracle_rate(n_sample, steps=args.warmup + args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / (args.warmup + args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "large-electrode VHF reactor 256x384, R=0.3 m, L=0.03 m, Ar 2 Pa, "
                                   "100 MHz 200 V (oracle on a %d-per-species sample)" % n_sample},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d macro-particles per species on the full 256x384 grid, "
                                       "%d whole steps incl. Picard, field solves, MCC, sort"
                                       % (n_sample, args.warmup + args.steps)},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    dist = ws > 1
    if dist:
        import torch.distributed as D

        D.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2212_08836_gb300 as P

    P.lib()
    cfg = P.large_reactor(seed=1 + rank)
    pic = P.Pic(cfg, device=dev)
    pic.load_particles()
    stream = pic.stream

    def barrier():
        torch.cuda.synchronize(dev)
        if dist:
            D.barrier()

    for _ in range(args.warmup):
        pic.step(1)

    # ---------------- timed region (device-resident state)
    pic.profile(True)
    barrier()
    pushes = 0
    launches = 0
    iters = []
    with ClockSampler(local) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            _, st = pic.step(1)
            pushes += st["pushes"]
            launches += st["launches"]
            iters.append(st["picard_iters"])
        ev1.record(stream)
        barrier()
    t_ms = ev0.elapsed_time(ev1)
    push_ms, push_launches = pic.profile_read()
    pic.profile(False)
    clocks = clk.summary()

    # ---------------- end to end through the C ABI with host buffers
    v = pic.view()
    host = []
    for s in range(2):
        n = v["cap"][s]
        host.append({k: torch.empty_like(v["species"][s][k], device="cpu").pin_memory()
                     for k in P.FIELDS})
    hf = {k: torch.empty_like(v[k], device="cpu").pin_memory() for k in ("er", "ez", "h")}
    for s in range(2):
        for k in P.FIELDS:
            host[s][k].copy_(v["species"][s][k])
    for k in hf:
        hf[k].copy_(v[k])
    torch.cuda.synchronize(dev)
    barrier()
    e2e_pushes = 0
    h2d = d2h = 0
    t0 = time.perf_counter()
    ev2 = torch.cuda.Event(enable_timing=True)
    ev3 = torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    for _ in range(args.steps):
        v = pic.view()
        with torch.cuda.stream(stream):
            for s in range(2):
                n = v["n"][s]
                for k in P.FIELDS:
                    v["species"][s][k][:n].copy_(host[s][k][:n], non_blocking=True)
                    h2d += host[s][k][:n].numel() * host[s][k].element_size()
            for k in hf:
                v[k].copy_(hf[k], non_blocking=True)
                h2d += hf[k].numel() * hf[k].element_size()
        _, st = pic.step(1)
        e2e_pushes += st["pushes"]
        v = pic.view()
        with torch.cuda.stream(stream):
            for s in range(2):
                n = v["n"][s]
                for k in P.FIELDS:
                    host[s][k][:n].copy_(v["species"][s][k][:n], non_blocking=True)
                    d2h += host[s][k][:n].numel() * host[s][k].element_size()
            for k in hf:
                hf[k].copy_(v[k], non_blocking=True)
                d2h += hf[k].numel() * hf[k].element_size()
    ev3.record(stream)
    barrier()
    e2e_ms = ev2.elapsed_time(ev3)

    # max over ranks
    t_max, e2e_max = t_ms, e2e_ms
    tot_pushes, tot_e2e = pushes, e2e_pushes
    if dist:
        tt = torch.tensor([t_ms, e2e_ms], dtype=torch.float64, device=dev)
        D.all_reduce(tt, op=D.ReduceOp.MAX)
        pp = torch.tensor([pushes, e2e_pushes], dtype=torch.float64, device=dev)
        D.all_reduce(pp)
        t_max, e2e_max = tt.tolist()
        tot_pushes, tot_e2e = pp.tolist()
    value = tot_pushes / (t_max * 1e-3)

    pk, pk_kind = peaks()
    avg_launch_ms = push_ms / max(push_launches, 1)
    pushes_per_launch = pushes / max(push_launches, 1)
    if FP64_FLOP_PER_PUSH is not None:
        fp64_peak = args.fp64_peak_tflops
        achieved = FP64_FLOP_PER_PUSH * pushes_per_launch / (avg_launch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "traffic": TRAFFIC_PER_LAUNCH,
                "kernel": "k_push_fp64", "peak_kind": "FP64 FMA rate (see DESIGN.md)"}
    else:
        achieved = BYTES_PER_PUSH_FP64 * pushes_per_launch / (avg_launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": TRAFFIC_PER_LAUNCH,
                "kernel": "k_push_fp64", "peak_kind": pk_kind}
    roof["avg_launch_ms"] = avg_launch_ms
    roof["launches"] = push_launches

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "large-electrode VHF reactor 256x384, R=0.3 m, L=0.03 m, Ar 2 Pa, "
                                   "100 MHz 200 V, 16M macro-particles/species, FP64 plain, tol 1e-8",
                       "l2": "inputs larger than L2 (particle store ~1.9 GB)",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "picard_iters": iters},
            "clocks": clocks,
            "e2e": {"value": tot_e2e / (e2e_max * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps},
            "gpu_launches": launches,
            "roofline": roof}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, secs, npush = cpu_oracle_rate(args.cpu_sample, steps=1)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "%d macro-particles per species on the 256x384 grid, 1 whole "
                                          "step (%d pushes, %.1f s)" % (args.cpu_sample, npush, secs)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        D.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=1 << 22)
    ap.add_argument("--ref-sample", type=int, default=1 << 20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-peak-tflops", type=float, default=1.25)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
