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
# FP64 peak of GB300: ncu reports 304 thread-DFMA per cycle GPU-wide
# (sm__sass_thread_inst_executed_op_dfma_pred_on.sum.peak_sustained), 2 flops each,
# at the maximum SM clock of MEASURED_PEAKS.json.
DFMA_PER_CYCLE = 304
# algorithmic bytes per push of the FP64 kernel: cell (4) + a, b, vr, vt, vz, w (48)
BYTES_PER_PUSH_FP64 = 52
# ncu DRAM bytes (read + write) per push of the current FP64 kernel, from the
# profile in profiles/ (None when the kernel changed after the capture)
TRAFFIC_PER_PUSH = 85.7  # DRAM bytes per push of the FP64 push kernels: ncu dram__bytes_read + write, 4M/species case
TRAFFIC_PER_PUSH_FP32 = 34.6  # the same for the FP32 push kernels of the mixed form


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
                                          "-i", str(self.idx), "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts once the sampler is running (its first
            # line), so that a short region still gets samples; that first
            # line, taken before the region, is dropped
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.skip = len(self.lines)
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
        skip = getattr(self, "skip", 0)
        for ln in (self.lines[skip:] if len(self.lines) > skip else self.lines):
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


def replica_seed(seed, rank):
    """Seed of the replica on `rank`: N > 1 runs N independent discharges
    (replicas only: the path needs no exchange between GPUs)."""
    return seed + rank


def reduce_replicas(D, t_ms, pushes, device):
    """Whole-job figures of the replicas: the slowest rank's time and the pushes
    of all ranks (value = all pushes / that time)."""
    import torch

    tt = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    D.all_reduce(tt, op=D.ReduceOp.MAX)
    nn = torch.tensor([float(pushes)], dtype=torch.float64, device=device)
    D.all_reduce(nn)
    return tt.item(), nn.item()


def bind_near_gpu(torch, dev):
    """Run this process on the host cores next to the GPU (its PCI device's
    local_cpulist), so that pinned host buffers come from the GPU's NUMA node
    and host transfers do not cross the link between host sockets.  Returns
    the core list, or None where the platform does not expose it."""
    try:
        p = torch.cuda.get_device_properties(dev)
        bus = "%04x:%02x:%02x.0" % (getattr(p, "pci_domain_id"), getattr(p, "pci_bus_id"),
                                    getattr(p, "pci_device_id"))
        with open("/sys/bus/pci/devices/%s/local_cpulist" % bus) as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            if "-" in part:
                lo, hi = part.split("-")
                cpus.update(range(int(lo), int(hi) + 1))
            elif part:
                cpus.add(int(part))
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return spec
    except (AttributeError, OSError, ValueError):
        return None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def host_cores():
    """Host cores this process may run on (the oracle's push threads)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_oracle_rate(n_sample, steps=1, seed=1, threads=1):
    """FP64 oracle on a bounded sample: the same reactor and grid with n_sample
    particles per species, its push split over `threads` host threads (per-
    thread crossed-charge arrays); returns (pushes/s, seconds, pushes)."""
    import oracle as O
    import paper_2212_08836_gb300 as P

    O.set_threads(threads)

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
    cores = host_cores()
    # warm-up steps and timed steps, each a fresh bounded sample step
    rate, secs, pushes = cpu_oracle_rate(n_sample, steps=args.warmup + args.steps, threads=cores)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / (args.warmup + args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "large-electrode VHF reactor 256x384, R=0.3 m, L=0.03 m, Ar 2 Pa, "
                                   "100 MHz 200 V (oracle on a %d-per-species sample)" % n_sample},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d macro-particles per species on the full 256x384 grid, "
                                       "%d whole steps incl. Picard, field solves, MCC, sort; "
                                       "push over %d threads (OpenMP, per-thread crossed charge), "
                                       "the rest serial"
                                       % (n_sample, args.warmup + args.steps, cores)},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def measure(P, torch, dev, cfg, args, dist, D, do_e2e, sample_clocks, local):
    """Load, warm up, then time args.steps whole steps (device-resident state)
    and optionally the same through the C ABI with pinned host buffers."""
    # the library's own stream, its Picard passes replayed from captured graphs
    pic = P.Pic(cfg, device=dev, stream=torch.cuda.Stream(device=dev))
    P.set_graphs(pic, True)
    pic.load_particles()
    stream = pic.stream

    def barrier():
        torch.cuda.synchronize(dev)
        if dist:
            D.barrier()

    # timing on during the warm-up too, so that the passes are captured with
    # their timing events before the timed region (the second call resets the
    # totals)
    pic.profile(True)
    for _ in range(args.warmup):
        pic.step(1)
    pic.profile(True)
    barrier()
    r = {"pushes": 0, "launches": 0, "iters": [], "flops": 0, "commit_pushes": 0,
         "bytes": 0, "substep_cap": 0}
    clk = ClockSampler(local) if sample_clocks else None
    if clk:
        clk.__enter__()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        _, st = pic.step(1)
        k = st["picard_iters"]
        # passes: k Picard passes, plus the commit push unless the converged
        # pass already wrote the state (out of place: every field)
        n_commit = st["pushes"] // (k + (0 if st["spec_final"] else 1))
        r["pushes"] += st["pushes"]
        r["launches"] += st["launches"]
        r["iters"].append(k)
        r["flops"] += st["push_flops"]
        r["commit_pushes"] += n_commit
        r["substep_cap"] += st["substep_err"]
        rb, wb = (28, 24) if cfg["precision"] == P.PIC_MIXED else (52, 48)
        if st["spec_final"]:
            wb += 8  # cell and id (4 B each) written too
        r["bytes"] += st["pushes"] * rb + n_commit * wb
    ev1.record(stream)
    barrier()
    if clk:
        clk.__exit__()
        r["clocks"] = clk.summary()
    r["t_ms"] = ev0.elapsed_time(ev1)
    r["push_ms"], r["push_launches"] = pic.profile_read()
    pic.profile(False)
    # the same steps with timing off, the Picard iteration run from the host
    # (one wait per pass) and on the device (one conditional graph and one
    # wait per step), alternating step by step so that both see the same
    # discharge (its iteration count changes as it develops); each step timed
    # alone, after one step of each that captures the graphs
    for on in (False, True):
        P.set_device_picard(pic, on)
        pic.step(1)
    barrier()
    loop = {"host": [], "device": []}
    its = {"host": [], "device": []}
    for i in range(2 * args.steps):
        on = i % 2 == 1
        P.set_device_picard(pic, on)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st = pic.step(1)
        e1.record(stream)
        e1.synchronize()
        key = "device" if on else "host"
        loop[key].append(e0.elapsed_time(e1))
        its[key].append(st["picard_iters"])
    barrier()
    r["picard_loop"] = {k: {"ms_per_step": sum(v) / len(v), "picard_iters": its[k]}
                        for k, v in loop.items()}
    # sub-step histogram of one more step, outside the timed region
    pic.substep_histogram(1)
    pic.step(1, check=False)
    r["substep_hist"] = [int(v) for v in pic.substep_histogram(0)]
    r["e2e_ms"] = None
    if do_e2e:
        # the whole state lives in pinned host memory between steps: every
        # step uploads it through the C ABI, steps, and reads the new state
        # back (pic_step_host: each step's download overlapped piece by piece
        # with the next step's upload)
        hs = pic.host_state(pinned=True)
        pic.state_download(hs)
        rs = pic.view()["species"][0]["a"].element_size()
        nf = sum(hs[k].numel() * 8 for k in ("er", "ez", "h"))
        n_start = sum(hs["n"])
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        _, st = pic.step_host(hs, args.steps)
        t1 = time.perf_counter()
        barrier()
        n_end = sum(hs["n"])
        # bytes per step: every step moves the whole state both ways (counts
        # change by the step's ionization and wall losses: their mean)
        per = 0.5 * (n_start + n_end) * (8 + 6 * rs) + nf
        r["e2e_ms"] = (t1 - t0) * 1e3
        r["e2e_pushes"] = st["pushes"]
        r["h2d"] = int(per)
        r["d2h"] = int(per)
    pic.close()
    del pic
    torch.cuda.empty_cache()
    return r


def ensemble_configs(P, rank):
    """16 discharges spanning 64x96..256x384 grids, 1M..16M macro-particles per
    species, 1-10 Pa, 40-100 MHz, 100-300 V, seeds 100-115 (mixed form)."""
    cfgs = []
    order_p = [3, 11, 6, 14, 0, 9, 5, 12, 2, 15, 7, 10, 1, 13, 4, 8]
    order_f = [9, 2, 13, 5, 15, 0, 7, 11, 4, 14, 1, 8, 12, 3, 10, 6]
    order_v = [6, 14, 1, 10, 3, 12, 8, 0, 15, 5, 11, 2, 13, 7, 4, 9]
    for i in range(16):
        u = i / 15.0
        nr = int(round((64 + u * 192) / 8.0)) * 8
        nz = nr * 3 // 2
        f = 40e6 + order_f[i] / 15.0 * 60e6
        cfgs.append(P.large_reactor(
            nr=nr, nz=nz, np_init=int(round((1 + 15 * u) * (1 << 20))),
            gas_pressure=1.0 + order_p[i] / 15.0 * 9.0, freq=f, dt=1.0 / (400 * f),
            volt=100.0 + order_v[i] / 15.0 * 200.0, seed=100 + i + 16 * rank,
            precision=P.PIC_MIXED, capacity_factor=1.5))
    return cfgs


def timed_cycle(P, torch, dev, pic, nsteps, relaxed):
    """nsteps steps of pic, wall clock with the device synchronised at both
    ends (host work between the steps included); returns (s, iterations,
    pushes, statuses)."""
    from paper_2212_08836_gb300.dispersion import advance

    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    iters, pushes, rcs = [], 0, []
    for k in range(nsteps):
        st = advance(pic, pic.cfg["picard_tol"], relaxed, k)
        iters.append(st["picard_iters"])
        pushes += st["pushes"]
    torch.cuda.synchronize(dev)
    return time.perf_counter() - t0, iters, pushes


def run_developed_form(P, torch, dev, args, rank, cycles=5):
    """The developed discharge: the 256 x 384 reactor after `cycles` RF cycles
    of the mixed form (sheaths, sheath-accelerated electrons, more face
    crossings than the Maxwellian start).  From that one state, one whole RF
    cycle (1/(f dt) steps) is timed for each form at the converged Picard
    tolerance 1e-8: the plain FP64 form, the mixed form with the plain start,
    and the mixed form with the learned start (the network trained on
    snapshots of the same discharge).  Wall-seconds per RF cycle with the
    device synchronised at both ends; the FP64 form's pushes/s too."""
    from paper_2212_08836_gb300 import guess as GS
    from paper_2212_08836_gb300.dispersion import advance

    seed = replica_seed(1, rank)
    cfgm = P.large_reactor(seed=seed, precision=P.PIC_MIXED, capacity_factor=3.0)
    if args.np:
        cfgm["np_init"] = args.np
    steps_cycle = int(round(1.0 / (cfgm["freq"] * cfgm["dt"])))
    n_dev = cycles * steps_cycle
    pic = P.Pic(cfgm, device=dev)
    pic.load_particles()
    relaxed = []
    t0 = time.perf_counter()
    try:
        for k in range(n_dev):
            advance(pic, cfgm["picard_tol"], relaxed, k)
    except RuntimeError as e:
        pic.close()
        return {"failed": str(e)}
    t_develop = time.perf_counter() - t0
    species = [pic.get_state(s) for s in range(2)]
    er, ez, h = pic.fields()
    v = pic.view()
    step, next_ids = v["step"], list(v["next_id"])

    def fresh(cfg):
        q = P.Pic(cfg, device=dev, stream=torch.cuda.Stream(device=dev))
        P.set_graphs(q, True)
        q.set_state(species, er, ez, h, next_ids=next_ids, step=step)
        return q

    out = {"workload": "256x384 reactor after %d RF cycles (%d steps of the mixed form, %.1f s), "
                       "then one RF cycle (%d steps) of each form from that state, tol %.0e"
                       % (cycles, n_dev, t_develop, steps_cycle, cfgm["picard_tol"]),
           "steps_per_rf_cycle": steps_cycle, "develop_steps_relaxed": len(relaxed)}
    walls, iters = {}, {}
    # ---- learned start: snapshots of this discharge (extrapolated start), training
    X, T = GS.collect(pic, args.guess_samples)
    pic.close()
    net = P.Cnn(cfgm["nr"], cfgm["nz"], batch=8, device=dev)
    t1 = time.perf_counter()
    loss, val, zero = GS.train(net, X, T, args.guess_epochs)
    t_train = time.perf_counter() - t1
    del X, T
    for name, mode in (("mixed", P.PIC_GUESS_PLAIN), ("mixed_learned_start", P.PIC_GUESS_CNN)):
        q = fresh(cfgm)
        P.set_guess(q, mode, net if mode == P.PIC_GUESS_CNN else None)
        q.step(4, check=False)  # the field history of the learned start refills
        rel = []
        w, it, _ = timed_cycle(P, torch, dev, q, steps_cycle, rel)
        walls[name], iters[name] = w, float(np.mean(it))
        out[name + "_relaxed_steps"] = len(rel)
        q.close()
    net.close()
    # ---- the plain FP64 form
    cfg = P.large_reactor(seed=seed, capacity_factor=3.0)
    if args.np:
        cfg["np_init"] = args.np
    q = fresh(cfg)
    q.step(4, check=False)
    rel = []
    w, it, pushes = timed_cycle(P, torch, dev, q, steps_cycle, rel)
    walls["plain_fp64"], iters["plain_fp64"] = w, float(np.mean(it))
    n = q.view()["n"]
    q.substep_histogram(1)
    q.step(1, check=False)
    hist = [int(x) for x in q.substep_histogram(0)]
    q.close()
    out.update({"wall_s_per_rf_cycle": walls, "picard_iters_mean": iters,
                "plain_fp64_relaxed_steps": len(rel),
                "value": pushes / w, "unit": UNIT, "ms_per_step": w * 1e3 / steps_cycle, "n": n,
                "substep_histogram": hist,
                "learned_start": {"samples": args.guess_samples, "adam_steps": args.guess_epochs,
                                  "train_s": t_train, "heldout_loss": val,
                                  "heldout_loss_no_correction": zero}})
    return out


def run_cnn_form(P, torch, dev, warm=3, steps=10):
    """The learned start's network alone on the 256 x 384 grid: batch 8 of
    random inputs and targets, `warm` + `steps` Adam steps, then `steps`
    forward passes, each phase timed with CUDA events on the network's stream."""
    net = P.Cnn(256, 384, batch=8, device=dev)
    x = torch.randn(8, P.CNN_IN, 257, 385, device=dev)
    t = torch.randn(8, P.CNN_OUT, 257, 385, device=dev)
    for _ in range(warm):
        net.train_step(x, t, 1e-4)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        net.train_step(x, t, 1e-4)
    e1.record()
    torch.cuda.synchronize(dev)
    train_ms = e0.elapsed_time(e1) / steps
    e0.record()
    for _ in range(steps):
        net.forward(x[:1])
    e1.record()
    torch.cuda.synchronize(dev)
    fwd_ms = e0.elapsed_time(e1) / steps
    n = net.num_params
    net.close()
    return {"params": n, "train_step_ms_batch8": train_ms, "forward_ms_batch1": fwd_ms}


def run_ensemble_form(P, torch, dev, args, rank):
    cfgs = ensemble_configs(P, rank)
    mem = []
    for c in cfgs:
        pic = P.Pic(c, device=dev, stream=torch.cuda.Stream(device=dev))
        pic.load_particles()
        mem.append(pic)
    torch.cuda.synchronize(dev)
    E = P.Ensemble(mem)
    E.step(args.warmup)
    frac, pers, ms_round = E.tune(rounds=3)
    E.step(1)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    _, st = E.step(1)
    pushes = sum(s["pushes"] for s in st)
    for _ in range(args.steps - 1):
        _, st = E.step(1)
        pushes += sum(s["pushes"] for s in st)
    torch.cuda.synchronize(dev)
    t_ens = time.perf_counter() - t0
    # the same discharges one after another (kernel-by-kernel launches, one
    # wave of the push kernels: the single-run configuration)
    t_seq, p_seq = 0.0, 0
    for pic in mem:
        P.set_graphs(pic, False)
        pic.step(1)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _, s1 = pic.step(1)
            p_seq += s1["pushes"]
        torch.cuda.synchronize(dev)
        t_seq += time.perf_counter() - t0
    npart = sum(c["np_init"] for c in cfgs)
    out = {"members": len(cfgs), "steps": args.steps,
           "workload": "16 discharges, grids %dx%d..%dx%d, %.0fM..%.0fM macro-particles/species "
                       "(%.0fM in all), 1-10 Pa, 40-100 MHz, 100-300 V, seeds 100-115, mixed form"
                       % (cfgs[0]["nr"], cfgs[0]["nz"], cfgs[-1]["nr"], cfgs[-1]["nz"],
                          cfgs[0]["np_init"] / 2 ** 20, cfgs[-1]["np_init"] / 2 ** 20,
                          2 * npart / 2 ** 20),
           "value": pushes / t_ens, "unit": UNIT, "ms_per_step": t_ens * 1e3 / args.steps,
           "sequential_value": p_seq / t_seq, "sequential_ms_per_step": t_seq * 1e3 / args.steps,
           "speedup_vs_sequential": (pushes / t_ens) / (p_seq / t_seq),
           "tuner": {"push_grid_fraction": frac, "persistent": pers,
                     "ms_per_round": {"per_member": ms_round[:3], "persistent": ms_round[3:],
                                      "fractions": [1.0, 0.5, 0.25]}},
           "timing": "host clock around whole ensemble steps (device synchronised)"}
    E.close()
    for pic in mem:
        pic.close()
    return out


def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    dist = ws > 1
    D = None
    if dist:
        import torch.distributed as D

        D.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    host_cpus = bind_near_gpu(torch, dev)
    import paper_2212_08836_gb300 as P

    P.lib()
    pk, pk_kind = peaks()
    sm_max = pk.get("sm_max_mhz", 2070.0)

    def maxsum(t, n):
        return reduce_replicas(D, t, n, dev) if dist else (t, n)

    forms = args.forms.split(",")
    if "plain" not in forms:
        # profiling aids (no headline line is printed): the mixed form alone,
        # the learned start's network alone, and/or the ensemble alone
        out = {"profiling_only": True}
        if "mixed" in forms:
            cfgm = P.large_reactor(seed=replica_seed(1, rank), precision=P.PIC_MIXED)
            if args.np:
                cfgm["np_init"] = args.np
            rm = measure(P, torch, dev, cfgm, args, dist, D, False, False, local)
            out.update({"ms_per_step": rm["t_ms"] / args.steps,
                        "push_ms_per_launch": rm["push_ms"] / max(rm["push_launches"], 1)})
        if "cnn" in forms:
            out["cnn"] = run_cnn_form(P, torch, dev)
        if "ensemble" in forms:
            out["ensemble"] = run_ensemble_form(P, torch, dev, args, rank)
        if rank == 0:
            print(json.dumps(out))
        return 0
    # ---- plain FP64 method on the 256 x 384 reactor (the headline workload)
    cfg = P.large_reactor(seed=replica_seed(1, rank))
    if args.np:
        cfg["np_init"] = args.np
    r = measure(P, torch, dev, cfg, args, dist, D, not args.no_e2e, True, local)
    t_max, tot = maxsum(r["t_ms"], r["pushes"])
    value = tot / (t_max * 1e-3)
    avg_launch_ms = r["push_ms"] / max(r["push_launches"], 1)
    pushes_per_launch = r["pushes"] / max(r["push_launches"], 1)
    flop_per_push = r["flops"] / max(r["commit_pushes"], 1)
    # the FP64 FMA pipe's throughput, measured on this GPU (pic_probe_dfma);
    # the unit count times the maximum clock for context
    _, fp64_peak = P.probe_dfma(4, 1 << 14)
    fp64_nominal = DFMA_PER_CYCLE * 2 * sm_max * 1e6 / 1e12
    achieved = flop_per_push * pushes_per_launch / (avg_launch_ms * 1e-3) / 1e12
    hbm_achieved = r["bytes"] / (r["push_ms"] * 1e-3) / 1e9
    roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": achieved / fp64_peak,
            "traffic": TRAFFIC_PER_PUSH * pushes_per_launch if TRAFFIC_PER_PUSH else None,
            "kernel": "k_push_fp64 (mover+deposit, FP64)",
            "peak_kind": "FP64 FMA pipe, measured (pic_probe_dfma: independent DFMA chains on "
                         "every SM); unit count 304 DFMA/cycle x 2 x max SM clock = %.3f TFLOP/s"
                         % fp64_nominal,
            "flop_per_push": flop_per_push, "avg_launch_ms": avg_launch_ms,
            "launches": r["push_launches"],
            "hbm": {"achieved_gbs": hbm_achieved, "peak_gbs": pk["hbm_gbs"],
                    "frac": hbm_achieved / pk["hbm_gbs"], "peak_kind": pk_kind}}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "large-electrode VHF reactor 256x384, R=0.3 m, L=0.03 m, Ar 2 Pa, "
                                   "100 MHz 200 V, %d macro-particles/species, FP64 plain, tol 1e-8"
                                   % cfg["np_init"],
                       "l2": "inputs larger than L2 (particle store ~1.9 GB)",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "picard_iters": r["iters"],
                       "substep_cap_hits": r["substep_cap"]},
            "clocks": r.get("clocks"),
            "gpu_launches": r["launches"],
            "roofline": roof,
            "picard_loop": {"plain_fp64": r["picard_loop"],
                            "note": "steps after the timed region with timing off, "
                                    "alternating: the iteration from the host (a wait per "
                                    "pass) against the device loop (pic_set_device_picard; "
                                    "one wait per step), each step timed alone"},
            "substep_histogram": {"bins": r["substep_hist"],
                                  "note": "particles with k+1 accepted sub-steps in bin k "
                                          "(bin 15: 16 or more), one step after the timed region"}}
    if r["e2e_ms"] is not None:
        te, ne = maxsum(r["e2e_ms"], r["e2e_pushes"])
        line["e2e"] = {"value": ne / (te * 1e-3), "unit": UNIT, "host_cpus": host_cpus,
                       "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"]}
    steps_per_cycle = 1.0 / (cfg["dt"] * cfg["freq"])
    wall = {"plain_fp64": t_max / args.steps * 1e-3 * steps_per_cycle}

    # ---- mixed-precision form on the same reactor (FP32 push/deposit)
    if "mixed" in forms:
        cfgm = P.large_reactor(seed=replica_seed(1, rank), precision=P.PIC_MIXED)
        if args.np:
            cfgm["np_init"] = args.np
        rm = measure(P, torch, dev, cfgm, args, dist, D, False, False, local)
        tm, totm = maxsum(rm["t_ms"], rm["pushes"])
        alm = rm["push_ms"] / max(rm["push_launches"], 1)
        hbm_m = rm["bytes"] / (rm["push_ms"] * 1e-3) / 1e9
        fp32_peak = 128 * 2 * 152 * sm_max * 1e6 / 1e12
        flm = rm["flops"] / max(rm["commit_pushes"], 1)
        ppl = rm["pushes"] / max(rm["push_launches"], 1)
        line["mixed_form"] = {
            "value": totm / (tm * 1e-3), "unit": UNIT, "ms_per_step": tm / args.steps,
            "dtype": "f32 particles / f64 fields", "picard_iters": rm["iters"],
            "gpu_launches": rm["launches"],
            "roofline": {"bound": "hbm", "achieved": hbm_m, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": hbm_m / pk["hbm_gbs"],
                         "traffic": TRAFFIC_PER_PUSH_FP32 * ppl if TRAFFIC_PER_PUSH_FP32 else None,
                         "kernel": "k_push_fp32 (mover+deposit, FP32)", "peak_kind": pk_kind,
                         "bytes_per_push": "28 read (+24 written in the commit pass)",
                         "avg_launch_ms": alm, "launches": rm["push_launches"],
                         "alu": {"flop_per_push": flm,
                                 "achieved_tflops": flm * ppl / (alm * 1e-3) / 1e12,
                                 "peak_tflops": fp32_peak,
                                 "peak_kind": "FP32: 128 lanes x 152 SMs x 2 x max SM clock"}}}
        wall["mixed"] = tm / args.steps * 1e-3 * steps_per_cycle
        line["picard_loop"]["mixed"] = rm["picard_loop"]
    # ---- the paper's feed: the axial dielectric port below a 0.2 m electrode
    # (quartz, 16 rows graded over 6.5 cm) with the blocking capacitor, FP64
    if "port" in forms:
        cfgp = P.large_reactor(seed=replica_seed(1, rank), feed=P.PIC_FEED_AXIAL, port_rin=171,
                               port_cells=16, port_len=0.065, eps_port=3.8, port_grade=1.15,
                               cblock=1e-9)
        if args.np:
            cfgp["np_init"] = args.np
        rp = measure(P, torch, dev, cfgp, args, dist, D, False, False, local)
        tp, totp = maxsum(rp["t_ms"], rp["pushes"])
        line["axial_port_form"] = {
            "value": totp / (tp * 1e-3), "unit": UNIT, "ms_per_step": tp / args.steps,
            "picard_iters": rp["iters"], "gpu_launches": rp["launches"],
            "config": "256x384 reactor, electrode r_p = 0.2 m fed through the axial port "
                      "(R = 0.3 m, quartz, 16 rows graded 1.15 over 6.5 cm), blocking "
                      "capacitor 1 nF, FP64, %d macro-particles/species" % cfgp["np_init"]}
    # ---- electrostatic field model (Eq. 8) on the same reactor, mixed form
    if "es" in forms:
        cfge = P.large_reactor(seed=replica_seed(1, rank), precision=P.PIC_MIXED, field_model=P.PIC_FIELD_ES)
        if args.np:
            cfge["np_init"] = args.np
        re_ = measure(P, torch, dev, cfge, args, dist, D, False, False, local)
        te, tote = maxsum(re_["t_ms"], re_["pushes"])
        line["es_form"] = {"value": tote / (te * 1e-3), "unit": UNIT, "ms_per_step": te / args.steps,
                           "picard_iters": re_["iters"], "gpu_launches": re_["launches"],
                           "field_model": "electrostatic (Eq. 8), mixed-precision push"}
        wall["mixed_es"] = te / args.steps * 1e-3 * steps_per_cycle

    # ---- learned Picard start (mixed form): trained on the discharge's own fields
    if "guess" in forms:
        from paper_2212_08836_gb300 import guess as GS
        cfgg = P.large_reactor(seed=replica_seed(1, rank), precision=P.PIC_MIXED, capacity_factor=2.5)
        if args.np:
            cfgg["np_init"] = args.np
        pic = P.Pic(cfgg, device=dev)
        pic.load_particles()
        pic.step(args.guess_warmup)
        X, T = GS.collect(pic, args.guess_samples)
        net = P.Cnn(cfgg["nr"], cfgg["nz"], batch=8, device=dev)
        t0 = time.perf_counter()
        loss, val, zero = GS.train(net, X, T, args.guess_epochs)
        t_train = time.perf_counter() - t0
        del X, T
        rs = GS.run_starts(pic, net, args.guess_steps)
        line["learned_guess"] = {
            "workload": "mixed form, 256x384 reactor after %d steps (%d samples, %d Adam steps "
                        "of batch 8, %.0f s)" % (args.guess_warmup, args.guess_samples,
                                                 args.guess_epochs, t_train),
            "network": "5 x conv3x3, 14-64-64-64-64-2, BF16 weights/activations, FP32 accumulate, "
                       "%d parameters" % net.num_params,
            "heldout_loss": val, "heldout_loss_no_correction": zero,
            "starts": rs, "tol": cfgg["picard_tol"]}
        wall["mixed_learned_start"] = rs["cnn"]["ms_per_step"] * 1e-3 * steps_per_cycle
        wall["mixed_plain_start_same_state"] = rs["plain"]["ms_per_step"] * 1e-3 * steps_per_cycle
        pic.close()
        net.close()
    # the Maxwellian start's step times scaled to an RF cycle (context only)
    line["wall_s_per_rf_cycle_maxwellian_extrapolated"] = wall

    # ---- the developed discharge (5 RF cycles): one RF cycle of each form timed
    if "developed" in forms:
        dv = run_developed_form(P, torch, dev, args, rank)
        line["developed_state"] = dv
        if "wall_s_per_rf_cycle" in dv:
            line["wall_s_per_rf_cycle"] = dict(dv["wall_s_per_rf_cycle"],
                                               note="measured over one RF cycle of the developed "
                                                    "discharge, tol 1e-8, device synchronised")

    # ---- batched ensemble of 16 uneven discharges (mixed form) vs the same
    # discharges stepped one after another
    if "ensemble" in forms:
        line["ensemble"] = run_ensemble_form(P, torch, dev, args, rank)

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        rate, secs, npush = cpu_oracle_rate(args.cpu_sample, steps=1, threads=cores)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "%d macro-particles per species on the 256x384 grid, 1 whole "
                                          "step (%d pushes, %.1f s); push over %d threads (OpenMP, "
                                          "per-thread crossed charge), field solve, MCC and sort serial"
                                          % (args.cpu_sample, npush, secs, cores)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        D.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=1 << 22)
    ap.add_argument("--ref-sample", type=int, default=1 << 20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--np", type=int, default=0, help="macro-particles per species (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--forms", default="plain,mixed,es,port,developed,ensemble",
                    help="comma list of plain (FP64), mixed (FP32 push), es (electrostatic "
                         "model), port (the axial port with the capacitor), guess (mixed form "
                         "with the learned Picard start), developed (the FP64 form after 5 RF "
                         "cycles) and ensemble (16 uneven discharges) to time")
    ap.add_argument("--guess-warmup", type=int, default=400)
    ap.add_argument("--guess-samples", type=int, default=600)
    ap.add_argument("--guess-epochs", type=int, default=1500)
    ap.add_argument("--guess-steps", type=int, default=100)
    args = ap.parse_args()
    args.steps_e2e = args.steps
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
