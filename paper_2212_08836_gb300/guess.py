"""Training of the learned Picard start on data the method generates.

Runs a discharge with the extrapolated start (PIC_GUESS_EXTRAP), keeps each
step's (inputs, target) pair on the GPU, and trains the network with Adam on
random mini-batches; the network then serves as the start of pic_step
(PIC_GUESS_CNN).  Usage as a script writes the trained parameters:

    python -m paper_2212_08836_gb300.guess --out weights.npy [--steps 800]
        [--epochs 1500] [--pressure 2] [--volt 200] [--np 16777216]

With --campaign the pairs come from one discharge per (pressure, voltage) of
the grid 1/2/5 Pa x 100/200/300 V (the same reactor, each developed first),
all kept on the GPU, and the trained network is then compared with the plain
start over whole RF cycles of developed discharges at 1, 2 and 5 Pa (200 V)
and at one condition outside the training grid (3 Pa, 150 V):

    python -m paper_2212_08836_gb300.guess --campaign --out weights.npy
        [--per-run 2222] [--warmup 1500] [--epochs 8000] [--depth 7]
"""
from __future__ import annotations

import argparse

import numpy as np

from . import (PIC_E_CAPACITY, PIC_GUESS_CNN, PIC_GUESS_EXTRAP, PIC_GUESS_PLAIN, PIC_MIXED, Cnn,
               Pic, PicError, guess_sample, large_reactor, set_guess)


def collect(pic, steps):
    """Steps pic with the extrapolated start; returns the stacked (X, T) pairs."""
    import torch
    set_guess(pic, PIC_GUESS_EXTRAP)
    xs, ts = [], []
    for _ in range(steps):
        pic.step(1)
        s = guess_sample(pic)
        if s is not None:
            xs.append(s[0].clone())
            ts.append(s[1].clone())
    return torch.stack(xs), torch.stack(ts)


def train(net, X, T, epochs, batch=8, lr=1e-3, seed=0, holdout=0.2, log=None, order=None):
    """Adam on random mini-batches of the first (1 - holdout) of the pairs (in
    `order`, a permutation of their indices, if given; X may be stored in
    bfloat16, which the network's input packing rounds to anyway); returns
    (last training loss, held-out loss, held-out loss of a zero correction)."""
    import torch
    n = X.shape[0]
    ntr = max(1, int((1.0 - holdout) * n))
    if order is None:
        order = torch.arange(n)
    g = torch.Generator(device="cpu").manual_seed(seed)
    loss = float("nan")
    for ep in range(epochs):
        idx = order[torch.randint(0, ntr, (min(batch, net.batch),), generator=g)].to(X.device)
        loss = net.train_step(X[idx].float(), T[idx], lr if ep < 0.7 * epochs else 0.3 * lr)
        if log and ep % 500 == 0:
            log("epoch %d loss %.3e" % (ep, loss))
    val, zero = [], []
    for k in range(ntr, n, net.batch):
        idx = order[k:k + net.batch].to(X.device)
        xb, tb = X[idx].float(), T[idx]
        val.append(net.loss_grad(xb, tb, grad=False)[0] * xb.shape[0])
        zero.append(float(tb.pow(2).sum().item()) / _nvalid(net))
    nv = max(n - ntr, 1)
    return loss, sum(val) / nv, sum(zero) / nv


def _nvalid(net):
    return net.nr * (net.nz + 1) + (net.nr + 1) * net.nz


def run_starts(pic, net, steps):
    """Picard iterations, first residuals and wall time per step for each start, in turn."""
    import time
    import torch
    out = {}
    for name, mode in (("plain", PIC_GUESS_PLAIN), ("extrap", PIC_GUESS_EXTRAP),
                       ("cnn", PIC_GUESS_CNN)):
        set_guess(pic, mode, net if mode == PIC_GUESS_CNN else None)
        it, fr, used = [], [], []
        pic.step(4)  # the history of the extrapolated starts refills
        torch.cuda.synchronize(pic.device)
        t0 = time.perf_counter()
        for _ in range(steps):
            _, st = pic.step(1)
            it.append(st["picard_iters"])
            fr.append(st["first_res"])
            used.append(st["guess"])
        torch.cuda.synchronize(pic.device)
        ms = (time.perf_counter() - t0) * 1e3 / steps
        used = np.array(used)
        keep = used == mode
        out[name] = {"picard_iters": float(np.mean(np.array(it)[keep])) if keep.any() else None,
                     "first_res_median": float(np.median(np.array(fr)[keep])) if keep.any() else None,
                     "steps": int(keep.sum()), "fallbacks": int(((used == 0) & (mode != 0)).sum()),
                     "ms_per_step": ms}
    return out


def _step(pic, n, capped):
    """n steps; a step that could not append all ionization pairs (the store is
    full) is committed all the same and counted in capped[0]."""
    for _ in range(n):
        try:
            st = pic.step(1)[1]
        except PicError as e:
            if e.code != PIC_E_CAPACITY:
                raise
            capped[0] += 1
            st = None
    return st


def campaign(a, log=print):
    """Pairs from 9 discharges (1/2/5 Pa x 100/200/300 V), training, then
    Picard iterations and wall time per RF cycle, plain against learned start."""
    import time
    import torch
    runs = [(p, v) for p in (1.0, 2.0, 5.0) for v in (100.0, 200.0, 300.0)]
    base = large_reactor(precision=PIC_MIXED, np_init=a.np, capacity_factor=a.capacity)
    capped = [0]
    H, W = base["nr"] + 1, base["nz"] + 1
    n = a.per_run * len(runs)
    X = torch.empty((n, 14, H, W), dtype=torch.bfloat16, device="cuda")
    T = torch.empty((n, 2, H, W), dtype=torch.float32, device="cuda")
    k = 0
    t0 = time.perf_counter()
    for p, v in runs:
        cfg = dict(base, gas_pressure=p, volt=v, seed=int(10 * p + v))
        pic = Pic(cfg)
        pic.load_particles()
        _step(pic, a.warmup, capped)
        set_guess(pic, PIC_GUESS_EXTRAP)
        got = 0
        while got < a.per_run:
            _step(pic, 1, capped)
            smp = guess_sample(pic)
            if smp is not None:
                X[k].copy_(smp[0])
                T[k].copy_(smp[1])
                k += 1
                got += 1
        log("collected %d pairs at %.0f Pa %.0f V (%.0f s, %d M / %d M particles)"
            % (got, p, v, time.perf_counter() - t0, pic.diag()["n"][0] >> 20,
               pic.diag()["n"][1] >> 20))
        pic.close()
    # one permutation, so that the held-out fifth mixes every discharge
    order = torch.randperm(n, generator=torch.Generator().manual_seed(0))
    net = Cnn(base["nr"], base["nz"], depth=a.depth, batch=8)
    t1 = time.perf_counter()
    loss, val, zero = train(net, X, T, a.epochs, log=log, order=order)
    t_train = time.perf_counter() - t1
    log("train %.3e held-out %.3e (no correction %.3e), %.0f s" % (loss, val, zero, t_train))
    del X, T
    torch.cuda.empty_cache()
    res = {"pairs": n, "params": net.num_params, "np_init": a.np, "capacity_factor": a.capacity, "depth": a.depth, "adam_steps": a.epochs,
           "train_s": t_train, "heldout_loss": val, "heldout_loss_no_correction": zero,
           "cycles": []}
    steps_cycle = int(round(1.0 / (base["freq"] * base["dt"])))
    for p, v in ((1.0, 200.0), (2.0, 200.0), (5.0, 200.0), (3.0, 150.0)):
        cfg = dict(base, gas_pressure=p, volt=v, seed=int(10 * p + v) + 7)
        pic = Pic(cfg)
        pic.load_particles()
        _step(pic, a.warmup, capped)
        row = {"pressure_pa": p, "volt": v}
        for name, mode in (("plain", PIC_GUESS_PLAIN), ("learned", PIC_GUESS_CNN)):
            set_guess(pic, mode, net if mode == PIC_GUESS_CNN else None)
            _step(pic, 4, capped)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            it, used = [], []
            for _ in range(steps_cycle):
                st = _step(pic, 1, capped)
                if st is None:
                    continue
                it.append(st["picard_iters"])
                used.append(st["guess"])
            torch.cuda.synchronize()
            row[name] = {"wall_s": time.perf_counter() - t2,
                         "picard_iters_mean": float(np.mean(it)),
                         "steps_on_this_start": int(np.sum(np.array(used) == mode))}
        log(str(row))
        res["cycles"].append(row)
        pic.close()
    res["capacity_limited_steps"] = capped[0]
    net_params = net.get_params()
    net.close()
    return res, net_params


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--steps", type=int, default=800)
    ap.add_argument("--warmup", type=int, default=400)
    ap.add_argument("--epochs", type=int, default=1500)
    ap.add_argument("--pressure", type=float, default=2.0)
    ap.add_argument("--volt", type=float, default=200.0)
    ap.add_argument("--np", type=int, default=16 * 1024 * 1024)
    ap.add_argument("--depth", type=int, default=5)
    ap.add_argument("--campaign", action="store_true")
    ap.add_argument("--per-run", type=int, default=2222)
    ap.add_argument("--capacity", type=float, default=2.5)
    a = ap.parse_args()
    if a.campaign:
        import json
        res, params = campaign(a)
        print(json.dumps(res))
        np.save(a.out, params)
        return
    cfg = large_reactor(precision=PIC_MIXED, np_init=a.np, gas_pressure=a.pressure, volt=a.volt,
                        capacity_factor=2.5)
    pic = Pic(cfg)
    pic.load_particles()
    pic.step(a.warmup)
    X, T = collect(pic, a.steps)
    net = Cnn(cfg["nr"], cfg["nz"], depth=a.depth, batch=8)
    loss, val, zero = train(net, X, T, a.epochs, log=print)
    print("train %.3e held-out %.3e (no correction %.3e)" % (loss, val, zero))
    np.save(a.out, net.get_params())


if __name__ == "__main__":
    main()
