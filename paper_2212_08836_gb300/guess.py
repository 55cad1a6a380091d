"""Training of the learned Picard start on data the method generates.

Runs a discharge with the extrapolated start (PIC_GUESS_EXTRAP), keeps each
step's (inputs, target) pair on the GPU, and trains the network with Adam on
random mini-batches; the network then serves as the start of pic_step
(PIC_GUESS_CNN).  Usage as a script writes the trained parameters:

    python -m paper_2212_08836_gb300.guess --out weights.npy [--steps 800]
        [--epochs 1500] [--pressure 2] [--volt 200] [--np 16777216]
"""
from __future__ import annotations

import argparse

import numpy as np

from . import (PIC_GUESS_CNN, PIC_GUESS_EXTRAP, PIC_GUESS_PLAIN, PIC_MIXED, Cnn, Pic,
               guess_sample, large_reactor, set_guess)


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


def train(net, X, T, epochs, batch=8, lr=1e-3, seed=0, holdout=0.2, log=None):
    """Adam on random mini-batches of the first (1 - holdout) of the pairs;
    returns (last training loss, held-out loss, held-out loss of a zero correction)."""
    import torch
    n = X.shape[0]
    ntr = max(1, int((1.0 - holdout) * n))
    g = torch.Generator(device="cpu").manual_seed(seed)
    loss = float("nan")
    for ep in range(epochs):
        idx = torch.randint(0, ntr, (min(batch, net.batch),), generator=g)
        loss = net.train_step(X[idx], T[idx], lr if ep < 0.7 * epochs else 0.3 * lr)
        if log and ep % 500 == 0:
            log("epoch %d loss %.3e" % (ep, loss))
    val, zero = [], []
    for k in range(ntr, n, net.batch):
        xb, tb = X[k:k + net.batch], T[k:k + net.batch]
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
    a = ap.parse_args()
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
