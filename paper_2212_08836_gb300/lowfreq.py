"""The low-frequency comparison of the electrostatic and electromagnetic
models (Sec. 3.2), run on the GPU.

At 13.56 MHz the wavelength is far larger than the reactor, so the two field
models must give the same discharge.  The reactor is asymmetric: the powered
electrode is the disc r <= r_p of z = 0, fed through the axial port (the
electromagnetic model's coaxial dielectric port, Eqs. 5 and 7; the
electrostatic model's Dirichlet port, Sec. 2.2), while the grounded top plate
and side wall are larger, and the blocking capacitor (Eq. 6) between the
generator and the electrode lets the discharge build the negative self-bias
that balances the electron and ion currents to the small electrode.  Both
models start from the same particles; per RF cycle the run records the mean
electrode potential (the self-bias) and its RF amplitude, and over the last
cycles the time-averaged electron and ion densities.  Usage as a script:

    python -m paper_2212_08836_gb300.lowfreq --out lowfreq.npz [--cycles 6]
"""
from __future__ import annotations

import argparse
import time

import numpy as np

from . import (PIC_DIAG_DENSITY_AVG, PIC_FEED_AXIAL, PIC_FIELD_EM, PIC_FIELD_ES, Pic,
               set_graphs, small_reactor)


def config(model, f=13.56e6, steps_per_cycle=400, volt=200.0, cblock=50e-12, port_rin=21,
           np_init=40000, seed=3, **kw):
    """The small reactor (32 x 64, R = 0.1 m, L = 0.03 m, argon 2 Pa) fed at f
    through the axial port of inner radius r(port_rin) with the blocking
    capacitor cblock; model: "es" or "em"."""
    fm = PIC_FIELD_ES if model == "es" else PIC_FIELD_EM
    args = dict(freq=f, dt=1.0 / (steps_per_cycle * f), volt=volt, field_model=fm,
                cblock=cblock, feed=PIC_FEED_AXIAL, port_rin=port_rin, port_cells=4,
                port_len=0.02, eps_port=3.8, np_init=np_init, mcc_on=1, seed=seed,
                capacity_factor=3.0)
    args.update(kw)   # e.g. feed=PIC_FEED_GAP: the same discharge between equal plates
    return small_reactor(**args)


def run(model, cycles=6, avg_cycles=2, device="cuda:0", **kw):
    """Runs `cycles` RF cycles from the loaded Maxwellian plasma; returns the
    self-bias and the RF amplitude of the electrode potential per cycle, the
    Picard iterations per step, and the electron and ion node densities
    ((nr+1) x (nz+1) each) averaged over the last avg_cycles cycles."""
    import torch
    cfg = config(model, **kw)
    spc = int(round(1.0 / (cfg["dt"] * cfg["freq"])))
    pic = Pic(cfg, device=device, stream=torch.cuda.Stream(device=device))
    set_graphs(pic, True)
    pic.load_particles()
    bias, amp, iters = [], [], []
    t0 = time.time()
    for c in range(cycles):
        if c == cycles - avg_cycles:
            pic.diag_average(True)
        phi = np.empty(spc)
        for k in range(spc):
            rc, st = pic.step(1, check=False)
            if rc not in (0, -4):   # PIC_E_SUBSTEP is reported and kept
                raise RuntimeError("pic_step failed with %d in cycle %d, step %d" % (rc, c, k))
            phi[k] = st["v_electrode"]
            iters.append(st["picard_iters"])
        bias.append(float(phi.mean()))
        amp.append(float(0.5 * (phi.max() - phi.min())))
    dens = np.asarray(pic.diag_get(PIC_DIAG_DENSITY_AVG), dtype=np.float64).ravel()
    nn = (cfg["nr"] + 1) * (cfg["nz"] + 1)
    out = {"model": model, "bias": np.array(bias), "amp": np.array(amp),
           "picard_iters_mean": float(np.mean(iters)),
           "ne": dens[:nn].reshape(cfg["nr"] + 1, cfg["nz"] + 1),
           "ni": dens[nn:2 * nn].reshape(cfg["nr"] + 1, cfg["nz"] + 1),
           "n": list(pic.view()["n"]), "wall_s": time.time() - t0, "port_rin": cfg["port_rin"]}
    pic.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--cycles", type=int, default=6)
    a = ap.parse_args()
    res = {m: run(m, cycles=a.cycles) for m in ("es", "em")}
    np.savez(a.out, **{"%s_%s" % (m, k): np.asarray(v) for m, r in res.items()
                      for k, v in r.items() if k != "model"})
    for m, r in res.items():
        print("%s: self-bias per cycle %s V, RF amplitude %.1f V, %.2f Picard iterations/step, "
              "%.1f s" % (m, np.round(r["bias"], 1), r["amp"][-1], r["picard_iters_mean"],
                          r["wall_s"]))


if __name__ == "__main__":
    main()
