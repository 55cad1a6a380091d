"""Surface-mode spectrum of a uniform plasma between two sheaths, the
verification problem of Sec. 3.1, run on the GPU.

Ions are held at a uniform density n0; a sinusoidal generator voltage forms
the sheaths, then it is replaced by the sawtooth-like excitation
V(t) = A sum_{n=1..N} sin(2 pi n f (t - t_s)) / n.  Every step E_z at a fixed
distance from the powered electrode is decomposed along r into Fourier-Bessel
modes (App. A, alpha = 0); an FFT in time of each mode's coefficient gives
the spectrum, whose peaks follow the surface-mode dispersion curves at
k_m = chi_{0,m}/R (symmetric) and chi_{1,m}/R (antisymmetric).  The sheath
width is read from the time-averaged electron density on the nodes.  Usage as
a script writes the spectrum to an .npz file:

    python -m paper_2212_08836_gb300.dispersion --out spectrum.npz [--model es|em]
"""
from __future__ import annotations

import argparse
import time

import numpy as np

from . import PIC_FIELD_EM, PIC_FIELD_ES, PIC_FP64, PIC_MIXED, Pic, small_reactor

QE = 1.602176634e-19


def run(model="es", nr=64, nz=128, R=0.1, L=0.03, n0=1e16, ppc=64, f=106e6, v_form=100.0,
        form_cycles=20, amp=1.0, nharm=20, obs_cycles=64, z_sample=1e-3, nmodes=10,
        dt=1e-10, mu=0.0, te_ev=3.0, seed=0, device="cuda:0", precision=PIC_FP64,
        profile_every=10):
    import torch
    fm = PIC_FIELD_ES if model == "es" else PIC_FIELD_EM
    npart = int(ppc * nr * nz)
    cfg = small_reactor(nr=nr, nz=nz, R=R, L=L, dt=dt, freq=f, volt=v_form, n0=n0, te_ev=te_ev,
                        np_init=npart, capacity_factor=1.0, mcc_on=0, ions_fixed=1,
                        field_model=fm, precision=precision, mu=mu, seed=seed,
                        picard_tol=1e-5 if precision == PIC_MIXED else 1e-8)
    pic = Pic(cfg, device=device, stream=torch.cuda.Stream(device=device))
    pic.load_particles()
    t0 = time.time()
    n_form = int(round(form_cycles / (f * dt)))
    iters = []
    for _ in range(n_form):
        iters.append(pic.step(1)[1]["picard_iters"])
    # sawtooth from t_s on: phases make every harmonic start at zero
    ts = n_form * dt
    harm = np.arange(1, nharm + 1)
    pic.set_drive(list(amp / harm), list(harm * f), list(-2 * np.pi * harm * f * ts))
    n_obs = int(round(obs_cycles / (f * dt)))
    dz, dr = L / nz, R / nr
    row = int(round(z_sample / dz - 0.5))
    coef = torch.empty((n_obs, nmodes), dtype=torch.float64, device=device)
    # node charge summed over the inner half radius per axial node (the ions
    # stay uniform, so the electron density follows from the net charge)
    qsum = torch.zeros(nz + 1, dtype=torch.float64, device=device)
    nprof = 0
    for k in range(n_obs):
        iters.append(pic.step(1)[1]["picard_iters"])
        pic.fourier_bessel(0, row, nmodes, out=coef[k])
        if k % profile_every == 0:
            qsum += pic.node_charge().reshape(nr + 1, nz + 1)[: nr // 2].sum(0)
            nprof += 1
    wall = time.time() - t0
    az = 2 * np.pi * np.arange(nr // 2) * dr * dr
    az[0] = np.pi * (0.5 * dr) ** 2
    ne = 1.0 - qsum.cpu().numpy() / max(nprof, 1) / (QE * n0 * az.sum() * dz)
    c = coef.cpu().numpy()
    c -= c.mean(axis=0)
    win = np.hanning(n_obs)[:, None]
    spec = np.abs(np.fft.rfft(c * win, axis=0)) ** 2
    freqs = np.fft.rfftfreq(n_obs, dt)
    inner = ne[1:nz]
    half = inner > 0.5
    s0 = (np.argmax(half) + 1) * dz if half.any() else np.nan
    s1 = (np.argmax(half[::-1]) + 1) * dz if half.any() else np.nan
    return {"freqs": freqs, "spectrum": spec.T, "ne_profile": ne, "sheath": (s0, s1),
            "n0": n0, "R": R, "L": L, "dz": dz, "row": row, "z_sample": (row + 0.5) * dz,
            "steps": n_form + n_obs, "wall_s": wall, "model": model, "mu": mu,
            "picard_iters_mean": float(np.mean(iters))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--model", default="es")
    ap.add_argument("--obs-cycles", type=int, default=64)
    ap.add_argument("--form-cycles", type=int, default=20)
    ap.add_argument("--ppc", type=int, default=64)
    ap.add_argument("--mu", type=float, default=0.0)
    a = ap.parse_args()
    r = run(model=a.model, obs_cycles=a.obs_cycles, form_cycles=a.form_cycles, ppc=a.ppc,
            mu=a.mu)
    np.savez(a.out, **{k: np.asarray(v) for k, v in r.items()})
    print("model %s sheaths %.3f / %.3f mm, %d steps in %.1f s, %.2f Picard iterations/step" %
          (r["model"], r["sheath"][0] * 1e3, r["sheath"][1] * 1e3, r["steps"], r["wall_s"],
           r["picard_iters_mean"]))


if __name__ == "__main__":
    main()
