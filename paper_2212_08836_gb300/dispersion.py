"""Surface-mode spectrum of a uniform plasma between two sheaths, the
verification problem of Sec. 3.1, run on the GPU.

Ions are held at a uniform density n0 over the whole gap; electrons of the
same density fill the slab s < z < L - s, so that both electrodes carry an
electron-free (matrix) sheath of width s, which the electrons, confined by the
sheath potential, keep.  (Sec. 3.1 forms the sheaths with a sinusoidal drive
first; loading them formed gives the same configuration with s known and
avoids the formation phase, whose wall losses make the Picard iteration
stall at a few 1e-4.)  The plasma is then driven by the sawtooth-like voltage
V(t) = A sum_{n=1..N} sin(2 pi n f t) / n.  Every step E_z at a fixed distance
from the powered electrode (inside its sheath) is decomposed along r into
Fourier-Bessel modes (App. A, alpha = 0); an FFT in time of each mode's
coefficient gives the spectrum, whose peaks follow the surface-mode
dispersion curves at k_m = chi_{0,m}/R (symmetric) and chi_{1,m}/R
(antisymmetric).  Usage as a script writes the spectrum to an .npz file:

    python -m paper_2212_08836_gb300.dispersion --out spectrum.npz [--model es|em]
"""
from __future__ import annotations

import argparse
import time

import numpy as np

from . import PIC_FIELD_EM, PIC_FIELD_ES, PIC_FP64, Pic, small_reactor

QE = 1.602176634e-19
ME = 9.1093837015e-31


def advance(pic, tol, relaxed, k):
    """One step; a step whose Picard iteration stalls above tol (a few
    particles switch between sub-step paths) is retried with a tolerance ten
    times looser, down to 1e-3, and recorded in relaxed.  A particle at the
    sub-step cap is reported (PIC_E_SUBSTEP) and kept."""
    rc, st = pic.step(1, check=False)
    t = tol
    while rc == -3 and t < 1e-3:
        t *= 10.0
        pic.set_picard(t, 100)
        rc, st = pic.step(1, check=False)
        pic.set_picard(tol, 100)
        relaxed.append((k, t))
    if rc not in (0, -4):
        raise RuntimeError("pic_step failed with %d at step %d (iterations %d, residual %.3g)"
                           % (rc, k, st["picard_iters"], st["last_res"]))
    return st


def slab_plasma(nr, nz, R, L, n0, ppc, s, te_ev, seed):
    """Electrons uniform over s < z < L - s and ions uniform over the gap, both
    at density n0 (uniform in the logical coordinates, weights proportional
    to r); electron velocities Maxwellian at te_ev, ions at rest."""
    rng = np.random.default_rng(seed)
    out = []
    for sp, (z0, z1) in enumerate(((s, L - s), (0.0, L))):
        n = int(ppc * nr * nz * (z1 - z0) / L)
        xi = rng.random(n) * nr
        eta = (z0 + rng.random(n) * (z1 - z0)) / (L / nz)
        ic = np.minimum(xi.astype(np.int64), nr - 1)
        jc = np.minimum(eta.astype(np.int64), nz - 1)
        w = n0 * 2 * np.pi * xi * (R / nr) * R * (z1 - z0) / n
        v = rng.normal(size=(3, n)) * np.sqrt(te_ev * QE / ME) if sp == 0 else np.zeros((3, n))
        cell = (ic * nz + jc).astype(np.int32)
        o = np.argsort(cell, kind="stable")
        out.append({"cell": cell[o], "a": (xi - ic)[o], "b": (eta - jc)[o], "vr": v[0][o],
                    "vt": v[1][o], "vz": v[2][o], "w": w[o],
                    "id": np.arange(n, dtype=np.uint32)})
    return out


def run(model="es", nr=64, nz=128, R=0.1, L=0.03, n0=1e16, ppc=64, sheath=1.8e-3, f=106e6,
        amp=10.0, nharm=20, obs_cycles=64, z_sample=1e-3, nmodes=10, dt=1e-10, mu=0.0,
        te_ev=3.0, seed=0, device="cuda:0", precision=PIC_FP64, tol=1e-7):
    import torch
    fm = PIC_FIELD_ES if model == "es" else PIC_FIELD_EM
    cfg = small_reactor(nr=nr, nz=nz, R=R, L=L, dt=dt, freq=f, volt=0.0, n0=n0, te_ev=te_ev,
                        np_init=int(ppc * nr * nz), capacity_factor=1.0, mcc_on=0,
                        ions_fixed=1, field_model=fm, precision=precision, mu=mu, seed=seed,
                        picard_tol=tol, picard_max=100)
    pic = Pic(cfg, device=device, stream=torch.cuda.Stream(device=device))
    sp = slab_plasma(nr, nz, R, L, n0, ppc, sheath, te_ev, seed)
    pic.set_state(sp)
    # Gauss-consistent start: the electrostatic field of the loaded charge
    er = torch.zeros(nr * (nz + 1), dtype=torch.float64, device=device)
    ez = torch.zeros((nr + 1) * nz, dtype=torch.float64, device=device)
    pic.es_solve(pic.node_charge(), 0.0, er, ez)
    torch.cuda.synchronize(device)
    pic.set_state(sp, er=er.cpu().numpy(), ez=ez.cpu().numpy())
    harm = np.arange(1, nharm + 1)
    pic.set_drive(list(amp / harm), list(harm * f), [0.0] * nharm)
    n_obs = int(round(obs_cycles / (f * dt)))
    dz = L / nz
    row = int(round(z_sample / dz - 0.5))
    coef = torch.empty((n_obs, nmodes), dtype=torch.float64, device=device)
    iters, sub_err, relaxed = [], [], []
    t0 = time.time()
    for k in range(n_obs):
        st = advance(pic, tol, relaxed, k)
        iters.append(st["picard_iters"])
        if st["substep_err"]:
            sub_err.append((k, st["substep_err"]))
        pic.fourier_bessel(0, row, nmodes, out=coef[k])
    wall = time.time() - t0
    c = coef.cpu().numpy()
    c -= c.mean(axis=0)
    win = np.hanning(n_obs)[:, None]
    spec = np.abs(np.fft.rfft(c * win, axis=0)) ** 2
    freqs = np.fft.rfftfreq(n_obs, dt)
    return {"freqs": freqs, "spectrum": spec.T, "sheath": sheath, "n0": n0, "R": R, "L": L,
            "dz": dz, "row": row, "z_sample": (row + 0.5) * dz, "steps": n_obs, "wall_s": wall,
            "model": model, "mu": mu, "picard_iters_mean": float(np.mean(iters)),
            "substep_errors": np.array(sub_err, dtype=np.int64).reshape(-1, 2), "coef": c,
            "relaxed": np.array(relaxed, dtype=np.float64).reshape(-1, 2)}


def bessel_zero0(m):
    """m-th positive zero of J_0 (scipy)."""
    from scipy import special as sp
    return float(sp.jn_zeros(0, m)[m - 1])


def ring(model="es", mode="symmetric", m=1, nr=64, nz=128, R=0.1, L=0.03, n0=1e16, ppc=64,
         sheath=1.8e-3, u0=5e4, steps=800, z_sample=1e-3, dt=1e-10, mu=0.0, te_ev=3.0, seed=0,
         device="cuda:0", precision=PIC_FP64, tol=1e-7, base=None, band=None):
    """Free oscillation of one surface mode: the electrons of the loaded slab
    get the axial velocity u0 J_0(chi_{0,m} r / R), uniform in z (symmetric
    mode: the slab moves between the two sheaths, the plasma series resonance
    at k -> 0) or of opposite sign in the two halves of the gap (antisymmetric
    mode); the ringing of the Fourier-Bessel coefficient c_m of E_z in the
    sheaths gives the mode's frequency at k = chi_{0,m} / R (the perturbed
    potential vanishes on the side wall, so both symmetries use the zeros of
    J_0).  Symmetric: c_m in the powered sheath.  Antisymmetric: half the
    difference of c_m in the two sheaths, at the same distance from either
    plate, in which the symmetric mode (E_z even about the midplane) cancels
    and the antisymmetric one (E_z odd) adds.  base: the series of the same
    run with u0 = 0, which is subtracted so that only the response to the kick
    remains.  band: (f_lo, f_hi) [Hz] to which the peak search is limited
    (None: the whole spectrum).  Returns the frequency from the FFT peak
    (parabolic interpolation on a 16x zero-padded spectrum) and the raw
    series."""
    import torch
    fm = PIC_FIELD_ES if model == "es" else PIC_FIELD_EM
    cfg = small_reactor(nr=nr, nz=nz, R=R, L=L, dt=dt, freq=1e6, volt=0.0, n0=n0,
                        te_ev=te_ev, np_init=int(ppc * nr * nz), capacity_factor=1.0, mcc_on=0,
                        ions_fixed=1, field_model=fm, precision=precision, mu=mu, seed=seed,
                        picard_tol=tol, picard_max=100)
    pic = Pic(cfg, device=device, stream=torch.cuda.Stream(device=device))
    sp = slab_plasma(nr, nz, R, L, n0, ppc, sheath, te_ev, seed)
    e = sp[0]
    chi = bessel_zero0(m)
    from scipy import special as ss
    xi = e["cell"] // nz + e["a"]   # r / dr on the uniform mesh
    eta = e["cell"] % nz + e["b"]
    prof = ss.j0(chi * xi / nr)     # J_0(chi r / R)
    sign = np.ones_like(eta) if mode == "symmetric" else np.where(eta < 0.5 * nz, -1.0, 1.0)
    e["vz"] = e["vz"] + u0 * prof * sign
    pic.set_state(sp)
    er = torch.zeros(nr * (nz + 1), dtype=torch.float64, device=device)
    ez = torch.zeros((nr + 1) * nz, dtype=torch.float64, device=device)
    pic.es_solve(pic.node_charge(), 0.0, er, ez)
    torch.cuda.synchronize(device)
    pic.set_state(sp, er=er.cpu().numpy(), ez=ez.cpu().numpy())
    row = int(round(z_sample / (L / nz) - 0.5))
    anti = mode != "symmetric"
    coef = torch.empty((steps, m), dtype=torch.float64, device=device)
    coef2 = torch.empty((steps, m), dtype=torch.float64, device=device) if anti else None
    iters, relaxed = [], []
    for k in range(steps):
        st = advance(pic, tol, relaxed, k)
        iters.append(st["picard_iters"])
        pic.fourier_bessel(0, row, m, out=coef[k])
        if anti:   # the mirror row in the grounded sheath
            pic.fourier_bessel(0, nz - 1 - row, m, out=coef2[k])
    c = coef[:, m - 1].cpu().numpy()
    if anti:
        c = 0.5 * (c - coef2[:, m - 1].cpu().numpy())
    series = c.copy()
    if base is not None:
        # the response to the kick alone: the unkicked run with the same
        # particles carries the loaded slab's own oscillation and the noise
        c = c - base
    c = c - c.mean()
    pad = 16 * len(c)
    P = np.abs(np.fft.rfft(c * np.hanning(len(c)), n=pad)) ** 2
    f = np.fft.rfftfreq(pad, dt)
    lo, hi = (1, len(P)) if band is None else (max(1, int(np.ceil(band[0] / f[1]))),
                                               min(len(P), int(band[1] / f[1]) + 1))
    k0 = int(np.argmax(P[lo:hi])) + lo
    if 1 <= k0 < len(P) - 1:
        a, b, cc = np.log(P[k0 - 1]), np.log(P[k0]), np.log(P[k0 + 1])
        k0 = k0 + 0.5 * (a - cc) / (a - 2 * b + cc)
    return {"freq": float(k0 * (f[1] - f[0])), "series": series,
            "k": chi / R, "model": model,
            "mode": mode, "m": m, "picard_iters_mean": float(np.mean(iters)),
            "relaxed_steps": len(relaxed)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--model", default="es")
    ap.add_argument("--obs-cycles", type=int, default=64)
    ap.add_argument("--ppc", type=int, default=64)
    ap.add_argument("--mu", type=float, default=0.0)
    a = ap.parse_args()
    r = run(model=a.model, obs_cycles=a.obs_cycles, ppc=a.ppc, mu=a.mu)
    np.savez(a.out, **{k: np.asarray(v) for k, v in r.items()})
    ne = int(r["substep_errors"][:, 1].sum())
    print("model %s: %d steps in %.1f s, %.2f Picard iterations/step, sub-step cap reached %d "
          "times, %d steps retried with a looser tolerance" %
          (r["model"], r["steps"], r["wall_s"], r["picard_iters_mean"], ne, len(r["relaxed"])))


if __name__ == "__main__":
    main()
