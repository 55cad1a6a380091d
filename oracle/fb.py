"""Fourier-Bessel decomposition along r (App. A, Eq. A2) and the surface-mode
dispersion relations (Sec. 3.1, Eqs. 9-10 of the paper's numbering eq3_1 /
eq3_2), plain numpy / scipy.  Test infrastructure only.

Eq. A2 on the mesh: the radial integrals are evaluated by the trapezoid rule
on the nodes r_i = i dr for quantities on the nodes (E_z, alpha = 0) and by
the midpoint rule on r_{i+1/2} for quantities on the radial edges (E_r,
alpha = 1); numerator and denominator use the same rule.
"""
from __future__ import annotations

import numpy as np
from scipy import special as sp


def basis_points(nr, R, alpha, xa=0):
    """Sample radii and quadrature weights of int_0^R dr (.) for a field with
    Bessel order alpha (0: nodes, trapezoid; 1: cell centres, midpoint), on
    the uniform mesh or the mapped one (xa > 0, r = 2 dr sqrt(xa xi) for
    xi <= xa, dr (xi + xa) beyond, dr = R / (nr + xa))."""
    dr = R / (nr + xa)
    i = np.arange(nr + 1, dtype=np.float64)
    rn = np.where(i < xa, 2.0 * dr * np.sqrt(xa * i), (i + xa) * dr)
    h = np.diff(rn)
    if alpha == 0:
        w = np.zeros(nr + 1)
        w[:-1] += 0.5 * h
        w[1:] += 0.5 * h
        return rn, w
    return 0.5 * (rn[:-1] + rn[1:]), h


def coefficients(f, nr, R, alpha, nmodes, xa=0):
    """c_m, m = 1..nmodes, of f sampled at basis_points(nr, R, alpha, xa):
    c_m = int r f F_m dr / int r F_m^2 dr, F_m = J_alpha(chi_{alpha,m} r / R)."""
    r, w = basis_points(nr, R, alpha, xa)
    chi = sp.jn_zeros(alpha, nmodes)
    F = sp.jv(alpha, np.outer(chi, r) / R)
    num = F @ (w * r * np.asarray(f, dtype=np.float64))
    den = (F * F) @ (w * r)
    return num / den


# ------------------------------------------------------------ dispersion
def es_omega(k, wpe, s, d, mode="symmetric"):
    """Electrostatic surface-mode dispersion (the c -> infinity form, eq3_2):
    uniform plasma of half width d between two sheaths of width s."""
    t = 1.0 / np.tanh(k * d) if mode == "symmetric" else np.tanh(k * d)
    return wpe * np.sqrt(t / (1.0 / np.tanh(k * s) + t))


def em_residual(w, k, wpe, s, d, c, mode="symmetric"):
    """Electromagnetic surface-mode relation (eq3_1) as
    beta cosh(a s) X(b d) + a eps_p sinh(a s) Y(b d) = 0, the relation
    multiplied by sinh(a s) and by sinh or cosh of (b d), with
    a = sqrt(k^2 - w^2/c^2) (sheath, vacuum), b = sqrt(k^2 - eps_p w^2/c^2)
    (plasma), eps_p = 1 - wpe^2/w^2; real for real or imaginary a."""
    ep = 1.0 - (wpe / w) ** 2
    a = np.sqrt(complex(k * k - (w / c) ** 2))
    b = np.sqrt(complex(k * k - ep * (w / c) ** 2))
    if mode == "symmetric":      # beta coth(a s) = -a eps_p coth(b d)
        g = b * np.cosh(a * s) * np.sinh(b * d) + a * ep * np.sinh(a * s) * np.cosh(b * d)
    else:                        # beta coth(a s) = -a eps_p tanh(b d)
        g = b * np.cosh(a * s) * np.cosh(b * d) + a * ep * np.sinh(a * s) * np.sinh(b * d)
    return float(np.real(g))


def em_omega(k, wpe, s, d, c, mode="symmetric", n=4000):
    """Lowest root in (0, wpe) of em_residual by a sign scan and bisection
    (NaN if none)."""
    ws = np.linspace(wpe * 1e-4, wpe * (1 - 1e-9), n)
    g = np.array([em_residual(w, k, wpe, s, d, c, mode) for w in ws])
    idx = np.where(np.sign(g[:-1]) * np.sign(g[1:]) < 0)[0]
    if len(idx) == 0:
        return float("nan")
    lo, hi = ws[idx[0]], ws[idx[0] + 1]
    glo = g[idx[0]]
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        gm = em_residual(mid, k, wpe, s, d, c, mode)
        if np.sign(gm) == np.sign(glo):
            lo, glo = mid, gm
        else:
            hi = mid
    return 0.5 * (lo + hi)
