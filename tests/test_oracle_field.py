"""Pins of the oracle's implicit Maxwell solve (row a4).

Fixed by the mathematics, not by the oracle: CN conserves the discrete field
energy exactly in a closed PEC box (adjoint curls); the discrete divergence
of the curl vanishes (Gauss unchanged without charge); the vacuum TM010
pill-box mode oscillates at (2/dt)*atan(w dt/2) with w = chi01*c/R (CN phase
error, closed form; continuum frequency to O(dr^2)); a slow gap drive gives
the quasi-static capacitor field V/L between the plates; with the drive the
field-energy change equals the energy delivered through the gap edges.
"""
import numpy as np
import pytest
from scipy.special import jn_zeros, j0

import oracle as O


def test_vacuum_energy_conserved_closed_box():
    g = O.Grid(12, 20, 0.05, 0.03)
    dt = 1e-11
    F = O.FieldSolver(g, dt)
    rng = np.random.default_rng(0)
    er, ez, h = g.zeros_fields()
    er[:] = rng.normal(size=g.n_er)
    er.reshape(g.nr, g.nz + 1)[:, [0, -1]] = 0.0
    ez[:] = rng.normal(size=g.n_ez)
    ez.reshape(g.nr + 1, g.nz)[-1, :] = 0.0
    h[:] = rng.normal(size=g.n_h) * 1e-3
    zr, zz = np.zeros(g.n_er), np.zeros(g.n_ez)
    W0 = O.field_energy(g, er, ez, h)
    for _ in range(10):
        er, ez, h, src = F.solve(er, ez, h, zr, zz)
        assert src == 0.0
    W1 = O.field_energy(g, er, ez, h)
    assert abs(W1 - W0) <= 1e-12 * W0
    assert np.max(np.abs(h)) > 1e-3  # fields actually evolved


def test_vacuum_gauss_unchanged():
    g = O.Grid(12, 20, 0.05, 0.03)
    F = O.FieldSolver(g, 2e-11)
    rng = np.random.default_rng(1)
    er, ez, h = g.zeros_fields()
    er[:] = rng.normal(size=g.n_er)
    er.reshape(g.nr, g.nz + 1)[:, [0, -1]] = 0.0
    ez[:] = rng.normal(size=g.n_ez)
    ez.reshape(g.nr + 1, g.nz)[-1, :] = 0.0
    Q = np.zeros(g.n_node)
    G0 = O.gauss_residual(g, er, ez, Q)
    for _ in range(5):
        er, ez, h, _ = F.solve(er, ez, h, np.zeros(g.n_er), np.zeros(g.n_ez))
    G1 = O.gauss_residual(g, er, ez, Q)
    scale = np.max(np.abs(G0))
    assert scale > 0
    assert np.max(np.abs(G1 - G0)) <= 1e-12 * scale


def _zero_crossing_freq(x, dt):
    s = np.sign(x)
    idx = np.where(s[:-1] * s[1:] < 0)[0]
    t = (idx + x[idx] / (x[idx] - x[idx + 1])) * dt
    half_periods = (t[-1] - t[0]) / (len(t) - 1)
    return np.pi / half_periods


def test_tm010_cavity_cn_frequency():
    nr = 64
    R = 0.1
    g = O.Grid(nr, 2, R, 0.03)
    c = 1.0 / np.sqrt(O.EPS0 * O.MU0)
    chi = jn_zeros(0, 1)[0]
    w = chi * c / R
    dt = 1.0 / w  # w dt = 1: CN phase error atan is 7 %
    F = O.FieldSolver(g, dt)
    er, ez, h = g.zeros_fields()
    ri = np.arange(nr + 1) * g.dr
    EZ = ez.reshape(nr + 1, g.nz)
    EZ[:, :] = j0(chi * ri / R)[:, None]
    EZ[-1, :] = 0.0
    zr, zz = np.zeros(g.n_er), np.zeros(g.n_ez)
    trace = []
    for _ in range(240):
        er, ez, h, _ = F.solve(er, ez, h, zr, zz)
        trace.append(ez[0])
    w_num = _zero_crossing_freq(np.array(trace), dt)
    w_cn = (2.0 / dt) * np.arctan(w * dt / 2.0)
    assert abs(w_num - w_cn) / w_cn < 3e-3
    assert abs(w_num - w) / w > 0.05  # CN, not the continuum frequency


def test_quasistatic_gap_drive_gives_capacitor_field_and_energy_balance():
    g = O.Grid(16, 12, 0.1, 0.03)
    f = 1e6
    V0 = 100.0
    dt = 1.0 / (200 * f)
    F = O.FieldSolver(g, dt)
    er, ez, h = g.zeros_fields()
    zr, zz = np.zeros(g.n_er), np.zeros(g.n_ez)
    W = O.field_energy(g, er, ez, h)
    worst = 0.0
    # smooth start (V, dV/dt, d2V/dt2 = 0 at t = 0) so H = 0 is a consistent initial state
    volt = lambda t: V0 * 0.25 * (1.0 - np.cos(2 * np.pi * f * t)) ** 2
    for n in range(60):
        v0 = volt(n * dt)
        v1 = volt((n + 1) * dt)
        er, ez, h, src = F.solve(er, ez, h, zr, zz, v0, v1)
        W1 = O.field_energy(g, er, ez, h)
        worst = max(worst, abs((W1 - W) - src) / max(W1, 1e-30))
        W = W1
        EZ = ez.reshape(g.nr + 1, g.nz)
        np.testing.assert_allclose(EZ[: g.nr // 2], v1 / g.L, rtol=1e-4, atol=1e-6 * V0 / g.L)
        assert v1 > 0 or n == 0
    assert worst < 1e-10
    assert W > 0
