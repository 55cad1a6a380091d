"""Pins of the oracle's wave port on r = R (the first-order absorbing
condition E_z + eta H_theta = 2 E_in of Eq. 5, read for the side feed):

* a slow drive gives the quasi-static capacitor field V/L inside (the
  incident wave E_in = V/(2L) doubles at the open end);
* the discrete energy identity W^{n+1} - W^n = energy through the boundary
  edges holds every step (absorbed and injected power included);
* a pulse leaves the domain: after it has crossed out, the field energy left is
  a few per cent of what the reflecting prescribed gap keeps.
"""
import numpy as np

import oracle as O


def slow_drive_error(f):
    g = O.Grid(16, 12, 0.1, 0.03)
    V0 = 100.0
    dt = 1.0 / (200 * f)
    F = O.FieldSolver(g, dt, wave=True)
    er, ez, h = g.zeros_fields()
    zr, zz = np.zeros(g.n_er), np.zeros(g.n_ez)
    volt = lambda t: V0 * 0.25 * (1.0 - np.cos(2 * np.pi * f * t)) ** 2
    W = O.field_energy(g, er, ez, h)
    worst = 0.0
    for n in range(60):
        v0, v1 = volt(n * dt), volt((n + 1) * dt)
        er, ez, h, src = F.solve(er, ez, h, zr, zz, v0, v1)
        W1 = O.field_energy(g, er, ez, h)
        worst = max(worst, abs((W1 - W) - src) / max(W1, 1e-30))
        W = W1
    EZ = ez.reshape(g.nr + 1, g.nz)
    return np.max(np.abs(EZ / (volt(60 * dt) / g.L) - 1.0)), worst


def test_slow_drive_gives_the_capacitor_field():
    """The charging current of the reactor capacitance flows through the
    port's wave impedance: the field lags the open-circuit value by a relative
    amount proportional to the frequency (an RC lag), which vanishes as f -> 0."""
    e1, w1 = slow_drive_error(1e6)
    e4, w4 = slow_drive_error(0.25e6)
    assert e1 < 3e-3 and w1 < 1e-10 and w4 < 1e-10
    assert 3.0 < e1 / e4 < 5.0, (e1, e4)


def pulse_energy(wave):
    nr, R = 64, 0.1
    g = O.Grid(nr, 2, R, 0.03)
    dt = 2e-12
    F = O.FieldSolver(g, dt, wave=wave)
    er, ez, h = g.zeros_fields()
    zr, zz = np.zeros(g.n_er), np.zeros(g.n_ez)
    f0, tau, t0 = 15e9, 0.1e-9, 0.3e-9
    volt = lambda t: 50.0 * np.exp(-((t - t0) / tau) ** 2) * np.sin(2 * np.pi * f0 * t)
    W, Wmax, bal = [], 0.0, 0.0
    Wp = 0.0
    for n in range(1000):
        v0, v1 = volt(n * dt), volt((n + 1) * dt)
        er, ez, h, src = F.solve(er, ez, h, zr, zz, v0, v1)
        w = O.field_energy(g, er, ez, h)
        bal = max(bal, abs((w - Wp) - src))
        Wp = w
        W.append(w)
    W = np.array(W)
    return W, bal


def test_pulse_leaves_through_the_port():
    Ww, balw = pulse_energy(True)
    Wg, _ = pulse_energy(False)
    peak = Ww.max()
    assert balw <= 1e-10 * peak
    # 2 ns = 6 transit times across R after the pulse: the port has let it out
    assert Ww[-1] < 0.03 * peak
    assert Wg[-1] > 0.2 * Wg.max()          # the prescribed gap (a wall) keeps it
    assert Ww[-1] < 0.05 * Wg[-1]
