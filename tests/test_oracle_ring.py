"""Pins of the oracle's dielectric ring (the outer cells of the mesh filled
with a dielectric of relative permittivity erd, particles moving inside it and
sticking at its inner face):

* Gauss's law of the electrostatic solver (oracle/es.py, its own weighted
  areas) through the C oracle's discrete divergence (its own);
* the electrostatic vacuum divider with the blocking capacitor is exact with
  the closed-form capacitance eps0 [pi R_d^2 + erd pi (r_{nr-1/2}^2 - R_d^2)] / L;
* the electromagnetic solve: quasi-static field V/L and the energy identity;
* particles stop at the ring face: node-wise continuity with the wall tally
  there, none beyond it, and the loaded density fills r < R_d only.
"""
import numpy as np
import pytest

import oracle as O
from oracle import es as ES
from tests import inputs

QE, ME = O.QE, O.ME
ND, ERD = 3, 3.8


def grid(nr=16, nz=20, R=0.1, L=0.03, xa=0):
    return O.Grid(nr, nz, R, L, xa=xa, nd=ND, erd=ERD)


@pytest.mark.parametrize("xa", [0, 3])
def test_es_solver_and_c_oracle_agree_on_gauss_law(xa):
    g = grid(nr=11, nz=9, xa=xa)
    rng = np.random.default_rng(3)
    Q = rng.normal(size=g.n_node) * 1e-12
    Q.reshape(g.nr + 1, g.nz + 1)[g.nr - ND:, :] = 0.0   # no charge in the dielectric
    _, er, ez = ES.solve(g.nr, g.nz, g.dr, g.dz, Q, 25.0, xa=xa, nd=ND, erd=ERD)
    G = O.gauss_residual(g, er, ez, Q).reshape(g.nr + 1, g.nz + 1)
    assert np.max(np.abs(G[:g.nr, 1:g.nz])) <= 1e-10 * np.max(np.abs(Q))


def test_es_vacuum_divider_with_the_ring():
    g = grid(nr=10, nz=12)
    dt, C, f, V = 1e-10, 4e-11, 60e6, 100.0
    rn = g.r_nodes()
    Rd, rh = rn[g.nr - ND], 0.5 * (rn[-2] + rn[-1])
    Cr = O.EPS0 * (np.pi * Rd ** 2 + ERD * np.pi * (rh ** 2 - Rd ** 2)) / g.L
    s = ES.Sim(g, dt, freq=f, volt=V, tol=1e-12, cblock=C)
    for k in range(1, 5):
        assert s.step()[0] == 0
        np.testing.assert_allclose(s.circ[1], C / (C + Cr) * V * np.sin(2 * np.pi * f * k * dt),
                                   rtol=1e-12)


def test_em_quasistatic_field_and_energy_identity():
    g = grid(nr=16, nz=12)
    f, V0 = 1e6, 100.0
    dt = 1.0 / (200 * f)
    F = O.FieldSolver(g, dt)
    er, ez, h = g.zeros_fields()
    zr, zz = np.zeros(g.n_er), np.zeros(g.n_ez)
    volt = lambda t: V0 * 0.25 * (1.0 - np.cos(2 * np.pi * f * t)) ** 2
    W, worst = 0.0, 0.0
    for n in range(60):
        er, ez, h, src = F.solve(er, ez, h, zr, zz, volt(n * dt), volt((n + 1) * dt))
        W1 = O.field_energy(g, er, ez, h)
        worst = max(worst, abs((W1 - W) - src) / max(W1, 1e-30))
        W = W1
    np.testing.assert_allclose(ez.reshape(g.nr + 1, g.nz)[: g.nr], volt(60 * dt) / g.L,
                               rtol=1e-4)
    assert worst < 1e-10


def test_particles_stick_at_the_ring_face():
    g = grid()
    n = 6000
    rng = np.random.default_rng(5)
    ic = rng.integers(g.nr - ND - 3, g.nr - ND, size=n)   # the last plasma cells
    jc = rng.integers(2, g.nz - 2, size=n)
    sp = inputs.particles(g.nr, g.nz, n, 5, 8e5, cells=ic * g.nz + jc)
    sp["vr"] = np.abs(sp["vr"]) + 3e5                    # all move outward
    er, ez = inputs.smooth_fields(g.nr, g.nz, 5, 1e3)
    Q0 = O.node_charge(g, -QE, sp)
    walls = (np.zeros(g.nr + 1), np.zeros(g.nr + 1), np.zeros(g.nz + 1))
    ir, iz, cnt, _ = O.push(g, 2e-9, -QE, ME, sp, er, ez, write=True, walls=walls)
    assert cnt[0] == 0 and cnt[1] > 300                  # many reached the face
    alive = sp["cell"] >= 0
    assert np.all(sp["cell"][alive] // g.nz < g.nr - ND)  # none inside the dielectric
    Q1 = O.node_charge(g, -QE, sp)
    Wl = np.zeros((g.nr + 1, g.nz + 1))
    Wl[g.nr - ND, :] += walls[2]                         # the r-wall tally sits on the face
    Wl[:, 0] += walls[0]
    Wl[:, -1] += walls[1]
    IR = ir.reshape(g.nr, g.nz + 1)
    IZ = iz.reshape(g.nr + 1, g.nz)
    D = np.zeros((g.nr + 1, g.nz + 1))
    D[:-1, :] += IR
    D[1:, :] -= IR
    D[:, :-1] += IZ
    D[:, 1:] -= IZ
    res = Q1.reshape(g.nr + 1, g.nz + 1) + Wl - Q0.reshape(g.nr + 1, g.nz + 1) + D
    assert np.max(np.abs(res)) <= 1e-13 * np.max(np.abs(Q0))


def test_loading_fills_the_plasma_region_only():
    g = grid(nr=12, nz=4)
    n0, n = 1e15, 200000
    e, _ = O.load(g, n, n0, 3.0, 0.026, 3)
    ic = e["cell"] // g.nz
    assert ic.max() == g.nr - ND - 1
    Rd = g.r_nodes()[g.nr - ND]
    assert np.sum(e["w"]) == pytest.approx(n0 * np.pi * Rd ** 2 * g.L, rel=0.01)


def test_es_step_keeps_the_stuck_charge_in_gauss_law():
    """Electrons stick at the ring face; the electrostatic step's field obeys
    Gauss's law with the moved particles plus the charge stuck on the face."""
    g = grid(nr=12, nz=16)
    e, i = O.load(g, 4000, 1e15, 30.0, 0.026, 9)
    s = ES.Sim(g, 2e-10, volt=0.0, tol=1e-12, species=[e, i])
    for _ in range(3):
        rc, st = s.step()
        assert rc == 0
    stuck = s.wall[2][: g.nz + 1] + s.wall[2][g.nz + 1:]
    assert np.sum(np.abs(stuck)) > 0
    Q = np.zeros(g.n_node)
    for sp in range(2):
        O.node_charge(g, (-QE, O.QE)[sp], s.state(sp), Q)
    Q.reshape(g.nr + 1, g.nz + 1)[g.nr - ND, :] += stuck
    G = O.gauss_residual(g, s.er, s.ez, Q).reshape(g.nr + 1, g.nz + 1)
    assert np.max(np.abs(G)) <= 1e-9 * np.max(np.abs(Q))
