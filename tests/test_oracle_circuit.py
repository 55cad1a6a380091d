"""Pins of the oracle's blocking-capacitor circuit (Eq. 6) and of its
electrostatic whole step, against things other than the code under test:

* electrostatic vacuum: the divider phi = C/(C + C_r) V exactly, C_r the
  closed-form discrete capacitance eps pi (R - dr/2)^2 / L of the first row of
  E_z dual faces (the vacuum potential is linear in z);
* C -> infinity reduces both models to the electrode driven at V(t);
* electromagnetic: Ampere's law summed over the first row of E_z edges
  telescopes to 2 pi r_{nr-1/2} H^{n+1/2}(nr-1/2, 1/2), an expression of the
  current that the oracle's Eq. 6 never uses: it must equal the change of the
  capacitor charge every step, and vanish for a floating electrode (C -> 0);
* electromagnetic vacuum: the divider error vanishes like mu (the c -> inf
  limit of Sec. 3.3);
* electrostatic step: Gauss's law with the charge of the moved particles
  (continuity) and, with the electrodes grounded, conservation of kinetic +
  field energy to the Picard tolerance (Sec. 2.2).
"""
import numpy as np
import pytest

import oracle as O
from oracle import es as ES

F, V0 = 60e6, 100.0


def cr_closed(g):
    return O.EPS0 * np.pi * (g.R - 0.5 * g.dr) ** 2 / g.L


def volt(k, dt):
    return V0 * np.sin(2 * np.pi * F * k * dt)


def plasma(g, n=3000, seed=4, te=3.0):
    return O.load(g, n, 1e15, te, 0.026, seed)


def test_es_vacuum_divider_is_exact():
    g = O.Grid(8, 12, 0.1, 0.03)
    dt, C = 1e-10, 5e-11
    s = ES.Sim(g, dt, freq=F, volt=V0, tol=1e-12, cblock=C)
    for k in range(1, 6):
        rc, st = s.step()
        assert rc == 0
        v = volt(k, dt)
        np.testing.assert_allclose(s.circ[1], C / (C + cr_closed(g)) * v, rtol=1e-12)
        np.testing.assert_allclose(s.circ[0], C * (v - s.circ[1]), rtol=1e-12)


def test_es_large_capacitor_reduces_to_the_driven_electrode():
    g = O.Grid(12, 16, 0.1, 0.03)
    e, i = plasma(g)
    a = ES.Sim(g, 1e-10, freq=F, volt=V0, tol=1e-12, species=[e, i])
    b = ES.Sim(g, 1e-10, freq=F, volt=V0, tol=1e-12, cblock=1e3, species=[e, i])
    for k in range(1, 4):
        assert a.step()[0] == 0 and b.step()[0] == 0
        assert abs(b.circ[1] - volt(k, 1e-10)) <= 1e-12 * V0
        for x, y in ((a.er, b.er), (a.ez, b.ez)):
            assert np.max(np.abs(x - y)) <= 1e-9 * np.max(np.abs(x))


def test_es_superposition_matches_the_final_solve():
    """The flow of the field solved at the circuit's phi (with the crossed
    charge of the iteration that fed it) equals the capacitor's charge change:
    the affine decomposition used to find phi is exact."""
    g = O.Grid(12, 16, 0.1, 0.03)
    e, i = plasma(g)
    s = ES.Sim(g, 1e-10, freq=F, volt=V0, tol=1e-13, cblock=2e-11, species=[e, i])
    q0 = 0.0
    for k in range(1, 4):
        ez0 = s.ez.copy()
        rc, st = s.step()
        assert rc == 0
        flow = ES.electrode_charge_flow(g.nr, g.nz, g.dr, g.dz, s.ez, ez0, st["iz"])
        assert abs(flow - (s.circ[0] - q0)) <= 1e-10 * abs(s.circ[0] - q0)
        q0 = s.circ[0]


def test_es_step_gauss_with_the_moved_particles():
    g = O.Grid(12, 16, 0.1, 0.03)
    e, i = plasma(g, te=8.0)
    s = ES.Sim(g, 2e-10, freq=F, volt=V0, tol=1e-12, cblock=3e-11, species=[e, i])
    for k in range(3):
        rc, st = s.step()
        assert rc == 0
        Q = np.zeros(g.n_node)
        for sp in range(2):
            O.node_charge(g, (-O.QE, O.QE)[sp], s.state(sp), Q)
        G = O.gauss_residual(g, s.er, s.ez, Q).reshape(g.nr + 1, g.nz + 1)
        assert np.max(np.abs(G)) <= 1e-9 * np.max(np.abs(Q)), k


def test_es_step_conserves_energy_with_grounded_electrodes():
    g = O.Grid(12, 16, 0.1, 0.03)
    e, i = plasma(g, n=4000, te=5.0)
    s = ES.Sim(g, 2e-10, volt=0.0, tol=1e-12, species=[e, i])
    h0 = np.zeros(g.n_h)

    def energy():
        return (O.kinetic_energy(O.ME, s.state(0)) + O.kinetic_energy(O.M_AR, s.state(1))
                + O.field_energy(g, s.er, s.ez, h0))
    # Gauss-consistent start: the field of the loaded charge (zero for pairs)
    W0, lost = energy(), 0.0
    for k in range(4):
        rc, st = s.step()
        assert rc == 0
        lost += st["ke_lost"]
        assert abs(energy() + lost - W0) <= 1e-8 * W0, k


def test_em_large_capacitor_reduces_to_the_driven_electrode():
    g = O.Grid(12, 16, 0.1, 0.03)
    e, i = plasma(g)
    a = O.Sim(g, 1e-10, freq=F, volt=V0, tol=1e-12, species=[e, i])
    b = O.Sim(g, 1e-10, freq=F, volt=V0, tol=1e-12, species=[e, i], cblock=1e3)
    for k in range(1, 4):
        assert a.step()[0] == 0 and b.step()[0] == 0
        assert abs(b.circ[1] - volt(k, 1e-10)) <= 1e-12 * V0
        for x, y in ((a.er, b.er), (a.ez, b.ez), (a.h, b.h)):
            assert np.max(np.abs(x - y)) <= 1e-9 * np.max(np.abs(x))


def ampere_flow(g, h0, h1, dt):
    """dt 2 pi r_{nr-1/2} H^{n+1/2} at the H node (nr-1/2, 1/2)."""
    c = (g.nr - 1) * g.nz
    return dt * 2 * np.pi * (g.nr - 0.5) * g.dr * 0.5 * (h0[c] + h1[c])


@pytest.mark.parametrize("C", [3e-11, 1e-30])
def test_em_capacitor_charge_follows_amperes_law(C):
    g = O.Grid(12, 16, 0.1, 0.03)
    e, i = plasma(g, te=8.0)
    dt = 1e-10
    s = O.Sim(g, dt, freq=F, volt=V0, tol=1e-13, species=[e, i], cblock=C)
    free = O.Sim(g, dt, freq=F, volt=V0, tol=1e-13, species=[e, i])
    for k in range(1, 5):
        h0, q0 = s.h.copy(), s.circ[0]
        fh0 = free.h.copy()
        assert s.step()[0] == 0 and free.step()[0] == 0
        flow = ampere_flow(g, h0, s.h, dt)
        scale = abs(ampere_flow(g, fh0, free.h, dt))
        assert scale > 0
        # Kirchhoff at the electrode: the capacitor charge changes by the current
        assert abs(flow - (s.circ[0] - q0)) <= 1e-6 * scale, (k, flow, s.circ[0] - q0)
        if C < 1e-20:   # floating electrode: no current, q stays ~0
            assert abs(flow) <= 1e-6 * scale
        np.testing.assert_allclose(s.circ[0], C * (volt(k, dt) - s.circ[1]), rtol=1e-12,
                                   atol=1e-40)


def test_em_vacuum_divider_tends_to_the_electrostatic_one_like_mu():
    g = O.Grid(8, 12, 0.1, 0.03)
    dt, C = 1e-10, 1e-10
    div = C / (C + cr_closed(g))
    errs = []
    for mu in (O.MU0 * 1e-4, O.MU0 * 1e-6):
        s = O.Sim(g, dt, freq=F, volt=V0, tol=1e-13, mu=mu, cblock=C)
        e = 0.0
        for k in range(1, 13):
            assert s.step()[0] == 0
            e = max(e, abs(s.circ[1] / volt(k, dt) - div))
        errs.append(e)
    assert errs[1] < 0.02 * errs[0] and errs[1] < 1e-5, errs


# ---- the electrostatic model's axial port (Sec. 2.2): the electrode is the
# disc r <= r_p, its circuit current the flow through the E_z faces over it

def test_es_port_large_capacitor_reduces_to_the_driven_electrode():
    g = O.Grid(12, 16, 0.1, 0.03)
    e, i = plasma(g)
    a = ES.Sim(g, 1e-10, freq=F, volt=V0, tol=1e-12, species=[e, i], port=8)
    b = ES.Sim(g, 1e-10, freq=F, volt=V0, tol=1e-12, cblock=1e3, species=[e, i], port=8)
    for k in range(1, 4):
        assert a.step()[0] == 0 and b.step()[0] == 0
        assert abs(b.circ[1] - volt(k, 1e-10)) <= 1e-12 * V0
        for x, y in ((a.er, b.er), (a.ez, b.ez)):
            assert np.max(np.abs(x - y)) <= 1e-9 * np.max(np.abs(x))


def test_es_port_step_gauss_with_the_moved_particles():
    g = O.Grid(12, 16, 0.1, 0.03)
    e, i = plasma(g, te=8.0)
    s = ES.Sim(g, 2e-10, freq=F, volt=V0, tol=1e-12, cblock=3e-11, species=[e, i], port=8)
    for k in range(3):
        rc, st = s.step()
        assert rc == 0
        Q = np.zeros(g.n_node)
        for sp in range(2):
            O.node_charge(g, (-O.QE, O.QE)[sp], s.state(sp), Q)
        G = O.gauss_residual(g, s.er, s.ez, Q).reshape(g.nr + 1, g.nz + 1)
        assert np.max(np.abs(G)) <= 1e-9 * np.max(np.abs(Q)), k
        # the side wall is grounded: no E_z on it
        assert np.max(np.abs(s.ez.reshape(g.nr + 1, g.nz)[g.nr])) == 0.0
