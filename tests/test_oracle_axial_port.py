"""Axial dielectric port (Sec. 2.2, Fig. 1; Eqs. 5 and 7) in the oracle's
field solve: a coaxial port filled with a dielectric below the powered
electrode, fed by an incoming TEM wave of half the electrode potential
through Mur's condition at its end.

Pins, none of which retypes the solver:
  * the discrete energy identity of the CN scheme: with no particles, the
    field energy of reactor and port changes by exactly the energy the port's
    end delivers (what the solve reports as src), from random fields;
  * the coaxial TEM mode: with a slowly varying drive the port's fields are
    E_r, H_theta proportional to 1/r across the annulus and E_z ~ 0;
  * the quasi-static limit: a drive slow against the transit time gives the
    electrode potential the drive's, i.e. E_z = phi / L between the plates on
    the axis side, and the incident wave of half the potential doubles at the
    (open, capacitive) reactor end.
"""
import numpy as np
import pytest

import oracle as O


def setup(nr=16, nz=12, R=0.1, L=0.02, ip=10, nzp=6, Lp=0.03, erq=3.8, dt=2e-11):
    g = O.Grid(nr, nz, R, L)
    P = O.PortSolver(g, dt, ip, nzp, Lp / nzp, erq)
    return g, P


def test_energy_identity_from_random_fields():
    g, P = setup()
    rng = np.random.default_rng(5)
    er, ez, h = (rng.normal(size=g.n_er) * 1e3, rng.normal(size=g.n_ez) * 1e3,
                 rng.normal(size=g.nr * g.nz))
    erp, ezp, hp = P.zeros_port()
    erp[:] = rng.normal(size=erp.size) * 1e3
    ezp[:] = rng.normal(size=ezp.size) * 1e3
    hp[:] = rng.normal(size=hp.size)
    # fields on conductors and plates are zero
    er.reshape(g.nr, g.nz + 1)[:, g.nz] = 0.0
    er.reshape(g.nr, g.nz + 1)[: P.ip, 0] = 0.0
    ez.reshape(g.nr + 1, g.nz)[g.nr, :] = 0.0
    m = g.nr - P.ip
    ezp.reshape(m + 1, P.nzp)[0, :] = 0.0
    ezp.reshape(m + 1, P.nzp)[m, :] = 0.0
    ir, iz = np.zeros(g.n_er), np.zeros(g.n_ez)
    for phi0, phi1 in ((0.0, 0.0), (3.0, 7.5), (-40.0, 12.0)):
        W0 = P.energy(er, ez, h, erp, ezp, hp)
        er1, ez1, h1, erp1, ezp1, hp1, src = P.solve(er, ez, h, erp, ezp, hp, ir, iz, phi0, phi1)
        W1 = P.energy(er1, ez1, h1, erp1, ezp1, hp1)
        assert abs(W1 - W0 - src) <= 1e-11 * W0, (W1 - W0, src)
        if phi0 == phi1 == 0.0:
            assert src <= 0.0  # Mur's condition only lets energy out


def drive(P, g, steps, omega, V):
    er, ez, h = g.zeros_fields()
    erp, ezp, hp = P.zeros_port()
    ir, iz = np.zeros(g.n_er), np.zeros(g.n_ez)
    for n in range(steps):
        phi0, phi1 = V * np.sin(omega * n * P.dt), V * np.sin(omega * (n + 1) * P.dt)
        er, ez, h, erp, ezp, hp, _ = P.solve(er, ez, h, erp, ezp, hp, ir, iz, phi0, phi1)
    return er, ez, h, erp, ezp, hp, V * np.sin(omega * steps * P.dt)


def test_quasi_static_tem_mode_and_gap_field():
    # a port twice the reactor's height, as the paper's (6.5 against 3 cm), so
    # that its end is well away from the junction's fringing field
    g, P = setup(dt=1e-11, nzp=12, Lp=0.06)
    # a period of 4000 steps (25 MHz, wavelength 12 m against a 5 cm domain)
    omega = 2 * np.pi / (4000 * P.dt)
    er, ez, h, erp, ezp, hp, phi = drive(P, g, 1000, omega, 100.0)  # a quarter period: phi = V
    m = g.nr - P.ip
    rh = 0.5 * (g.r_nodes()[P.ip:-1] + g.r_nodes()[P.ip + 1:])   # r_{i+1/2} of the port columns
    # TEM at the port's end (the junction with the reactor, a few cells above,
    # adds the fringing field): r E_r constant across the annulus, E_z small
    Erp = erp.reshape(m, P.nzp)
    Ezp = ezp.reshape(m + 1, P.nzp)
    for q in (0, 1):
        rE = rh * Erp[:, q]
        assert np.max(np.abs(rE - rE.mean())) <= 1e-2 * np.abs(rE.mean()), q
    assert np.max(np.abs(Ezp[:, 0])) <= 5e-2 * np.max(np.abs(Erp[:, 0]))
    # the coaxial voltage across the annulus equals the electrode potential at
    # every height of the port (the incident wave of phi / 2, doubled)
    dr = np.diff(g.r_nodes()[P.ip:])
    for q in range(P.nzp):
        Vc = Erp[:, q] @ dr
        assert abs(Vc - phi) <= 1e-2 * phi, (q, Vc, phi)
    # gap field on the axis side: E_z = phi / L (directed from the powered plate)
    Ez = ez.reshape(g.nr + 1, g.nz)
    assert np.max(np.abs(Ez[: P.ip // 2] * g.L - phi)) <= 1e-2 * phi


# ---- the axial port with the blocking capacitor (Eq. 6 feeding Eq. 7) --------

F, V0 = 60e6, 100.0
PORT = (10, 6, 0.03, 3.8)


def volt(k, dt):
    return V0 * np.sin(2 * np.pi * F * k * dt)


def port_plasma(g, seed=4):
    return O.load(g, 2000, 1e15, 8.0, 0.026, seed)


def test_port_large_capacitor_reduces_to_the_driven_port():
    g = O.Grid(16, 12, 0.1, 0.02)
    e, i = port_plasma(g)
    dt = 2e-11
    a = O.Sim(g, dt, freq=F, volt=V0, tol=1e-12, species=[e, i], port=PORT)
    b = O.Sim(g, dt, freq=F, volt=V0, tol=1e-12, species=[e, i], port=PORT, cblock=1e3)
    for k in range(1, 4):
        assert a.step()[0] == 0 and b.step()[0] == 0
        assert abs(b.circ[1] - volt(k, dt)) <= 1e-12 * V0
        for x, y in ((a.er, b.er), (a.ez, b.ez), (a.h, b.h), (a.erp, b.erp), (a.hp, b.hp)):
            assert np.max(np.abs(x - y)) <= 1e-9 * np.max(np.abs(x))


@pytest.mark.parametrize("C,grade", [(3e-11, 1.0), (1e-30, 1.0), (3e-11, 1.3)])
def test_port_capacitor_charge_follows_amperes_law(C, grade):
    """Ampere's law summed over the E_z edges of the first row over the
    electrode (i < ip) telescopes to dt 2 pi r_{ip-1/2} H^{n+1/2}(ip-1/2, 1/2),
    an expression of the electrode current that the oracle's circuit never
    evaluates: the capacitor charge must change by it every step."""
    g = O.Grid(16, 12, 0.1, 0.02)
    e, i = port_plasma(g)
    dt = 2e-11
    ip = PORT[0]
    c = (ip - 1) * g.nz
    rh = 2 * np.pi * (ip - 0.5) * g.dr
    port = PORT + (grade,)
    s = O.Sim(g, dt, freq=F, volt=V0, tol=1e-13, species=[e, i], port=port, cblock=C)
    free = O.Sim(g, dt, freq=F, volt=V0, tol=1e-13, species=[e, i], port=port)
    for k in range(1, 5):
        h0, q0, fh0 = s.h.copy(), s.circ[0], free.h.copy()
        assert s.step()[0] == 0 and free.step()[0] == 0
        flow = dt * rh * 0.5 * (h0[c] + s.h[c])
        scale = abs(dt * rh * 0.5 * (fh0[c] + free.h[c]))
        assert scale > 0
        assert abs(flow - (s.circ[0] - q0)) <= 1e-6 * scale, (k, flow, s.circ[0] - q0)
        if C < 1e-20:  # floating electrode: no current
            assert abs(flow) <= 1e-6 * scale
        np.testing.assert_allclose(s.circ[0], C * (volt(k, dt) - s.circ[1]), rtol=1e-12,
                                   atol=1e-40)


# ---- a graded port (rows growing from the junction down: Sec. 2.1's
# nonuniform mesh, which lengthens the waveguide in few cells) ----------------

def graded(nzp=12, Lp=0.06, grade=1.2, nr=16, nz=12, ip=10, erq=3.8, dt=2e-11):
    g = O.Grid(nr, nz, 0.1, 0.02)
    return g, O.PortSolver(g, dt, ip, nzp, Lp / nzp, erq, heights=O.port_heights(nzp, Lp, grade))


def test_port_heights_are_a_geometric_progression_summing_to_the_length():
    h = O.port_heights(12, 0.06, 1.2)
    assert abs(h.sum() - 0.06) <= 1e-15
    np.testing.assert_allclose(h[:-1] / h[1:], 1.2, rtol=1e-13)   # q = 0 (the end) largest
    np.testing.assert_allclose(O.port_heights(5, 0.03, 1.0), 0.006, rtol=1e-15)


def test_graded_port_energy_identity_from_random_fields():
    g, P = graded()
    rng = np.random.default_rng(9)
    er, ez, h = (rng.normal(size=g.n_er) * 1e3, rng.normal(size=g.n_ez) * 1e3,
                 rng.normal(size=g.nr * g.nz))
    erp, ezp, hp = P.zeros_port()
    erp[:] = rng.normal(size=erp.size) * 1e3
    ezp[:] = rng.normal(size=ezp.size) * 1e3
    hp[:] = rng.normal(size=hp.size)
    er.reshape(g.nr, g.nz + 1)[:, g.nz] = 0.0
    er.reshape(g.nr, g.nz + 1)[: P.ip, 0] = 0.0
    ez.reshape(g.nr + 1, g.nz)[g.nr, :] = 0.0
    m = g.nr - P.ip
    ezp.reshape(m + 1, P.nzp)[0, :] = 0.0
    ezp.reshape(m + 1, P.nzp)[m, :] = 0.0
    ir, iz = np.zeros(g.n_er), np.zeros(g.n_ez)
    for phi0, phi1 in ((0.0, 0.0), (3.0, 7.5)):
        W0 = P.energy(er, ez, h, erp, ezp, hp)
        er1, ez1, h1, erp1, ezp1, hp1, src = P.solve(er, ez, h, erp, ezp, hp, ir, iz, phi0, phi1)
        W1 = P.energy(er1, ez1, h1, erp1, ezp1, hp1)
        assert abs(W1 - W0 - src) <= 1e-11 * W0, (W1 - W0, src)


def test_graded_port_carries_the_electrode_potential_at_every_height():
    """Quasi-static drive: the coaxial voltage across the annulus equals the
    electrode potential in every row, coarse or fine."""
    g, P = graded(dt=1e-11)
    omega = 2 * np.pi / (4000 * P.dt)
    er, ez, h, erp, ezp, hp, phi = drive(P, g, 1000, omega, 100.0)
    m = g.nr - P.ip
    Erp = erp.reshape(m, P.nzp)
    dr = np.diff(g.r_nodes()[P.ip:])
    for q in range(P.nzp):
        assert abs(Erp[:, q] @ dr - phi) <= 1e-2 * phi, q


def test_graded_port_transit_time_matches_a_fine_uniform_port():
    """A smooth rise of the potential reaches the junction after the port's
    transit time L_p sqrt(eps_q) / c: the half-rise time of E_r in the top
    port row through 12 graded rows (1.5 to 11 mm) agrees with that through
    48 uniform rows of 1.25 mm to 3 %."""
    c = 1.0 / np.sqrt(O.EPS0 * O.MU0)
    Lp, erq, dt = 0.06, 3.8, 2e-12
    T = Lp * np.sqrt(erq) / c

    def half_rise(P, g):
        er, ez, h = g.zeros_fields()
        erp, ezp, hp = P.zeros_port()
        ir, iz = np.zeros(g.n_er), np.zeros(g.n_ez)
        V = lambda t: 50.0 * (1.0 - np.cos(np.pi * min(t, T) / T))
        m, y = g.nr - P.ip, []
        for n in range(900):
            er, ez, h, erp, ezp, hp, _ = P.solve(er, ez, h, erp, ezp, hp, ir, iz, V(n * dt),
                                                 V((n + 1) * dt))
            y.append(erp.reshape(m, P.nzp)[0, P.nzp - 1])
        y = np.array(y)
        return np.argmax(y > 0.5 * y.max()) * dt

    tg = half_rise(*graded(nzp=12, Lp=Lp, grade=1.2, dt=dt)[::-1])
    tu = half_rise(*graded(nzp=48, Lp=Lp, grade=1.0, dt=dt)[::-1])
    assert tu > T  # the rise has crossed the port
    assert abs(tg / tu - 1.0) <= 0.03, (tg, tu)
