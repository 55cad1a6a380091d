"""Pins of the oracle's conducting ring (Eq. 2's sigma E term, with which
Sec. 2.1 models metals in electromagnetic runs): the outer cells of the mesh
carry a conductivity sgd besides their permittivity.

* DC steady state in closed form: under a constant gap voltage V the field is
  E_z = V/L everywhere and Ampere's law makes 2 pi r H_theta at r_{i+1/2} equal
  to the conduction current sgd (V/L) pi (r_{i+1/2}^2 - R_d^2) through the
  annulus inside r_{i+1/2}; one solve leaves that state unchanged;
* energy: field energy change = energy in through the gap - Ohmic heat
  dt sum sgd A (E^{n+1/2})^2 L, the heat summed here from the test's own areas
  (the time centring of the sigma term is what makes this exact);
* sgd -> infinity: the ring becomes a perfect conductor, and the fields inside
  it follow those of the smaller grid that ends at the ring's face;
* Gauss's law after whole steps with particles sticking at the face holds
  with the charge carried by the conduction current added to the nodes.
"""
import numpy as np
import pytest

import oracle as O

QE = O.QE
ND, ERD = 3, 2.0


def grid(nr=14, nz=12, R=0.1, L=0.03, xa=0, sgd=5.0, erd=ERD):
    return O.Grid(nr, nz, R, L, xa=xa, nd=ND, erd=erd, sgd=sgd)


def ring_areas(g):
    """Conducting part of each dual face, from the node radii: the E_r face of
    row i is the cylinder 2 pi r_{i+1/2} dz, the E_z face of node i the annulus
    between the neighbouring cell centres, cut at the ring's face r_{nr-nd}."""
    rn = g.r_nodes()
    rh = 0.5 * (rn[:-1] + rn[1:])
    Rd = rn[g.nr - ND]
    ar = np.where(np.arange(g.nr) >= g.nr - ND, 2 * np.pi * rh * g.dz, 0.0)
    az = np.zeros(g.nr + 1)
    for i in range(g.nr):
        lo = rh[i - 1] if i > 0 else 0.0
        lo = max(lo, Rd)
        if rh[i] > lo:
            az[i] = np.pi * (rh[i] ** 2 - lo ** 2)
    return g.sgd * ar, g.sgd * az, rh


@pytest.mark.parametrize("xa", [0, 3])
def test_dc_steady_state_is_a_fixed_point(xa):
    g = grid(xa=xa, sgd=40.0)
    V, dt = 150.0, 2e-11
    F = O.FieldSolver(g, dt)
    er, ez, h = g.zeros_fields()
    ez[:] = V / g.L
    rn = g.r_nodes()
    rh = 0.5 * (rn[:-1] + rn[1:])
    Rd = rn[g.nr - ND]
    H = np.where(rh > Rd, g.sgd * V / g.L * np.pi * (rh ** 2 - Rd ** 2) / (2 * np.pi * rh), 0.0)
    h.reshape(g.nr, g.nz)[:] = H[:, None]
    zr, zz = np.zeros(g.n_er), np.zeros(g.n_ez)
    er1, ez1, h1, _ = F.solve(er, ez, h, zr, zz, V, V)
    np.testing.assert_allclose(ez1, ez, rtol=1e-11)
    assert np.max(np.abs(er1)) <= 1e-11 * V / g.L
    np.testing.assert_allclose(h1, h, rtol=1e-11, atol=1e-11 * np.max(H))
    # and a ring with no conductivity carries no current: H stays at zero
    g0 = grid(xa=xa, sgd=0.0)
    _, ez0, h0, _ = O.FieldSolver(g0, dt).solve(er, ez, np.zeros(g.n_h), zr, zz, V, V)
    assert np.max(np.abs(h0)) <= 1e-12 * np.max(H)


@pytest.mark.parametrize("xa,sgd", [(0, 2.0), (3, 0.3), (0, 300.0)])
def test_energy_identity_with_ohmic_heat(xa, sgd):
    g = grid(xa=xa, sgd=sgd)
    f, V0 = 2e9, 80.0
    dt = 1.0 / (40 * f)
    F = O.FieldSolver(g, dt)
    rng = np.random.default_rng(11)
    er, ez, h = g.zeros_fields()
    er[:] = rng.normal(size=g.n_er) * 300.0
    er.reshape(g.nr, g.nz + 1)[:, [0, -1]] = 0.0
    ez[:] = rng.normal(size=g.n_ez) * 300.0
    ez.reshape(g.nr + 1, g.nz)[-1] = V0 * np.sin(0.0) / g.L
    h[:] = rng.normal(size=g.n_h) * 1.0
    zr, zz = np.zeros(g.n_er), np.zeros(g.n_ez)
    sr, sz, rh = ring_areas(g)
    rn = g.r_nodes()
    wr = np.diff(rn)
    volt = lambda t: V0 * np.sin(2 * np.pi * f * t)
    W = O.field_energy(g, er, ez, h)
    heat_total, worst, qc = 0.0, 0.0, np.zeros(g.n_node)
    for n in range(40):
        er1, ez1, h1, src = F.solve(er, ez, h, zr, zz, volt(n * dt), volt((n + 1) * dt))
        erh = 0.5 * (er + er1).reshape(g.nr, g.nz + 1)[:, 1:-1]
        ezh = 0.5 * (ez + ez1).reshape(g.nr + 1, g.nz)[:-1]
        heat = dt * (np.sum(sr[:, None] * erh ** 2 * wr[:, None])
                     + np.sum(sz[:-1, None] * ezh ** 2 * g.dz))
        heat_c = F.conduction(er, ez, er1, ez1, qc)
        assert heat_c == pytest.approx(heat, rel=1e-12)
        W1 = O.field_energy(g, er1, ez1, h1)
        worst = max(worst, abs((W1 - W) - (src - heat)) / W)
        heat_total += heat
        er, ez, h, W = er1, ez1, h1, W1
    assert heat_total > 1e-3 * W      # the ring does dissipate
    assert worst < 1e-11


def test_perfect_conductor_limit_matches_the_smaller_grid():
    """sgd -> infinity: the ring is a perfect conductor, E_z at its face goes to
    zero, and the fields inside follow the grid of nr - nd cells whose outer
    edge carries zero gap voltage."""
    g = grid(nr=14, nz=12, sgd=1e9, erd=1.0)
    i0 = g.nr - ND
    gs = O.Grid(i0, g.nz, g.dr * i0, g.L)
    assert np.allclose(gs.r_nodes(), g.r_nodes()[: i0 + 1], rtol=1e-15)
    dt = 1e-12
    F, Fs = O.FieldSolver(g, dt), O.FieldSolver(gs, dt)
    er, ez, h = g.zeros_fields()
    ers, ezs, hs = gs.zeros_fields()
    rh = 0.5 * (g.r_nodes()[:-1] + g.r_nodes()[1:])
    zc = (np.arange(g.nz) + 0.5) / g.nz
    bump = np.where(rh < g.r_nodes()[i0], np.sin(np.pi * rh / g.r_nodes()[i0]), 0.0)
    h.reshape(g.nr, g.nz)[:] = bump[:, None] * np.sin(np.pi * zc)[None, :]
    hs[:] = h.reshape(g.nr, g.nz)[:i0].ravel()
    zr, zz = np.zeros(g.n_er), np.zeros(g.n_ez)
    zrs, zzs = np.zeros(gs.n_er), np.zeros(gs.n_ez)
    for _ in range(30):
        er, ez, h, _ = F.solve(er, ez, h, zr, zz, 0.0, 0.0)
        ers, ezs, hs, _ = Fs.solve(ers, ezs, hs, zrs, zzs, 0.0, 0.0)
    Hs = np.max(np.abs(hs))
    np.testing.assert_allclose(h.reshape(g.nr, g.nz)[:i0].ravel(), hs, atol=1e-6 * Hs)
    Es = np.max(np.abs(ezs))
    np.testing.assert_allclose(ez.reshape(g.nr + 1, g.nz)[: i0 + 1].ravel(), ezs, atol=1e-6 * Es)
    np.testing.assert_allclose(er.reshape(g.nr, g.nz + 1)[:i0].ravel(), ers, atol=1e-6 * Es)
    assert np.max(np.abs(h.reshape(g.nr, g.nz)[i0:])) <= 1e-6 * Hs


@pytest.mark.parametrize("xa", [0, 2])
def test_gauss_law_after_steps_with_conduction_and_sticking(xa):
    g = grid(nr=12, nz=16, xa=xa, sgd=0.5)
    e, i = O.load(g, 3000, 1e15, 30.0, 0.026, 21)
    s = O.Sim(g, 5e-11, freq=60e6, volt=50.0, tol=1e-12, species=[e, i])
    for _ in range(4):
        rc, st = s.step()
        assert rc == 0
    assert np.max(np.abs(s.qcond)) > 0 and s.ohmic > 0
    nz1 = g.nz + 1
    stuck = s.wall_r[:nz1] + s.wall_r[nz1:]
    assert np.sum(np.abs(stuck)) > 0
    Q = np.zeros(g.n_node)
    for sp in range(2):
        O.node_charge(g, (-QE, QE)[sp], s.state(sp), Q)
    Qn = Q.reshape(g.nr + 1, nz1)
    Qn[g.nr - ND, :] += stuck
    G = O.gauss_residual(g, s.er, s.ez, Q + s.qcond)
    scale = max(np.max(np.abs(Q)), np.max(np.abs(s.qcond)))
    assert np.max(np.abs(G)) <= 1e-9 * scale
    # without the conduction charge the ring's nodes do not balance
    G0 = O.gauss_residual(g, s.er, s.ez, Q)
    assert np.max(np.abs(G0)) > 1e3 * np.max(np.abs(G))


def test_electrostatic_model_refuses_a_conducting_ring():
    from oracle import es as ES
    with pytest.raises(ValueError):
        ES.Sim(grid(sgd=1.0), 1e-10)
