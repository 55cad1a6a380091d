"""Pins of the oracle on the mapped radial mesh (Sec. 2.1: r proportional to
sqrt(xi) in the first xa cells, linear beyond, J_r constant per cell):

* the mapping's closed form (r^2 linear in xi near the axis, continuous slope,
  r(nr) = R);
* exact single-particle motion across cells of different widths: free flight
  and a constant radial force give the exact parabola in physical r, and the
  inertial terms keep |v| and r v_theta exactly;
* node-wise charge continuity of the deposit;
* loading: weights proportional to r J_r give the density n0 in every ring;
* the field operator: Gauss's law of the electrostatic solver (oracle/es.py,
  its own areas) through the C oracle's discrete divergence (its own areas),
  the vacuum TM010 frequency, and whole-step energy conservation to the Picard
  tolerance.
"""
import numpy as np
import pytest
from scipy.special import jn_zeros, j0

import oracle as O
from oracle import es as ES
from tests import inputs

QE, ME = O.QE, O.ME
XA = 3


def grid(nr=16, nz=24, R=0.05, L=0.03, xa=XA):
    return O.Grid(nr, nz, R, L, xa=xa)


def phys_r(g, sp):
    rn = g.r_nodes()
    ic = sp["cell"] // g.nz
    return rn[ic] + sp["a"] * (rn[ic + 1] - rn[ic])


def test_mapping_closed_form():
    g = grid(nr=20, R=0.1, xa=4)
    rn = g.r_nodes()
    assert rn[-1] == pytest.approx(0.1, rel=1e-15)
    i = np.arange(5)
    np.testing.assert_allclose(rn[:5] ** 2, 4 * g.dr ** 2 * g.xa * i, rtol=1e-14, atol=0)
    np.testing.assert_allclose(np.diff(rn)[4:], g.dr, rtol=1e-13)
    # r J_r at the axis (continuous mapping): d(r^2)/dxi / 2 = 2 dr^2 xa
    assert (rn[1] ** 2 - rn[0] ** 2) / 2 == pytest.approx(2 * g.dr ** 2 * g.xa, rel=1e-14)


def radial_particles(g, n, seed, v):
    rng = np.random.default_rng(seed)
    ic = rng.integers(1, g.nr - 4, size=n)
    jc = rng.integers(4, g.nz - 4, size=n)
    return inputs.particles(g.nr, g.nz, n, seed, v, cells=ic * g.nz + jc)


@pytest.mark.parametrize("E0", [0.0, 60.0, -60.0])
def test_radial_parabola_exact_across_mapped_cells(E0):
    g = grid()
    dt = 1e-9
    sp = radial_particles(g, 3000, 2, 1.2e5)
    sp["vt"][:] = 0.0
    er, ez, _ = g.zeros_fields()
    er[:] = E0
    r0, vr0 = phys_r(g, sp), sp["vr"].copy()
    acc = -QE / ME * E0
    keep = r0 + vr0 * dt + 0.5 * acc * dt * dt > 0.2 * r0  # stay clear of the axis
    _, _, cnt, _ = O.push(g, dt, -QE, ME, sp, er, ez, write=True)
    assert cnt[0] == 0 and cnt[2] > 3000  # crossings happened
    r1 = phys_r(g, sp)
    np.testing.assert_allclose(r1[keep], (r0 + vr0 * dt + 0.5 * acc * dt * dt)[keep], rtol=0,
                               atol=1e-12 * g.R)
    np.testing.assert_allclose(sp["vr"][keep], (vr0 + acc * dt)[keep], rtol=1e-12, atol=1e-9)


def test_inertial_terms_conserve_speed_and_angular_momentum():
    g = grid()
    dt = 2e-9
    sp = inputs.particles(g.nr, g.nz, 3000, 4, 2e5)
    er, ez, _ = g.zeros_fields()
    v2 = sp["vr"] ** 2 + sp["vt"] ** 2 + sp["vz"] ** 2
    L0 = phys_r(g, sp) * sp["vt"]
    _, _, cnt, _ = O.push(g, dt, -QE, ME, sp, er, ez, write=True)
    alive = sp["cell"] >= 0
    assert cnt[0] == 0 and alive.sum() > 2500
    v2n = sp["vr"] ** 2 + sp["vt"] ** 2 + sp["vz"] ** 2
    np.testing.assert_allclose(v2n[alive], v2[alive], rtol=1e-11)
    np.testing.assert_allclose((phys_r(g, sp) * sp["vt"])[alive], L0[alive], rtol=1e-10,
                               atol=1e-12 * np.max(np.abs(L0)))


def divergence(g, ir, iz):
    IR = ir.reshape(g.nr, g.nz + 1)
    IZ = iz.reshape(g.nr + 1, g.nz)
    D = np.zeros((g.nr + 1, g.nz + 1))
    D[:-1, :] += IR
    D[1:, :] -= IR
    D[:, :-1] += IZ
    D[:, 1:] -= IZ
    return D.ravel()


def test_charge_continuity_per_node():
    g = grid()
    sp = inputs.particles(g.nr, g.nz, 6000, 7, 8e5, edge_frac=0.05)
    er, ez = inputs.smooth_fields(g.nr, g.nz, 7, 3e3)
    Q0 = O.node_charge(g, -QE, sp)
    walls = (np.zeros(g.nr + 1), np.zeros(g.nr + 1), np.zeros(g.nz + 1))
    ir, iz, cnt, _ = O.push(g, 1e-9, -QE, ME, sp, er, ez, write=True, walls=walls)
    assert cnt[0] == 0 and cnt[1] > 0
    Q1 = O.node_charge(g, -QE, sp)
    W = np.zeros((g.nr + 1, g.nz + 1))
    W[:, 0] += walls[0]
    W[:, -1] += walls[1]
    W[-1, :] += walls[2]
    res = Q1 + W.ravel() - Q0 + divergence(g, ir, iz)
    assert np.max(np.abs(res)) <= 1e-13 * np.max(np.abs(Q0))


def test_loading_gives_uniform_density_in_every_ring():
    g = grid(nr=12, nz=4, R=0.1, L=0.03, xa=4)
    n0, n = 1e15, 400000
    e, _ = O.load(g, n, n0, 3.0, 0.026, 3)
    rn = g.r_nodes()
    ic = e["cell"] // g.nz
    wsum = np.bincount(ic, weights=e["w"], minlength=g.nr)
    vol = np.pi * (rn[1:] ** 2 - rn[:-1] ** 2) * g.L
    cnt = np.bincount(ic, minlength=g.nr)
    dens = wsum / vol / n0
    # weights vary inside a cell, so allow a few sigma of the count noise
    np.testing.assert_allclose(dens, 1.0, atol=5.0 / np.sqrt(cnt.min()) + 0.01)
    assert np.sum(e["w"]) == pytest.approx(n0 * np.pi * 0.1 ** 2 * 0.03, rel=0.01)


def test_es_solver_and_c_oracle_agree_on_gauss_law():
    g = grid(nr=9, nz=11, R=0.05, xa=3)
    rng = np.random.default_rng(2)
    Q = rng.normal(size=g.n_node) * 1e-12
    phi, er, ez = ES.solve(g.nr, g.nz, g.dr, g.dz, Q, 37.0, xa=g.xa)
    G = O.gauss_residual(g, er, ez, Q).reshape(g.nr + 1, g.nz + 1)
    assert np.max(np.abs(G[:g.nr, 1:g.nz])) <= 1e-10 * np.max(np.abs(Q))


def _zero_crossing_freq(x, dt):
    s = np.sign(x)
    idx = np.where(s[:-1] * s[1:] < 0)[0]
    t = (idx + x[idx] / (x[idx] - x[idx + 1])) * dt
    return np.pi / ((t[-1] - t[0]) / (len(t) - 1))


def test_tm010_frequency_on_the_mapped_mesh():
    nr, R = 64, 0.1
    g = O.Grid(nr, 2, R, 0.03, xa=4)
    c = 1.0 / np.sqrt(O.EPS0 * O.MU0)
    chi = jn_zeros(0, 1)[0]
    w = chi * c / R
    dt = 1.0 / w
    F = O.FieldSolver(g, dt)
    er, ez, h = g.zeros_fields()
    EZ = ez.reshape(nr + 1, g.nz)
    EZ[:, :] = j0(chi * g.r_nodes() / R)[:, None]
    EZ[-1, :] = 0.0
    zr, zz = np.zeros(g.n_er), np.zeros(g.n_ez)
    trace = []
    for _ in range(240):
        er, ez, h, _ = F.solve(er, ez, h, zr, zz)
        trace.append(ez[0])
    w_num = _zero_crossing_freq(np.array(trace), dt)
    w_cn = (2.0 / dt) * np.arctan(w * dt / 2.0)
    assert abs(w_num - w_cn) / w_cn < 3e-3


def test_whole_step_energy_conserved_to_the_picard_tolerance():
    g = O.Grid(10, 16, 0.05, 0.03, xa=3)
    e, i = O.load(g, 3000, 1e15, 3.0, 0.026, 5)
    sim = O.Sim(g, 5e-10, tol=1e-11, species=[e, i])

    def total():
        W = O.field_energy(g, sim.er, sim.ez, sim.h)
        return W + O.kinetic_energy(O.ME, sim.state(0)) + O.kinetic_energy(O.M_AR, sim.state(1))
    W0, lost = total(), 0.0
    for _ in range(4):
        rc, st = sim.step()
        assert rc == 0
        lost += st.ke_lost
    assert abs(total() + lost - W0) <= 1e-8 * W0
