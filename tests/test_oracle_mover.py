"""Pins of the oracle's CN mover + charge-conserving deposit (rows a2, a3).

Each check is fixed by the mathematics of Eq. 4 / Eq. 3 rather than by the
oracle itself: exact ballistic and constant-force orbits (CN is exact for a
constant acceleration, so sub-stepping must not change them), discrete charge
continuity per node (Villasenor-Buneman for S1 shapes), the work-energy
identity between gather and deposit, exact conservation of (canonical)
angular momentum and |v| under CN, the CN gyration angle 2*atan(w dt/2),
and the E x B drift.
"""
import numpy as np
import pytest

import oracle as O
from tests import inputs

QE, ME = O.QE, O.ME


def grid():
    return O.Grid(16, 24, 0.05, 0.03)


def xi_eta(g, sp):
    ic = sp["cell"] // g.nz
    jc = sp["cell"] % g.nz
    return ic + sp["a"], jc + sp["b"]


def divergence(g, ir, iz):
    """node-wise net charge flux out of each node's dual cell"""
    IR = ir.reshape(g.nr, g.nz + 1)
    IZ = iz.reshape(g.nr + 1, g.nz)
    D = np.zeros((g.nr + 1, g.nz + 1))
    D[:-1, :] += IR
    D[1:, :] -= IR
    D[:, :-1] += IZ
    D[:, 1:] -= IZ
    return D.ravel()


def interior_particles(g, n, seed, vth):
    """particles in cells away from axis and walls"""
    rng = np.random.default_rng(seed + 99)
    ic = rng.integers(4, g.nr - 4, size=n)
    jc = rng.integers(5, g.nz - 5, size=n)
    return inputs.particles(g.nr, g.nz, n, seed, vth, cells=ic * g.nz + jc)


def test_ballistic_free_flight_exact():
    g = grid()
    dt = 2e-9
    sp = interior_particles(g, 2000, 1, 3e5)  # |v dt| up to ~2 cells
    sp["vt"][:] = 0.0
    x0, y0 = xi_eta(g, sp)
    v0 = (sp["vr"].copy(), sp["vz"].copy())
    er, ez, _ = g.zeros_fields()
    _, _, cnt, _ = O.push(g, dt, -QE, ME, sp, er, ez, write=True)
    x1, y1 = xi_eta(g, sp)
    assert cnt[0] == 0 and cnt[3] == 0
    np.testing.assert_allclose(x1, x0 + v0[0] * dt / g.dr, rtol=0, atol=1e-12)
    np.testing.assert_allclose(y1, y0 + v0[1] * dt / g.dz, rtol=0, atol=1e-12)
    assert np.array_equal(sp["vr"], v0[0]) and np.array_equal(sp["vz"], v0[1])
    assert cnt[2] > 2000  # cell crossings happened


@pytest.mark.parametrize("comp", ["z", "r"])
def test_constant_force_parabola_exact(comp):
    g = grid()
    dt = 2e-9
    sp = interior_particles(g, 2000, 2, 1e5)
    sp["vt"][:] = 0.0
    er, ez, _ = g.zeros_fields()
    E0 = 40.0
    if comp == "z":
        ez[:] = E0
    else:
        er[:] = E0
    qm = -QE / ME
    x0, y0 = xi_eta(g, sp)
    vr0, vz0 = sp["vr"].copy(), sp["vz"].copy()
    _, _, cnt, _ = O.push(g, dt, -QE, ME, sp, er, ez, write=True)
    x1, y1 = xi_eta(g, sp)
    acc = qm * E0
    if comp == "z":
        np.testing.assert_allclose(y1 * g.dz, y0 * g.dz + vz0 * dt + 0.5 * acc * dt * dt,
                                   rtol=0, atol=1e-12 * g.dz)
        np.testing.assert_allclose(sp["vz"], vz0 + acc * dt, rtol=1e-12, atol=1e-9)
        np.testing.assert_allclose(x1 * g.dr, x0 * g.dr + vr0 * dt, rtol=0, atol=1e-12 * g.dr)
    else:
        np.testing.assert_allclose(x1 * g.dr, x0 * g.dr + vr0 * dt + 0.5 * acc * dt * dt,
                                   rtol=0, atol=1e-12 * g.dr)
        np.testing.assert_allclose(sp["vr"], vr0 + acc * dt, rtol=1e-12, atol=1e-9)
    assert cnt[0] == 0


def test_grazing_crossings_land_on_the_first_crossing():
    """Electrons decelerated by a uniform E_z whose parabola peaks just beyond
    the upper z-face of their cell and ends beyond it: each crosses that face
    exactly once.  The sub-step must end on that (first) crossing and the
    rest of the step runs in the next cell: two sub-steps per particle, no
    halving fallback, and the end state of the exact parabola (CN is exact for
    a constant acceleration).  A landing started on the far side of the
    crossing time can converge past the first root and fall back to halving."""
    g = grid()
    dt = 1e-9
    n = 400
    rng = np.random.default_rng(5)
    k = 1.0                                   # deceleration, cells per step^2
    Ez = k * g.dz / (QE / ME * dt * dt)      # electrons: a_z = -k dz / dt^2
    sp_ = rng.uniform(0.85, 1.0, size=n)      # peak time [steps]
    graze = 0.5 * k * (1.0 - sp_) ** 2        # the peak's height above the end point
    delta = graze + rng.uniform(1e-5, 5e-3, size=n)  # peak above the face
    u = k * sp_                               # initial z velocity [cells per step]
    b0 = 1.0 + delta - 0.5 * k * sp_ ** 2
    ic = rng.integers(4, g.nr - 4, size=n)
    jc = rng.integers(5, g.nz - 6, size=n)
    order = np.argsort(ic * g.nz + jc, kind="stable")
    sp = {"cell": (ic * g.nz + jc)[order].astype(np.int32), "a": rng.random(n)[order],
          "b": b0[order], "vr": np.zeros(n), "vt": np.zeros(n), "vz": (u * g.dz / dt)[order],
          "w": np.ones(n), "id": np.arange(n, dtype=np.uint32)}
    x0, y0 = xi_eta(g, sp)
    vz0 = sp["vz"].copy()
    er, ez, _ = g.zeros_fields()
    ez[:] = Ez
    _, _, cnt, _ = O.push(g, dt, -QE, ME, sp, er, ez, write=True)
    x1, y1 = xi_eta(g, sp)
    assert cnt[0] == 0 and cnt[3] == 0, cnt
    assert cnt[2] == 2 * n, cnt
    acc = -QE / ME * Ez
    np.testing.assert_allclose(y1 * g.dz, y0 * g.dz + vz0 * dt + 0.5 * acc * dt * dt,
                               rtol=0, atol=1e-12 * g.dz)
    np.testing.assert_allclose(sp["vz"], vz0 + acc * dt, rtol=1e-12, atol=1e-9)
    assert np.array_equal(sp["cell"], (ic * g.nz + jc + 1)[order])
    np.testing.assert_array_equal(x1, x0)


def test_inertial_terms_conserve_energy_and_angular_momentum():
    """E = 0: CN keeps vr^2+vt^2+vz^2 and r*vt exact (arithmetic-mean identity)."""
    g = grid()
    dt = 2e-9
    sp = inputs.particles(g.nr, g.nz, 3000, 3, 4e5)
    # keep them off the walls in z and r (axis allowed)
    sp["cell"] = (sp["cell"] // g.nz).clip(0, g.nr - 6) * g.nz + (sp["cell"] % g.nz).clip(6, g.nz - 7)
    x0, _ = xi_eta(g, sp)
    L0 = x0 * g.dr * sp["vt"]
    K0 = sp["vr"] ** 2 + sp["vt"] ** 2 + sp["vz"] ** 2
    er, ez, _ = g.zeros_fields()
    for _ in range(3):
        _, _, cnt, _ = O.push(g, dt, -QE, ME, sp, er, ez, write=True)
        assert cnt[0] == 0
    alive = sp["cell"] >= 0
    x1, _ = xi_eta(g, sp)
    L1 = x1 * g.dr * sp["vt"]
    K1 = sp["vr"] ** 2 + sp["vt"] ** 2 + sp["vz"] ** 2
    np.testing.assert_allclose(K1[alive], K0[alive], rtol=1e-12)
    np.testing.assert_allclose(L1[alive], L0[alive], rtol=1e-11, atol=1e-30)
    # CN orbit approximates the Cartesian straight line to second order
    near = alive & (x0 > 3)
    assert near.sum() > 500


def test_free_flight_matches_cartesian_line_far_from_axis():
    g = O.Grid(16, 24, 0.05, 0.03)
    dt = 1e-10
    sp = interior_particles(g, 500, 4, 3e5)  # v dt ~ 0.01 dr, r >= 4 dr
    x0, y0 = xi_eta(g, sp)
    r0, vr, vt = x0 * g.dr, sp["vr"].copy(), sp["vt"].copy()
    er, ez, _ = g.zeros_fields()
    O.push(g, dt, -QE, ME, sp, er, ez, write=True)
    x1, _ = xi_eta(g, sp)
    r_exact = np.sqrt((r0 + vr * dt) ** 2 + (vt * dt) ** 2)
    step = np.sqrt(vr ** 2 + vt ** 2) * dt
    assert np.max(np.abs(x1 * g.dr - r_exact) / step) < 1e-3


@pytest.mark.parametrize("seed", [5, 6])
def test_discrete_charge_continuity_per_node(seed):
    """Q^{n+1} - Q^n + div(dQ) + wall tallies = 0 at every node (Eq. 3 with
    S1 shapes on sub-step segments), incl. cell crossings and wall losses."""
    g = grid()
    dt = 1e-9
    sp = inputs.particles(g.nr, g.nz, 6000, seed, 8e5, edge_frac=0.05)
    er, ez = inputs.smooth_fields(g.nr, g.nz, seed, 3e3)
    q = -QE
    Q0 = O.node_charge(g, q, sp)
    walls = (np.zeros(g.nr + 1), np.zeros(g.nr + 1), np.zeros(g.nz + 1))
    ir, iz, cnt, _ = O.push(g, dt, q, ME, sp, er, ez, write=True, walls=walls)
    assert cnt[0] == 0
    assert cnt[1] > 0  # some absorbed
    assert cnt[2] > 1.3 * 6000  # many crossings
    Q1 = O.node_charge(g, q, sp)
    W = np.zeros((g.nr + 1, g.nz + 1))
    W[:, 0] += walls[0]
    W[:, -1] += walls[1]
    W[-1, :] += walls[2]
    res = Q1 + W.ravel() - Q0 + divergence(g, ir, iz)
    assert np.max(np.abs(res)) <= 1e-13 * np.max(np.abs(Q0))


def test_work_energy_identity_gather_deposit():
    """Sum of kinetic-energy changes equals sum over edges of E * length * dQ
    (the gather and the deposit use the same S0 x S1 weights)."""
    g = grid()
    dt = 1e-9
    m = ME
    q = -QE
    sp = inputs.particles(g.nr, g.nz, 6000, 7, 6e5)
    er, ez = inputs.smooth_fields(g.nr, g.nz, 7, 5e3)
    K0 = O.kinetic_energy(m, sp)
    ir, iz, cnt, kel = O.push(g, dt, q, m, sp, er, ez, write=True)
    K1 = O.kinetic_energy(m, sp) + kel
    work = np.sum(er * ir) * g.dr + np.sum(ez * iz) * g.dz
    assert cnt[0] == 0
    assert abs((K1 - K0) - work) <= 1e-9 * abs(K1 - K0) + 1e-12 * K0


def test_axis_reflection_zero_angular_momentum():
    g = grid()
    dt = 2e-9
    n = 200
    rng = np.random.default_rng(8)
    sp = inputs.particles(g.nr, g.nz, n, 8, 1.0, cells=np.full(n, 0 * g.nz + 10))
    sp["a"] = rng.random(n) * 0.8 + 0.1
    sp["b"][:] = 0.5
    sp["vt"][:] = 0.0
    sp["vz"][:] = 0.0
    sp["vr"] = -(0.5 + rng.random(n)) * g.dr / dt  # crosses the axis within the step
    r0 = sp["a"] * g.dr
    vr0 = sp["vr"].copy()
    er, ez, _ = g.zeros_fields()
    O.push(g, dt, -QE, ME, sp, er, ez, write=True)
    x1, _ = xi_eta(g, sp)
    np.testing.assert_allclose(x1 * g.dr, np.abs(r0 + vr0 * dt), rtol=0, atol=1e-13 * g.dr)
    crossed = r0 + vr0 * dt < 0
    assert crossed.sum() > 50
    np.testing.assert_array_equal(sp["vr"], np.where(crossed, -vr0, vr0))


def test_wall_absorption_and_tally():
    g = grid()
    dt = 1e-9
    sp = inputs.particles(g.nr, g.nz, 50, 9, 1.0, cells=np.full(50, 5 * g.nz + g.nz - 1))
    sp["vr"][:] = 0.0
    sp["vt"][:] = 0.0
    sp["vz"][:] = 2.0 * g.dz / dt
    walls = (np.zeros(g.nr + 1), np.zeros(g.nr + 1), np.zeros(g.nz + 1))
    q = QE
    O.push(g, dt, q, O.M_AR, sp, *g.zeros_fields()[:2], write=True, walls=walls)
    assert np.all(sp["cell"] == -1)
    np.testing.assert_allclose(walls[1][5], np.sum(q * sp["w"] * (1 - sp["a"])), rtol=1e-13)
    np.testing.assert_allclose(walls[1][6], np.sum(q * sp["w"] * sp["a"]), rtol=1e-13)
    assert walls[0].sum() == 0 and walls[2].sum() == 0


def test_near_axis_centrifugal_barrier_robust():
    """Particles close to the axis with L != 0 never reach r = 0; energy and
    angular momentum stay exact (no fallback needed for a modest swing)."""
    g = grid()
    dt = 5e-10
    n = 500
    rng = np.random.default_rng(10)
    sp = inputs.particles(g.nr, g.nz, n, 10, 1.0, cells=np.full(n, 0 * g.nz + 12))
    sp["a"] = 10 ** rng.uniform(-4, -1, size=n)
    v = 1e6
    ang = rng.uniform(0, 2 * np.pi, size=n)
    sp["vr"] = v * np.cos(ang)
    sp["vt"] = v * np.sin(ang)
    sp["vz"][:] = 0.0
    r0 = sp["a"] * g.dr
    L0 = r0 * sp["vt"]
    er, ez, _ = g.zeros_fields()
    _, _, cnt, _ = O.push(g, dt, -QE, ME, sp, er, ez, write=True)
    assert cnt[0] == 0
    x1, _ = xi_eta(g, sp)
    np.testing.assert_allclose(x1 * g.dr * sp["vt"], L0, rtol=1e-10)
    np.testing.assert_allclose(np.hypot(sp["vr"], sp["vt"]), v, rtol=1e-12)
    assert np.all(x1 > 0)


# ------------------------------------------------------------- external B_z
def test_bz_canonical_momentum_speed_and_fixed_orbit():
    g = O.Grid(16, 24, 0.05, 0.03)
    dt = 1e-10
    B = 0.01
    qm = -QE / ME
    wc = qm * B
    sp = interior_particles(g, 400, 11, 2e5)
    er, ez, _ = g.zeros_fields()
    x0, _ = xi_eta(g, sp)
    P0 = x0 * g.dr * sp["vt"] + 0.5 * wc * (x0 * g.dr) ** 2
    S0 = sp["vr"] ** 2 + sp["vt"] ** 2 + sp["vz"] ** 2
    for _ in range(4):
        _, _, cnt, _ = O.push(g, dt, -QE, ME, sp, er, ez, write=True, bz=B)
    x1, _ = xi_eta(g, sp)
    P1 = x1 * g.dr * sp["vt"] + 0.5 * wc * (x1 * g.dr) ** 2
    np.testing.assert_allclose(P1, P0, rtol=1e-10, atol=1e-12 * np.max(np.abs(P0)))
    np.testing.assert_allclose(sp["vr"] ** 2 + sp["vt"] ** 2 + sp["vz"] ** 2, S0, rtol=1e-12)
    # centred circular orbit vr = 0, vt = -wc r0 is an exact fixed point of CN
    orb = inputs.particles(g.nr, g.nz, 20, 12, 1.0, cells=np.arange(20) % 10 * g.nz + 12 + 0 * np.arange(20))
    orb["vr"][:] = 0.0
    orb["vz"][:] = 0.0
    xo, _ = xi_eta(g, orb)
    orb["vt"] = -wc * xo * g.dr
    for _ in range(5):
        O.push(g, dt, -QE, ME, orb, er, ez, write=True, bz=B)
    xo1, _ = xi_eta(g, orb)
    np.testing.assert_allclose(xo1, xo, rtol=0, atol=1e-13)
    assert np.max(np.abs(orb["vr"])) <= 1e-9 * np.max(np.abs(orb["vt"]))


def test_bz_gyration_angle_is_cn_rotation():
    """At r >> rho_L the velocity rotates by 2*atan(wc*dt/2) per step
    (exact CN rotation) up to the frame rotation O(v dt / r)."""
    g = O.Grid(16, 24, 0.05, 0.03)
    B = 0.05
    qm = -QE / ME
    wc = qm * B
    dt = 1.2 / abs(wc)  # large angle: the atan correction is 10 %
    n = 50
    sp = inputs.particles(g.nr, g.nz, n, 13, 1.0, cells=np.full(n, 12 * g.nz + 12))
    v = 2e3  # rho_L = v/wc ~ 2e-7 m << r ~ 0.04 m
    sp["vr"][:] = v
    sp["vt"][:] = 0.0
    sp["vz"][:] = 0.0
    er, ez, _ = g.zeros_fields()
    O.push(g, dt, -QE, ME, sp, er, ez, write=True, bz=B)
    ang = np.arctan2(sp["vt"], sp["vr"])
    expect = -2.0 * np.arctan(wc * dt / 2.0)
    np.testing.assert_allclose(ang, expect, rtol=1e-4)
    assert abs(expect - (-wc * dt)) > 0.04  # distinguishes CN from exact rotation


def test_exb_drift():
    """Uniform E_r and B_z: guiding centre drifts with v_theta = -E_r/B_z."""
    g = O.Grid(16, 24, 0.05, 0.03)
    B = 0.05
    E0 = 100.0
    qm = -QE / ME
    wc = abs(qm * B)
    dt = 0.3 / wc
    n = 10
    sp = inputs.particles(g.nr, g.nz, n, 14, 1.0, cells=np.full(n, 12 * g.nz + 12))
    sp["vr"][:] = 0.0
    sp["vt"][:] = 0.0
    sp["vz"][:] = 0.0
    er, ez, _ = g.zeros_fields()
    er[:] = E0
    vts = []
    for _ in range(400):
        O.push(g, dt, -QE, ME, sp, er, ez, write=True, bz=B)
        vts.append(sp["vt"].copy())
    vmean = np.mean(np.array(vts), axis=0)
    vE = -E0 / B
    r = 12.5 * g.dr
    assert np.all(np.abs(vmean - vE) <= 0.02 * abs(vE) + 10 * vE ** 2 / (wc * r))


def test_threaded_timing_form_matches_serial():
    """The oracle's threaded push (the CPU baseline's timing form) gives the
    serial form's particles bit for bit and its crossed charge, wall tallies
    and counters up to the summation order."""
    g = grid()
    dt = 1e-9
    sp0 = inputs.particles(g.nr, g.nz, 20000, 9, 8e5, edge_frac=0.02)
    er, ez = inputs.smooth_fields(g.nr, g.nz, 4, 3e3)
    outs = []
    for nt in (1, 4):
        O.set_threads(nt)
        sp = {k: v.copy() for k, v in sp0.items()}
        walls = (np.zeros(g.nr + 1), np.zeros(g.nr + 1), np.zeros(g.nz + 1))
        ir, iz, cnt, kel = O.push(g, dt, -QE, ME, sp, er, ez, write=True, walls=walls)
        outs.append((sp, ir, iz, cnt, kel, walls))
    O.set_threads(1)
    (s1, ir1, iz1, c1, k1, w1), (s4, ir4, iz4, c4, k4, w4) = outs
    for k in s1:
        assert np.array_equal(s1[k], s4[k]), k
    assert np.array_equal(c1, c4)
    scale = np.max(np.abs(np.concatenate([ir1, iz1])))
    np.testing.assert_allclose(ir4, ir1, rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(iz4, iz1, rtol=0, atol=1e-13 * scale)
    for a, b in zip(w1, w4):
        np.testing.assert_allclose(b, a, rtol=1e-13, atol=1e-30)
    assert abs(k4 - k1) <= 1e-13 * abs(k1)
