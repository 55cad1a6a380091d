"""Pins of the oracle's whole implicit step (rows a2-a8, a5 Picard).

Fixed by the method's guarantees (Sec. 2.1): charge conservation makes the
Gauss residual at interior nodes constant to roundoff over full steps (with
drive, wall losses and ionization); total particle + field energy is
conserved to the nonlinear tolerance and the error shrinks with it; a cold
plasma oscillates at the CN frequency (2/dt)*atan(w_pe*dt/2); a step that
fails to converge leaves the state untouched; on a tiny grid the Picard step
equals the fixed point found by Newton with a finite-difference Jacobian on
the full nonlinear system (brute force).
"""
import numpy as np
import pytest

import oracle as O

QE, ME, M_AR = O.QE, O.ME, O.M_AR


def node_Q(sim):
    g = sim.grid
    Q = np.zeros(g.n_node)
    for s in range(len(sim.sp)):
        O.node_charge(g, sim.sp[s]["q"], sim.state(s), Q)
    return Q


def small_sim(n=4000, volt=0.0, mcc=False, tol=1e-10, te=3.0, seed=3, dt=None, nr=12, nz=24):
    g = O.Grid(nr, nz, 0.05, 0.03)
    f = 60e6
    dt = dt or 1.0 / (200 * f)
    e, i = O.load(g, n, 1e15, te, 0.026, seed)
    sim = O.Sim(g, dt, freq=f, volt=volt, tol=tol, kmax=60, mcc_on=mcc, ng=2.0 / (O.KB * 300),
                seed=seed, species=[e, i])
    return sim


def test_gauss_residual_constant_over_steps_with_drive_and_mcc():
    sim = small_sim(volt=300.0, mcc=True, te=6.0)
    g = sim.grid
    G0 = O.gauss_residual(g, sim.er, sim.ez, node_Q(sim))
    qscale = np.max(np.abs(node_Q(sim))) + np.sum(np.abs(sim.state(0)["w"])) * QE / g.n_node
    absorbed = 0
    iz = 0
    for _ in range(12):
        rc, st = sim.step()
        assert rc == 0 and st.converged
        absorbed += st.counters[1]
        iz += st.mcc[3]
        G = O.gauss_residual(g, sim.er, sim.ez, node_Q(sim))
        assert np.max(np.abs(G - G0)) <= 1e-11 * qscale
    assert absorbed > 0
    assert np.max(np.abs(sim.ez)) > 1.0  # the drive is on


def _energy_errors(tol):
    sim = small_sim(volt=0.0, mcc=False, tol=tol, te=3.0)
    g = sim.grid

    def total():
        K = sum(O.kinetic_energy(sim.sp[s]["m"], sim.state(s)) for s in range(2))
        return K + O.field_energy(g, sim.er, sim.ez, sim.h)

    W0 = total()
    lost = 0.0
    errs = []
    for _ in range(10):
        Wb = total()
        rc, st = sim.step()
        assert rc == 0
        lost += st.ke_lost
        errs.append(abs(total() + st.ke_lost - Wb - st.src_energy) / W0)
    assert lost > 0  # wall losses are part of the balance
    return max(errs)


def test_energy_conserved_to_nonlinear_tolerance():
    """|dW_total|/W per step is bounded by the Picard tolerance and falls with it."""
    loose = _energy_errors(1e-5)
    tight = _energy_errors(1e-11)
    assert loose < 1e-4
    assert tight < 1e-9
    assert tight < loose


def quiet_lattice(g, n0, na, nb):
    """Quiet start: na x nb particles on a regular lattice in every cell,
    weight = n0 * (cell-fraction of the annular volume 2 pi r dr dz)."""
    ic, jc, ka, kb = np.meshgrid(np.arange(g.nr), np.arange(g.nz), np.arange(na), np.arange(nb),
                                 indexing="ij")
    ic, jc, ka, kb = [x.ravel() for x in (ic, jc, ka, kb)]
    a = (ka + 0.5) / na
    b = (kb + 0.5) / nb
    r = (ic + a) * g.dr
    n = len(a)
    sp = {"cell": (ic * g.nz + jc).astype(np.int32), "a": a, "b": b, "vr": np.zeros(n),
          "vt": np.zeros(n), "vz": np.zeros(n), "w": n0 * 2 * np.pi * r * g.dr * g.dz / (na * nb),
          "id": np.arange(n, dtype=np.uint32)}
    o = np.argsort(sp["cell"], kind="stable")
    return {k: v[o].copy() for k, v in sp.items()}


def test_cold_plasma_oscillation_cn_frequency():
    """Uniform cold electrons over immobile ions (quiet lattice start),
    v_z = u0 sin(2 pi z/L): each fluid element oscillates at w_pe; CN turns
    it into (2/dt) atan(w_pe dt/2), 7 % below w_pe at w_pe dt = 1."""
    nr, nz = 4, 64
    g = O.Grid(nr, nz, 0.2, 0.03)
    n0 = 1e15
    wpe = np.sqrt(n0 * QE ** 2 / (O.EPS0 * ME))
    dt = 1.0 / wpe
    e = quiet_lattice(g, n0, 2, 4)
    i = {k: v.copy() for k, v in e.items()}
    z0 = ((e["cell"] % nz) + e["b"]) * g.dz
    e["vz"] = 1e3 * np.sin(2 * np.pi * z0 / g.L)
    sim = O.Sim(g, dt, tol=1e-12, kmax=80, species=[e, i], masses=(ME, M_AR * 1e9))
    r0 = ((e["cell"] // nz) + e["a"]) * g.dr
    sel = r0 < 0.4 * g.R
    ids = e["id"][sel]
    w = np.sin(2 * np.pi * z0[sel] / g.L)
    xs = []
    for _ in range(60):
        rc, _ = sim.step()
        assert rc == 0
        st = sim.state(0)
        order = np.argsort(st["id"])
        k = order[np.searchsorted(st["id"][order], ids)]
        z = ((st["cell"][k] % nz) + st["b"][k]) * g.dz
        xs.append(np.sum((z - z0[sel]) * w))
    xs = np.array(xs)
    s = np.sign(xs)
    idx = np.where(s[:-1] * s[1:] < 0)[0]
    t = (idx + 1 + xs[idx] / (xs[idx] - xs[idx + 1])) * dt
    w_num = np.pi / ((t[-1] - t[0]) / (len(t) - 1))
    w_cn = 2.0 / dt * np.arctan(wpe * dt / 2.0)
    assert abs(w_num - w_cn) / w_cn < 0.01
    assert abs(w_num - wpe) / wpe > 0.05


def test_noconv_leaves_state_unchanged():
    sim = small_sim(n=500, tol=1e-300)
    sim.cfg.kmax = 2
    before = sim.state(0)
    er = sim.er.copy()
    rc, st = sim.step()
    assert rc == -3 and not st.converged and st.picard_iters == 2
    after = sim.state(0)
    for k in before:
        np.testing.assert_array_equal(before[k], after[k])
    np.testing.assert_array_equal(er, sim.er)
    assert sim.step_index == 0


def test_picard_step_equals_newton_brute_force_on_a_tiny_grid():
    """The implicit step is the fixed point E = G(E) of push + field solve
    (Sec. 2.1).  On a 3x4 grid with 8 strongly weighted electrons (so that the
    field couples back), Newton with a finite-difference Jacobian on the full
    nonlinear system, no Picard, reaches the same E^{n+1} and particle state as
    the oracle's Picard step."""
    nr, nz = 3, 4
    g = O.Grid(nr, nz, 0.01, 0.01)
    dt, f, V = 2e-10, 60e6, 30.0
    rng = np.random.default_rng(11)
    n = 8
    sp = O.empty_species(n)
    ic, jc = rng.integers(0, nr, n), rng.integers(0, nz, n)
    sp["cell"][:] = ic * nz + jc
    sp["a"][:] = 0.3 + 0.4 * rng.random(n)
    sp["b"][:] = 0.3 + 0.4 * rng.random(n)
    sp["vr"][:], sp["vt"][:], sp["vz"][:] = rng.normal(size=(3, n)) * 2e5
    sp["w"][:] = 3e7
    sp["id"][:] = np.arange(n)
    ions = {k: v.copy() for k, v in sp.items()}
    ions["vr"][:] = ions["vt"][:] = ions["vz"][:] = 0.0
    sim = O.Sim(g, dt, freq=f, volt=V, tol=1e-14, kmax=200, species=[sp, ions])
    er0, ez0, h0 = sim.er.copy(), sim.ez.copy(), sim.h.copy()
    F = O.FieldSolver(g, dt)
    v1 = V * np.sin(2 * np.pi * f * dt)
    mr = np.ones((nr, nz + 1), bool)
    mr[:, [0, nz]] = False
    ur = np.flatnonzero(mr.ravel())            # unknown E_r edges
    uz = np.arange(nr * nz)                     # unknown E_z edges (i < nr)

    def fields(x):
        er, ez = np.zeros(g.n_er), np.zeros(g.n_ez)
        er[ur], ez[uz] = x[:len(ur)], x[len(ur):]
        ez[nr * nz:] = v1 / g.L
        return er, ez

    def G(x):
        er1, ez1 = fields(x)
        ir, iz = np.zeros(g.n_er), np.zeros(g.n_ez)
        for s, (q, m) in enumerate(((-QE, ME), (QE, M_AR))):
            O.push(g, dt, q, m, sim.state(s), 0.5 * (er0 + er1), 0.5 * (ez0 + ez1), ir=ir, iz=iz)
        ern, ezn, _, _ = F.solve(er0, ez0, h0, ir, iz, 0.0, v1)
        return np.concatenate([ern[ur], ezn[uz]])

    x = G(np.concatenate([er0[ur], ez0[uz]]))
    for _ in range(20):
        r = x - G(x)
        if np.linalg.norm(r) <= 1e-14 * np.linalg.norm(x):
            break
        J = np.eye(len(x))
        for k in range(len(x)):
            hk = 1e-6 * max(abs(x[k]), 1e-3 * np.max(np.abs(x)))
            e = np.zeros(len(x))
            e[k] = hk
            J[:, k] -= (G(x + e) - G(x - e)) / (2 * hk)
        x = x - np.linalg.solve(J, r)
    assert np.linalg.norm(x - G(x)) <= 1e-12 * np.linalg.norm(x)
    rc, st = sim.step()
    assert rc == 0 and st.picard_iters > 2  # the coupling is strong enough to iterate
    ern, ezn = fields(x)
    scale = np.max(np.abs(x))
    assert np.max(np.abs(sim.er[ur] - ern[ur])) <= 1e-10 * scale
    assert np.max(np.abs(sim.ez[uz] - ezn[uz])) <= 1e-10 * scale
    # the committed particles follow the Newton half field
    ref = O.empty_species(n)
    for k in O.FIELDS:
        ref[k][:] = sp[k]
    O.push(g, dt, -QE, ME, ref, 0.5 * (er0 + ern), 0.5 * (ez0 + ezn), write=True)
    got = sim.state(0)
    o = np.argsort(got["id"])
    for k in ("a", "b", "vr", "vz"):
        np.testing.assert_allclose(got[k][o], ref[k], rtol=1e-9, atol=1e-12 * np.max(np.abs(ref[k])))
