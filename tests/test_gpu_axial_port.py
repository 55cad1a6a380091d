"""Axial dielectric port (PIC_FEED_AXIAL; Sec. 2.2, Eqs. 5 and 7) on the GPU
against the oracle's banded solve of the same system.

The GPU solve is exact, not iterative: the reactor's separable solver and the
port block's dense inverse, coupled through the interface edges on z = 0 by
the Woodbury identity.  So every field of a solve equals the oracle's to
rounding (1e-10 of the largest value), for the three transforms along z (FFT,
even/odd split, dense), and a vacuum run of whole steps (pic_step, no
particles) follows the oracle's solves step by step.  With particles, the
energy of fields and particles changes by what the port delivers and the
walls absorb (to the Picard tolerance), and Gauss's law holds on the
reactor's interior nodes (charge conservation of the deposit).
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as G
    G.build()


def P():
    import paper_2212_08836_gb300 as M
    return M


def make(nr, nz, ip, nzp, Lp=0.03, erq=3.8, dt=2e-11, **kw):
    M = P()
    cfg = M.small_reactor(nr=nr, nz=nz, R=0.1, L=0.02, dt=dt, feed=M.PIC_FEED_AXIAL,
                          port_cells=nzp, port_len=Lp, port_rin=ip, eps_port=erq, **kw)
    return M.Pic(cfg, device=DEV), cfg


def tg(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def close(a, b, tol=1e-10):
    return np.max(np.abs(a - b)) <= tol * max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("nr,nz,ip,nzp,grade,xa", [(16, 12, 10, 6, 1.0, 0), (20, 20, 13, 8, 1.0, 0),
                                                   (18, 15, 11, 5, 1.0, 0), (16, 12, 10, 9, 1.3, 0),
                                                   (16, 12, 10, 6, 1.0, 2)],
                         ids=["fft", "split", "dense", "graded", "mapped"])
def test_port_field_solve_matches_oracle(nr, nz, ip, nzp, grade, xa):
    pic, cfg = make(nr, nz, ip, nzp, port_grade=grade, axis_cells=xa)
    g = O.Grid(nr, nz, cfg["R"], cfg["L"], xa)
    S = O.PortSolver(g, cfg["dt"], ip, nzp, cfg["port_len"] / nzp, cfg["eps_port"],
                     heights=O.port_heights(nzp, cfg["port_len"], grade))
    rng = np.random.default_rng(nr + nz)
    er, ez, h = rng.normal(size=g.n_er) * 1e3, rng.normal(size=g.n_ez) * 1e3, rng.normal(size=nr * nz)
    er.reshape(nr, nz + 1)[:, nz] = 0.0
    er.reshape(nr, nz + 1)[:ip, 0] = 0.0
    ez.reshape(nr + 1, nz)[nr, :] = 0.0
    erp, ezp, hp = S.zeros_port()
    erp[:] = rng.normal(size=erp.size) * 1e3
    ezp[:] = rng.normal(size=ezp.size) * 1e3
    hp[:] = rng.normal(size=hp.size)
    m = nr - ip
    ezp.reshape(m + 1, nzp)[[0, m], :] = 0.0
    ir, iz = rng.normal(size=g.n_er) * 1e-12, rng.normal(size=g.n_ez) * 1e-12
    phi0, phi1 = 37.0, -12.5
    ref = S.solve(er, ez, h, erp, ezp, hp, ir, iz, phi0, phi1)
    out = [torch.zeros(n, dtype=torch.float64, device=DEV)
           for n in (g.n_er, g.n_ez, nr * nz, m * nzp, m * nzp, (m + 1) * nzp)]
    src = torch.zeros(1, dtype=torch.float64, device=DEV)
    pic.port_field_solve(tg(er), tg(ez), tg(h), tg(hp), tg(erp), tg(ezp), tg(ir), tg(iz), phi0,
                         phi1, out[0], out[1], out[2], out[3], out[4], out[5], src)
    got = [t.cpu().numpy() for t in out]
    # order of the oracle's outputs: er, ez, h, erp, ezp, hp
    for k, (a, b) in enumerate(zip((got[0], got[1], got[2], got[4], got[5], got[3]), ref[:6])):
        assert close(a, b), k
    assert abs(src.item() - ref[6]) <= 1e-9 * max(abs(ref[6]), 1e-30)


def test_vacuum_steps_follow_the_oracle():
    """pic_step with no particles: each step is one field solve driven by the
    electrode potential V(t) (the Picard iteration converges at its second
    pass), the same as the oracle's solves."""
    nr, nz, ip, nzp = 16, 12, 10, 6
    pic, cfg = make(nr, nz, ip, nzp, freq=200e6, volt=80.0, mcc_on=0, picard_tol=1e-12)
    g = O.Grid(nr, nz, cfg["R"], cfg["L"])
    S = O.PortSolver(g, cfg["dt"], ip, nzp, cfg["port_len"] / nzp, cfg["eps_port"])
    er, ez, h = g.zeros_fields()
    erp, ezp, hp = S.zeros_port()
    ir, iz = np.zeros(g.n_er), np.zeros(g.n_ez)
    V = lambda n: cfg["volt"] * np.sin(2 * np.pi * cfg["freq"] * n * cfg["dt"])
    for n in range(30):
        rc, st = pic.step(1)
        assert rc == 0
        er, ez, h, erp, ezp, hp, src = S.solve(er, ez, h, erp, ezp, hp, ir, iz, V(n), V(n + 1))
    v = pic.view()
    for a, b in ((v["er"], er), (v["ez"], ez), (v["h"], h), (v["port_h"], hp),
                 (v["port_er"], erp), (v["port_ez"], ezp)):
        assert close(a.cpu().numpy(), b, 1e-9)


def test_vacuum_capacitor_energy_and_charge():
    """The capacitor-fed port with no particles: the field energy of reactor
    and port changes by exactly what the port's end delivers, and the
    capacitor charge by the electrode current dt 2 pi r_{ip-1/2} H^{n+1/2}
    at the electrode's rim, the telescoped Ampere law over its first row of
    E_z edges (an expression the step's circuit solve does not evaluate)."""
    nr, nz, ip, nzp = 16, 12, 10, 6
    pic, cfg = make(nr, nz, ip, nzp, freq=200e6, volt=80.0, mcc_on=0, picard_tol=1e-12,
                    cblock=8e-12)
    g = O.Grid(nr, nz, cfg["R"], cfg["L"])
    S = O.PortSolver(g, cfg["dt"], ip, nzp, cfg["port_len"] / nzp, cfg["eps_port"])
    c, rh, dt = (ip - 1) * nz, 2 * np.pi * (ip - 0.5) * g.dr, cfg["dt"]

    def fields():
        v = pic.view()
        return [v[k].cpu().numpy().copy() for k in ("er", "ez", "h", "port_er", "port_ez", "port_h")]

    W = S.energy(*fields())
    for n in range(40):
        f0 = fields()
        q0, _ = pic.circuit()
        rc, st = pic.step(1)
        assert rc == 0
        f1 = fields()
        W1 = S.energy(*f1)
        assert abs(W1 - W - st["src_energy"]) <= 1e-9 * max(W1, 1e-300) + 1e-24, n
        W = W1
        q1, phi = pic.circuit()
        flow = dt * rh * 0.5 * (f0[2][c] + f1[2][c])
        assert abs(flow - (q1 - q0)) <= 1e-7 * max(abs(q1 - q0), 1e-300), n
    v = cfg["volt"] * np.sin(2 * np.pi * cfg["freq"] * 40 * dt)
    assert abs(phi - v) > 0.05 * abs(v)


def test_discharge_energy_and_gauss():
    M = P()
    nr, nz, ip, nzp = 32, 24, 22, 12
    pic, cfg = make(nr, nz, ip, nzp, Lp=0.04, dt=5e-11, freq=100e6, volt=150.0, mcc_on=0,
                    np_init=20000, picard_tol=1e-10)
    pic.load_particles()
    g = O.Grid(nr, nz, cfg["R"], cfg["L"])
    S = O.PortSolver(g, cfg["dt"], ip, nzp, cfg["port_len"] / nzp, cfg["eps_port"])

    def energy():
        v = pic.view()
        f = [v[k].cpu().numpy() for k in ("er", "ez", "h", "port_er", "port_ez", "port_h")]
        d = pic.diag()
        return S.energy(*f) + sum(d["kinetic"])

    def gauss_interior():
        er, ez, _ = pic.fields()
        res = O.gauss_residual(g, er, ez, pic.node_charge().cpu().numpy())
        return res.reshape(nr + 1, nz + 1)[1:nr, 1:nz]

    W0, G0 = energy(), gauss_interior()
    src = lost = 0.0
    for _ in range(20):
        rc, st = pic.step(1)
        assert rc == 0
        src += st["src_energy"]
        lost += st["ke_lost"]
    W1 = energy()
    assert abs((W1 - W0) - (src - lost)) <= 1e-6 * max(W0, W1), (W1 - W0, src, lost)
    qs = np.max(np.abs(pic.node_charge().cpu().numpy()))
    assert np.max(np.abs(gauss_interior() - G0)) <= 1e-9 * qs


@pytest.mark.parametrize("cblock,grade", [(0.0, 1.0), (1e-11, 1.0), (0.0, 1.4)],
                         ids=["driven", "capacitor", "graded"])
def test_full_steps_with_the_port_match_the_oracle(cblock, grade):
    """Whole steps (Picard iteration of push, deposit and the port's field
    solve, commit, sort) of a small discharge fed through the axial port,
    against the oracle's steps with the same port: same iteration counts,
    fields of reactor and port and every particle to 1e-10.  With the blocking
    capacitor (Eq. 6) the electrode potential and the capacitor charge too."""
    from tests.test_gpu_parity import assert_state_close, by_id
    M = P()
    nr, nz, ip, nzp, n = 24, 32, 16, 10, 30000
    pic, cfg = make(nr, nz, ip, nzp, Lp=0.04, dt=5e-11, freq=100e6, volt=200.0, mcc_on=0,
                    np_init=n, capacity_factor=1.5, picard_tol=1e-10, cblock=cblock,
                    port_grade=grade)
    g = O.Grid(nr, nz, cfg["R"], cfg["L"])
    e, i = O.load(g, n, 1e15, 6.0, 0.026, 23)
    pic.set_state([e, i])
    sim = O.Sim(g, cfg["dt"], freq=cfg["freq"], volt=cfg["volt"], tol=cfg["picard_tol"],
                kmax=cfg["picard_max"], species=[e, i], cap=int(n * 1.5), cblock=cblock,
                port=(ip, nzp, cfg["port_len"], cfg["eps_port"], grade))
    for step in range(3):
        rc, st = pic.step(1)
        rco, sto = sim.step()
        assert rc == 0 and rco == 0
        assert st["picard_iters"] == sto.picard_iters
        v = pic.view()
        for k, ref in (("er", sim.er), ("ez", sim.ez), ("h", sim.h), ("port_h", sim.hp),
                       ("port_er", sim.erp), ("port_ez", sim.ezp)):
            assert close(v[k].cpu().numpy(), ref), (step, k)
        for s in range(2):
            got, ref = by_id(pic.get_state(s)), by_id(sim.state(s))
            assert len(got["id"]) == len(ref["id"])
            assert_state_close(got, ref, rtol=1e-10, what="step %d species %d " % (step, s), nz=nz)
        assert st["absorbed"] == sto.counters[1]
        assert abs(st["src_energy"] - sto.src_energy) <= 1e-9 * max(abs(sto.src_energy), 1e-30)
        if cblock > 0:
            q, phi = pic.circuit()
            np.testing.assert_allclose(phi, sim.circ[1], rtol=1e-10)
            np.testing.assert_allclose(q, sim.circ[0], rtol=1e-8)
            assert q != 0.0
