"""Mixed-precision form (FP32 particle state, push and deposit; FP64 field
solve, current accumulation and diagnostics) against the FP64 oracle.

The oracle receives the same FP32-rounded state (as FP64).  Stated
tolerance of the FP32 path: 1e-5 relative per pass/step, every particle; positions are
compared in global logical coordinates (xi = ic + a), because a particle
within ~1e-7 of a face may end on either side of it in FP32.
"""
import numpy as np
import pytest

import oracle as O
from tests import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

QE, ME, M_AR = O.QE, O.ME, O.M_AR
DEV = "cuda:0"
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as G
    G.build()


def P():
    import paper_2212_08836_gb300 as M
    return M


def f32(sp):
    out = {k: v.copy() for k, v in sp.items()}
    for k in ("a", "b", "vr", "vt", "vz", "w"):
        out[k] = out[k].astype(np.float32).astype(np.float64)
    return out


def make_pic(nr, nz, R, L, dt, cap, **kw):
    M = P()
    cfg = M.small_reactor(nr=nr, nz=nz, R=R, L=L, dt=dt, np_init=cap, capacity_factor=1.0,
                          mcc_on=0, precision=M.PIC_MIXED)
    cfg.update(kw)
    return M.Pic(cfg, device=DEV)


def tgpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def gxy(sp, nz):
    alive = sp["cell"] >= 0
    return ((sp["cell"] // nz) + sp["a"].astype(np.float64)), \
           ((sp["cell"] % nz) + sp["b"].astype(np.float64)), alive


@pytest.mark.parametrize("nr,nz,n,dt", [(16, 24, 6000, 1e-9), (32, 64, 40000, 5e-10)])
def test_mixed_push_deposit_parity(nr, nz, n, dt):
    g = O.Grid(nr, nz, 0.05, 0.03)
    e = f32(inputs.particles(nr, nz, n, 1, 8e5))
    i = f32(inputs.particles(nr, nz, n, 2, 3e3))
    er, ez = inputs.smooth_fields(nr, nz, 3, 3e3)
    pic = make_pic(nr, nz, 0.05, 0.03, dt, n)
    pic.set_state([e, i])
    ir = torch.zeros(g.n_er, dtype=torch.float64, device=DEV)
    iz = torch.zeros(g.n_ez, dtype=torch.float64, device=DEV)
    cnt = torch.zeros(5, dtype=torch.int64, device=DEV)
    pic.push_deposit(tgpu(er), tgpu(ez), ir, iz, write=True, counters=cnt)
    assert cnt[0].item() == 0
    ir_o, iz_o = np.zeros(g.n_er), np.zeros(g.n_ez)
    refs = []
    for sp, q, m in ((e, -QE, ME), (i, QE, M_AR)):
        s = {k: v.copy() for k, v in sp.items()}
        O.push(g, dt, q, m, s, er, ez, write=True, ir=ir_o, iz=iz_o)
        refs.append(s)
    # crossed charge per edge: 1e-5 of the largest edge, and in the L2 norm
    got_i = np.concatenate([ir.cpu().numpy(), iz.cpu().numpy()])
    ref_i = np.concatenate([ir_o, iz_o])
    assert np.linalg.norm(got_i - ref_i) <= TOL32 * np.linalg.norm(ref_i)
    assert np.max(np.abs(got_i - ref_i)) <= TOL32 * np.max(np.abs(ref_i))
    for s in range(2):
        got = pic.get_state(s)
        x1, y1, al1 = gxy(got, nz)
        x0, y0, al0 = gxy(refs[s], nz)
        assert np.array_equal(al1, al0)
        # every particle, near-axis starts included: positions within 1e-5 cells,
        # velocities within 1e-5 of the largest speed
        for d in (np.abs(x1 - x0)[al0], np.abs(y1 - y0)[al0]):
            assert np.max(d) <= TOL32
        vs = max(np.max(np.abs(refs[s]["vr"])), np.max(np.abs(refs[s]["vz"])))
        for k in ("vr", "vt", "vz"):
            d = np.abs(got[k].astype(np.float64) - refs[s][k])[al0] / vs
            assert np.max(d) <= TOL32


def test_mixed_continuity_and_gauss_on_gpu():
    """Charge conservation of the FP32 deposit, node by node, over full steps:
    the Gauss residual stays constant to FP32 rounding of the particle state."""
    M = P()
    cfg = M.small_reactor(np_init=40000, volt=300.0, mcc_on=1, picard_tol=1e-8,
                          precision=M.PIC_MIXED)
    pic = M.Pic(cfg, device=DEV)
    pic.load_particles()
    g = O.Grid(cfg["nr"], cfg["nz"], cfg["R"], cfg["L"])

    def gauss():
        er, ez, _ = pic.fields()
        return O.gauss_residual(g, er, ez, pic.node_charge().cpu().numpy())

    G0 = gauss()
    st = pic.get_state(0)
    qs = np.max(np.abs(O.node_charge(g, -QE, {k: v.astype(np.float64) if v.dtype == np.float32 else v
                                              for k, v in st.items()})))
    for _ in range(5):
        rc, stt = pic.step(1)
        assert rc == 0
    drift = np.max(np.abs(gauss() - G0)) / qs
    assert drift <= 1e-6, drift


def test_mixed_full_step_vs_oracle():
    M = P()
    nr, nz, n = 32, 64, 40000
    cfg = M.small_reactor(np_init=n, capacity_factor=1.5, mcc_on=0, picard_tol=1e-8,
                          volt=300.0, precision=M.PIC_MIXED)
    g = O.Grid(nr, nz, cfg["R"], cfg["L"])
    e, i = O.load(g, n, 1e15, 8.0, 0.026, 21)
    e, i = f32(e), f32(i)
    pic = M.Pic(cfg, device=DEV)
    pic.set_state([e, i])
    sim = O.Sim(g, cfg["dt"], freq=cfg["freq"], volt=cfg["volt"], tol=1e-10,
                kmax=cfg["picard_max"], species=[e, i], cap=int(n * 1.5))
    for step in range(3):
        rc, st = pic.step(1)
        rco, sto = sim.step()
        assert rc == 0 and rco == 0
        er, ez, h = pic.fields()
        for got, ref in ((er, sim.er), (ez, sim.ez), (h, sim.h)):
            assert np.max(np.abs(got - ref)) <= TOL32 * np.max(np.abs(ref)), step
        for s in range(2):
            got, ref = pic.get_state(s), sim.state(s)
            og, orr = np.argsort(got["id"]), np.argsort(ref["id"])
            assert len(og) == len(orr)
            G = {k: v[og] for k, v in got.items()}
            Rf = {k: v[orr] for k, v in ref.items()}
            xg, yg, _ = gxy(G, nz)
            xo, yo, _ = gxy(Rf, nz)
            assert np.max(np.abs(xg - xo)) <= TOL32
            assert np.max(np.abs(yg - yo)) <= TOL32
            vs = max(np.max(np.abs(Rf["vr"])), np.max(np.abs(Rf["vz"])))
            for k in ("vr", "vt", "vz"):
                assert np.max(np.abs(G[k].astype(np.float64) - Rf[k])) <= TOL32 * vs


def test_mixed_energy_balance_on_gpu():
    M = P()
    cfg = M.small_reactor(np_init=40000, volt=0.0, mcc_on=0, picard_tol=1e-8,
                          precision=M.PIC_MIXED)
    pic = M.Pic(cfg, device=DEV)
    pic.load_particles()
    d0 = pic.diag()
    W0 = sum(d0["kinetic"]) + d0["field"]
    lost = 0.0
    for _ in range(5):
        _, st = pic.step(1)
        lost += st["ke_lost"]
    d1 = pic.diag()
    W1 = sum(d1["kinetic"]) + d1["field"]
    assert abs(W1 + lost - W0) / W0 <= 5 * 1e-6


def test_mixed_near_axis_invariants():
    """Particles within 1e-4..1e-1 cells of the axis with angular momentum,
    no field: the FP32 CN sub-steps keep |v| and r*v_theta exact to FP32
    rounding and never cross the axis (centrifugal barrier), and every
    particle ends where the FP64 oracle puts it (1e-5)."""
    nr, nz, n, dt = 16, 24, 4000, 5e-10
    g = O.Grid(nr, nz, 0.05, 0.03)
    rng = np.random.default_rng(44)
    e = inputs.particles(nr, nz, n, 45, 1.0, cells=np.sort(rng.integers(4, nz - 4, size=n)))
    e["a"] = 10 ** rng.uniform(-4, -1, size=n)
    v = 1e6
    ang = rng.uniform(0, 2 * np.pi, size=n)
    e["vr"], e["vt"] = v * np.cos(ang), v * np.sin(ang)
    e["vz"] = rng.normal(size=n) * 3e5
    e = f32(e)
    i = f32(inputs.particles(nr, nz, 16, 46, 1e3))
    pic = make_pic(nr, nz, 0.05, 0.03, dt, n)
    pic.set_state([e, i])
    ir = torch.zeros(g.n_er, dtype=torch.float64, device=DEV)
    iz = torch.zeros(g.n_ez, dtype=torch.float64, device=DEV)
    cnt = torch.zeros(5, dtype=torch.int64, device=DEV)
    zr, zz = torch.zeros_like(ir), torch.zeros_like(iz)
    pic.push_deposit(zr, zz, ir, iz, write=True, counters=cnt)
    assert cnt[0].item() == 0
    got = pic.get_state(0)
    x0 = (e["cell"] // nz) + e["a"]
    x1 = (got["cell"] // nz) + got["a"].astype(np.float64)
    assert np.all(x1 > 0)
    s0 = e["vr"] ** 2 + e["vt"] ** 2 + e["vz"] ** 2
    s1 = got["vr"].astype(np.float64) ** 2 + got["vt"].astype(np.float64) ** 2 + \
        got["vz"].astype(np.float64) ** 2
    # FP32 rounding is amplified by the centrifugal term when r' is tiny
    np.testing.assert_allclose(s1, s0, rtol=1e-4)
    L0 = x0 * e["vt"]
    L1 = x1 * got["vt"].astype(np.float64)
    np.testing.assert_allclose(L1, L0, rtol=1e-4, atol=1e-6 * np.max(np.abs(L0)))
    ref = {k: v.copy() for k, v in e.items()}
    er0, ez0, _ = g.zeros_fields()
    O.push(g, dt, -QE, ME, ref, er0, ez0, write=True)
    xr = (ref["cell"] // nz) + ref["a"]
    yr = (ref["cell"] % nz) + ref["b"]
    y1 = (got["cell"] % nz) + got["b"].astype(np.float64)
    assert np.max(np.abs(x1 - xr)) <= TOL32
    assert np.max(np.abs(y1 - yr)) <= TOL32
    for k in ("vr", "vt", "vz"):
        assert np.max(np.abs(got[k].astype(np.float64) - ref[k])) <= TOL32 * v
