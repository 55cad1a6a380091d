"""GPU (sm_103a) parity of every hot-path row against the FP64 oracle.

All calls go through the C ABI (ctypes binding); inputs are seeded synthetic
arrays from tests/inputs.py or the oracle's own loader.  Tolerances: FP64
path 1e-12 relative unless a reason is given at the assertion.
"""
import numpy as np
import pytest

import oracle as O
from tests import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

QE, ME, M_AR = O.QE, O.ME, O.M_AR
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as G
    G.build()


def P():
    import paper_2212_08836_gb300 as M
    return M


def make_pic(nr, nz, R, L, dt, cap, **kw):
    M = P()
    cfg = M.small_reactor(nr=nr, nz=nz, R=R, L=L, dt=dt, np_init=cap, capacity_factor=1.0,
                          mcc_on=0)
    cfg.update(kw)
    return M.Pic(cfg, device=DEV)


def tgpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def by_id(sp):
    o = np.argsort(sp["id"], kind="stable")
    return {k: v[o] for k, v in sp.items()}


def assert_state_close(gs, os_, rtol=1e-12, what="", nz=None):
    """Same particles in the same state.  Positions are compared in global
    logical coordinates: a particle that ends within roundoff of a face may
    sit in either adjacent cell (counted, at most two per comparison)."""
    if nz is None:
        assert np.array_equal(gs["cell"], os_["cell"]), what + " cell"
    else:
        assert np.array_equal(gs["cell"] >= 0, os_["cell"] >= 0), what + " absorbed set"
        bad = np.where(gs["cell"] != os_["cell"])[0]
        info = [(int(gs["id"][k]), int(gs["cell"][k]), float(gs["a"][k]), float(gs["b"][k]),
                 int(os_["cell"][k]), float(os_["a"][k]), float(os_["b"][k])) for k in bad[:5]]
        assert len(bad) <= 2, what + " %d face-side flips %s" % (len(bad), info)
        alive = gs["cell"] >= 0
        for name, x_g, x_o in (("xi", gs["cell"] // nz + gs["a"], os_["cell"] // nz + os_["a"]),
                               ("eta", gs["cell"] % nz + gs["b"], os_["cell"] % nz + os_["b"])):
            np.testing.assert_allclose(x_g[alive], x_o[alive], rtol=0, atol=rtol * 64,
                                       err_msg=what + name)
        # the in-cell offsets and velocities of the particles on the same side
        # of every face (one mask for both sides, so the arrays stay aligned)
        same = gs["cell"] == os_["cell"]
        gs = {k: v[same] for k, v in gs.items()}
        os_ = {k: v[same] for k, v in os_.items()}
    for k in ("a", "b"):
        np.testing.assert_allclose(gs[k], os_[k], rtol=0, atol=rtol, err_msg=what + k)
    vs = max(np.max(np.abs(os_["vr"])), np.max(np.abs(os_["vz"])), 1e-300)
    for k in ("vr", "vt", "vz"):
        np.testing.assert_allclose(gs[k], os_[k], rtol=rtol, atol=rtol * vs, err_msg=what + k)


# ------------------------------------------------------------ a2 + a3 (+a6)
@pytest.mark.parametrize("nr,nz,n,dt", [(16, 24, 6000, 1e-9), (32, 64, 40000, 5e-10),
                                        (5, 7, 333, 2e-9)])
def test_push_deposit_parity(nr, nz, n, dt):
    g = O.Grid(nr, nz, 0.05, 0.03)
    e = inputs.particles(nr, nz, n, 1, 8e5, edge_frac=0.02)
    i = inputs.particles(nr, nz, n, 2, 3e3)
    er, ez = inputs.smooth_fields(nr, nz, 3, 3e3)
    pic = make_pic(nr, nz, 0.05, 0.03, dt, n)
    pic.set_state([e, i])
    ir = torch.zeros(g.n_er, dtype=torch.float64, device=DEV)
    iz = torch.zeros(g.n_ez, dtype=torch.float64, device=DEV)
    cnt = torch.zeros(5, dtype=torch.int64, device=DEV)
    kel = torch.zeros(1, dtype=torch.float64, device=DEV)
    pic.push_deposit(tgpu(er), tgpu(ez), ir, iz, write=True, counters=cnt, ke_lost=kel)
    ir_o, iz_o = np.zeros(g.n_er), np.zeros(g.n_ez)
    cnt_o = np.zeros(4, dtype=np.int64)
    kel_o = 0.0
    states = []
    for sp, q, m in ((e, -QE, ME), (i, QE, M_AR)):
        s = {k: v.copy() for k, v in sp.items()}
        _, _, c, kl = O.push(g, dt, q, m, s, er, ez, write=True, ir=ir_o, iz=iz_o)
        cnt_o += c
        kel_o += kl
        states.append(s)
    scale = max(np.max(np.abs(ir_o)), np.max(np.abs(iz_o)))
    assert np.max(np.abs(ir.cpu().numpy() - ir_o)) <= 1e-12 * scale
    assert np.max(np.abs(iz.cpu().numpy() - iz_o)) <= 1e-12 * scale
    assert list(cnt.cpu().numpy()[:4]) == list(cnt_o)
    assert cnt.cpu().numpy()[4] > 100 * 2 * n  # algorithmic FP64 operations counted
    np.testing.assert_allclose(kel.item(), kel_o, rtol=1e-12)
    assert cnt_o[2] > 1.2 * 2 * n / 2  # crossings exercised
    for s in range(2):
        assert_state_close(pic.get_state(s), states[s], what="species %d " % s)


def test_push_deposit_only_leaves_state():
    nr, nz, n = 16, 24, 3000
    e = inputs.particles(nr, nz, n, 4, 5e5)
    i = inputs.particles(nr, nz, n, 5, 3e3)
    er, ez = inputs.smooth_fields(nr, nz, 6, 1e3)
    pic = make_pic(nr, nz, 0.05, 0.03, 1e-9, n)
    pic.set_state([e, i])
    before = pic.get_state(0)
    ir = torch.zeros(nr * (nz + 1), dtype=torch.float64, device=DEV)
    iz = torch.zeros((nr + 1) * nz, dtype=torch.float64, device=DEV)
    pic.push_deposit(tgpu(er), tgpu(ez), ir, iz, write=False)
    after = pic.get_state(0)
    for k in before:
        np.testing.assert_array_equal(before[k], after[k])
    assert torch.count_nonzero(ir).item() > 0


# ------------------------------------------------------------------ a4
@pytest.mark.parametrize("nr,nz,R,L,dt", [(32, 64, 0.1, 0.03, 1.0 / (200 * 60e6)),
                                          (7, 5, 0.05, 0.03, 1e-10),
                                          (256, 384, 0.3, 0.03, 2.5e-11)])
def test_field_solve_parity(nr, nz, R, L, dt):
    g = O.Grid(nr, nz, R, L)
    rng = np.random.default_rng(nr * 1000 + nz)
    er0 = rng.normal(size=g.n_er) * 100
    er0.reshape(nr, nz + 1)[:, [0, -1]] = 0.0
    ez0 = rng.normal(size=g.n_ez) * 100
    h0 = rng.normal(size=g.n_h) * 0.1
    ir = rng.normal(size=g.n_er) * 1e-12
    iz = rng.normal(size=g.n_ez) * 1e-12
    v0, v1 = 37.0, -12.0
    ez0.reshape(nr + 1, nz)[-1, :] = v0 / L
    F = O.FieldSolver(g, dt)
    er1, ez1, h1, src = F.solve(er0, ez0, h0, ir, iz, v0, v1)
    pic = make_pic(nr, nz, R, L, dt, 16)
    out = [torch.empty(k, dtype=torch.float64, device=DEV) for k in (g.n_er, g.n_ez, g.n_h)]
    s_dev = torch.zeros(1, dtype=torch.float64, device=DEV)
    pic.field_solve(tgpu(er0), tgpu(ez0), tgpu(h0), tgpu(ir), tgpu(iz), v0, v1, *out, src=s_dev)
    torch.cuda.synchronize()
    # separable direct solve vs banded Cholesky of the same SPD system:
    # both exact up to rounding amplified by the condition number
    for got, ref in zip(out, (er1, ez1, h1)):
        got = got.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
    np.testing.assert_allclose(s_dev.item(), src, rtol=1e-9, atol=1e-12 * abs(src))


# ------------------------------------------------------------------ a1
def test_load_parity():
    M = P()
    cfg = M.small_reactor(np_init=20000)
    pic = M.Pic(cfg, device=DEV)
    pic.load_particles()
    g = O.Grid(cfg["nr"], cfg["nz"], cfg["R"], cfg["L"])
    e, i = O.load(g, 20000, cfg["n0"], cfg["te_ev"], cfg["ti_ev"], cfg["seed"])
    for s, ref in enumerate((e, i)):
        got = by_id(pic.get_state(s))
        ref = by_id(ref)
        for k in ("cell", "a", "b", "w", "id"):
            np.testing.assert_array_equal(got[k], ref[k])
        for k in ("vr", "vt", "vz"):  # device log/cos/sin vs libm: a few ulp
            np.testing.assert_allclose(got[k], ref[k], rtol=1e-13, atol=1e-13 * np.max(np.abs(ref[k])))
        # sorted by cell
        assert np.all(np.diff(pic.get_state(s)["cell"]) >= 0)


# ------------------------------------------------------------------ a7
def test_mcc_parity():
    M = P()
    nr, nz = 16, 24
    cfg = M.small_reactor(nr=nr, nz=nz, np_init=30000, capacity_factor=1.5, gas_pressure=20.0)
    pic = M.Pic(cfg, device=DEV)
    g = O.Grid(nr, nz, cfg["R"], cfg["L"])
    e, i = O.load(g, 30000, 1e15, 20.0, 0.5, 9)  # hot electrons: all processes occur
    pic.set_state([e, i])
    ng = 20.0 / (O.KB * 300)
    numax = O.numax_e(ng)
    vthg = np.sqrt(O.KB * 300.0 / M_AR)
    gmax = np.sqrt(2.0 * QE * 1000.0 / M_AR) + 5.0 * vthg
    pe = -np.expm1(-numax * cfg["dt"])
    pi = -np.expm1(-(ng * 5e-19 * gmax) * cfg["dt"])
    # the library derives the same constants on its own
    np.testing.assert_allclose(pic.mcc_constants(), (numax, gmax, pe, pi), rtol=1e-14)
    step = 123
    rc, counts, de = pic.mcc(step)
    assert rc == 0
    cap = int(30000 * 1.5)
    eo, io = O.empty_species(cap), O.empty_species(cap)
    for k in O.FIELDS:
        eo[k][:30000] = e[k]
        io[k][:30000] = i[k]
    rco, ne, ni, nid, co, deo = O.mcc(cfg["seed"], step, ng, 300.0, numax, pe,
                                      pi, gmax, eo, 30000, 30000, io, (30000, 30000))
    assert rco == 0
    assert counts[:7] == list(co[:7])
    assert counts[3] > 10 and counts[5] > 0
    for s, (ref, n) in enumerate(((eo, ne), (io, ni))):
        got = by_id(pic.get_state(s))
        r = by_id({k: v[:n] for k, v in ref.items()})
        assert len(got["id"]) == n
        assert_state_close(got, r, rtol=1e-12, what="mcc species %d " % s)
    np.testing.assert_allclose(de, deo, rtol=1e-10)


# ------------------------------------------------------------------ a8
def test_sort_parity():
    nr, nz, n = 16, 24, 50000
    rng = np.random.default_rng(11)
    e = inputs.particles(nr, nz, n, 12, 1e5, sorted_=False)
    e["cell"][rng.random(n) < 0.05] = -1
    i = inputs.particles(nr, nz, n, 13, 1e3, sorted_=False)
    pic = make_pic(nr, nz, 0.05, 0.03, 1e-9, n)
    pic.set_state([e, i])
    pic.sort()
    g = O.Grid(nr, nz, 0.05, 0.03)
    for s, sp in enumerate((e, i)):
        ref = {k: v.copy() for k, v in sp.items()}
        m = O.sort(g, ref, n)
        got = pic.get_state(s)
        assert len(got["cell"]) == m
        assert np.all(np.diff(got["cell"]) >= 0)
        # within a cell the GPU order is not defined: compare ordered by (cell, id)
        og = np.lexsort((got["id"], got["cell"]))
        oo = np.lexsort((ref["id"][:m], ref["cell"][:m]))
        for k in O.FIELDS:
            np.testing.assert_array_equal(got[k][og], ref[k][:m][oo])


# -------------------------------------------------------- whole step (a2-a8)
def _pair_state(nr, nz, R, L, n, te, seed):
    g = O.Grid(nr, nz, R, L)
    return g, O.load(g, n, 1e15, te, 0.026, seed)


@pytest.mark.parametrize("mcc", [0, 1])
def test_full_step_parity(mcc):
    M = P()
    nr, nz, n = 32, 64, 40000
    cfg = M.small_reactor(np_init=n, capacity_factor=1.5, mcc_on=mcc, picard_tol=1e-10,
                          volt=300.0, gas_pressure=5.0)
    g, (e, i) = _pair_state(nr, nz, cfg["R"], cfg["L"], n, 8.0, 21)
    pic = M.Pic(cfg, device=DEV)
    pic.set_state([e, i])
    sim = O.Sim(g, cfg["dt"], freq=cfg["freq"], volt=cfg["volt"], tol=cfg["picard_tol"],
                kmax=cfg["picard_max"], mcc_on=bool(mcc), ng=cfg["gas_pressure"] / (O.KB * 300),
                seed=cfg["seed"], species=[e, i], cap=int(n * 1.5))
    if mcc:  # each side derives its MCC constants itself
        c = sim.cfg
        np.testing.assert_allclose(pic.mcc_constants(), (c.numax_e, c.gmax, c.pnull_e, c.pnull_i),
                                   rtol=1e-14)
    for step in range(3):
        rc, st = pic.step(1)
        rco, sto = sim.step()
        assert rc == 0 and rco == 0
        # same number of Picard iterations, so the comparison is at roundoff level
        assert st["picard_iters"] == sto.picard_iters
        er, ez, h = pic.fields()
        for got, ref in ((er, sim.er), (ez, sim.ez), (h, sim.h)):
            assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))
        for s in range(2):
            got = by_id(pic.get_state(s))
            ref = by_id(sim.state(s))
            assert len(got["id"]) == len(ref["id"])
            assert_state_close(got, ref, rtol=1e-11, what="step %d species %d " % (step, s),
                               nz=nz)
        assert st["absorbed"] == sto.counters[1]
        if mcc:
            assert st["mcc"][:7] == list(sto.mcc[:7])


def test_gauss_and_energy_on_gpu_over_steps():
    """Properties at any size: Gauss residual constant (charge conservation)
    and the energy balance to the Picard tolerance, on the GPU alone."""
    M = P()
    cfg = M.small_reactor(np_init=40000, volt=0.0, mcc_on=0, picard_tol=1e-10)
    pic = M.Pic(cfg, device=DEV)
    pic.load_particles()
    g = O.Grid(cfg["nr"], cfg["nz"], cfg["R"], cfg["L"])

    def gauss():
        er, ez, _ = pic.fields()
        return O.gauss_residual(g, er, ez, pic.node_charge().cpu().numpy())

    G0 = gauss()
    # pair loading: net node charge ~0; the scale is one species' node charge
    qs = np.max(np.abs(O.node_charge(g, -QE, pic.get_state(0))))
    d0 = pic.diag()
    W0 = sum(d0["kinetic"]) + d0["field"]
    lost = 0.0
    for _ in range(5):
        _, st = pic.step(1)
        lost += st["ke_lost"]
    d1 = pic.diag()
    W1 = sum(d1["kinetic"]) + d1["field"]
    assert np.max(np.abs(gauss() - G0)) <= 1e-11 * qs
    assert abs(W1 + lost - W0) <= 5 * 5e-10 * W0


# ------------------------------------------ full size (256 x 384, 16M/species)
def test_full_size_push_sampled_parity_and_continuity():
    """The bench configuration: the whole store is pushed on the GPU; the
    oracle recomputes a random sample of particles one by one, and node-wise
    charge continuity is checked for the whole store on the GPU."""
    M = P()
    cfg = M.large_reactor()
    pic = M.Pic(cfg, device=DEV)
    pic.load_particles()
    nr, nz = cfg["nr"], cfg["nz"]
    g = O.Grid(nr, nz, cfg["R"], cfg["L"])
    er, ez = inputs.smooth_fields(nr, nz, 31, 2e4)
    v = pic.view()
    rng = np.random.default_rng(5)
    samples = []
    for s in range(2):
        n = v["n"][s]
        idx = np.sort(rng.choice(n, size=3000, replace=False))
        it = torch.from_numpy(idx).to(DEV)
        sp = {k: v["species"][s][k][:n][it].cpu().numpy() for k in O.FIELDS}
        sp["id"] = sp["id"].view(np.uint32)
        samples.append((idx, sp))
    q0 = pic.node_charge()
    ir = torch.zeros(g.n_er, dtype=torch.float64, device=DEV)
    iz = torch.zeros(g.n_ez, dtype=torch.float64, device=DEV)
    pic.push_deposit(tgpu(er), tgpu(ez), ir, iz, write=True)
    q1 = pic.node_charge()  # absorbed particles excluded: their charge is at wall nodes
    v = pic.view()
    for s, (idx, sp) in enumerate(samples):
        q, m = (-QE, ME) if s == 0 else (QE, M_AR)
        ref = {k: x.copy() for k, x in sp.items()}
        O.push(g, cfg["dt"], q, m, ref, er, ez, write=True)
        it = torch.from_numpy(idx).to(DEV)
        got = {k: v["species"][s][k][it].cpu().numpy() for k in O.FIELDS}
        got["id"] = got["id"].view(np.uint32)
        assert_state_close(got, ref, rtol=1e-12, what="full-size species %d " % s)
    # continuity at interior nodes (wall nodes also receive absorbed charge)
    IR = ir.view(nr, nz + 1)
    IZ = iz.view(nr + 1, nz)
    D = torch.zeros(nr + 1, nz + 1, dtype=torch.float64, device=DEV)
    D[:-1, :] += IR
    D[1:, :] -= IR
    D[:, :-1] += IZ
    D[:, 1:] -= IZ
    res = (q1 - q0).view(nr + 1, nz + 1) + D
    # pair loading: the net node charge is ~0, so the scale is the crossed charge
    scale = max(torch.max(torch.abs(ir)).item(), torch.max(torch.abs(iz)).item())
    assert scale > 0
    assert torch.max(torch.abs(res[:-1, 1:-1])).item() <= 1e-12 * scale
