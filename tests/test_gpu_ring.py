"""Dielectric ring (ring_cells, eps_ring) on the GPU against the FP64 oracle:
field solve, loading, whole steps of both field models (particles sticking
at the ring face), and the Gauss residual with the permittivity-weighted
faces."""
import numpy as np
import pytest

import oracle as O
from oracle import es as ES
from tests.test_gpu_parity import assert_state_close, by_id

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
ND, ERD = 3, 3.8


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as G
    G.build()


def P():
    import paper_2212_08836_gb300 as M
    return M


def tgpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


@pytest.mark.parametrize("xa,wave", [(0, 0), (3, 1)])
def test_field_solve_parity(xa, wave):
    M = P()
    nr, nz, R, L, dt = 24, 48, 0.1, 0.03, 1.0 / (200 * 60e6)
    g = O.Grid(nr, nz, R, L, xa=xa, nd=ND, erd=ERD)
    rng = np.random.default_rng(7 + xa)
    er0 = rng.normal(size=g.n_er) * 100
    er0.reshape(nr, nz + 1)[:, [0, -1]] = 0.0
    ez0 = rng.normal(size=g.n_ez) * 100
    h0 = rng.normal(size=g.n_h) * 0.1
    ir = rng.normal(size=g.n_er) * 1e-12
    iz = rng.normal(size=g.n_ez) * 1e-12
    v0, v1 = 37.0, -12.0
    er1, ez1, h1, src = O.FieldSolver(g, dt, wave=bool(wave)).solve(er0, ez0, h0, ir, iz, v0, v1)
    cfg = M.small_reactor(nr=nr, nz=nz, R=R, L=L, dt=dt, np_init=16, axis_cells=xa,
                          ring_cells=ND, eps_ring=ERD, feed=wave)
    pic = M.Pic(cfg, device=DEV)
    out = [torch.empty(k, dtype=torch.float64, device=DEV) for k in (g.n_er, g.n_ez, g.n_h)]
    s_dev = torch.zeros(1, dtype=torch.float64, device=DEV)
    pic.field_solve(tgpu(er0), tgpu(ez0), tgpu(h0), tgpu(ir), tgpu(iz), v0, v1, *out, src=s_dev)
    torch.cuda.synchronize()
    for got, ref in zip(out, (er1, ez1, h1)):
        assert np.max(np.abs(got.cpu().numpy() - ref)) <= 1e-10 * np.max(np.abs(ref))
    np.testing.assert_allclose(s_dev.item(), src, rtol=1e-9)


def test_load_parity():
    M = P()
    cfg = M.small_reactor(np_init=20000, ring_cells=ND, eps_ring=ERD)
    pic = M.Pic(cfg, device=DEV)
    pic.load_particles()
    g = O.Grid(cfg["nr"], cfg["nz"], cfg["R"], cfg["L"], nd=ND, erd=ERD)
    e, i = O.load(g, 20000, cfg["n0"], cfg["te_ev"], cfg["ti_ev"], cfg["seed"])
    for s, ref in enumerate((e, i)):
        got, ref = by_id(pic.get_state(s)), by_id(ref)
        for k in ("cell", "a", "b", "id"):
            np.testing.assert_array_equal(got[k], ref[k])
        np.testing.assert_allclose(got["w"], ref["w"], rtol=1e-14)


@pytest.mark.parametrize("field_model", [0, 1])
def test_step_parity_with_sticking(field_model):
    M = P()
    n = 30000
    cfg = M.small_reactor(np_init=n, capacity_factor=1.5, mcc_on=0, picard_tol=1e-10,
                          volt=300.0, ring_cells=ND, eps_ring=ERD, field_model=field_model)
    g = O.Grid(cfg["nr"], cfg["nz"], cfg["R"], cfg["L"], nd=ND, erd=ERD)
    e, i = O.load(g, n, 1e15, 20.0, 0.026, 21)  # hot electrons: many reach the ring face
    pic = M.Pic(cfg, device=DEV)
    pic.set_state([e, i])
    if field_model == 1:
        sim = ES.Sim(g, cfg["dt"], freq=cfg["freq"], volt=cfg["volt"], tol=1e-10,
                     species=[e, i], cap=int(1.5 * n))
    else:
        sim = O.Sim(g, cfg["dt"], freq=cfg["freq"], volt=cfg["volt"], tol=1e-10,
                    kmax=cfg["picard_max"], species=[e, i], cap=int(1.5 * n))
    for step in range(3):
        rc, st = pic.step(1)
        rco, sto = sim.step()
        assert rc == 0 and rco == 0
        its = sto["picard_iters"] if isinstance(sto, dict) else sto.picard_iters
        assert st["picard_iters"] == its
        er, ez, _ = pic.fields()
        for got, ref in ((er, sim.er), (ez, sim.ez)):
            assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref)), step
        for s in range(2):
            assert_state_close(by_id(pic.get_state(s)), by_id(sim.state(s)), rtol=1e-10,
                               what="step %d species %d " % (step, s), nz=cfg["nz"])
    wall = pic.wall_charge()[0]["r"]
    assert np.sum(np.abs(wall)) > 0  # electrons stuck at the ring face
    r = pic.gauss_residual().cpu().numpy()
    Q = pic.node_charge().cpu().numpy()
    assert np.max(np.abs(r)) <= 1e-9 * np.max(np.abs(Q)) + 1e-30
