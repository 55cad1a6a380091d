"""Conducting ring (ring_cells, eps_ring, sigma_ring: Eq. 2's sigma E in the
outer cells) on the GPU against the FP64 oracle: field solve, whole steps with
particles sticking at the ring face (with and without the blocking
capacitor), the conduction charge tally, Gauss's law with it, the
checkpoint, and the configurations the library refuses."""
import numpy as np
import pytest

import oracle as O
from tests.test_gpu_parity import assert_state_close, by_id

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
ND, ERD = 3, 2.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as G
    G.build()


def P():
    import paper_2212_08836_gb300 as M
    return M


def tgpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


@pytest.mark.parametrize("xa,wave,sgd", [(0, 0, 5.0), (3, 1, 0.4), (0, 0, 1e7)])
def test_field_solve_parity(xa, wave, sgd):
    M = P()
    nr, nz, R, L, dt = 24, 48, 0.1, 0.03, 1.0 / (200 * 60e6)
    g = O.Grid(nr, nz, R, L, xa=xa, nd=ND, erd=ERD, sgd=sgd)
    rng = np.random.default_rng(17 + xa)
    er0 = rng.normal(size=g.n_er) * 100
    er0.reshape(nr, nz + 1)[:, [0, -1]] = 0.0
    ez0 = rng.normal(size=g.n_ez) * 100
    h0 = rng.normal(size=g.n_h) * 0.1
    ir = rng.normal(size=g.n_er) * 1e-12
    iz = rng.normal(size=g.n_ez) * 1e-12
    v0, v1 = 37.0, -12.0
    er1, ez1, h1, src = O.FieldSolver(g, dt, wave=bool(wave)).solve(er0, ez0, h0, ir, iz, v0, v1)
    cfg = M.small_reactor(nr=nr, nz=nz, R=R, L=L, dt=dt, np_init=16, axis_cells=xa,
                          ring_cells=ND, eps_ring=ERD, sigma_ring=sgd, feed=wave)
    pic = M.Pic(cfg, device=DEV)
    out = [torch.empty(k, dtype=torch.float64, device=DEV) for k in (g.n_er, g.n_ez, g.n_h)]
    s_dev = torch.zeros(1, dtype=torch.float64, device=DEV)
    pic.field_solve(tgpu(er0), tgpu(ez0), tgpu(h0), tgpu(ir), tgpu(iz), v0, v1, *out, src=s_dev)
    torch.cuda.synchronize()
    for got, ref in zip(out, (er1, ez1, h1)):
        assert np.max(np.abs(got.cpu().numpy() - ref)) <= 1e-10 * np.max(np.abs(ref))
    np.testing.assert_allclose(s_dev.item(), src, rtol=1e-9)


@pytest.mark.parametrize("xa,cblock", [(0, 0.0), (2, 0.0), (0, 2e-10)])
def test_step_parity_with_conduction_and_sticking(xa, cblock):
    M = P()
    n, sgd = 30000, 0.05
    cfg = M.small_reactor(np_init=n, capacity_factor=1.5, mcc_on=0, picard_tol=1e-10,
                          volt=300.0, ring_cells=ND, eps_ring=ERD, sigma_ring=sgd,
                          axis_cells=xa, cblock=cblock)
    g = O.Grid(cfg["nr"], cfg["nz"], cfg["R"], cfg["L"], xa=xa, nd=ND, erd=ERD, sgd=sgd)
    e, i = O.load(g, n, 1e15, 20.0, 0.026, 23)  # hot electrons: many reach the ring face
    pic = M.Pic(cfg, device=DEV)
    pic.set_state([e, i])
    sim = O.Sim(g, cfg["dt"], freq=cfg["freq"], volt=cfg["volt"], tol=1e-10,
                kmax=cfg["picard_max"], species=[e, i], cap=int(1.5 * n), cblock=cblock)
    for step in range(3):
        rc, st = pic.step(1)
        rco, sto = sim.step()
        assert rc == 0 and rco == 0
        assert st["picard_iters"] == sto.picard_iters
        er, ez, _ = pic.fields()
        for got, ref in ((er, sim.er), (ez, sim.ez)):
            assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref)), step
        for s in range(2):
            assert_state_close(by_id(pic.get_state(s)), by_id(sim.state(s)), rtol=1e-10,
                               what="step %d species %d " % (step, s), nz=cfg["nz"])
        if cblock > 0:
            np.testing.assert_allclose(pic.circuit(), sim.circ, rtol=1e-9)
    qc = pic.view()["qcond"].cpu().numpy()
    assert np.max(np.abs(sim.qcond)) > 0
    assert np.max(np.abs(qc - sim.qcond)) <= 1e-9 * np.max(np.abs(sim.qcond))
    assert np.sum(np.abs(pic.wall_charge()[0]["r"])) > 0  # electrons stuck at the ring face
    r = pic.gauss_residual().cpu().numpy()
    Q = pic.node_charge().cpu().numpy()
    assert np.max(np.abs(r)) <= 1e-9 * max(np.max(np.abs(Q)), np.max(np.abs(qc)))


def test_checkpoint_keeps_the_conduction_tally(tmp_path):
    M = P()
    cfg = M.small_reactor(np_init=8000, mcc_on=0, volt=200.0, ring_cells=ND, eps_ring=ERD,
                          sigma_ring=0.2)
    a = M.Pic(cfg, device=DEV)
    a.load_particles()
    for _ in range(3):
        assert a.step(1)[0] == 0
    path = str(tmp_path / "ck.bin")
    a.save(path)
    b = M.Pic(cfg, device=DEV)
    b.load(path)
    qa = a.view()["qcond"].cpu().numpy()
    assert np.max(np.abs(qa)) > 0
    np.testing.assert_array_equal(b.view()["qcond"].cpu().numpy(), qa)
    for _ in range(2):
        assert a.step(1)[0] == 0 and b.step(1)[0] == 0
    # continued runs agree up to the order of the deposit's atomic additions
    qa, qb = a.view()["qcond"].cpu().numpy(), b.view()["qcond"].cpu().numpy()
    assert np.max(np.abs(qb - qa)) <= 1e-12 * np.max(np.abs(qa))
    # a context without the conducting ring, or with another ring, refuses it
    for other in (dict(sigma_ring=0.0), dict(ring_cells=ND + 1)):
        c = M.Pic(dict(cfg, **other), device=DEV)
        with pytest.raises(M.PicError) as e:
            c.load(path)
        assert e.value.code == M.PIC_E_STATE


@pytest.mark.parametrize("kw", [dict(sigma_ring=1.0),                                   # no ring
                                dict(ring_cells=ND, sigma_ring=1.0, field_model=1),      # ES
                                dict(ring_cells=ND, sigma_ring=-1.0),
                                dict(ring_cells=ND, sigma_ring=float("inf"))])
def test_refused_configurations(kw):
    M = P()
    cfg = M.small_reactor(np_init=16, eps_ring=ERD, **kw)
    with pytest.raises(M.PicError) as e:
        M.Pic(cfg, device=DEV)
    assert e.value.code == M.PIC_E_CONFIG
