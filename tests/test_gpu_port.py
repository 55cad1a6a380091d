"""Wave port on r = R (PIC_FEED_WAVE) on the GPU against the FP64 oracle:
the field solve and whole steps with particles."""
import numpy as np
import pytest

import oracle as O
from tests.test_gpu_parity import assert_state_close, by_id

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


def tgpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


@pytest.mark.parametrize("nr,nz,xa", [(32, 64, 0), (24, 48, 3)])
def test_field_solve_parity(nr, nz, xa):
    M = P()
    R, L, dt = 0.1, 0.03, 1.0 / (200 * 60e6)
    g = O.Grid(nr, nz, R, L, xa=xa)
    rng = np.random.default_rng(nr + xa)
    er0 = rng.normal(size=g.n_er) * 100
    er0.reshape(nr, nz + 1)[:, [0, -1]] = 0.0
    ez0 = rng.normal(size=g.n_ez) * 100
    h0 = rng.normal(size=g.n_h) * 0.1
    ir = rng.normal(size=g.n_er) * 1e-12
    iz = rng.normal(size=g.n_ez) * 1e-12
    v0, v1 = 37.0, -12.0
    er1, ez1, h1, src = O.FieldSolver(g, dt, wave=True).solve(er0, ez0, h0, ir, iz, v0, v1)
    cfg = M.small_reactor(nr=nr, nz=nz, R=R, L=L, dt=dt, np_init=16, feed=M.PIC_FEED_WAVE,
                          axis_cells=xa)
    pic = M.Pic(cfg, device=DEV)
    out = [torch.empty(k, dtype=torch.float64, device=DEV) for k in (g.n_er, g.n_ez, g.n_h)]
    s_dev = torch.zeros(1, dtype=torch.float64, device=DEV)
    pic.field_solve(tgpu(er0), tgpu(ez0), tgpu(h0), tgpu(ir), tgpu(iz), v0, v1, *out, src=s_dev)
    torch.cuda.synchronize()
    for got, ref in zip(out, (er1, ez1, h1)):
        assert np.max(np.abs(got.cpu().numpy() - ref)) <= 1e-10 * np.max(np.abs(ref))
    np.testing.assert_allclose(s_dev.item(), src, rtol=1e-9)


def test_step_parity():
    M = P()
    n = 30000
    cfg = M.small_reactor(np_init=n, capacity_factor=1.5, mcc_on=0, picard_tol=1e-10,
                          volt=300.0, feed=M.PIC_FEED_WAVE)
    g = O.Grid(cfg["nr"], cfg["nz"], cfg["R"], cfg["L"])
    e, i = O.load(g, n, 1e15, 8.0, 0.026, 21)
    pic = M.Pic(cfg, device=DEV)
    pic.set_state([e, i])
    sim = O.Sim(g, cfg["dt"], freq=cfg["freq"], volt=cfg["volt"], tol=1e-10,
                kmax=cfg["picard_max"], species=[e, i], cap=int(1.5 * n), wave=True)
    for step in range(3):
        rc, st = pic.step(1)
        rco, sto = sim.step()
        assert rc == 0 and rco == 0 and st["picard_iters"] == sto.picard_iters
        er, ez, h = pic.fields()
        for got, ref in ((er, sim.er), (ez, sim.ez), (h, sim.h)):
            assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref)), step
        np.testing.assert_allclose(st["src_energy"], sto.src_energy, rtol=1e-8)
        for s in range(2):
            assert_state_close(by_id(pic.get_state(s)), by_id(sim.state(s)), rtol=1e-10,
                               what="step %d species %d " % (step, s), nz=cfg["nz"])
