"""Edge cases of the hot path on the GPU against the oracle: species with no
particles or a single one, a store whose particles have all been absorbed,
and whole steps of an empty reactor (the field solve alone), in both forms.
The kernels' launch guards, the queue with nothing in it and the sort of an
empty store must give what the oracle gives."""
import numpy as np
import pytest

import oracle as O
from tests import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
QE, ME, M_AR = O.QE, O.ME, O.M_AR


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as G
    G.build()


def P():
    import paper_2212_08836_gb300 as M
    return M


def make(nr, nz, cap, precision=0, **kw):
    M = P()
    cfg = M.small_reactor(nr=nr, nz=nz, R=0.05, L=0.03, dt=1e-9, np_init=cap,
                          capacity_factor=1.0, mcc_on=0, precision=precision, **kw)
    return M.Pic(cfg, device=DEV), cfg


def empty_species():
    return {k: np.zeros(0, dtype=np.int32 if k == "cell" else
                        (np.uint32 if k == "id" else np.float64)) for k in O.FIELDS}


@pytest.mark.parametrize("precision", [0, 1])
def test_single_electron_and_no_ions(precision):
    """One electron crossing a face and an empty ion species: the same crossed
    charge and new state as the oracle's push (FP64 to 1e-12, FP32 particles
    to 1e-5)."""
    nr, nz = 8, 12
    g = O.Grid(nr, nz, 0.05, 0.03)
    e = inputs.particles(nr, nz, 1, 3, 8e5)
    e["b"][:] = 0.97  # close to the upper z-face: the step crosses it
    e["vz"][:] = 2e6
    i = empty_species()
    er, ez = inputs.smooth_fields(nr, nz, 5, 3e2)
    pic, _ = make(nr, nz, 4, precision)
    pic.set_state([e, i])
    ir = torch.zeros(g.n_er, dtype=torch.float64, device=DEV)
    iz = torch.zeros(g.n_ez, dtype=torch.float64, device=DEV)
    pic.push_deposit(torch.tensor(er, device=DEV), torch.tensor(ez, device=DEV), ir, iz,
                     write=True)
    s = {k: v.copy() for k, v in e.items()}
    if precision == 1:  # the oracle starts from the FP32-rounded state
        for k in ("a", "b", "vr", "vt", "vz", "w"):
            s[k] = s[k].astype(np.float32).astype(np.float64)
    ir_o, iz_o = np.zeros(g.n_er), np.zeros(g.n_ez)
    O.push(g, 1e-9, -QE, ME, s, er, ez, write=True, ir=ir_o, iz=iz_o)
    tol = 1e-12 if precision == 0 else 1e-5
    scale = max(np.max(np.abs(ir_o)), np.max(np.abs(iz_o)))
    assert scale > 0
    assert np.max(np.abs(ir.cpu().numpy() - ir_o)) <= tol * scale
    assert np.max(np.abs(iz.cpu().numpy() - iz_o)) <= tol * scale
    got = pic.get_state(0)
    assert got["cell"][0] == s["cell"][0] and s["cell"][0] != e["cell"][0]
    for k in ("a", "b"):
        assert abs(got[k][0] - s[k][0]) <= tol
    assert len(pic.get_state(1)["cell"]) == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_empty_reactor_steps_follow_the_oracle(precision):
    """No particles at all: each step is the field solve driven by V(t); the
    same fields as the oracle's whole steps with no species."""
    M = P()
    nr, nz = 16, 24
    pic, cfg = make(nr, nz, 0, precision, volt=80.0, picard_tol=1e-12)
    pic.load_particles()
    g = O.Grid(nr, nz, cfg["R"], cfg["L"])
    sim = O.Sim(g, cfg["dt"], freq=cfg["freq"], volt=cfg["volt"], tol=1e-12,
                kmax=cfg["picard_max"], species=[])
    for k in range(3):
        rc, st = pic.step(1)
        rco, sto = sim.step()
        assert rc == 0 and rco == 0
        assert st["pushes"] == 0
    er, ez, h = pic.fields()
    # (E_r is rounding noise in both: the driven vacuum field is axial, so the
    # bound is taken on the whole electric field)
    se = max(np.max(np.abs(sim.er)), np.max(np.abs(sim.ez)))
    for a, b, sc in ((er, sim.er, se), (ez, sim.ez, se), (h, sim.h, np.max(np.abs(sim.h)))):
        assert np.max(np.abs(a - b)) <= 1e-10 * sc
    assert list(pic.view()["n"]) == [0, 0]


@pytest.mark.parametrize("precision", [0, 1])
def test_store_with_every_particle_absorbed(precision):
    """A store whose particles all carry cell -1 (absorbed): the sort leaves
    it empty and the next step pushes nothing."""
    nr, nz, n = 8, 12, 500
    e = inputs.particles(nr, nz, n, 7, 1e5)
    i = inputs.particles(nr, nz, n, 8, 1e3)
    e["cell"][:] = -1
    i["cell"][:] = -1
    pic, _ = make(nr, nz, n, precision)
    pic.set_state([e, i])
    pic.sort()
    assert list(pic.view()["n"]) == [0, 0]
    rc, st = pic.step(1)
    assert rc == 0 and st["pushes"] == 0 and st["absorbed"] == 0
