"""Row a9 on the GPU: the device Gauss residual against the oracle's discrete
divergence (same fields, same charges), and its conservation over steps of
both forms (charge-conserving deposit: the residual of the pair-loaded start,
zero, stays at rounding level)."""
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


@pytest.mark.parametrize("xa", [0, 3])
def test_gauss_residual_matches_oracle(xa):
    M = P()
    cfg = M.small_reactor(np_init=20000, mcc_on=0, axis_cells=xa)
    pic = M.Pic(cfg, device=DEV)
    g = O.Grid(cfg["nr"], cfg["nz"], cfg["R"], cfg["L"], xa=xa)
    e, i = O.load(g, 20000, 1e15, 3.0, 0.026, 4)
    rng = np.random.default_rng(1)
    e["b"] = rng.random(len(e["b"]))  # separate the pairs: a charged state
    er = rng.normal(size=g.n_er) * 50
    ez = rng.normal(size=g.n_ez) * 50
    pic.set_state([e, i], er=er, ez=ez)
    got = pic.gauss_residual().cpu().numpy()
    Q = O.node_charge(g, -O.QE, e)
    O.node_charge(g, O.QE, i, Q)
    ref = O.gauss_residual(g, er, ez, Q)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("precision", [0, 1])
def test_gauss_residual_stays_at_rounding_over_steps(precision):
    M = P()
    cfg = M.small_reactor(np_init=40000, volt=200.0, precision=precision,
                          picard_tol=1e-8 if precision == 0 else 1e-5)
    pic = M.Pic(cfg, device=DEV)
    pic.load_particles()
    q_scale = O.QE * float(np.max(pic.get_state(0)["w"])) * 20  # ~ charge of a cell's electrons
    for _ in range(5):
        pic.step(1)
    r = np.max(np.abs(pic.gauss_residual().cpu().numpy()))
    assert r <= (1e-12 if precision == 0 else 1e-6) * q_scale, r
