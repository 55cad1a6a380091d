"""Electrostatic field model (Eq. 8) on the GPU against the FP64 oracle
(oracle/es.py), and the limit of the electromagnetic model as the speed of
light grows (mu -> 0), where its fields must approach the electrostatic ones
with a difference of order mu (1/c^2), the paper's third verification test."""
import numpy as np
import pytest

import oracle as O
from tests.drive import drive_voltage
from oracle import es as ES

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


def rel(a, b):
    return float(np.max(np.abs(np.ravel(a) - np.ravel(b))) / max(np.max(np.abs(np.ravel(b))), 1e-300))


@pytest.mark.parametrize("nr,nz", [(8, 12), (32, 64), (37, 50)])
def test_es_solve_matches_oracle(nr, nz):
    M = P()
    cfg = M.small_reactor(nr=nr, nz=nz, np_init=100, field_model=M.PIC_FIELD_ES)
    pic = M.Pic(cfg, device=DEV)
    rng = np.random.default_rng(nr + nz)
    Q = rng.normal(size=(nr + 1) * (nz + 1)) * 1e-13
    er = torch.zeros(nr * (nz + 1), dtype=torch.float64, device=DEV)
    ez = torch.zeros((nr + 1) * nz, dtype=torch.float64, device=DEV)
    pic.es_solve(torch.tensor(Q, device=DEV), 57.0, er, ez)
    torch.cuda.synchronize()
    _, ero, ezo = ES.solve(nr, nz, cfg["R"] / nr, cfg["L"] / nz, Q, 57.0)
    scale = max(np.max(np.abs(ero)), np.max(np.abs(ezo)))
    assert np.max(np.abs(er.cpu().numpy() - ero)) <= 1e-10 * scale
    assert np.max(np.abs(ez.cpu().numpy() - ezo)) <= 1e-10 * scale


@pytest.mark.parametrize("nr,nz,ip,xa", [(8, 12, 5, 0), (32, 64, 20, 0), (37, 50, 30, 0),
                                          (32, 64, 20, 3)],
                         ids=["small", "fft", "dense", "mapped"])
def test_es_port_solve_matches_oracle(nr, nz, ip, xa):
    """The electrostatic model's axial port (Sec. 2.2): the electrode disc, the
    port's opening at the coaxial line's potential and the grounded side wall
    as Dirichlet values of the same solve (three transform paths)."""
    M = P()
    cfg = M.small_reactor(nr=nr, nz=nz, np_init=100, field_model=M.PIC_FIELD_ES,
                          feed=M.PIC_FEED_AXIAL, port_rin=ip, port_cells=4, port_len=0.02,
                          eps_port=3.8, axis_cells=xa)
    pic = M.Pic(cfg, device=DEV)
    rng = np.random.default_rng(nr + nz + ip)
    Q = rng.normal(size=(nr + 1) * (nz + 1)) * 1e-13
    er = torch.zeros(nr * (nz + 1), dtype=torch.float64, device=DEV)
    ez = torch.zeros((nr + 1) * nz, dtype=torch.float64, device=DEV)
    pic.es_solve(torch.tensor(Q, device=DEV), -41.0, er, ez)
    torch.cuda.synchronize()
    _, ero, ezo = ES.solve(nr, nz, cfg["R"] / (nr + xa), cfg["L"] / nz, Q, -41.0, xa=xa,
                           port=ip)
    scale = max(np.max(np.abs(ero)), np.max(np.abs(ezo)))
    assert np.max(np.abs(er.cpu().numpy() - ero)) <= 1e-10 * scale
    assert np.max(np.abs(ez.cpu().numpy() - ezo)) <= 1e-10 * scale


@pytest.mark.parametrize("precision", [0, 1])
def test_es_steps_solve_gauss_with_the_moved_charge(precision):
    """Each step's field is the oracle's electrostatic solution for the node
    charge of the particles after the step (continuity inside the passes)."""
    M = P()
    cfg = M.small_reactor(np_init=20000, mcc_on=1, volt=150.0, field_model=M.PIC_FIELD_ES,
                          precision=precision)
    pic = M.Pic(cfg, device=DEV)
    pic.load_particles()
    nr, nz = cfg["nr"], cfg["nz"]
    for k in range(4):
        rc, st = pic.step(1)
        assert rc == 0 and st["converged"] == 1
        Q = pic.node_charge().cpu().numpy()
        er, ez, h = pic.fields()
        assert np.all(h == 0.0)
        v1 = drive_voltage(cfg, k + 1)
        _, ero, ezo = ES.solve(nr, nz, cfg["R"] / nr, cfg["L"] / nz, Q, v1)
        tol = 1e-9 if precision == 0 else 1e-5
        assert rel(er, ero) <= tol and rel(ez, ezo) <= tol, k


def test_em_fields_approach_es_fields_as_c_grows():
    M = P()
    errs = []
    for s in (1e-2, 1e-4, 1e-6):
        cfg = M.small_reactor(np_init=20000, mcc_on=0, volt=100.0, mu=O.MU0 * s, seed=2)
        pic = M.Pic(cfg, device=DEV)
        pic.load_particles()
        for _ in range(3):
            rc, st = pic.step(1)
            assert rc == 0
        Q = pic.node_charge().cpu().numpy()
        er, ez, _ = pic.fields()
        v1 = drive_voltage(cfg, 3)
        nr, nz = cfg["nr"], cfg["nz"]
        _, ero, ezo = ES.solve(nr, nz, cfg["R"] / nr, cfg["L"] / nz, Q, v1)
        errs.append(max(rel(er, np.concatenate([ero])), rel(ez, ezo)))
    # difference of order mu (1/c^2): each hundredfold smaller mu brings the fields
    # more than twentyfold closer
    assert errs[1] < 0.05 * errs[0] and errs[2] < 0.05 * errs[1], errs
    assert errs[2] < 1e-5, errs
