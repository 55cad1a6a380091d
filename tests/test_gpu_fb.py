"""Fourier-Bessel sampling (App. A, Eq. A2), the multi-harmonic generator
waveform and fixed ions (the ingredients of the dispersion test of Sec. 3.1)
on the GPU against the oracle (oracle/fb.py, oracle/es.py)."""
import numpy as np
import pytest

import oracle as O
from oracle import es as ES
from oracle import fb as FB
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


@pytest.mark.parametrize("alpha,row", [(0, 2), (0, 31), (1, 5), (1, 64)])
def test_fourier_bessel_matches_oracle(alpha, row):
    M = P()
    cfg = M.small_reactor(np_init=20000, mcc_on=0, volt=150.0)
    pic = M.Pic(cfg, device=DEV)
    pic.load_particles()
    pic.step(3)
    er, ez, _ = pic.fields()
    nr, nz = cfg["nr"], cfg["nz"]
    f = ez.reshape(nr + 1, nz)[:, row] if alpha == 0 else er.reshape(nr, nz + 1)[:, row]
    ref = FB.coefficients(f, nr, cfg["R"], alpha, 24)
    got = pic.fourier_bessel(alpha, row, 24).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_single_harmonic_drive_equals_the_configured_sine():
    M = P()
    out = []
    for harm in (0, 1):
        cfg = M.small_reactor(np_init=20000, mcc_on=1)
        pic = M.Pic(cfg, device=DEV)
        pic.load_particles()
        if harm:
            pic.set_drive([cfg["volt"]], [cfg["freq"]], [0.0])
        pic.step(3)
        out.append(pic.fields())
    # equal up to the order of the FP64 atomic additions of the deposit
    for a, b in zip(*out):
        assert np.max(np.abs(a - b)) <= 1e-10 * max(np.max(np.abs(a)), 1e-300)


def test_sawtooth_drive_and_fixed_ions_match_the_es_oracle():
    """Sawtooth-like excitation sum_n A sin(2 pi n f t)/n with ions held in
    place, electrostatic model, FP64, against the oracle's whole step."""
    M = P()
    f, A, N = 106e6, 20.0, 6
    cfg = M.small_reactor(np_init=30000, mcc_on=0, picard_tol=1e-10, field_model=M.PIC_FIELD_ES,
                          ions_fixed=1, dt=1e-10)
    g = O.Grid(cfg["nr"], cfg["nz"], cfg["R"], cfg["L"])
    e, i = O.load(g, 30000, 1e15, 6.0, 0.026, 5)
    pic = M.Pic(cfg, device=DEV)
    pic.set_state([e, i])
    amp = [A / n for n in range(1, N + 1)]
    fr = [n * f for n in range(1, N + 1)]
    pic.set_drive(amp, fr, [0.0] * N)
    drive = lambda t: sum(a * np.sin(2 * np.pi * q * t) for a, q in zip(amp, fr))
    sim = ES.Sim(g, cfg["dt"], tol=1e-10, species=[e, i], drive=drive, fixed=(1,),
                 cap=45000)
    ions0 = by_id(pic.get_state(1))
    for step in range(3):
        rc, st = pic.step(1)
        rco, sto = sim.step()
        assert rc == 0 and rco == 0 and st["picard_iters"] == sto["picard_iters"]
        assert st["v_electrode"] == pytest.approx(drive((step + 1) * cfg["dt"]), rel=1e-14)
        er, ez, _ = pic.fields()
        for got, ref in ((er, sim.er), (ez, sim.ez)):
            assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))
        assert_state_close(by_id(pic.get_state(0)), by_id(sim.state(0)), rtol=1e-10,
                           what="electrons step %d " % step, nz=cfg["nz"])
        ions = by_id(pic.get_state(1))
        for k in ions0:
            assert np.array_equal(ions[k], ions0[k]), k
