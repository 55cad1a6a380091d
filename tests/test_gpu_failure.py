"""Failure detection on the GPU, with every failure made on the host: the
library's error codes of pic_step (include/pic.h) for a nonlinear iteration
that does not converge, a store without room for the ionization pairs, and a
non-finite field, each checked for the state it leaves behind.  No kernel is
made to fault, trap or hang."""
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


def snapshot(pic):
    st = [pic.get_state(s) for s in range(2)]
    return st, pic.fields(), pic.view()["wall"].cpu().numpy(), pic.view()["step"]


def same(a, b):
    (sa, fa, wa, ka), (sb, fb, wb, kb) = a, b
    assert ka == kb
    for s in range(2):
        for k in sa[s]:
            assert np.array_equal(sa[s][k], sb[s][k]), (s, k)
    for x, y in zip(fa, fb):
        assert np.array_equal(x, y)
    assert np.array_equal(wa, wb)


@pytest.mark.parametrize("precision,graphs", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_noconv_leaves_state_n(precision, graphs):
    """Sec. 2.1's convergence test cannot be met (tol 1e-30) within K_max = 2:
    PIC_E_NOCONV, and particles, fields, wall tallies and the step index are
    those of step n, bit for bit (no pass of the failed step wrote them).
    With graph replay the iteration runs on the device (after the first step)."""
    M = P()
    cfg = M.small_reactor(np_init=20000, volt=200.0, precision=precision)
    pic = M.Pic(cfg, device=DEV, stream=torch.cuda.Stream(device=DEV) if graphs else None)
    M.set_graphs(pic, bool(graphs))
    pic.load_particles()
    pic.step(3)
    before = snapshot(pic)
    pic.set_picard(1e-30, 2)
    rc, st = pic.step(1, check=False)
    assert rc == M.PIC_E_NOCONV
    assert st["converged"] == 0 and st["picard_iters"] == 2
    same(before, snapshot(pic))
    # the context stays usable: the step goes through at the usual tolerance
    pic.set_picard(cfg["picard_tol"], cfg["picard_max"])
    rc, st = pic.step(1)
    assert rc == 0 and st["converged"] == 1


@pytest.mark.parametrize("precision", [0, 1])
def test_capacity_appends_no_pair(precision):
    """A store filled to capacity (capacity factor 1) with 50 eV electrons in
    20 Pa argon: the collisions of the step ionize, there is no room for the
    pairs, the step reports PIC_E_CAPACITY after committing and appends none
    (the counts fall by the absorbed particles only, the ids do not move)."""
    M = P()
    n = 20000
    cfg = M.small_reactor(np_init=n, capacity_factor=1.0, gas_pressure=20.0, precision=precision)
    pic = M.Pic(cfg, device=DEV)
    g = O.Grid(cfg["nr"], cfg["nz"], cfg["R"], cfg["L"])
    e, i = O.load(g, n, 1e15, 50.0, 0.026, 8)
    pic.set_state([e, i])
    v0 = pic.view()
    n0, ids0 = list(v0["n"]), list(v0["next_id"])
    rc, st = pic.step(1, check=False)
    assert rc == M.PIC_E_CAPACITY
    assert st["converged"] == 1
    v1 = pic.view()
    assert list(v1["next_id"]) == ids0
    assert v1["n"][0] + v1["n"][1] == n0[0] + n0[1] - st["absorbed"]
    assert v1["n"][0] <= n0[0] and v1["n"][1] <= n0[1]
    for s in range(2):
        ids = pic.get_state(s)["id"]
        assert ids.max() < ids0[s]


@pytest.mark.parametrize("precision,graphs", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_nan_field_reports_nan(precision, graphs):
    """A NaN written into E^n from the host (through pic_state_upload): the
    Picard residual is not finite, pic_step returns PIC_E_NAN without
    committing, and after a clean upload the context steps again.  With graph
    replay the iteration runs on the device and stops at the first pass."""
    M = P()
    cfg = M.small_reactor(np_init=20000, volt=200.0, precision=precision)
    pic = M.Pic(cfg, device=DEV, stream=torch.cuda.Stream(device=DEV) if graphs else None)
    M.set_graphs(pic, bool(graphs))
    pic.load_particles()
    pic.step(2)
    hs = pic.host_state(pinned=True)
    pic.state_download(hs)
    clean = hs["er"].clone()
    step0 = hs["step"]
    # an interior E_r edge (the plate edges j = 0, nz are prescribed by the PEC
    # condition and never reach the field solve)
    nz = cfg["nz"]
    hs["er"][(cfg["nr"] // 2) * (nz + 1) + nz // 2] = float("nan")
    pic.state_upload(hs)
    rc, st = pic.step(1, check=False)
    assert rc == M.PIC_E_NAN
    assert pic.view()["step"] == step0
    if graphs:
        assert st["picard_iters"] == 1
    hs["er"].copy_(clean)
    pic.state_upload(hs)
    rc, st = pic.step(1)
    assert rc == 0 and st["converged"] == 1
