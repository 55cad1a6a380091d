"""Checkpoint and resume (pic_save / pic_load): a run resumed from a
checkpoint takes the same steps as the uninterrupted run, for the FP64 and
mixed forms, the electrostatic model and the blocking capacitor, up to the
order of the FP64 atomic additions of the deposit; mismatched contexts and
unreadable files are refused."""
import os

import numpy as np
import pytest

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


def by_id(sp):
    o = np.argsort(sp["id"], kind="stable")
    return {k: v[o] for k, v in sp.items()}


@pytest.mark.parametrize("kw", [dict(), dict(precision=1), dict(field_model=1, cblock=3e-11),
                                dict(cblock=3e-11, axis_cells=3)])
def test_resumed_run_matches_the_uninterrupted_one(kw, tmp_path):
    M = P()
    cfg = M.small_reactor(np_init=20000, mcc_on=1, volt=200.0, gas_pressure=10.0,
                          picard_tol=1e-8 if kw.get("precision", 0) == 0 else 1e-5, **kw)
    path = str(tmp_path / "ckpt.bin")
    a = M.Pic(cfg, device=DEV)
    a.load_particles()
    a.step(3)
    a.save(path)
    for _ in range(3):
        a.step(1)
    b = M.Pic(cfg, device=DEV)
    b.load(path)
    for _ in range(3):
        b.step(1)
    fa, fb = a.fields(), b.fields()
    ftol = 1e-10 if kw.get("precision", 0) == 0 else 1e-5
    for x, y in zip(fa, fb):
        assert np.max(np.abs(x - y)) <= ftol * max(np.max(np.abs(x)), 1e-300)
    assert a.circuit() == pytest.approx(b.circuit(), rel=1e-9, abs=1e-30)
    for s in range(2):
        ga, gb = by_id(a.get_state(s)), by_id(b.get_state(s))
        assert np.array_equal(ga["id"], gb["id"])  # same ionizations, same new ids
        assert np.mean(ga["cell"] == gb["cell"]) > 0.999
        for k in ("vr", "vz"):
            d = np.abs(ga[k].astype(np.float64) - gb[k])
            assert np.quantile(d, 0.999) <= 1e-6 * np.max(np.abs(ga[k]))


def test_refused_checkpoints(tmp_path):
    M = P()
    path = str(tmp_path / "c.bin")
    a = M.Pic(M.small_reactor(np_init=5000), device=DEV)
    a.load_particles()
    a.save(path)
    other = M.Pic(M.small_reactor(np_init=5000, nz=48), device=DEV)
    with pytest.raises(M.PicError) as e:
        other.load(path)
    assert e.value.code == M.PIC_E_STATE
    with pytest.raises(M.PicError) as e:
        other.load(str(tmp_path / "missing.bin"))
    assert e.value.code == M.PIC_E_IO
    with open(path, "r+b") as f:
        f.write(b"XXXX")
    with pytest.raises(M.PicError) as e:
        a.load(path)
    assert e.value.code == M.PIC_E_IO


def test_host_state_round_trip():
    """pic_state_download / pic_state_upload move the whole state through
    host memory: a context stepped after a round trip matches one stepped
    without it, and an undersized host buffer is refused."""
    M = P()
    cfg = M.small_reactor(np_init=6000, mcc_on=1)
    a = M.Pic(cfg, device=DEV)
    a.load_particles()
    for _ in range(2):
        a.step(1)
    hs = a.host_state(pinned=True)
    a.state_download(hs)
    assert hs["n"] == a.view()["n"] and hs["step"] == a.view()["step"]
    b = M.Pic(cfg, device=DEV)
    b.state_upload(hs)
    for _ in range(2):
        a.step(1)
        b.step(1)
    for s in range(2):
        # the same particles; the order inside a cell is not fixed by the sort
        ga, gb = a.get_state(s), b.get_state(s)
        oa, ob = np.argsort(ga["id"]), np.argsort(gb["id"])
        np.testing.assert_array_equal(ga["id"][oa], gb["id"][ob])
        np.testing.assert_array_equal(ga["cell"][oa], gb["cell"][ob])
        for k in ("a", "b", "vr", "vt", "vz"):
            np.testing.assert_allclose(gb[k][ob], ga[k][oa], rtol=1e-9,
                                       atol=1e-9 * np.max(np.abs(ga[k])))
    small = a.host_state(pinned=False)
    small["species"][0] = {k: v[:10] for k, v in small["species"][0].items()}
    with pytest.raises(M.PicError) as e:
        a.state_download(small)
    assert e.value.code == M.PIC_E_STATE


@pytest.mark.parametrize("precision", [0, 1])
def test_step_host_matches_upload_step_download(precision):
    """pic_step_host (download of each step overlapped with the next step's
    upload) gives the host state that the same steps give through
    pic_state_upload / pic_step / pic_state_download, step counters and the
    summed pushes included."""
    M = P()
    cfg = M.small_reactor(np_init=20000, mcc_on=1, gas_pressure=10.0, precision=precision,
                          picard_tol=1e-8 if precision == 0 else 1e-5)
    a, b = M.Pic(cfg, device=DEV), M.Pic(cfg, device=DEV)
    a.load_particles()
    b.load_particles()
    ha, hb = a.host_state(pinned=True), b.host_state(pinned=True)
    a.state_download(ha)
    b.state_download(hb)
    pushes = 0
    for _ in range(4):
        b.state_upload(hb)
        _, st = b.step(1)
        pushes += st["pushes"]
        b.state_download(hb)
    rc, sa = a.step_host(ha, 4)
    assert rc == 0 and sa["pushes"] == pushes
    assert ha["n"] == hb["n"] and ha["next_id"] == hb["next_id"] and ha["step"] == hb["step"]
    for s in range(2):
        n = ha["n"][s]
        ga = {k: ha["species"][s][k][:n].numpy() for k in ("id", "cell", "a", "b", "vr", "vt", "vz")}
        gb = {k: hb["species"][s][k][:n].numpy() for k in ("id", "cell", "a", "b", "vr", "vt", "vz")}
        oa, ob = np.argsort(ga["id"]), np.argsort(gb["id"])
        np.testing.assert_array_equal(ga["id"][oa], gb["id"][ob])
        np.testing.assert_array_equal(ga["cell"][oa], gb["cell"][ob])
        tol = 1e-9 if precision == 0 else 1e-5
        for k in ("a", "b", "vr", "vt", "vz"):
            x, y = ga[k][oa].astype(np.float64), gb[k][ob].astype(np.float64)
            np.testing.assert_allclose(x, y, rtol=tol, atol=tol * np.max(np.abs(y)))
    for k in ("er", "ez", "h"):
        x, y = ha[k].numpy(), hb[k].numpy()
        assert np.max(np.abs(x - y)) <= 1e-6 * max(np.max(np.abs(y)), 1e-300)
