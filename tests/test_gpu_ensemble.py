"""Ensembles of independent discharges and CUDA-graph replay of the Picard
passes give the results of stepping each discharge alone (to the rounding of
the order of FP64 atomic additions in the deposit: 1e-10 relative after
three steps)."""
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


CFGS = [dict(nr=16, nz=24, np_init=8000, seed=3, volt=150.0),
        dict(nr=32, nz=64, np_init=40000, seed=4, freq=80e6, dt=1.0 / (200 * 80e6)),
        # the FP32 form at a tolerance well above its rounding floor, where the
        # iteration count does not depend on the order of the deposit's atomics
        dict(nr=24, nz=48, np_init=20000, seed=5, gas_pressure=5.0, precision=1, picard_tol=1e-6)]


def make(c):
    M = P()
    cfg = M.small_reactor(**c)
    s = torch.cuda.Stream(device=DEV)
    pic = M.Pic(cfg, device=DEV, stream=s)
    pic.load_particles()
    return pic


def compare(a, b, what):
    ea, eza, ha = a.fields()
    eb, ezb, hb = b.fields()
    # mixed form: a field difference at FP64 rounding can move an FP32 state by an ulp
    ftol = 1e-6 if a.cfg.get("precision", 0) == 1 else 1e-10
    for x, y in ((ea, eb), (eza, ezb), (ha, hb)):
        assert np.max(np.abs(x - y)) <= ftol * max(np.max(np.abs(y)), 1e-300), what
    for s in range(2):
        ga, gb = a.get_state(s), b.get_state(s)
        assert len(ga["id"]) == len(gb["id"]), what
        oa, ob = np.argsort(ga["id"]), np.argsort(gb["id"])
        assert np.array_equal(ga["cell"][oa], gb["cell"][ob]), what
        for k in ("a", "b", "vr", "vt", "vz"):
            x, y = ga[k][oa].astype(np.float64), gb[k][ob].astype(np.float64)
            tol = 1e-10 if ga[k].dtype == np.float64 else 1e-4
            assert np.max(np.abs(x - y)) <= tol * max(np.max(np.abs(y)), 1e-300), (what, k)


def test_graph_replay_matches_kernel_launches():
    a, b = make(CFGS[1]), make(CFGS[1])
    P().set_graphs(b, True)
    for _ in range(3):
        ra, sa = a.step(1)
        rb, sb = b.step(1)
        assert ra == rb == 0 and sa["picard_iters"] == sb["picard_iters"]
    compare(a, b, "graphs")


# members of one precision, for persistent rounds (one push launch per species
# over every member)
CFGS64 = [dict(nr=16, nz=24, np_init=8000, seed=3, volt=150.0),
          dict(nr=32, nz=64, np_init=40000, seed=4, freq=80e6, dt=1.0 / (200 * 80e6)),
          dict(nr=24, nz=48, np_init=20000, seed=6, gas_pressure=5.0)]
CFGS32 = [dict(c, precision=1, picard_tol=1e-6) for c in CFGS64]


@pytest.mark.parametrize("cfgs,persistent", [(CFGS, False), (CFGS64, True), (CFGS64, False),
                                             (CFGS32, True)],
                         ids=["mixed-precisions", "fp64-persistent", "fp64-per-member",
                              "fp32-persistent"])
def test_ensemble_matches_members_stepped_alone(cfgs, persistent):
    M = P()
    alone = [make(c) for c in cfgs]
    ens_m = [make(c) for c in cfgs]
    E = M.Ensemble(ens_m)
    E.set_persistent(persistent)
    for _ in range(3):
        rc, st = E.step(1)
        assert rc == 0
        for p, s in zip(alone, st):
            r, sa = p.step(1)
            assert r == 0 and sa["picard_iters"] == s["picard_iters"]
            assert sa["n"] == s["n"]
    for i, (a, b) in enumerate(zip(alone, ens_m)):
        compare(a, b, "member %d" % i)


def test_tune_changes_no_state_and_keeps_results():
    M = P()
    ens_m = [make(c) for c in CFGS]
    ref = [make(c) for c in CFGS]
    E = M.Ensemble(ens_m)
    frac, pers, ms = E.tune(rounds=2)
    # members of two precisions: no persistent candidates
    assert frac in (1.0, 0.5, 0.25) and not pers
    assert all(t > 0 for t in ms[:3]) and all(t == -1.0 for t in ms[3:])
    for a, b in zip(ens_m, ref):
        compare(a, b, "after tune")
    E.step(2)
    for p in ref:
        p.step(2)
    for i, (a, b) in enumerate(zip(ens_m, ref)):
        compare(a, b, "tuned member %d" % i)


def test_persistent_tune_and_rejection():
    """Members of one precision offer all six candidates; members of two
    precisions refuse persistent rounds."""
    M = P()
    ens_m = [make(c) for c in CFGS64]
    ref = [make(c) for c in CFGS64]
    E = M.Ensemble(ens_m)
    frac, pers, ms = E.tune(rounds=2)
    assert frac in (1.0, 0.5, 0.25) and all(t > 0 for t in ms)
    E.step(2)
    for p in ref:
        p.step(2)
    for i, (a, b) in enumerate(zip(ens_m, ref)):
        compare(a, b, "tuned persistent=%s member %d" % (pers, i))
    E2 = M.Ensemble([make(c) for c in CFGS])
    with pytest.raises(M.PicError):
        E2.set_persistent(True)
