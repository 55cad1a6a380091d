"""The Picard iteration of Sec. 2.1 run on the device (pic_set_device_picard):
one conditional graph per step repeats the pass, tests convergence and
chooses the speculative final pass on the device, so the host waits once for
the whole iteration.  It runs the same kernels in the same order as the host
loop, so two contexts started from the same state, one per loop, take the
same iteration counts, the same speculation outcomes and the same launches,
and their fields and particles agree to the rounding of the deposit's
atomic sums (their order is not fixed; with FP32 particles that rounding
reaches the FP32 push, so the bound is the FP32 one)."""
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


def pair(guess=0, **kw):
    M = P()
    if kw.get("precision", 0) == 1:
        # FP32 particles: a step converged at 1e-8 sits near the rounding floor
        # of the FP32 push, where the order of the atomic sums can cost one pass
        # more or less; at 1e-6 the loops' decisions are the same in both
        kw.setdefault("picard_tol", 1e-6)
    cfg = M.small_reactor(np_init=30000, volt=200.0, **kw)
    out = []
    for dev_loop in (False, True):
        pic = M.Pic(cfg, device=DEV, stream=torch.cuda.Stream(device=DEV))
        M.set_graphs(pic, True)
        M.set_device_picard(pic, dev_loop)
        if guess:
            M.set_guess(pic, guess)
        pic.load_particles()
        out.append(pic)
    return cfg, out


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize(
    "kw,guess",
    [(dict(), 0), (dict(precision=1), 0), (dict(precision=1, field_model=1), 0),
     (dict(cblock=4e-11), 0), (dict(precision=1), 1)],
    ids=["fp64", "mixed", "mixed-es", "fp64-capacitor", "mixed-extrapolated-start"])
def test_device_loop_follows_the_host_loop(kw, guess):
    from tests.test_gpu_parity import by_id
    cfg, (host, dev) = pair(guess, **kw)
    fp64 = kw.get("precision", 0) == 0
    spec_seen = 0
    for step in range(12):
        rc_h, sh = host.step(1, check=False)
        rc_d, sd = dev.step(1, check=False)
        assert rc_h == rc_d and rc_h in (0,), (step, rc_h, rc_d)
        for k in ("picard_iters", "converged", "spec_final", "guess", "pushes"):
            assert sh[k] == sd[k], (step, k, sh[k], sd[k])
        # the same launches plus the device loop's convergence test per pass
        # (from the second step: the context's first pass is never captured)
        assert sd["launches"] == sh["launches"] + (sd["picard_iters"] if step > 0 else 0), step
        assert abs(sh["first_res"] - sd["first_res"]) <= 1e-6 * sh["first_res"] + 1e-300
        if fp64:
            assert abs(sh["last_res"] - sd["last_res"]) <= 1e-6 * sh["last_res"] + 1e-300
        # (FP32 particles: the converged residual sits near the rounding floor of
        # the FP32 push, which the order of the atomic sums moves)
        spec_seen += sd["spec_final"]
        for a, b in zip(dev.fields(), host.fields()):
            assert rel(a, b) <= (1e-9 if fp64 else 1e-6), step
    assert spec_seen > 0  # the speculative branch of the if-node ran and was adopted
    vh, vd = host.view(), dev.view()
    assert list(vh["n"]) == list(vd["n"])
    for s in range(2):
        gh, gd = by_id(host.get_state(s)), by_id(dev.get_state(s))
        assert np.array_equal(gh["id"], gd["id"])
        for k in ("a", "b", "vr", "vt", "vz"):
            tol = 1e-9 if fp64 else 1e-5
            assert np.max(np.abs(gh[k] - gd[k])) <= tol * max(np.max(np.abs(gh[k])), 1e-30), (s, k)
    if kw.get("cblock", 0) > 0:
        qh, ph = host.circuit()
        qd, pd = dev.circuit()
        assert abs(ph - pd) <= 1e-9 * abs(ph) and abs(qh - qd) <= 1e-8 * abs(qh)


def test_iteration_limit_and_switching():
    """K_max reached on the device ends the loop with PIC_E_NOCONV after exactly
    K_max passes; switching the loop off and on between steps keeps the
    contraction estimate that steers the speculative pass."""
    M = P()
    cfg, (host, dev) = pair()
    for pic in (host, dev):
        pic.step(3)
        pic.set_picard(1e-30, 3)
        rc, st = pic.step(1, check=False)
        assert rc == M.PIC_E_NOCONV and st["picard_iters"] == 3 and st["converged"] == 0
        pic.set_picard(cfg["picard_tol"], cfg["picard_max"])
    for on in (False, True, False, True):
        M.set_device_picard(dev, on)
        rc_h, sh = host.step(1)
        rc_d, sd = dev.step(1)
        assert sh["picard_iters"] == sd["picard_iters"] and sh["spec_final"] == sd["spec_final"]
