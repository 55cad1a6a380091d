"""Pins of the FP64 oracle of the learned Picard guess (oracle/cnn.py) against
things other than itself: scipy's 2-D correlation, central finite
differences, Adam's closed-form first step, exactness of the quadratic
extrapolation on quadratic-in-time fields, and invariances of the inputs."""
import numpy as np
import pytest

from oracle import cnn as Q

scipy_signal = pytest.importorskip("scipy.signal")


def test_conv3x3_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 7, 9))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = Q.conv3x3(x, w, b)
    for o in range(4):
        ref = b[o] + sum(scipy_signal.correlate2d(x[c], w[o, c], mode="same", boundary="fill")
                         for c in range(3))
        np.testing.assert_allclose(y[o], ref, rtol=1e-12, atol=1e-12)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(1)
    ch = [3, 5, 4, 2]
    ps = Q.init_params(ch, 2)
    ps = [(w, rng.normal(size=b.shape) * 0.1) for w, b in ps]
    x = rng.normal(size=(3, 6, 7))
    t = rng.normal(size=(2, 6, 7))
    m = (rng.uniform(size=(2, 6, 7)) > 0.2).astype(float)
    out, cache = Q.forward(ps, x)
    g = Q.flatten(Q.backward(ps, cache, out, t, m))
    v = Q.flatten(ps)
    idx = rng.choice(v.size, size=60, replace=False)
    h = 1e-6
    for k in idx:
        vp, vm = v.copy(), v.copy()
        vp[k] += h
        vm[k] -= h
        lp = Q.loss(Q.forward(Q.unflatten(vp, ch), x)[0], t, m)
        lm = Q.loss(Q.forward(Q.unflatten(vm, ch), x)[0], t, m)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_loss_zero_at_target_and_adam_first_step():
    rng = np.random.default_rng(3)
    t = rng.normal(size=(2, 4, 5))
    m = np.ones_like(t)
    assert Q.loss(t, t, m) == 0.0
    ps = Q.init_params([2, 3, 2], 4)
    gs = [(rng.normal(size=w.shape), rng.normal(size=b.shape)) for w, b in ps]
    new = Q.adam(ps, gs, {}, lr=1e-3, eps=0.0)
    # first step: m_hat = g, v_hat = g^2, so every parameter moves by -lr * sign(g)
    for (w, b), (w1, b1), (gw, gb) in zip(ps, new, gs):
        np.testing.assert_allclose(w1 - w, -1e-3 * np.sign(gw), rtol=1e-12)
        np.testing.assert_allclose(b1 - b, -1e-3 * np.sign(gb), rtol=1e-12)


def test_extrapolation_exact_for_quadratic_time_dependence():
    rng = np.random.default_rng(5)
    A, B, C = (rng.normal(size=20) for _ in range(3))
    f = lambda t: A + B * t + C * t * t
    er_hist = [f(0.0), f(-1.0), f(-2.0)]
    ez_hist = [2 * f(0.0), 2 * f(-1.0), 2 * f(-2.0)]
    er, ez = Q.extrapolate(er_hist, ez_hist)
    np.testing.assert_allclose(er, f(1.0), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(ez, 2 * f(1.0), rtol=1e-12, atol=1e-12)


def test_features_scale_invariant_and_masked():
    nr, nz = 4, 6
    rng = np.random.default_rng(6)
    er = [rng.normal(size=nr * (nz + 1)) for _ in range(4)]
    ez = [rng.normal(size=(nr + 1) * nz) for _ in range(4)]
    h = rng.normal(size=nr * nz)
    ir, iz = rng.normal(size=nr * (nz + 1)), rng.normal(size=(nr + 1) * nz)
    x, sd = Q.features(nr, nz, er, ez, h, ir, iz)
    x3, sd3 = Q.features(nr, nz, [3 * a for a in er], [3 * a for a in ez], 5 * h, 7 * ir, 7 * iz)
    np.testing.assert_allclose(x3, x, rtol=1e-12, atol=1e-12)
    assert abs(sd3 / sd - 3.0) < 1e-12
    # padding points of E_r (row nr) and E_z (column nz) are zero in every field channel
    for c in (0, 2, 4, 6, 9):
        assert np.all(x[c][nr, :] == 0.0)
    for c in (1, 3, 5, 7, 10):
        assert np.all(x[c][:, nz] == 0.0)
    assert x[11].sum() == nr * (nz + 1) and x[12].sum() == (nr + 1) * nz
    np.testing.assert_allclose(x[13][:, 0], np.arange(nr + 1) / nr)
    # increments are RMS-normalised: channels 0-1 have unit RMS over the valid points
    v = np.concatenate([x[0][:nr, :].ravel(), x[1][:, :nz].ravel()])
    assert abs(np.sqrt(np.mean(v * v)) - 1.0) < 1e-9


def test_bf16_rounding_matches_torch():
    """round_bf16 against torch's float32 -> bfloat16 conversion (round to
    nearest even), including ties, subnormals, zeros and large values."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    a = np.concatenate([rng.normal(size=5000) * 10 ** rng.uniform(-30, 30, size=5000),
                        [0.0, -0.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1e-40, -1e-39, 3e38]])
    a = a.astype(np.float32)
    ref = torch.tensor(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(Q.round_bf16(a), ref)


def test_forward_bf16_bound_holds_under_perturbed_sums():
    """forward_bf16's element-wise bound: the same network evaluated with
    every sum perturbed by up to the FP32 allowance (random signs) and the
    hidden activations rounded to bfloat16 from the perturbed sums stays
    within the bound of the unperturbed pass (and does differ from it)."""
    rng = np.random.default_rng(11)
    ps = Q.init_params([14, 16, 16, 2], 4)
    ps = [(Q.round_bf16(w), rng.normal(size=b.shape) * 0.05) for w, b in ps]
    x = Q.round_bf16(rng.normal(size=(14, 9, 13)))
    ref, bound = Q.forward_bf16(ps, x)
    worst = 0.0
    for trial in range(20):
        h = x
        for k, (w, b) in enumerate(ps):
            z = Q.conv3x3(h, w, b)
            scale = Q.FP32_SUM * Q.conv3x3(np.abs(h), np.abs(w), np.abs(b))
            z = z + scale * rng.uniform(-1, 1, size=z.shape)
            h = Q.round_bf16(np.maximum(z, 0.0)) if k + 1 < len(ps) else z
        assert np.all(np.abs(h - ref) <= bound), np.max(np.abs(h - ref) / bound)
        worst = max(worst, float(np.max(np.abs(h - ref))))
    assert worst > 0.0
