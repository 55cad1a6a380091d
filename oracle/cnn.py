"""FP64 CPU oracle of the learned Picard initial guess (test infrastructure only).

The learned guess predicts the field iterate E^{n+1,0} that starts the
nonlinear (Picard) iteration of a step (Sec. 2.1 leaves the start open; the
plain start is E^n).  It is the quadratic time extrapolation
    G = 3 E^n - 3 E^{n-1} + E^{n-2}
plus a learned correction s_d * f(x), where f is a stack of 3x3 convolutions
with ReLU between them and x are the 14 input channels built below on the
padded (nr+1) x (nz+1) grid that holds the staggered points of E_r
(nr x (nz+1)), E_z ((nr+1) x nz) and H_theta (nr x nz) at their own indices.

Everything here is plain numpy in float64, written from the definitions:
convolution as the sum over taps and input channels, the chain rule for the
gradients, Adam as published (Kingma & Ba, ICLR 2015, Algorithm 1).  Only
tests/ and bench.py's reference legs may import it.
"""
from __future__ import annotations

import numpy as np

N_IN = 14
TINY = 1e-30


# --------------------------------------------------------------------------
# input channels and the extrapolated start
def _rms(*arrays):
    s = sum(float(np.sum(a * a)) for a in arrays)
    n = sum(a.size for a in arrays)
    return np.sqrt(s / max(n, 1)) + TINY


def pad_er(er, nr, nz):
    out = np.zeros((nr + 1, nz + 1))
    out[:nr, :] = np.asarray(er).reshape(nr, nz + 1)
    return out


def pad_ez(ez, nr, nz):
    out = np.zeros((nr + 1, nz + 1))
    out[:, :nz] = np.asarray(ez).reshape(nr + 1, nz)
    return out


def pad_h(h, nr, nz):
    out = np.zeros((nr + 1, nz + 1))
    out[:nr, :nz] = np.asarray(h).reshape(nr, nz)
    return out


def extrapolate(er_hist, ez_hist):
    """Quadratic extrapolation from E^n, E^{n-1}, E^{n-2} (lists, newest first)."""
    er = 3.0 * er_hist[0] - 3.0 * er_hist[1] + er_hist[2]
    ez = 3.0 * ez_hist[0] - 3.0 * ez_hist[1] + ez_hist[2]
    return er, ez


def features(nr, nz, er_hist, ez_hist, h, ir, iz):
    """The 14 input channels and the increment scale s_d.

    er_hist / ez_hist: E^n, E^{n-1}, E^{n-2}, E^{n-3} (newest first, flat Yee
    layouts); h: H^n; ir / iz: charge crossed in the last step.
      0-5   successive increments E^{n-k} - E^{n-k-1} (k = 0, 1, 2; E_r, E_z) / s_d
      6-7   E^n / s_e          8  H^n / s_h          9-10  (ir, iz) / s_j
      11-12 validity masks of the E_r and E_z points   13   r / R of the row
    with s_d, s_e, s_h, s_j the RMS over the valid points of what they scale.
    """
    d = [(er_hist[k] - er_hist[k + 1], ez_hist[k] - ez_hist[k + 1]) for k in range(3)]
    sd = _rms(*d[0])
    se = _rms(er_hist[0], ez_hist[0])
    sh = _rms(h)
    sj = _rms(ir, iz)
    x = np.zeros((N_IN, nr + 1, nz + 1))
    for k in range(3):
        x[2 * k] = pad_er(d[k][0] / sd, nr, nz)
        x[2 * k + 1] = pad_ez(d[k][1] / sd, nr, nz)
    x[6] = pad_er(er_hist[0] / se, nr, nz)
    x[7] = pad_ez(ez_hist[0] / se, nr, nz)
    x[8] = pad_h(h / sh, nr, nz)
    x[9] = pad_er(ir / sj, nr, nz)
    x[10] = pad_ez(iz / sj, nr, nz)
    x[11] = pad_er(np.ones(nr * (nz + 1)), nr, nz)
    x[12] = pad_ez(np.ones((nr + 1) * nz), nr, nz)
    x[13] = (np.arange(nr + 1) / nr)[:, None] * np.ones((1, nz + 1))
    return x, sd


def target(nr, nz, er_next, ez_next, er_hist, ez_hist, sd):
    """Training target (E^{n+1} - G) / s_d on the padded grid, and its mask (2 channels)."""
    ger, gez = extrapolate(er_hist, ez_hist)
    t = np.zeros((2, nr + 1, nz + 1))
    t[0] = pad_er((er_next - ger) / sd, nr, nz)
    t[1] = pad_ez((ez_next - gez) / sd, nr, nz)
    m = np.zeros((2, nr + 1, nz + 1))
    m[0] = pad_er(np.ones(nr * (nz + 1)), nr, nz)
    m[1] = pad_ez(np.ones((nr + 1) * nz), nr, nz)
    return t, m


# --------------------------------------------------------------------------
# network
def init_params(channels, seed):
    """He-normal weights (std sqrt(2 / (9 c_in))), zero biases; channels e.g. [14, 64, 64, 64, 64, 2]."""
    rng = np.random.default_rng(seed)
    ps = []
    for ci, co in zip(channels[:-1], channels[1:]):
        w = rng.normal(size=(co, ci, 3, 3)) * np.sqrt(2.0 / (9 * ci))
        ps.append((w, np.zeros(co)))
    return ps


def conv3x3(x, w, b):
    """y[o, i, j] = b[o] + sum_{c, di, dj} w[o, c, di, dj] x[c, i + di - 1, j + dj - 1] (zero outside)."""
    ci, H, W = x.shape
    xp = np.zeros((ci, H + 2, W + 2))
    xp[:, 1:H + 1, 1:W + 1] = x
    y = np.zeros((w.shape[0], H, W)) + b[:, None, None]
    for di in range(3):
        for dj in range(3):
            y += np.tensordot(w[:, :, di, dj], xp[:, di:di + H, dj:dj + W], axes=(1, 0))
    return y


def forward(params, x):
    """Convolutions with ReLU between them (none after the last); returns (out, pre-activations)."""
    acts = [x]
    pres = []
    h = x
    for k, (w, b) in enumerate(params):
        z = conv3x3(h, w, b)
        pres.append(z)
        h = np.maximum(z, 0.0) if k + 1 < len(params) else z
        acts.append(h)
    return h, (acts, pres)


def round_bf16(a):
    """Nearest bfloat16 value of each element, as an FP64 array: the FP32 value
    cut to its top 16 bits, rounded to nearest with ties to even (bfloat16 is
    the upper half of the IEEE binary32 format)."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


# rounding allowances of forward_bf16's bound: an FP32 sum of K <= 9 x 64
# products is within K 2^-24 of the sum of their magnitudes (2^-14 covers it),
# and a bfloat16 step is at most 2^-7 of the value rounded
FP32_SUM = 2.0 ** -14
BF16_STEP = 2.0 ** -7


def forward_bf16(params, x):
    """The forward pass as the tensor-core kernels compute it: weights and
    inputs already bfloat16 values, every hidden activation rounded to
    bfloat16 after its ReLU, the last layer's output kept unrounded (sums in
    FP64 here).  Returns (out, bound): an element-wise bound on the difference
    from the same computation with FP32 sums in any order.  Per layer, a sum
    is within FP32_SUM x (|w| * |h| + |b|) of the exact one plus the carried
    difference of its inputs through |w|; the ReLU does not increase it; the
    bfloat16 rounding of a value off by that much lands within the same
    difference plus one bfloat16 step."""
    h = np.asarray(x, dtype=np.float64)
    e = np.zeros_like(h)
    for k, (w, b) in enumerate(params):
        z = conv3x3(h, w, b)
        aw = np.abs(w)
        ez = conv3x3(e, aw, np.zeros_like(b)) + FP32_SUM * conv3x3(np.abs(h), aw, np.abs(b))
        if k + 1 < len(params):
            h = round_bf16(np.maximum(z, 0.0))
            e = ez + BF16_STEP * np.abs(h)
        else:
            h, e = z, ez
    return h, e


def loss(out, t, m):
    """Mean squared error over the valid points: sum m (out - t)^2 / sum m."""
    return float(np.sum(m * (out - t) ** 2) / np.sum(m))


def backward(params, cache, out, t, m):
    """Gradients of loss() with respect to every (w, b), by the chain rule."""
    acts, pres = cache
    g = 2.0 * m * (out - t) / np.sum(m)
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        w, b = params[k]
        if k + 1 < len(params):
            g = g * (pres[k] > 0.0)
        h = acts[k]
        ci, H, W = h.shape
        hp = np.zeros((ci, H + 2, W + 2))
        hp[:, 1:H + 1, 1:W + 1] = h
        gw = np.zeros_like(w)
        for di in range(3):
            for dj in range(3):
                gw[:, :, di, dj] = np.tensordot(g, hp[:, di:di + H, dj:dj + W], axes=([1, 2], [1, 2]))
        gb = g.sum(axis=(1, 2))
        grads[k] = (gw, gb)
        # d/dh of sum_o g[o] * conv(h)[o]: correlation of g with the flipped kernel
        gp = np.zeros((w.shape[0], H + 2, W + 2))
        gp[:, 1:H + 1, 1:W + 1] = g
        gh = np.zeros((ci, H, W))
        for di in range(3):
            for dj in range(3):
                gh += np.tensordot(w[:, :, di, dj], gp[:, 2 - di:2 - di + H, 2 - dj:2 - dj + W],
                                   axes=(0, 0))
        g = gh
    return grads


def adam(params, grads, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015): m, v moments with bias correction; returns new params."""
    t = state.get("t", 0) + 1
    state["t"] = t
    out = []
    for k, ((w, b), (gw, gb)) in enumerate(zip(params, grads)):
        new = []
        for j, (p, g) in enumerate(((w, gw), (b, gb))):
            key = (k, j)
            m = state.get(("m",) + key, np.zeros_like(p))
            v = state.get(("v",) + key, np.zeros_like(p))
            m = b1 * m + (1 - b1) * g
            v = b2 * v + (1 - b2) * g * g
            state[("m",) + key] = m
            state[("v",) + key] = v
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            new.append(p - lr * mh / (np.sqrt(vh) + eps))
        out.append(tuple(new))
    return out


def flatten(params):
    """Parameters as one vector: per layer w (o, c, di, dj order), then b."""
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params])


def unflatten(vec, channels):
    ps = []
    k = 0
    for ci, co in zip(channels[:-1], channels[1:]):
        nw = co * ci * 9
        w = vec[k:k + nw].reshape(co, ci, 3, 3)
        k += nw
        b = vec[k:k + co]
        k += co
        ps.append((w.copy(), b.copy()))
    return ps
