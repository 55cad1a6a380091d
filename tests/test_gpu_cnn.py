"""The learned Picard start on the GPU against the FP64 oracle (oracle/cnn.py).

The network computes in BF16 (weights and activations) with FP32
accumulation, so forward outputs and gradients are compared in relative L2
norm at a tolerance set by BF16 rounding (8 significant bits, a few layers:
3e-2), with the oracle given the same BF16-rounded weights and inputs.
The inputs / target kernels of the step are compared with the oracle's
definitions at FP32 rounding."""
import numpy as np
import pytest

import oracle as O
from oracle import cnn as Q

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
CH = [14, 64, 64, 64, 64, 2]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as G
    G.build()


def M():
    import paper_2212_08836_gb300 as P
    return P


def bf16(a):
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def setup(nr, nz, batch, seed):
    P = M()
    net = P.Cnn(nr, nz, depth=len(CH) - 1, batch=batch, seed=seed, device=DEV)
    ps = Q.init_params(CH, seed)
    rng = np.random.default_rng(seed + 1)
    ps = [(w, rng.normal(size=b.shape) * 0.05) for w, b in ps]
    ps = [(bf16(w), b) for w, b in ps]
    net.set_params(Q.flatten(ps).astype(np.float32))
    return net, ps, rng


def masks(nr, nz):
    m = np.zeros((2, nr + 1, nz + 1))
    m[0, :nr, :] = 1.0
    m[1, :, :nz] = 1.0
    return m


@pytest.mark.parametrize("nr,nz,batch", [(8, 12, 1), (13, 70, 2)])
def test_forward_matches_oracle(nr, nz, batch):
    net, ps, rng = setup(nr, nz, batch, 3)
    x = bf16(rng.normal(size=(batch, 14, nr + 1, nz + 1)))
    y = net.forward(torch.tensor(x, dtype=torch.float32, device=DEV)).cpu().numpy()
    for b in range(batch):
        ref, _ = Q.forward(ps, x[b])
        assert rel(y[b], ref) <= 3e-2, rel(y[b], ref)


def test_gradient_matches_oracle():
    nr, nz, batch = 10, 21, 2
    net, ps, rng = setup(nr, nz, batch, 5)
    x = bf16(rng.normal(size=(batch, 14, nr + 1, nz + 1)))
    t = rng.normal(size=(batch, 2, nr + 1, nz + 1))
    m = masks(nr, nz)
    loss, g = net.loss_grad(torch.tensor(x, dtype=torch.float32, device=DEV),
                            torch.tensor(t, dtype=torch.float32, device=DEV))
    lref = 0.0
    gref = np.zeros(net.num_params)
    for b in range(batch):
        out, cache = Q.forward(ps, x[b])
        lref += Q.loss(out, t[b], m) / batch
        gref += Q.flatten(Q.backward(ps, cache, out, t[b], m)) / batch
    assert abs(loss - lref) <= 2e-2 * abs(lref)
    assert rel(g, gref) <= 5e-2, rel(g, gref)
    cos = float(np.dot(g, gref) / (np.linalg.norm(g) * np.linalg.norm(gref)))
    assert cos >= 0.998, cos
    # every layer's gradient, not only the largest one
    off = 0
    for ci, co in zip(CH[:-1], CH[1:]):
        n = co * ci * 9 + co
        assert rel(g[off:off + n], gref[off:off + n]) <= 8e-2
        off += n


def test_adam_first_step_and_training_reduces_loss():
    nr, nz, batch = 12, 20, 4
    net, ps, rng = setup(nr, nz, batch, 7)
    x = torch.tensor(bf16(rng.normal(size=(batch, 14, nr + 1, nz + 1))), dtype=torch.float32,
                     device=DEV)
    # a learnable target: a smooth function of the inputs
    xt = x.cpu().numpy()
    t = np.stack([0.5 * xt[:, 0] - 0.3 * xt[:, 6], 0.2 * xt[:, 1] + 0.4 * xt[:, 7]], axis=1)
    t = torch.tensor(t, dtype=torch.float32, device=DEV)
    p0 = net.get_params()
    _, g0 = net.loss_grad(x, t)
    lr = 1e-3
    l0 = net.train_step(x, t, lr)
    p1 = net.get_params()
    # Adam's first step moves every parameter by -lr * sign(g) (Kingma & Ba, bias-corrected)
    big = np.abs(g0) > 1e-4
    np.testing.assert_allclose((p1 - p0)[big], -lr * np.sign(g0[big]), rtol=1e-3, atol=1e-7)
    for _ in range(150):
        l = net.train_step(x, t, lr)
    assert l < 0.3 * l0, (l0, l)


def reactor(**kw):
    P = M()
    cfg = P.small_reactor(np_init=20000, mcc_on=0, volt=150.0, **kw)
    pic = P.Pic(cfg, device=DEV)
    pic.load_particles()
    return P, cfg, pic


def test_inputs_and_target_match_oracle_definitions():
    P, cfg, pic = reactor()
    nr, nz = cfg["nr"], cfg["nz"]
    P.set_guess(pic, P.PIC_GUESS_EXTRAP)
    ers, ezs = [], []
    rc, st = 0, None
    for k in range(6):
        er, ez, h = pic.fields()
        ers.insert(0, er)
        ezs.insert(0, ez)
        rc, st = pic.step(1)
        if k >= 3:
            assert st["guess"] == P.PIC_GUESS_EXTRAP
    # the sample of the last step: inputs at its start, target after it
    smp = P.guess_sample(pic)
    assert smp is not None
    xg, tg = (a.cpu().numpy() for a in smp)
    er1, ez1, _ = pic.fields()
    # inputs of the last step use E^n .. E^{n-3} = ers[0..3], H^n and the crossed
    # charge of the step before; compare the channels that need only the fields
    xo, sd = Q.features(nr, nz, ers[:4], ezs[:4], np.zeros(nr * nz), np.ones(nr * (nz + 1)),
                        np.ones((nr + 1) * nz))
    for c in list(range(8)) + [11, 12, 13]:
        assert rel(xg[c], xo[c]) <= 1e-6, c
    to, _ = Q.target(nr, nz, er1, ez1, ers[:4], ezs[:4], sd)
    assert rel(tg, to) <= 1e-6


@pytest.mark.parametrize("mode", [1, 2])
def test_steps_converge_from_each_start(mode):
    P, cfg, pic = reactor()
    net = P.Cnn(cfg["nr"], cfg["nz"], batch=1, seed=1, device=DEV) if mode == 2 else None
    P.set_guess(pic, mode, net)
    g = O.Grid(cfg["nr"], cfg["nz"], cfg["R"], cfg["L"])

    def gauss():
        er, ez, _ = pic.fields()
        return O.gauss_residual(g, er, ez, pic.node_charge().cpu().numpy())

    G0 = gauss()
    used = []
    for _ in range(8):
        rc, st = pic.step(1)
        assert rc == 0 and st["converged"] == 1
        used.append(st["guess"])
    assert used[:3] == [0, 0, 0]
    assert all(u in (0, mode) for u in used[3:])
    # the start does not touch charge conservation (Gauss residual unchanged to
    # roundoff of the electron node charge)
    qs = np.max(np.abs(O.node_charge(g, -O.QE, pic.get_state(0))))
    assert np.max(np.abs(gauss() - G0)) <= 1e-12 * qs


def test_trained_start_gains_over_the_plain_start():
    """What the trained network gains: trained on the pairs a discharge
    generates, its start lowers the first Picard residual below those of the
    plain and the extrapolated starts on later steps, with at most the plain
    start's iteration count and charge conservation untouched."""
    from paper_2212_08836_gb300 import guess as GS
    P = M()
    cfg = P.small_reactor(np_init=40000)
    pic = P.Pic(cfg, device=DEV)
    pic.load_particles()
    pic.step(150)
    X, T = GS.collect(pic, 400)
    net = P.Cnn(cfg["nr"], cfg["nz"], batch=8, seed=0, device=DEV)
    loss, val, zero = GS.train(net, X, T, 2000)
    assert val < 0.5 * zero, (val, zero)
    r = GS.run_starts(pic, net, 120)
    fp, fe, fc = (r[k]["first_res_median"] for k in ("plain", "extrap", "cnn"))
    assert r["cnn"]["steps"] >= 110
    assert fc < 0.7 * fp and fc < 0.7 * fe, r
    assert r["cnn"]["picard_iters"] <= r["plain"]["picard_iters"] + 0.05, r


@pytest.mark.parametrize("nr,nz,batch", [(8, 12, 1), (13, 70, 2), (33, 65, 1)])
def test_forward_elementwise_within_bf16_bound(nr, nz, batch):
    """Every output element of the tensor-core forward pass against the oracle
    pass that rounds each hidden activation to bfloat16 as the kernels do
    (oracle.cnn.forward_bf16), within that pass's element-wise bound (FP32
    sums in any order, one bfloat16 step per rounding decision taken from a
    slightly different sum, carried through the later layers)."""
    net, ps, rng = setup(nr, nz, batch, 13)
    x = bf16(rng.normal(size=(batch, 14, nr + 1, nz + 1)))
    y = net.forward(torch.tensor(x, dtype=torch.float32, device=DEV)).cpu().numpy()
    for b in range(batch):
        ref, bound = Q.forward_bf16(ps, x[b])
        err = np.abs(y[b] - ref)
        assert np.all(err <= bound + 1e-30), float(np.max(err / np.maximum(bound, 1e-300)))
