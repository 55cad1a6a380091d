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


@pytest.mark.parametrize("precision,graphs", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_substep_histogram_counts_every_push(precision, graphs):
    """Every particle of a state-writing pass lands in one bin, and the bins
    weighted by their sub-step counts give the step's accepted sub-steps.
    With graph replay the histogram is switched on after the passes have been
    captured with it off: the replayed speculative passes must still count."""
    M = P()
    cfg = M.small_reactor(np_init=20000, mcc_on=1, precision=precision)
    pic = M.Pic(cfg, device=DEV, stream=torch.cuda.Stream(device=DEV) if graphs else None)
    M.set_graphs(pic, bool(graphs))
    pic.load_particles()
    pic.step(2)
    assert pic.substep_histogram(1).sum() == 0  # off until enabled
    tot_n = tot_sub = 0
    for _ in range(3):
        n = sum(pic.view()["n"])
        rc, st = pic.step(1, check=False)
        assert rc in (0, M.PIC_E_SUBSTEP)
        tot_n += n
        tot_sub += st["substeps"]
    h = pic.substep_histogram(0)
    assert int(h.sum()) == tot_n
    w = int((np.arange(16, dtype=np.uint64) + 1) @ h)
    # bin 0 also holds particles absorbed before a first sub-step, bin 15 16 or more
    assert abs(w - tot_sub) <= 1e-3 * tot_sub + 64 * int(h[15])
    assert h[0] > 0.5 * h.sum() and h[1] > 0
    pic.step(1)
    assert np.array_equal(pic.substep_histogram(-1), h)  # stopped counting


@pytest.mark.parametrize("precision,xa,ring", [(0, 0, 0), (1, 0, 0), (0, 3, 0), (0, 0, 4)])
def test_energies_match_oracle(precision, xa, ring):
    """Row a9: pic_diag's kinetic energy per species and field energy against
    the oracle's sums on the same state (fields, particles); FP64 sums of the
    same values, so they agree to rounding of the summation order."""
    M = P()
    kw = dict(np_init=20000, mcc_on=0, axis_cells=xa, precision=precision)
    if ring:
        kw.update(ring_cells=ring, eps_ring=4.0)
    cfg = M.small_reactor(**kw)
    pic = M.Pic(cfg, device=DEV)
    g = O.Grid(cfg["nr"], cfg["nz"], cfg["R"], cfg["L"], xa=xa, nd=ring,
               erd=4.0 if ring else 1.0)
    e, i = O.load(g, 20000, 1e15, 3.0, 0.026, 5)
    if precision == 1:
        for sp in (e, i):
            for k in ("a", "b", "vr", "vt", "vz", "w"):
                sp[k] = sp[k].astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(2)
    er = rng.normal(size=g.n_er) * 3e3
    ez = rng.normal(size=g.n_ez) * 3e3
    h = rng.normal(size=cfg["nr"] * cfg["nz"]) * 5.0
    pic.set_state([e, i], er=er, ez=ez, h=h)
    d = pic.diag()
    for s, (sp, m) in enumerate(((e, O.ME), (i, O.M_AR))):
        ref = O.kinetic_energy(m, sp)
        assert abs(d["kinetic"][s] - ref) <= 1e-12 * ref, (s, d["kinetic"][s], ref)
    ref_f = O.field_energy(g, er, ez, h)
    assert abs(d["field"] - ref_f) <= 1e-12 * ref_f, (d["field"], ref_f)


def _dual_volume(g):
    """Node dual volumes on the uniform mesh, written from their definition:
    the ring between the neighbouring cell-centre radii (the axis disc, the
    half ring at r = R) times dz (half on the electrodes)."""
    dr, dz = g.R / g.nr, g.L / g.nz
    rc = (np.arange(g.nr) + 0.5) * dr
    lo = np.concatenate([[0.0], rc])
    hi = np.concatenate([rc, [g.R]])
    ring = np.pi * (hi ** 2 - lo ** 2)
    zext = np.full(g.nz + 1, dz)
    zext[0] = zext[-1] = 0.5 * dz
    return ring, ring[:, None] * zext[None, :]


@pytest.mark.parametrize("precision", [0, 1])
def test_averaged_density_and_ion_flux_match_their_definitions(precision):
    """pic_diag_get(DENSITY_AVG) after k steps equals the mean over those steps
    of the oracle's w S1 x S1 node sums of the states after each step divided
    by the dual volume; ION_FLUX_AVG equals the ions' wall tally gained on each
    electrode node over the window / (e dt k x its electrode ring)."""
    M = P()
    cfg = M.small_reactor(np_init=20000, volt=200.0, precision=precision, gas_pressure=5.0)
    pic = M.Pic(cfg, device=DEV)
    pic.load_particles()
    pic.step(5)
    g = O.Grid(cfg["nr"], cfg["nz"], cfg["R"], cfg["L"])
    ring, vol = _dual_volume(g)
    pic.diag_average(True)
    w0 = pic.wall_charge()[1]
    acc = np.zeros((2, g.nr + 1, g.nz + 1))
    k = 4
    for _ in range(k):
        pic.step(1)
        for s in range(2):
            st = pic.get_state(s)
            st = {kk: (v.astype(np.float64) if v.dtype == np.float32 else v) for kk, v in st.items()}
            acc[s] += O.node_charge(g, 1.0, st).reshape(g.nr + 1, g.nz + 1)
    dens = pic.diag_get(M.PIC_DIAG_DENSITY_AVG)
    ref = acc / (k * vol)
    np.testing.assert_allclose(dens, ref, rtol=1e-12, atol=1e-12 * ref.max())
    w1 = pic.wall_charge()[1]
    flux = pic.diag_get(M.PIC_DIAG_ION_FLUX_AVG)
    for e, key in enumerate(("z0", "zl")):
        fref = (w1[key] - w0[key]) / (O.QE * cfg["dt"] * k * ring)
        np.testing.assert_allclose(flux[e], fref, rtol=1e-12, atol=1e-12 * max(abs(fref).max(), 1.0))
    assert list(pic.diag_get(M.PIC_DIAG_COUNTS)[2:]) == [pic.view()["step"], k]


@pytest.mark.parametrize("precision,ring", [(0, 0), (1, 0), (0, 4)])
def test_continuity_residual_per_step(precision, ring):
    """The per-node charge balance of every committed step (drive, collisions,
    wall absorption, sticking on the ring's face): the particles' node charge
    change plus the wall tallies' change plus the net crossed charge out of the
    node's dual cell is zero to rounding (FP64: 1e-12, FP32 particles: 1e-6 of
    the charge of a cell's electrons)."""
    M = P()
    kw = dict(np_init=20000, volt=300.0, precision=precision, gas_pressure=5.0)
    if ring:
        kw.update(ring_cells=ring, eps_ring=4.0)
    cfg = M.small_reactor(**kw)
    pic = M.Pic(cfg, device=DEV)
    pic.load_particles()
    pic.step(3)
    pic.diag_average(True)
    with pytest.raises(M.PicError):
        pic.diag_get(M.PIC_DIAG_CONTINUITY)
    q_scale = O.QE * float(np.max(pic.get_state(0)["w"])) * 20
    absorbed = 0
    for _ in range(4):
        rc, st = pic.step(1, check=False)
        absorbed += st["absorbed"]
        res = pic.diag_get(M.PIC_DIAG_CONTINUITY)
        assert np.max(np.abs(res)) <= (1e-12 if precision == 0 else 1e-6) * q_scale
    assert absorbed > 0


def test_fp64_fma_probe_reports_a_plausible_peak():
    """pic_probe_dfma (the FP64 roofline's denominator): independent FMA chains
    on every SM; the rate lies between a tenth of and twice the GB300 unit
    count (304 DFMA per cycle at 2.07 GHz = 1.26 TFLOP/s), and a longer run
    takes proportionally longer."""
    M = P()
    s1, tf1 = M.probe_dfma(4, 1 << 12)
    s2, tf2 = M.probe_dfma(4, 1 << 14)
    assert 0.126 < tf2 < 2.52, tf2
    assert 2.0 < s2 / s1 < 8.0, (s1, s2)


@pytest.mark.parametrize("precision", [0, 1])
def test_push_timing_under_graph_replay(precision):
    """pic_profile's push timing while the Picard passes replay from captured
    graphs (the benchmark's configuration): every step completes, and the
    pushes of the replayed passes are timed (a positive total over the
    expected number of launches)."""
    M = P()
    cfg = M.small_reactor(np_init=20000, volt=200.0, precision=precision)
    pic = M.Pic(cfg, device=DEV, stream=torch.cuda.Stream(device=DEV))
    M.set_graphs(pic, True)
    pic.load_particles()
    pic.profile(True)
    pic.step(3)
    pic.profile(True)
    iters = 0
    for _ in range(3):
        rc, st = pic.step(1)
        assert rc == 0
        iters += st["picard_iters"]
    ms, nl = pic.profile_read()
    assert ms > 0.0
    assert nl >= 2 * iters
