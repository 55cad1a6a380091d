"""Pins of the oracle's RNG, particle loading (a1), null-collision MCC (a7)
and counting sort (a8).

Fixed independently of the oracle: Philox4x64-10 bit-for-bit against numpy's
own implementation; loading moments (total weight n0*pi*R^2*L, uniform node
density, Maxwellian second moments, zero net charge of the pairs); null-
collision statistics (Binomial candidate count, process fractions
nu_k/nu_max, exact threshold losses, equal ionization split, elastic recoil
mean 2m/M, isotropy, charge-exchange acceptance <g>/g_max for ions at rest);
the sort against numpy's stable argsort.
"""
import numpy as np
import pytest

import oracle as O

QE, ME, M_AR, KB = O.QE, O.ME, O.M_AR, O.KB


# -------------------------------------------------------------------- RNG
def test_philox4x64_matches_numpy_bit_for_bit():
    rng = np.random.default_rng(0)
    for _ in range(50):
        key = rng.integers(0, 2 ** 63, size=2, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
        ctr = rng.integers(1, 2 ** 63, size=4, dtype=np.uint64)
        mine = O.philox4x64(ctr, key)
        prev = ctr.copy()
        prev[0] -= np.uint64(1)  # numpy increments the counter before each block
        bg = np.random.Philox(key=key, counter=prev)
        np.testing.assert_array_equal(mine, bg.random_raw(4))


# ------------------------------------------------------------------- load
def test_load_moments_and_neutral_pairs():
    g = O.Grid(16, 24, 0.1, 0.03)
    n = 200000
    n0, te, ti = 1e15, 3.0, 0.026
    e, i = O.load(g, n, n0, te, ti, 7)
    # positions uniform in the logical box: chi^2 over cells
    counts = np.bincount(e["cell"], minlength=g.nr * g.nz)
    exp = n / (g.nr * g.nz)
    chi2 = np.sum((counts - exp) ** 2 / exp)
    dof = g.nr * g.nz - 1
    assert abs(chi2 - dof) < 5 * np.sqrt(2 * dof)
    # total weight: E = n0 pi R^2 L, relative std = 1/sqrt(3 n)
    tot = e["w"].sum()
    expect = n0 * np.pi * g.R ** 2 * g.L
    assert abs(tot / expect - 1) < 5 / np.sqrt(3 * n)
    # interior node density close to n0 (S1 volume 2 pi r_i dr dz)
    Q = O.node_charge(g, 1.0, e).reshape(g.nr + 1, g.nz + 1)
    ri = np.arange(g.nr + 1) * g.dr
    V = 2 * np.pi * ri[1:-1, None] * g.dr * g.dz
    dens = Q[1:-1, 1:-1] / V
    assert abs(dens.mean() / n0 - 1) < 0.01
    # Maxwellian second moments per component
    for sp, T, m in ((e, te, ME), (i, ti, M_AR)):
        for k in ("vr", "vt", "vz"):
            s2 = np.mean(sp[k] ** 2)
            target = T * QE / m
            assert abs(s2 / target - 1) < 5 * np.sqrt(2.0 / n)
            assert abs(np.mean(sp[k])) < 5 * np.sqrt(target / n)
    # pairs: identical positions and weights -> zero node charge
    Qe = O.node_charge(g, -QE, e)
    Qi = O.node_charge(g, QE, i)
    assert np.max(np.abs(Qe + Qi)) <= 1e-15 * np.max(np.abs(Qe))


# -------------------------------------------------------------------- MCC
def _beam(n, eps_ev, cap_factor=2, seed=0):
    cap = int(n * cap_factor)
    e = O.empty_species(cap)
    i = O.empty_species(cap)
    rng = np.random.default_rng(seed)
    v = np.sqrt(2 * eps_ev * QE / ME)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    e["cell"][:n] = rng.integers(0, 100, size=n)
    e["a"][:n], e["b"][:n] = rng.random(n), rng.random(n)
    e["vr"][:n], e["vt"][:n], e["vz"][:n] = v * d
    e["w"][:n] = 1.0 + rng.random(n)
    e["id"][:n] = np.arange(n)
    return e, i


def test_mcc_candidates_process_fractions_and_energetics():
    n = 200000
    eps = 50.0
    ng = 1e21
    dt = 1e-10
    e, i = _beam(n, eps)
    e0 = {k: v.copy() for k, v in e.items()}
    v = np.sqrt(2 * eps * QE / ME)
    nu = {k: ng * f(eps) * v for k, f in (("el", O.sigma_el), ("ex", O.sigma_ex),
                                          ("iz", O.sigma_iz))}
    numax = 1.5 * sum(nu.values())
    pnull = 0.3
    rc, ne, ni, nid, counts, _ = O.mcc(5, 17, ng, 300.0, numax, pnull, 0.0, 1.0, e, n, 0, i,
                                       (n, 0))
    assert rc == 0
    cand = counts[0]
    assert abs(cand - n * pnull) < 5 * np.sqrt(n * pnull * (1 - pnull))
    for k, idx in (("el", 1), ("ex", 2), ("iz", 3)):
        p = nu[k] / numax
        assert abs(counts[idx] - cand * p) < 5 * np.sqrt(cand * p * (1 - p)) + 1
    # ionization created pairs at the parent's position with its weight
    niz = counts[3]
    assert ne == n + niz and ni == niz and nid == (n + niz, niz)
    newe = slice(n, n + niz)
    assert np.array_equal(e["id"][newe], np.arange(n, n + niz, dtype=np.uint32))
    for k in ("cell", "a", "b", "w"):
        np.testing.assert_array_equal(e[k][newe], i[k][:niz])
    # exact energy bookkeeping per process
    E1 = 0.5 * ME * (e["vr"] ** 2 + e["vt"] ** 2 + e["vz"] ** 2) / QE
    changed = np.where(np.abs(E1[:n] - eps) > 1e-9)[0]
    ex_like = np.isclose(E1[changed], eps - 11.5, rtol=1e-12)
    iz_like = np.isclose(E1[changed], 0.5 * (eps - 15.76), rtol=1e-12)
    assert ex_like.sum() == counts[2]
    assert iz_like.sum() == niz
    np.testing.assert_allclose(E1[newe], 0.5 * (eps - 15.76), rtol=1e-12)
    # elastic: eps'/eps = 1 - 2 m/M (1 - cos chi), mean 1 - 2m/M for isotropic scattering
    el = changed[~(ex_like | iz_like)]
    assert len(el) == counts[1]
    ratio = E1[el] / eps
    mu = 2 * ME / M_AR
    assert np.all(ratio <= 1.0 + 1e-15) and np.all(ratio >= 1 - 2 * mu - 1e-15)
    assert abs(np.mean(1 - ratio) - mu) < 5 * mu / np.sqrt(3 * len(el))
    # isotropy of the new directions (elastic + excitation + ionization parents)
    vv = np.stack([e["vr"][changed], e["vt"][changed], e["vz"][changed]])
    nn = vv / np.linalg.norm(vv, axis=0)
    m = len(changed)
    assert np.all(np.abs(nn.mean(axis=1)) < 5 / np.sqrt(3 * m))
    assert abs(np.mean(nn[2] ** 2) - 1 / 3) < 5 * np.sqrt(4 / 45 / m)
    # new ions: 300 K Maxwellian
    vth2 = KB * 300.0 / M_AR
    for k in ("vr", "vt", "vz"):
        assert abs(np.mean(i[k][:niz] ** 2) / vth2 - 1) < 5 * np.sqrt(2.0 / niz)
    # untouched particles keep their state bit-for-bit
    same = np.setdiff1d(np.arange(n), changed)
    for k in ("vr", "vt", "vz"):
        np.testing.assert_array_equal(e[k][same], e0[k][same])


def test_mcc_thresholds_and_numax_bound():
    assert O.sigma_ex(11.5) == 0.0 and O.sigma_ex(11.6) > 0
    assert O.sigma_iz(15.76) == 0.0 and O.sigma_iz(15.9) > 0
    ng = 4.8e20
    numax = O.numax_e(ng)
    rng = np.random.default_rng(1)
    for eps in rng.uniform(0.01, 1000.0, size=2000):
        v = np.sqrt(2 * eps * QE / ME)
        tot = O.sigma_el(eps) + O.sigma_ex(eps) + O.sigma_iz(eps)
        assert ng * tot * v <= numax


def test_ion_charge_exchange_acceptance_and_velocity():
    n = 200000
    tg = 300.0
    i = O.empty_species(n)
    e = O.empty_species(1)
    i["cell"][:] = 3
    i["id"][:] = np.arange(n)
    i["w"][:] = 1.0
    vth = np.sqrt(KB * tg / M_AR)
    gmax = 8 * vth
    rc, ne, ni, _, counts, _ = O.mcc(9, 4, 1e21, tg, 1.0, 0.0, 1.0, gmax, e, 0, n, i, (0, n))
    assert rc == 0 and counts[4] == n
    mean_g = np.sqrt(8 * KB * tg / (np.pi * M_AR))
    p = mean_g / gmax
    assert abs(counts[5] - n * p) < 5 * np.sqrt(n * p * (1 - p))
    moved = i["vr"] != 0
    assert moved.sum() == counts[5]
    # accepted neutrals are speed-biased (weight g): <v^2> = 4 vth^2 for ions at rest
    v2 = i["vr"][moved] ** 2 + i["vt"][moved] ** 2 + i["vz"][moved] ** 2
    assert abs(np.mean(v2) / (4 * vth ** 2) - 1) < 0.02


# ------------------------------------------------------------------- sort
def test_counting_sort_matches_numpy_stable_argsort():
    g = O.Grid(8, 10, 0.1, 0.03)
    rng = np.random.default_rng(3)
    n = 5000
    sp = {k: rng.random(n) for k in ("a", "b", "vr", "vt", "vz", "w")}
    sp["cell"] = rng.integers(-1, g.nr * g.nz, size=n).astype(np.int32)
    sp["id"] = np.arange(n, dtype=np.uint32)
    ref = {k: v.copy() for k, v in sp.items()}
    m = O.sort(g, sp, n)
    keep = ref["cell"] >= 0
    order = np.argsort(ref["cell"][keep], kind="stable")
    assert m == keep.sum()
    for k in ref:
        np.testing.assert_array_equal(sp[k][:m], ref[k][keep][order])
