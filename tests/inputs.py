"""Seeded synthetic inputs shared by the oracle pins and the GPU parity tests.

Holds none of the method's arithmetic: only numpy random draws shaped like the
particle store (cell index, offsets in the cell, velocities, weight, id) and the
Yee field arrays (E_r on nr x (nz+1) edges, E_z on (nr+1) x nz edges).
"""
import numpy as np

QE = 1.602176634e-19
ME = 9.1093837015e-31
M_AR = 39.948 * 1.66053906660e-27


def particles(nr, nz, n, seed, vth, wmean=1e6, sorted_=True, cells=None, edge_frac=0.0):
    """n particles in random cells (or the given ``cells``), offsets in [0,1),
    Maxwellian-like velocities of scale ``vth``; weights around ``wmean``.
    ``edge_frac`` of them are put exactly on a cell face (a or b in {0, 1})."""
    rng = np.random.default_rng(seed)
    if cells is None:
        cells = rng.integers(0, nr * nz, size=n)
    cells = np.asarray(cells, dtype=np.int32)
    if sorted_:
        cells = np.sort(cells)
    a = rng.random(n)
    b = rng.random(n)
    if edge_frac > 0:
        k = int(edge_frac * n)
        idx = rng.choice(n, size=k, replace=False)
        which = rng.integers(0, 4, size=k)
        a[idx[which == 0]] = 0.0
        a[idx[which == 1]] = 1.0
        b[idx[which == 2]] = 0.0
        b[idx[which == 3]] = 1.0
    v = rng.normal(size=(3, n)) * vth
    w = wmean * (0.5 + rng.random(n))
    return {
        "cell": cells,
        "a": a,
        "b": b,
        "vr": v[0].copy(),
        "vt": v[1].copy(),
        "vz": v[2].copy(),
        "w": w,
        "id": np.arange(n, dtype=np.uint32),
    }


def fields(nr, nz, seed, scale):
    """Random Er (nr x (nz+1)) and Ez ((nr+1) x nz) edge fields, flattened."""
    rng = np.random.default_rng(seed)
    er = rng.normal(size=nr * (nz + 1)) * scale
    ez = rng.normal(size=(nr + 1) * nz) * scale
    return er, ez


def smooth_fields(nr, nz, seed, scale):
    """Smooth random edge fields (a few low Fourier modes)."""
    rng = np.random.default_rng(seed)
    ir = (np.arange(nr) + 0.5)[:, None] / nr
    jr = np.arange(nz + 1)[None, :] / nz
    iz = np.arange(nr + 1)[:, None] / nr
    jz = (np.arange(nz) + 0.5)[None, :] / nz
    er = np.zeros((nr, nz + 1))
    ez = np.zeros((nr + 1, nz))
    for _ in range(4):
        kx, ky = rng.integers(1, 4, size=2)
        ph = rng.random(2) * 6.283
        c = rng.normal(size=2) * scale
        er += c[0] * np.sin(np.pi * kx * ir + ph[0]) * np.cos(np.pi * ky * jr + ph[1])
        ez += c[1] * np.cos(np.pi * kx * iz + ph[0]) * np.sin(np.pi * ky * jz + ph[1])
    return er.ravel(), ez.ravel()
