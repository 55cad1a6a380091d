"""Pins of the electrostatic oracle (oracle/es.py) against things other than
itself: the exact vacuum solution between the plates, Gauss's law through the
C oracle's own discrete divergence, and the discrete energy identity
W = 1/2 sum Q phi through the C oracle's field energy."""
import numpy as np

import oracle as O
from oracle import es as ES


def grid(nr=6, nz=9, R=0.05, L=0.03):
    return nr, nz, R / nr, L / nz, R, L


def test_vacuum_field_is_uniform():
    nr, nz, dr, dz, R, L = grid()
    phi0 = -123.0
    phi, er, ez = ES.solve(nr, nz, dr, dz, np.zeros((nr + 1) * (nz + 1)), phi0)
    assert np.max(np.abs(er)) <= 1e-12 * abs(phi0) / L
    np.testing.assert_allclose(ez, phi0 / L, rtol=1e-12)
    z = np.arange(nz + 1) * dz
    np.testing.assert_allclose(phi, np.outer(np.ones(nr + 1), phi0 * (1 - z / L)), atol=1e-10)


def test_gauss_law_through_the_c_oracle():
    nr, nz, dr, dz, R, L = grid(7, 11)
    g = O.Grid(nr, nz, R, L)
    rng = np.random.default_rng(2)
    Q = rng.normal(size=(nr + 1) * (nz + 1)) * 1e-12
    phi, er, ez = ES.solve(nr, nz, dr, dz, Q, 37.0)
    G = O.gauss_residual(g, er, ez, Q).reshape(nr + 1, nz + 1)
    assert np.max(np.abs(G[:nr, 1:nz])) <= 1e-10 * np.max(np.abs(Q))


def test_energy_identity_through_the_c_oracle():
    nr, nz, dr, dz, R, L = grid(5, 8)
    g = O.Grid(nr, nz, R, L)
    rng = np.random.default_rng(3)
    Q = np.zeros((nr + 1, nz + 1))
    Q[:nr, 1:nz] = rng.normal(size=(nr, nz - 1)) * 1e-12
    phi, er, ez = ES.solve(nr, nz, dr, dz, Q.ravel(), 0.0)
    W = O.field_energy(g, er, ez, np.zeros(nr * nz))
    assert abs(W - 0.5 * np.sum(Q * phi)) <= 1e-10 * abs(W)
