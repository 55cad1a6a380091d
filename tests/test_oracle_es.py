"""Pins of the electrostatic oracle (oracle/es.py) against things other than
itself: the exact vacuum solution between the plates, Gauss's law through the
C oracle's own discrete divergence, and the discrete energy identity
W = 1/2 sum Q phi through the C oracle's field energy."""
import numpy as np
import pytest

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


# ---- the axial port of the electrostatic model (Sec. 2.2): the disc r <= r_p
# powered, the port's opening at the coaxial line's potential, side wall grounded

@pytest.mark.parametrize("xa", [0, 3])
def test_port_solve_keeps_gauss_law_through_the_c_oracle(xa):
    nr, nz, dr, dz, R, L = grid(12, 10, 0.1, 0.03)
    dr = R / (nr + xa)
    g = O.Grid(nr, nz, R, L, xa)
    rng = np.random.default_rng(4)
    Q = rng.normal(size=(nr + 1) * (nz + 1)) * 1e-12
    phi, er, ez = ES.solve(nr, nz, dr, dz, Q, 55.0, xa=xa, port=7)
    G = O.gauss_residual(g, er, ez, Q).reshape(nr + 1, nz + 1)
    assert np.max(np.abs(G[:nr, 1:nz])) <= 1e-10 * np.max(np.abs(Q))


def test_port_boundary_is_the_coaxial_tem_field():
    """Along the port's opening r E_r is the TEM constant phi0 / ln(R / r_p) (to
    the mesh's O(dr^2 / r^2)), the electrode disc is an equipotential (E_r = 0
    on it) and the grounded side wall carries no E_z."""
    nr, nz, dr, dz, R, L = grid(40, 12, 0.1, 0.03)
    ip, phi0 = 24, 80.0
    _, er, ez = ES.solve(nr, nz, dr, dz, np.zeros((nr + 1) * (nz + 1)), phi0, port=ip)
    Er0 = er.reshape(nr, nz + 1)[:, 0]
    rc = (np.arange(nr) + 0.5) * dr
    tem = phi0 / np.log(R / (ip * dr))
    np.testing.assert_allclose(rc[ip:] * Er0[ip:], tem, rtol=2e-3)
    assert np.max(np.abs(Er0[:ip])) == 0.0
    assert np.max(np.abs(ez.reshape(nr + 1, nz)[nr])) == 0.0


def test_port_field_near_the_axis_is_the_plate_field():
    """More than three gaps inside the electrode's rim the vacuum field is that
    of two infinite plates, phi0 / L, up to the rim's exp(-pi d / L) influence."""
    nr, nz, dr, dz, R, L = grid(48, 12, 0.16, 0.03)
    ip, phi0 = 36, -60.0           # r_p = 0.12 m = 4 L
    _, er, ez = ES.solve(nr, nz, dr, dz, np.zeros((nr + 1) * (nz + 1)), phi0, port=ip)
    Ez = ez.reshape(nr + 1, nz)
    d = ip * dr - 6 * dr            # distance of the outermost node checked from the rim
    assert d / L >= 3.0
    np.testing.assert_allclose(Ez[:7], phi0 / L, rtol=5e-4)
