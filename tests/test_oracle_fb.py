"""Pins of the Fourier-Bessel decomposition (App. A, Eq. A2) and of the
surface-mode dispersion relations (Sec. 3.1) in oracle/fb.py: closed-form
Fourier-Bessel coefficients, the orthogonality of the basis, the plasma
series resonance and surface-plasmon limits, and the electrostatic limit of
the electromagnetic relation as c grows."""
import numpy as np
from scipy import special as sp

from oracle import fb

R = 0.1


def test_single_mode_gives_a_unit_coefficient():
    for alpha in (0, 1):
        chi = sp.jn_zeros(alpha, 6)
        r, _ = fb.basis_points(256, R, alpha)
        for k in range(6):
            c = fb.coefficients(sp.jv(alpha, chi[k] * r / R), 256, R, alpha, 6)
            e = np.zeros(6)
            e[k] = 1.0
            assert np.max(np.abs(c - e)) < 2e-3, (alpha, k, c)


def test_constant_alpha0_closed_form_and_second_order():
    chi = sp.jn_zeros(0, 5)
    exact = 2.0 / (chi * sp.j1(chi))
    errs = []
    for nr in (64, 256):
        errs.append(np.max(np.abs(fb.coefficients(np.ones(nr + 1), nr, R, 0, 5) - exact)))
    assert errs[1] < errs[0] / 12 and errs[1] < 2e-3, errs


def test_linear_alpha1_closed_form():
    """f = r/R with alpha = 1: c_m = 2 J_2(chi) / (chi J_0(chi)^2)."""
    chi = sp.jn_zeros(1, 5)
    exact = 2.0 * sp.jv(2, chi) / (chi * sp.j0(chi) ** 2)
    nr = 400
    r, _ = fb.basis_points(nr, R, 1)
    c = fb.coefficients(r / R, nr, R, 1, 5)
    np.testing.assert_allclose(c, exact, rtol=2e-3, atol=1e-5)


WPE, S, D = 5.64e9, 1.8e-3, 13.2e-3


def test_es_symmetric_mode_cuts_off_at_the_series_resonance():
    w = fb.es_omega(1e-3, WPE, S, D)
    np.testing.assert_allclose(w, WPE * np.sqrt(S / (S + D)), rtol=1e-5)


def test_es_modes_tend_to_the_surface_plasmon():
    for mode in ("symmetric", "antisymmetric"):
        np.testing.assert_allclose(fb.es_omega(1e5, WPE, S, D, mode), WPE / np.sqrt(2),
                                   rtol=1e-8)


def test_es_antisymmetric_mode_is_acoustic_at_small_k():
    """tanh(kd) ~ kd: omega ~ wpe sqrt(k d s) for k s, k d << 1."""
    k = 0.01
    np.testing.assert_allclose(fb.es_omega(k, WPE, S, D, "antisymmetric"),
                               WPE * np.sqrt(k * D * k * S), rtol=1e-3)


def test_em_relation_tends_to_the_es_one_as_c_grows():
    for mode in ("symmetric", "antisymmetric"):
        for k in (20.0, 80.0, 300.0):
            es = fb.es_omega(k, WPE, S, D, mode)
            errs = [abs(fb.em_omega(k, WPE, S, D, c, mode) / es - 1) for c in (3e9, 3e11)]
            assert errs[1] < 1e-5 and errs[1] <= errs[0] + 1e-12, (mode, k, errs)


def test_em_symmetric_mode_drops_below_the_es_one_at_long_wavelength():
    """The knee of the electromagnetic symmetric branch: at k = 10 /m with the
    real speed of light the frequency is far below the ES cut-off."""
    k = 10.0
    assert fb.em_omega(k, WPE, S, D, 2.998e8) < 0.6 * fb.es_omega(k, WPE, S, D)
