"""Surface-mode dispersion (Sec. 3.1) measured with the GPU code.

A slab of electrons at n0 = 1e16 m^-3 between matrix sheaths of 1.8 mm (ions
fixed), 64x128 mesh, gets an axial velocity kick u0 J_0(chi_01 r / R),
uniform in z, which excites the symmetric surface mode at k = chi_01 / R (the
plasma series resonance branch).  The ringing of the m = 1 Fourier-Bessel
coefficient of E_z in the powered sheath, minus the same run without the kick,
gives its frequency.  Checked against the dispersion relations in the oracle
(oracle/fb.py): eq3_2 for the electrostatic model and eq3_1 for the
electromagnetic one, to 15 %, and the electromagnetic lowering of the
frequency (the long-wavelength knee of the symmetric branch), which the
theory puts at 19 %, to 5 % of the ratio.  The absolute values come out
about 10 % low: the Maxwellian electrons reach a few Debye lengths into the
loaded sheaths, so the vacuum gap is narrower than the loaded width.  The
antisymmetric branch is checked at m = 2 from the difference of the two
sheaths (test_antisymmetric_surface_mode)."""
import numpy as np
import pytest
from scipy import special as sp

import oracle as O
from oracle import fb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as G
    G.build()


def test_symmetric_surface_mode_and_its_electromagnetic_knee():
    from paper_2212_08836_gb300 import dispersion as D
    n0, s, L, R = 1e16, 1.8e-3, 0.03, 0.1
    wpe = np.sqrt(n0 * O.QE ** 2 / (O.EPS0 * O.ME))
    k = sp.jn_zeros(0, 1)[0] / R
    theory = {"es": fb.es_omega(k, wpe, s, L / 2 - s) / (2 * np.pi),
              "em": fb.em_omega(k, wpe, s, L / 2 - s, 1.0 / np.sqrt(O.EPS0 * O.MU0)) / (2 * np.pi)}
    got = {}
    for model in ("es", "em"):
        base = D.ring(model=model, m=1, steps=700, u0=0.0, n0=n0, sheath=s, L=L, R=R, device=DEV)
        r = D.ring(model=model, m=1, steps=700, u0=1e5, n0=n0, sheath=s, L=L, R=R, device=DEV,
                   base=base["series"])
        got[model] = r["freq"]
        assert abs(got[model] / theory[model] - 1.0) < 0.15, (model, got, theory)
    ratio, ratio_th = got["em"] / got["es"], theory["em"] / theory["es"]
    assert ratio_th < 0.85  # the knee is a sizeable effect at this k
    assert abs(ratio / ratio_th - 1.0) < 0.05, (ratio, ratio_th)


def test_antisymmetric_surface_mode():
    """The antisymmetric branch: a kick of opposite sign in the two halves of
    the gap, the m = 2 coefficient of E_z taken as half the difference of the
    two sheaths (the symmetric mode cancels in it).  At k = chi_02 / R (the
    perturbed potential vanishes on the side wall) eq3_2 and eq3_1 give 216
    and 214 MHz: the antisymmetric branch barely feels the electromagnetic
    terms at this size, and the two models must agree with each other (to 3 %)
    and with the theory (to 15 %).  The kick also excites the loaded slab's
    own oscillation near 135 MHz (present in every run of this slab, kicked
    or not), so the peak is searched above 160 MHz, a band that holds the
    symmetric m = 2 mode (306-333 MHz) as well: a wrong symmetry fails.  (At
    m = 1 the antisymmetric branch, near 103 MHz, lies under that line.)"""
    from paper_2212_08836_gb300 import dispersion as D
    n0, s, L, R, m = 1e16, 1.8e-3, 0.03, 0.1, 2
    wpe = np.sqrt(n0 * O.QE ** 2 / (O.EPS0 * O.ME))
    k = sp.jn_zeros(0, m)[m - 1] / R
    c = 1.0 / np.sqrt(O.EPS0 * O.MU0)
    theory = {"es": fb.es_omega(k, wpe, s, L / 2 - s, "antisymmetric") / (2 * np.pi),
              "em": fb.em_omega(k, wpe, s, L / 2 - s, c, "antisymmetric") / (2 * np.pi)}
    got = {}
    for model in ("es", "em"):
        kw = dict(model=model, mode="antisymmetric", m=m, steps=700, n0=n0, sheath=s, L=L, R=R,
                  device=DEV)
        base = D.ring(u0=0.0, **kw)
        r = D.ring(u0=1e5, base=base["series"], band=(160e6, 600e6), **kw)
        got[model] = r["freq"]
        assert abs(got[model] / theory[model] - 1.0) < 0.15, (model, got, theory)
    ratio, ratio_th = got["em"] / got["es"], theory["em"] / theory["es"]
    assert abs(ratio / ratio_th - 1.0) < 0.03, (ratio, ratio_th)
