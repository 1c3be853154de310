"""The shallow-water surface of Eq. shallow behind the dam-break validation
(Sec. 5.1) and the surface extraction from particles, checked on the CPU:

- the tip (y -> 0) advances at 2 sqrt(g H0) and the top of the rarefaction
  (y = H0) recedes at sqrt(g H0), the two edges of Ritter's solution;
- the area under the surface, the integral of x(y) over 0 <= y <= H0, stays
  L0 H0 at every time (the water's volume is conserved);
- the surface of a hand-built particle set.
"""
import numpy as np
import pytest

from paper_2507_04192_gb300 import validation


@pytest.mark.parametrize("L0,H0,g", [(1.0, 0.1, 9.8), (0.4, 0.25, 9.81)])
def test_shallow_water_surface_edges_and_volume(L0, H0, g):
    c0 = np.sqrt(g * H0)
    for t in (0.0, 0.1, 0.3, 0.7):
        x = lambda y: validation.shallow_water_x(y, t, length=L0, height=H0, g=g)
        assert float(x(0.0)) == pytest.approx(L0 + 2.0 * c0 * t, rel=1e-14)
        assert float(x(H0)) == pytest.approx(L0 - c0 * t, rel=1e-14)
        # the integrand has a sqrt(y) singularity in its derivative: integrate in s = sqrt(y), dy = 2 s ds
        s = np.linspace(0.0, np.sqrt(H0), 200001)
        f = x(s * s) * 2.0 * s
        area = float(np.sum(0.5 * (f[1:] + f[:-1]) * np.diff(s)))
        assert area == pytest.approx(L0 * H0, rel=1e-9)


def test_surface_of_a_hand_built_particle_set():
    x = np.array([[0.1, 0.05], [0.3, 0.01], [0.2, 0.2]])
    got = validation.surface_x(x, [0.0, 0.02, 0.1, 0.3])
    np.testing.assert_array_equal(got[:3], [0.3, 0.2, 0.2])
    assert np.isnan(got[3])
