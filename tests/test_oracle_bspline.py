"""Pins of the oracle's quadratic B-spline (Sec. 2.1) against values and
identities fixed by the mathematics, not by the oracle itself."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bspline_values.txt")


def cardinal_bspline(k, t):
    """Cardinal B-spline of degree k on knots 0..k+1 by the Cox-de Boor recursion."""
    if k == 0:
        return 1.0 if 0.0 <= t < 1.0 else 0.0
    return (t * cardinal_bspline(k - 1, t) + (k + 1 - t) * cardinal_bspline(k - 1, t - 1.0)) / k


def cardinal_bspline_deriv(k, t):
    return cardinal_bspline(k - 1, t) - cardinal_bspline(k - 1, t - 1.0)


def test_golden_values():
    rows = np.loadtxt(GOLDEN, comments="#")
    for xi, val, der in rows:
        assert oracle.phi_bar(xi) == pytest.approx(val, abs=1e-15)
        assert oracle.dphi_bar(xi) == pytest.approx(der, abs=1e-15)


def test_matches_cox_de_boor():
    rng = np.random.default_rng(1)
    for xi in rng.uniform(-2.0, 2.0, 500):
        assert oracle.phi_bar(xi) == pytest.approx(cardinal_bspline(2, xi + 1.5), abs=1e-14)
        assert oracle.dphi_bar(xi) == pytest.approx(cardinal_bspline_deriv(2, xi + 1.5), abs=1e-14)


def test_partition_of_unity_and_moments():
    rng = np.random.default_rng(2)
    for u in rng.uniform(-3.0, 3.0, 300):
        ks = np.arange(np.floor(u) - 3, np.floor(u) + 4)
        w = np.array([oracle.phi_bar(u - k) for k in ks])
        dw = np.array([oracle.dphi_bar(u - k) for k in ks])
        assert w.sum() == pytest.approx(1.0, abs=1e-15)                 # partition of unity
        assert dw.sum() == pytest.approx(0.0, abs=1e-14)                # gradient sum zero
        assert (w * ks).sum() == pytest.approx(u, abs=1e-13)            # linear reproduction
        assert (w * (ks - u) ** 2).sum() == pytest.approx(0.25, abs=1e-13)  # D_p = dx^2/4 I
        assert (dw * ks).sum() == pytest.approx(1.0, abs=1e-13)         # sum x_i grad phi_i = 1


def test_continuity_at_knots():
    for xi in (0.5, 1.5, -0.5, -1.5):
        for f in (oracle.phi_bar, oracle.dphi_bar):
            assert f(xi - 1e-12) == pytest.approx(f(xi + 1e-12), abs=1e-11)
