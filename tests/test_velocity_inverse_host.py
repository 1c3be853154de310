"""Host logic of the initial-velocity inversion driver: the coordinate network's
gradient (central differences) and the Adam update (a quadratic's minimum)."""
import numpy as np
import pytest

from paper_2507_04192_gb300.velocity_inverse import Adam, CoordinateMLP


def test_coordinate_network_gradient_matches_central_differences():
    net = CoordinateMLP(seed=3)
    rng = np.random.default_rng(0)
    s = rng.uniform(0, 1, 64)
    gout = rng.normal(size=64)
    out, h = net.forward(s)
    g = net.backward(h, gout)
    p0 = net.flat()
    d = rng.normal(size=p0.size)
    eps = 1e-6
    net.set_flat(p0 + eps * d)
    fp = float((net.forward(s)[0] * gout).sum())
    net.set_flat(p0 - eps * d)
    fm = float((net.forward(s)[0] * gout).sum())
    net.set_flat(p0)
    assert float((g * d).sum()) == pytest.approx((fp - fm) / (2 * eps), rel=1e-6)
    assert net.n_params == 2 * 30 + 2 * (30 * 30 + 30) + 31


def test_adam_reaches_the_minimum_of_a_quadratic():
    opt = Adam(2, lr0=0.1, decay=1.0)
    p = np.array([3.0, -2.0])
    for _ in range(2000):
        p = opt.step(p, 2.0 * (p - np.array([0.5, 1.5])))
    np.testing.assert_allclose(p, [0.5, 1.5], atol=1e-3)
