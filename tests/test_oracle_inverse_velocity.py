"""Pins of the oracle pieces of the initial-velocity inverse problems (Sec. 5.2):

- the velocity-monitor mean of a hand-built configuration;
- the monitor loss gradient in v equals central differences (the loss is
  quadratic in v at fixed positions);
- dL/d(alpha) from the initial-state adjoint (chain rule through
  v_x0 = alpha (H0 - y)) equals central differences of the oracle's own
  trajectory loss, for tracked positions and for the monitors.
"""
import numpy as np
import pytest

import oracle
from paper_2507_04192_gb300 import inputs
from velocity_inverse_oracle import loss_and_v0_adjoint, observe, small_problem


def test_monitor_mean_by_hand():
    x = np.array([[0.1, 0.1], [0.15, 0.12], [0.5, 0.5], [0.2, 0.1]])
    v = np.array([[1.0, 2.0], [3.0, -2.0], [9.0, 9.0], [5.0, 0.0]])
    Q, cnt = oracle.monitor_means(x, v, [((0.05, 0.05), (0.2, 0.2)), ((0.6, 0.6), (0.7, 0.7))])
    assert list(cnt) == [3, 0]                       # the box is closed: (0.2, 0.1) is inside
    np.testing.assert_allclose(Q[0], [3.0, 0.0])
    np.testing.assert_allclose(Q[1], [0.0, 0.0])


def test_monitor_seed_is_the_gradient_in_v():
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, (200, 2))
    v = rng.normal(size=(200, 2))
    boxes = [((0.1, 0.1), (0.4, 0.3)), ((0.5, 0.5), (0.9, 0.8)), ((2.0, 2.0), (3.0, 3.0))]
    z = rng.normal(size=(3, 2))
    loss, g = oracle.monitor_loss_and_seed(x, v, boxes, z)
    assert loss > 0
    dv = rng.normal(size=v.shape)
    eps = 1e-3
    lp = oracle.monitor_loss_and_seed(x, v + eps * dv, boxes, z)[0]
    lm = oracle.monitor_loss_and_seed(x, v - eps * dv, boxes, z)[0]
    assert float((g * dv).sum()) == pytest.approx((lp - lm) / (2 * eps), rel=1e-9)


@pytest.mark.parametrize("kind", ["tracked", "monitors"])
def test_alpha_gradient_matches_central_differences(kind):
    w = small_problem(inputs, steps=120, frames=4)
    H0 = w.extras["H0"]
    prof = lambda a: inputs.velocity_profile_linear(w.x, a, H0)
    zx, zv = observe(w, prof(2.0))
    args = dict(zx=zx) if kind == "tracked" else dict(zv=zv)
    alpha = 1.2
    loss, lam_v0 = loss_and_v0_adjoint(w, prof(alpha), **args)
    assert loss > 0
    grad = float((lam_v0[:, 0] * (H0 - w.x[:, 1])).sum())
    # central differences agree to about 1e-9 here; an adjoint that linearises each
    # step about the wrong state of the trajectory is off by about 4e-7
    eps = 1e-4
    lp = loss_and_v0_adjoint(w, prof(alpha + eps), **args)[0]
    lm = loss_and_v0_adjoint(w, prof(alpha - eps), **args)[0]
    assert grad == pytest.approx((lp - lm) / (2 * eps), rel=2e-8)
    # and along a random direction of every particle's initial velocity
    dv = np.random.default_rng(5).normal(size=lam_v0.shape)
    lp = loss_and_v0_adjoint(w, prof(alpha) + eps * dv, **args)[0]
    lm = loss_and_v0_adjoint(w, prof(alpha) - eps * dv, **args)[0]
    assert float((lam_v0 * dv).sum()) == pytest.approx((lp - lm) / (2 * eps), rel=2e-8)
