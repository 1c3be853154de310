"""Host logic of the friction inversion (Sec. 5.3) and of the warm-start
features, checked on the CPU with a stand-in problem whose loss and gradient
are a known quadratic (the GPU adjoint is what the real problem supplies):

- the autograd wrapper hands the problem's gradient to torch unchanged;
- Adam with the decaying rate reaches the minimum, records the rate
  lr0 decay^k, stops at the error target on the masked segments, and keeps
  mu inside [0, 1] when the minimum lies outside;
- the relative error by hand;
- the network features are the tracks' displacements along the floor over the
  column width, flattened time-major, for one run and for a batch.
"""
import types

import numpy as np
import pytest
import torch

from paper_2507_04192_gb300 import inverse, warmstart


class Quadratic:
    """Stand-in problem: L(mu) = sum_s a_s (mu_s - m_s)^2."""

    def __init__(self, m, a):
        self.m, self.a = np.asarray(m, dtype=np.float64), np.asarray(a, dtype=np.float64)
        self.calls = 0

    def loss_and_grad(self, mu):
        self.calls += 1
        e = np.asarray(mu, dtype=np.float64) - self.m
        return float((self.a * e * e).sum()), 2.0 * self.a * e


def test_autograd_wrapper_returns_the_problem_gradient():
    prob = Quadratic([0.2, 0.5, 0.7], [1.0, 3.0, 0.5])
    mu = torch.tensor([0.4, 0.1, 0.9], dtype=torch.float64, requires_grad=True)
    loss = inverse.friction_loss(mu, prob)
    (2.0 * loss).backward()
    ref_loss, ref_g = prob.loss_and_grad(mu.detach().numpy())
    assert float(loss.detach()) == ref_loss
    np.testing.assert_array_equal(mu.grad.numpy(), 2.0 * ref_g)


def test_adam_reaches_the_minimum_with_the_decaying_rate():
    m = np.array([0.15, 0.3, 0.45, 0.6])
    prob = Quadratic(m, [1.0, 2.0, 0.5, 4.0])
    res = inverse.invert(prob, np.full(4, warmstart.UNIFORM_GUESS), mu_true=m, tol=0.01, max_iters=400)
    assert res.converged and res.iterations < 400
    assert inverse.relative_error(res.mu, m) <= 0.01
    lrs = [h["lr"] for h in res.history]
    np.testing.assert_allclose(lrs, 0.1 * 0.97 ** np.arange(len(lrs)), rtol=1e-12)
    assert prob.calls == res.iterations


def test_masked_error_target_and_the_clamp():
    # the last segment's minimum lies above 1: it stays clamped at 1, and the
    # error target counts only the masked segments
    m = np.array([0.2, 0.4, 1.3])
    prob = Quadratic(m, [1.0, 1.0, 1.0])
    mask = np.array([True, True, False])
    res = inverse.invert(prob, np.full(3, 0.35), mu_true=m, mask=mask, tol=0.02, max_iters=400)
    assert res.converged
    assert inverse.relative_error(res.mu, m, mask) <= 0.02
    assert res.mu[2] == 1.0
    res = inverse.invert(prob, np.full(3, 0.35), mu_true=None, max_iters=60)
    assert not res.converged and res.iterations == 60 and len(res.history) == 60
    assert res.mu.min() >= 0.0 and res.mu.max() <= 1.0


def test_per_segment_rates_follow_torch_adam():
    # one rate per segment takes Adam's update element by element: a uniform
    # array gives torch.optim.Adam's trajectory, and a segment with a tenfold
    # smaller rate moves tenfold less in the first step
    m = np.array([0.15, 0.3, 0.45, 0.6])
    prob = Quadratic(m, [1.0, 2.0, 0.5, 4.0])
    ref = inverse.invert(prob, np.full(4, 0.35), mu_true=None, max_iters=40)
    vec = inverse.invert(prob, np.full(4, 0.35), mu_true=None, max_iters=40, lr0=np.full(4, 0.1))
    np.testing.assert_allclose(vec.mu, ref.mu, rtol=0, atol=1e-12)
    np.testing.assert_allclose([h["lr"] for h in vec.history], [h["lr"] for h in ref.history], rtol=1e-12)
    one = inverse.invert(prob, np.full(4, 0.35), mu_true=None, max_iters=1, lr0=np.array([0.1, 0.01, 0.1, 0.1]))
    step = np.abs(one.mu - 0.35)
    np.testing.assert_allclose(step, [0.1, 0.01, 0.1, 0.1], rtol=1e-6)


def test_refine_rate_per_segment_from_held_out_error():
    net = types.SimpleNamespace(val_rmse_seg=np.array([0.001, 0.03, 0.5]))
    rates = warmstart.WarmStartNet.refine_rate(net)
    np.testing.assert_allclose(rates, [2e-3, 0.03, 0.1])
    assert warmstart.WarmStartNet.refine_rate(types.SimpleNamespace(val_rmse_seg=None)) == 0.1


def test_relative_error_by_hand():
    assert inverse.relative_error([1.0, 2.0, 2.0], [1.0, 2.0, 4.0]) == pytest.approx(2.0 / np.sqrt(21.0))
    assert inverse.relative_error([0.0, 2.0, 9.0], [1.0, 2.0, 4.0], np.array([True, True, False])) == \
        pytest.approx(1.0 / np.sqrt(5.0))


def test_features_are_scaled_floor_displacements():
    setup = warmstart.Setup(n_track=3, n_obs=2)
    w = types.SimpleNamespace(x=np.array([[0.1, 0.0], [0.2, 0.05], [0.3, 0.1], [0.4, 0.2]]),
                              extras={"track_ids": np.array([2, 0, 3]), "body_lo": (0.05, 0.0),
                                      "body_hi": (0.45, 0.3)})
    z = np.array([[[0.34, 0.1], [0.1, 0.0], [0.52, 0.2]],
                  [[0.38, 0.1], [0.18, 0.0], [0.6, 0.2]]])
    f = warmstart.features(setup, w, z)
    np.testing.assert_allclose(f, np.array([0.04, 0.0, 0.12, 0.08, 0.08, 0.2]) / 0.4, rtol=1e-6)
    assert f.dtype == np.float32 and f.shape == (setup.n_features,)
    fb = warmstart.features(setup, w, np.stack([z, z]))
    assert fb.shape == (2, setup.n_features)
    np.testing.assert_array_equal(fb[1], f)
