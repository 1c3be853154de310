"""Pins of the FP64 oracle of the warm-start network (oracle/mlp.py).

The rounding helper against torch's bfloat16 cast (round to nearest even) and
hand-worked ties; GELU against torch's exact-erf GELU and its odd-part identity;
the loss gradient against central finite differences with rounding off; a
one-layer network against its closed form; with rounding on, the values the
tensor cores are fed are bfloat16: the loss and every gradient depend on the
weights and on the input only through their bfloat16 values, the hidden
activations are bfloat16 numbers, and the weight gradients depend on the output
error only through its bfloat16 value.
"""
import numpy as np
import pytest
import torch

from oracle import mlp


def test_bf16_rounding_is_round_to_nearest_even():
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.standard_normal(4096) * 10.0 ** rng.integers(-6, 6, 4096), [0.0, -0.0, 1e-40]])
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(a), ref)
    # ties: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 (even mantissa: 1);
    # 1 + 3 2^-8 halfway between 1 + 2^-7 and 1 + 2^-6 (even: 1 + 2^-6)
    assert mlp.bf16(np.array([1 + 2.0 ** -8]))[0] == 1.0
    assert mlp.bf16(np.array([1 + 3 * 2.0 ** -8]))[0] == 1 + 2.0 ** -6
    assert mlp.bf16(np.array([-(1 + 3 * 2.0 ** -8)]))[0] == -(1 + 2.0 ** -6)


def test_gelu_exact_erf_form():
    z = np.linspace(-6, 6, 241)
    ref = torch.nn.functional.gelu(torch.tensor(z, dtype=torch.float64), approximate="none").numpy()
    np.testing.assert_allclose(mlp.gelu(z), ref, rtol=0, atol=1e-14)
    # Phi(z) + Phi(-z) = 1  =>  gelu(z) - gelu(-z) = z
    np.testing.assert_allclose(mlp.gelu(z) - mlp.gelu(-z), z, rtol=0, atol=1e-14)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, rtol=0, atol=1e-8)


def test_one_layer_network_is_a_scaled_sigmoid_of_an_affine_map():
    rng = np.random.default_rng(1)
    W, b = rng.standard_normal((8, 16)), rng.standard_normal(8)
    x = rng.standard_normal((5, 16))
    y, _, _ = mlp.forward(mlp.pack([(W, b)]), [16, 8], x, 0.1, 0.6, bf16_round=False)
    ref = 0.1 + 0.5 * torch.sigmoid(torch.tensor(x @ W.T + b)).numpy()
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-14)
    # zero weights: the middle of the output range
    y0, _, _ = mlp.forward(np.zeros(8 * 16 + 8), [16, 8], x, 0.1, 0.6)
    np.testing.assert_allclose(y0, 0.35, rtol=0, atol=0)


@pytest.mark.parametrize("widths", [[16, 24, 8], [8, 16, 16, 8]])
def test_loss_gradient_matches_central_differences(widths):
    rng = np.random.default_rng(2)
    n_par = sum(widths[l + 1] * widths[l] + widths[l + 1] for l in range(len(widths) - 1))
    p = rng.standard_normal(n_par) * 0.5
    x = rng.standard_normal((6, widths[0]))
    t = rng.uniform(0.1, 0.6, (6, widths[-1]))
    loss, g = mlp.loss_and_grad(p, widths, x, t, bf16_round=False)
    h = 1e-6
    idx = rng.choice(n_par, 60, replace=False)
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_grad(pp, widths, x, t, bf16_round=False)[0] -
              mlp.loss_and_grad(pm, widths, x, t, bf16_round=False)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-10)
    # the loss is the mean squared error of the forward output
    y, _, _ = mlp.forward(p, widths, x, bf16_round=False)
    assert loss == pytest.approx(((y - t) ** 2).mean(), rel=1e-14)


def test_bf16_rounding_points_change_little():
    rng = np.random.default_rng(3)
    widths = [64, 32, 32, 8]
    n_par = sum(widths[l + 1] * widths[l] + widths[l + 1] for l in range(len(widths) - 1))
    p = rng.standard_normal(n_par) * 0.2
    x = rng.standard_normal((16, 64))
    t = rng.uniform(0.1, 0.6, (16, 8))
    l0, g0 = mlp.loss_and_grad(p, widths, x, t, bf16_round=False)
    l1, g1 = mlp.loss_and_grad(p, widths, x, t, bf16_round=True)
    assert l1 == pytest.approx(l0, rel=2e-2)
    assert np.linalg.norm(g1 - g0) <= 2e-2 * np.linalg.norm(g0)


def test_values_depend_on_the_weights_only_through_their_bf16_roundings():
    rng = np.random.default_rng(4)
    widths = [16, 24, 24, 8]
    n_par = sum(widths[l + 1] * widths[l] + widths[l + 1] for l in range(len(widths) - 1))
    p = rng.standard_normal(n_par) * 0.3
    x = rng.standard_normal((12, 16))
    t = rng.uniform(0.1, 0.6, (12, 8))
    layers = mlp.unpack(p, widths)
    # bf16-exact weights, then the same weights moved by a quarter of a bf16 unit in the last place
    exact = mlp.pack([(mlp.bf16(W), b) for W, b in layers])
    moved = mlp.pack([(mlp.bf16(W) * (1.0 + 2.0 ** -10), b) for W, b in layers])
    assert (mlp.bf16(moved) == moved).sum() < 0.5 * n_par
    l0, g0 = mlp.loss_and_grad(exact, widths, x, t)
    l1, g1 = mlp.loss_and_grad(moved, widths, x, t)
    assert l1 == l0
    np.testing.assert_array_equal(g1, g0)


def _net(seed):
    rng = np.random.default_rng(seed)
    widths = [16, 24, 24, 8]
    n_par = sum(widths[l + 1] * widths[l] + widths[l + 1] for l in range(len(widths) - 1))
    return widths, rng.standard_normal(n_par) * 0.3, rng.standard_normal((12, 16)), rng.uniform(0.1, 0.6, (12, 8))


def test_input_enters_only_through_its_bf16_value_and_activations_are_bf16():
    widths, p, x, t = _net(5)
    xe = mlp.bf16(x)
    xm = xe * (1.0 + 2.0 ** -10)
    assert (mlp.bf16(xm) == xm).sum() < 0.5 * xm.size
    l0, g0 = mlp.loss_and_grad(p, widths, xe, t)
    l1, g1 = mlp.loss_and_grad(p, widths, xm, t)
    assert l1 == l0
    np.testing.assert_array_equal(g1, g0)
    _, xs, _ = mlp.forward(p, widths, x)
    for a in xs:
        np.testing.assert_array_equal(mlp.bf16(a), a)


def test_weight_gradients_see_the_output_error_only_through_its_bf16_value():
    # targets moved by 1e-12 relative change the output error far below a bf16 unit:
    # every weight gradient and the hidden layers' bias gradients stay bit-identical,
    # while the output bias gradient (a sum of the unrounded error) moves
    widths, p, x, t = _net(6)
    _, g0 = mlp.loss_and_grad(p, widths, x, t)
    _, g1 = mlp.loss_and_grad(p, widths, x, t * (1.0 + 1e-12))
    n_out_bias = widths[-1]
    np.testing.assert_array_equal(g1[:-n_out_bias], g0[:-n_out_bias])
    assert (g1[-n_out_bias:] != g0[-n_out_bias:]).any()


# ---- the coordinate network's variants: ReLU hidden layers, linear output, a given output gradient

def test_relu_and_its_derivative():
    z = np.array([-2.0, -1e-300, 0.0, 1e-300, 3.5])
    np.testing.assert_array_equal(mlp.relu(z), [0.0, 0.0, 0.0, 1e-300, 3.5])
    np.testing.assert_array_equal(mlp.relu_grad(z), [0.0, 0.0, 0.0, 1.0, 1.0])


def test_linear_one_layer_network_and_its_gradient_in_closed_form():
    # y = x W^T + b, L = sum(c * y): dL/dW = c^T x, dL/db = sum over the batch of c
    rng = np.random.default_rng(7)
    W, b = rng.standard_normal((8, 16)), rng.standard_normal(8)
    x, c = rng.standard_normal((5, 16)), rng.standard_normal((5, 8))
    p = mlp.pack([(W, b)])
    y, _, _ = mlp.forward(p, [16, 8], x, bf16_round=False, out="linear")
    np.testing.assert_allclose(y, x @ W.T + b, rtol=0, atol=1e-13)
    g = mlp.backward(p, [16, 8], x, c, bf16_round=False, out="linear")
    np.testing.assert_allclose(g[:128].reshape(8, 16), c.T @ x, rtol=0, atol=1e-13)
    np.testing.assert_allclose(g[128:], c.sum(axis=0), rtol=0, atol=1e-13)


def test_relu_network_by_hand():
    # 1 -> 2 -> 1, ReLU, linear output: y = w2 . relu(w1 x + b1) + b2
    W1, b1 = np.array([[2.0], [-1.0]]), np.array([0.5, 0.25])
    W2, b2 = np.array([[3.0, 4.0]]), np.array([-1.0])
    p = mlp.pack([(W1, b1), (W2, b2)])
    x = np.array([[1.0], [2.0]])          # hidden: (2.5, 0) and (4.5, 0): the second unit is off
    y, _, _ = mlp.forward(p, [1, 2, 1], x, bf16_round=False, hidden="relu", out="linear")
    np.testing.assert_allclose(y[:, 0], [3 * 2.5 - 1, 3 * 4.5 - 1], rtol=0, atol=1e-14)
    g = mlp.backward(p, [1, 2, 1], x, np.ones((2, 1)), bf16_round=False, hidden="relu", out="linear")
    # dL/dW1 = sum_n W2_0 x_n for the active unit, 0 for the inactive one; dL/db1 likewise
    np.testing.assert_allclose(g, [3 * 3.0, 0.0, 3 * 2.0, 0.0, 2.5 + 4.5, 0.0, 2.0], rtol=0, atol=1e-14)


@pytest.mark.parametrize("out", ["linear", "sigmoid"])
def test_relu_network_gradient_matches_central_differences(out):
    widths = [8, 16, 16, 8]
    rng = np.random.default_rng(8)
    n_par = sum(widths[l + 1] * widths[l] + widths[l + 1] for l in range(len(widths) - 1))
    p = rng.standard_normal(n_par) * 0.5
    x = rng.standard_normal((6, widths[0]))
    c = rng.standard_normal((6, widths[-1]))

    def L(q):
        y, _, _ = mlp.forward(q, widths, x, bf16_round=False, hidden="relu", out=out)
        return float((c * y).sum())

    g = mlp.backward(p, widths, x, c, bf16_round=False, hidden="relu", out=out)
    h = 1e-6
    for i in rng.choice(n_par, 60, replace=False):
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        assert g[i] == pytest.approx((L(pp) - L(pm)) / (2 * h), rel=1e-5, abs=1e-9)


def test_zero_padded_units_stay_inert():
    # hidden units whose weights in and out are zero have zero gradients (ReLU is off
    # at 0, and nothing reads them), so padding a layer to a multiple of 8 changes nothing
    rng = np.random.default_rng(9)
    W1, b1 = rng.standard_normal((6, 8)), rng.standard_normal(6)
    W2, b2 = rng.standard_normal((8, 6)), rng.standard_normal(8)
    W1p, b1p = np.vstack([W1, np.zeros((2, 8))]), np.concatenate([b1, np.zeros(2)])
    W2p = np.hstack([W2, np.zeros((8, 2))])
    x, c = rng.standard_normal((4, 8)), rng.standard_normal((4, 8))
    p, pp = mlp.pack([(W1, b1), (W2, b2)]), mlp.pack([(W1p, b1p), (W2p, b2)])
    y, _, _ = mlp.forward(p, [8, 6, 8], x, bf16_round=False, hidden="relu", out="linear")
    yp, _, _ = mlp.forward(pp, [8, 8, 8], x, bf16_round=False, hidden="relu", out="linear")
    np.testing.assert_allclose(yp, y, rtol=0, atol=1e-14)
    gp = mlp.unpack(mlp.backward(pp, [8, 8, 8], x, c, bf16_round=False, hidden="relu", out="linear"), [8, 8, 8])
    assert np.all(gp[0][0][6:] == 0) and np.all(gp[0][1][6:] == 0) and np.all(gp[1][0][:, 6:] == 0)
