"""FP64 oracle of the fully connected networks (test infrastructure only).

Plain numpy, float64 arithmetic.  With ``bf16=True`` the values the tensor-core
path feeds to its GEMMs are rounded to bfloat16 (round to nearest even) at the
same points: the network input, the weights, the hidden activations and the
back-propagated pre-activation gradients.  Hidden layers use GELU (exact erf
form; the warm-start network) or ReLU (the coordinate network of Eq. nn_apprx,
Sec. 5.2); the output is lo + (hi - lo) sigmoid(z) or the affine map z itself.
"""
from __future__ import annotations

import math

import numpy as np

_erf = np.vectorize(math.erf)


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def relu(z):
    return np.maximum(z, 0.0)


def relu_grad(z):
    """Derivative of max(z, 0), taken as 0 at z = 0."""
    return (np.asarray(z) > 0.0).astype(np.float64)


_ACT = {"gelu": (gelu, gelu_grad), "relu": (relu, relu_grad)}


def unpack(params, widths):
    out, o = [], 0
    for l in range(len(widths) - 1):
        n_in, n_out = widths[l], widths[l + 1]
        W = np.asarray(params[o:o + n_out * n_in], dtype=np.float64).reshape(n_out, n_in)
        o += n_out * n_in
        b = np.asarray(params[o:o + n_out], dtype=np.float64)
        o += n_out
        out.append((W, b))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in layers])


def forward(params, widths, x, lo=0.1, hi=0.6, bf16_round=True, hidden="gelu", out="sigmoid"):
    """Output y and the layer inputs xs (as the GEMMs see them) and pre-activations zs."""
    r = bf16 if bf16_round else (lambda a: np.asarray(a, dtype=np.float64))
    act = _ACT[hidden][0]
    layers = unpack(params, widths)
    xs, zs = [r(x)], []
    for l, (W, b) in enumerate(layers):
        z = xs[-1] @ r(W).T + b
        zs.append(z)
        if l + 1 < len(layers):
            xs.append(r(act(z)))
    if out == "linear":
        return zs[-1].copy(), xs, zs
    s = 1.0 / (1.0 + np.exp(-zs[-1]))
    return lo + (hi - lo) * s, xs, zs


def backward(params, widths, x, dy, lo=0.1, hi=0.6, bf16_round=True, hidden="gelu", out="sigmoid"):
    """Gradient of a scalar L with respect to the parameters, given dL/dy (the
    output's shape): back-propagation through the layers of ``forward``."""
    r = bf16 if bf16_round else (lambda a: np.asarray(a, dtype=np.float64))
    dact = _ACT[hidden][1]
    layers = unpack(params, widths)
    _, xs, zs = forward(params, widths, x, lo, hi, bf16_round, hidden, out)
    if out == "linear":
        dz = np.asarray(dy, dtype=np.float64)
    else:
        s = 1.0 / (1.0 + np.exp(-zs[-1]))
        dz = np.asarray(dy, dtype=np.float64) * (hi - lo) * s * (1.0 - s)
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        dzr = r(dz)
        gW = dzr.T @ xs[l]
        gb = dz.sum(axis=0)
        grads[l] = (gW, gb)
        if l > 0:
            da = dzr @ r(W)
            dz = da * dact(zs[l - 1])
    return pack(grads)


def loss_and_grad(params, widths, x, t, lo=0.1, hi=0.6, bf16_round=True, hidden="gelu", out="sigmoid"):
    """Mean squared error L = mean (y - t)^2 and its gradient with respect to the parameters."""
    y, _, _ = forward(params, widths, x, lo, hi, bf16_round, hidden, out)
    n = y.size
    e = y - t
    loss = float((e * e).sum() / n)
    return loss, backward(params, widths, x, 2.0 * e / n, lo, hi, bf16_round, hidden, out)
