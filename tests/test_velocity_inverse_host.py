"""Host logic of the initial-velocity inversion driver: the coordinate network's
sizes and the Adam update (a quadratic's minimum).  The network itself runs on
the tensor cores; tests/test_gpu_mlp.py and tests/test_gpu_inverse_velocity.py
check it against the FP64 oracle of the network."""
import numpy as np
import pytest

from paper_2507_04192_gb300.velocity_inverse import Adam, CoordinateNet


def test_coordinate_network_sizes():
    # the paper's 1 -> 30 -> 30 -> 30 -> 1 network has 1,951 parameters (Table 3); the
    # tensor-core layout pads each width to a multiple of 8
    t, p = CoordinateNet.TRUE, CoordinateNet.PADDED
    assert sum(t[i] * t[i + 1] + t[i + 1] for i in range(4)) == 1951
    assert all(w % 8 == 0 and w >= v for w, v in zip(p, t))


def test_adam_reaches_the_minimum_of_a_quadratic():
    opt = Adam(2, lr0=0.1, decay=1.0)
    p = np.array([3.0, -2.0])
    for _ in range(2000):
        p = opt.step(p, 2.0 * (p - np.array([0.5, 1.5])))
    np.testing.assert_allclose(p, [0.5, 1.5], atol=1e-3)
