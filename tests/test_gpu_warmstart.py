"""Batched forward runs as training data, and the learned warm start of the
friction inversion against the uniform first guess (Sec. 5.3 inverse problem)."""
import numpy as np
import pytest

from paper_2507_04192_gb300 import inputs, mpm, warmstart

pytestmark = pytest.mark.gpu

SMALL = warmstart.Setup(n_cells=48, n_seg=16, n_track=32, n_obs=6, steps=300, checkpoint_every=50)


def test_batched_observations_match_single_runs_fp64():
    w = SMALL.workload()
    mus = np.stack([inputs.friction_field(SMALL.n_seg, 10 + i) for i in range(5)])
    zb = warmstart.observe_batch(w, mus, mpm.MPM_FP64)
    assert zb.shape == (5, SMALL.n_obs, SMALL.n_track, 2)
    for i in (0, 3):
        z1 = warmstart.observe_batch(w, mus[i:i + 1], mpm.MPM_FP64)[0]
        np.testing.assert_allclose(zb[i], z1, rtol=0, atol=1e-12)
    # runs with different friction differ; the features are displacements along the floor
    assert np.abs(zb[0] - zb[1]).max() > 1e-6
    f = warmstart.features(SMALL, w, zb)
    assert f.shape == (5, SMALL.n_features)
    x0 = w.x[w.extras["track_ids"]]
    np.testing.assert_allclose(f[2].reshape(SMALL.n_obs, SMALL.n_track),
                               (zb[2, :, :, 0] - x0[:, 0]) / SMALL.scale(w), rtol=1e-6, atol=1e-7)


def test_warm_start_beats_the_uniform_guess():
    X, Y = warmstart.generate(SMALL, 1536, batch=256)
    assert X.shape == (1536, SMALL.n_features) and np.isfinite(X).all()
    net = warmstart.WarmStartNet(SMALL.n_features, SMALL.n_seg, hidden=(128, 128), max_batch=256)
    hist = net.fit(X, Y, epochs=60, lr=1e-3)
    # segments the front never reaches are unpredictable (their best guess is the
    # mean), so the loss cannot fall far below the variance of U[0.1, 0.6)
    assert hist[-1] < 0.8 * hist[0]
    rows = warmstart.compare(SMALL, net, mu_seeds=[1, 2, 3], max_iters=60)
    net.close()
    e_u = np.mean([r["err0_uniform"] for r in rows])
    e_w = np.mean([r["err0_warm"] for r in rows])
    assert e_w < 0.7 * e_u, rows
    it_u = sum(r["iters_uniform"] for r in rows)
    it_w = sum(r["iters_warm"] for r in rows)
    assert it_w <= it_u, rows
