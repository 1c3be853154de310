"""The per-step adjoint (mpm_step_adjoint_1) chained backwards over stored
states gives the loss gradient of the whole-horizon adjoint (mpm_step_adjoint):
dL/dmu and the adjoint of the initial state, for the fluid in 2D (FP64) and
for Drucker-Prager sand in 3D (FP64, and FP32 with the cell-ordered v_bar scatter).

The sand starts moving (horizontal convergence, downward velocity) rather than at
rest: at rest every particle's stress is zero, the apex of the Drucker-Prager
cone, where the return mapping has a kink and rounding picks the branch; two
runs of the whole-horizon adjoint from rest already differ by about 1 % in the
v and C adjoints of S^0 (x, the loss and dL/dmu agree to rounding)."""
import numpy as np
import pytest

from paper_2507_04192_gb300 import inputs, mpm

pytestmark = pytest.mark.gpu


def chained(w, precision, wall, mu_shape, mu, T, track_ids, z, v0=None):
    """Loss at step T on the tracked positions, by T calls of mpm_step_adjoint_1."""
    sim = mpm.Simulation(w.dim, w.n_cells, w.dx, w.dt, w.gravity, w.material, precision, w.sort_every)
    sim.load(w.x, v0, w.particle_volume)
    sim.set_friction(wall, mu_shape, mu)
    for t in range(T):                           # S^0 .. S^{T-1} in slots 0 .. T-1
        mpm.mpm_save_state(sim.ctx, t)
        sim.step(1)
    x_T = sim.get("x")
    d = w.dim
    NA = mpm.mpm_adjoint_width(sim.ctx)
    lam = np.zeros((w.n, NA))
    e = x_T[track_ids] - z
    lam[track_ids, :d] = 2.0 * e                 # dL/dx^T of L = sum |x - z|^2
    grad = np.zeros(len(mu))
    for t in range(T - 1, -1, -1):
        mpm.mpm_restore_state(sim.ctx, t)
        lam, g = mpm.mpm_step_adjoint_1(sim.ctx, wall, lam, len(mu))
        grad += g
    sim.close()
    return float((e * e).sum()), grad, lam


def whole(w, precision, wall, mu_shape, mu, T, track_ids, z, K, v0=None):
    sim = mpm.Simulation(w.dim, w.n_cells, w.dx, w.dt, w.gravity, w.material, precision, w.sort_every)
    sim.load(w.x, v0, w.particle_volume)
    sim.set_friction(wall, mu_shape, mu)
    mpm.mpm_set_observations(sim.ctx, track_ids, [T], z[None])
    loss, grad = mpm.mpm_step_adjoint(sim.ctx, T, K, wall, len(mu))
    lam0 = {f: mpm.mpm_get_initial_adjoint(sim.ctx, f) for f in ("x", "v", "C", "rho")}
    sim.close()
    return loss, grad, lam0


def compare(w, precision, wall, mu_shape, mu, T, K, rtol, field_norm=None, v0=None):
    """field_norm: compare the initial adjoint's fields in relative L2 norm (FP32:
    the two runs sum the grid in different orders); else element-wise."""
    rng = np.random.default_rng(5)
    track_ids = np.sort(rng.choice(w.n, 48, replace=False)).astype(np.int64)
    z = w.x[track_ids] + rng.normal(scale=2 * w.dx, size=(48, w.dim))
    loss1, grad1, lam = chained(w, precision, wall, mu_shape, mu, T, track_ids, z, v0)
    loss, grad, lam0 = whole(w, precision, wall, mu_shape, mu, T, track_ids, z, K, v0)
    assert loss1 == pytest.approx(loss, rel=rtol)
    assert np.abs(grad).max() > 0
    np.testing.assert_allclose(grad1, grad, rtol=0, atol=rtol * np.abs(grad).max())
    d = w.dim
    cols = {"x": slice(0, d), "v": slice(d, 2 * d), "C": slice(2 * d, 2 * d + d * d),
            "rho": slice(2 * d + d * d, 2 * d + d * d + 1)}
    for f, sl in cols.items():
        ref = lam0[f].reshape(w.n, -1)
        if field_norm is not None:
            assert np.linalg.norm(lam[:, sl] - ref) <= field_norm * np.linalg.norm(ref), f
            continue
        scale = max(float(np.abs(ref).max()), 1e-30)
        np.testing.assert_allclose(lam[:, sl], ref, rtol=0, atol=rtol * scale, err_msg=f)


def test_chained_steps_match_the_whole_adjoint_fluid_2d_fp64():
    w = inputs.dam_break_inverse_2d(32, n_seg=8, steps=12)
    mu = inputs.friction_field(8, 7)
    compare(w, mpm.MPM_FP64, 2, (8, 1), mu, T=12, K=5, rtol=1e-9)


def sand_3d():
    w = inputs.granular_cylinder_3d((24, 24, 24), 5, 10, dx=1 / 24, dt=2e-4, floor_mu=0.0, steps=10)
    w.friction = [(4, (2, 2), np.array([0.2, 0.3, 0.4, 0.5]))]
    cx, cy = w.extras["axis"]
    v0 = np.zeros_like(w.x)
    v0[:, 0] = -2.0 * (w.x[:, 0] - cx)
    v0[:, 1] = -2.0 * (w.x[:, 1] - cy)
    v0[:, 2] = -0.2
    return w, v0


def test_chained_steps_match_the_whole_adjoint_sand_3d_fp32():
    w, v0 = sand_3d()
    compare(w, mpm.MPM_FP32, 4, (2, 2), w.friction[0][2], T=10, K=4, rtol=2e-3, field_norm=1e-4, v0=v0)


def test_chained_steps_match_the_whole_adjoint_sand_3d_fp64():
    w, v0 = sand_3d()
    compare(w, mpm.MPM_FP64, 4, (2, 2), w.friction[0][2], T=10, K=4, rtol=1e-8, v0=v0)
