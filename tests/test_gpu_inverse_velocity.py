"""The initial-velocity inverse problems of Sec. 5.2 on the GPU, through the
C-ABI: the adjoint of the initial velocity (mpm_get_initial_adjoint after
mpm_step_adjoint without a friction parameter) for tracked positions and for
velocity monitors against the oracle's reverse recursion, the monitor means
against the oracle's definition, and a short recovery of the velocity constant.

Tolerances: FP64 loss within 1e-9 relative, FP64 dL/dv0 within 1e-6 of its
largest entry (summation order of atomics only).
"""
import numpy as np
import pytest

import oracle
from paper_2507_04192_gb300 import inputs, mpm, velocity_inverse
from velocity_inverse_oracle import loss_and_v0_adjoint, observe, small_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    w = small_problem(inputs)
    H0 = w.extras["H0"]
    zx, zv = observe(w, inputs.velocity_profile_linear(w.x, 2.0, H0))
    v0 = inputs.velocity_profile_linear(w.x, 1.2, H0)
    return w, zx, zv, v0


def gpu_loss_and_v0(w, v0, zx=None, zv=None, precision=mpm.MPM_FP64, K=50):
    sim = mpm.Simulation(w.dim, w.n_cells, w.dx, w.dt, w.gravity, w.material, precision, w.sort_every)
    sim.load(w.x, v0, w.particle_volume)
    if zx is not None:
        mpm.mpm_set_observations(sim.ctx, w.extras["track_ids"], w.extras["obs_steps"], zx)
    if zv is not None:
        mpm.mpm_set_velocity_monitors(sim.ctx, w.extras["monitors"], w.extras["obs_steps"], zv)
    loss, _ = mpm.mpm_step_adjoint(sim.ctx, max(w.extras["obs_steps"]), K, -1, 0)
    g = mpm.mpm_get_initial_adjoint(sim.ctx, "v")
    sim.close()
    return loss, g


@pytest.mark.parametrize("kind", ["tracked", "monitors", "both"])
def test_initial_velocity_adjoint_matches_oracle(case, kind):
    w, zx, zv, v0 = case
    args = dict(zx=zx if kind in ("tracked", "both") else None, zv=zv if kind in ("monitors", "both") else None)
    ref_loss, ref_g = loss_and_v0_adjoint(w, v0, **args)
    loss, g = gpu_loss_and_v0(w, v0, **args)
    assert ref_loss > 0 and np.abs(ref_g).max() > 0
    assert loss == pytest.approx(ref_loss, rel=1e-9)
    np.testing.assert_allclose(g, ref_g, rtol=0, atol=1e-6 * np.abs(ref_g).max())


def test_adjoint_is_independent_of_checkpoint_interval(case):
    w, zx, zv, v0 = case
    a = gpu_loss_and_v0(w, v0, zx=zx, zv=zv, K=7)
    b = gpu_loss_and_v0(w, v0, zx=zx, zv=zv, K=240)
    assert a[0] == pytest.approx(b[0], rel=1e-12)
    np.testing.assert_allclose(a[1], b[1], rtol=0, atol=1e-9 * np.abs(b[1]).max())


def test_monitor_means_match_oracle(case):
    w, _, _, v0 = case
    sim = mpm.Simulation(w.dim, w.n_cells, w.dx, w.dt, w.gravity, w.material, mpm.MPM_FP64, w.sort_every)
    sim.load(w.x, v0, w.particle_volume)
    sim.step(100)
    Q, cnt = mpm.mpm_monitor_means(sim.ctx, w.extras["monitors"])
    x, v = sim.get("x"), sim.get("v")
    sim.close()
    Qr, cr = oracle.monitor_means(x, v, w.extras["monitors"])
    np.testing.assert_array_equal(cnt, cr)
    assert cnt.sum() > 0
    np.testing.assert_allclose(Q, Qr, rtol=0, atol=1e-12 * max(1.0, np.abs(Qr).max()))


def test_velocity_constant_recovered_from_monitors():
    w = inputs.dam_break_velocity_inverse(dx=0.02, steps=3000, n_frames=50, frame_every=10, checkpoint_every=100)
    H0 = w.extras["H0"]
    _, zv = velocity_inverse.record_observations(w, inputs.velocity_profile_linear(w.x, 2.0, H0))
    prob = velocity_inverse.VelocityInversion(w, zv=zv)
    res = velocity_inverse.invert_alpha(prob, alpha0=0.1, alpha_true=2.0, tol=0.02, max_iters=80)
    prob.close()
    assert res.converged, res.history[-3:]


def test_3d_monitors_and_initial_adjoint_match_oracle():
    # the 3D forms of the monitor kernels and of the initial-state adjoint
    w = inputs.dam_break_3d((16, 8, 8), dx=1 / 16, dt=2e-4, steps=0, obstacles=False)
    w.v = np.tile([0.6, 0.1, 0.0], (w.n, 1)) * (1.0 - w.x[:, 2:3] / 0.2)
    boxes = [((0.05, 0.1, 0.02), (0.2, 0.3, 0.12)), ((0.2, 0.2, 0.0), (0.35, 0.45, 0.1))]
    obs_steps = [20, 40]
    w.extras.update(obs_steps=obs_steps, monitors=boxes, track_ids=np.arange(0, w.n, 97, dtype=np.int64))
    zx, zv = observe(w, w.v * 0.8)
    ref_loss, ref_g = loss_and_v0_adjoint(w, w.v, zx=zx, zv=zv)
    loss, g = gpu_loss_and_v0(w, w.v, zx=zx, zv=zv, K=15)
    assert ref_loss > 0 and np.abs(ref_g).max() > 0
    assert loss == pytest.approx(ref_loss, rel=1e-9)
    np.testing.assert_allclose(g, ref_g, rtol=0, atol=1e-6 * np.abs(ref_g).max())
    sim = mpm.Simulation(3, w.n_cells, w.dx, w.dt, w.gravity, w.material, mpm.MPM_FP64, w.sort_every)
    sim.load(w.x, w.v, w.particle_volume)
    sim.step(30)
    Q, cnt = mpm.mpm_monitor_means(sim.ctx, boxes)
    x, v = sim.get("x"), sim.get("v")
    sim.close()
    Qr, cr = oracle.monitor_means(x, v, boxes)
    np.testing.assert_array_equal(cnt, cr)
    assert cnt.min() > 0
    np.testing.assert_allclose(Q, Qr, rtol=0, atol=1e-12 * max(1.0, np.abs(Qr).max()))


def test_velocity_field_recovered_by_the_tensor_core_coordinate_network():
    # Sec. 5.2 "initial velocity field": the coordinate network (1 -> 30 -> 30 -> 30 -> 1,
    # ReLU) on the library's tensor-core network, trained through the adjoint; a
    # coarse resolution and a short horizon keep this to seconds
    w = inputs.dam_break_velocity_inverse(dx=0.02, steps=3000, n_frames=50, frame_every=10, n_track=400,
                                          checkpoint_every=100)
    H0 = w.extras["H0"]
    v_true = np.zeros_like(w.x)
    v_true[:, 0] = inputs.velocity_profile_field(w.x[:, 1], H0)
    zx, _ = velocity_inverse.record_observations(w, v_true)
    prob = velocity_inverse.VelocityInversion(w, zx=zx)
    res = velocity_inverse.invert_field(prob, epochs=60, lr0=1e-2)
    prob.close()
    e0, e1 = res.history[0]["error"], res.history[-1]["error"]
    losses = [h["loss"] for h in res.history[:-1]]
    assert losses[-1] < 0.05 * losses[0], losses[::10]
    assert e1 < 0.5 * e0 and e1 < 0.35, (e0, e1)
    # the network's padding to multiples of 8 stayed inert: only the 1-30-30-30-1 block moved
    net = velocity_inverse.CoordinateNet
    p = res.params
    o = 0
    for i in range(4):
        W = p[o:o + net.PADDED[i + 1] * net.PADDED[i]].reshape(net.PADDED[i + 1], net.PADDED[i])
        o += W.size
        b = p[o:o + net.PADDED[i + 1]]
        o += b.size
        assert np.all(W[net.TRUE[i + 1]:, :] == 0) and np.all(W[:, net.TRUE[i]:] == 0)
        assert np.all(b[net.TRUE[i + 1]:] == 0)
