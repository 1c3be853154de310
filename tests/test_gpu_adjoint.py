"""The GPU adjoint (mpm_step_adjoint) against the oracle's hand-derived adjoint,
against central finite differences of the GPU loss, and for its invariances.

Loss of Eq. inverse_loss (Sec. 3.2): tracked particle positions at observation
steps; parameters: the basal Coulomb friction of Sec. 5.3 per floor segment.
Tolerances: FP64 gradient within 1e-6 of the oracle (relative to its largest
entry); FP32 cosine >= 0.99 and relative L2 error <= 5e-2.
"""
import numpy as np
import pytest

import oracle
from paper_2507_04192_gb300 import inputs, mpm

pytestmark = pytest.mark.gpu


def problem(n_cells=32, n_seg=8, steps=300, n_obs=4, n_track=32, seed=0):
    w = inputs.dam_break_inverse_2d(n_cells, n_seg=n_seg, n_track=n_track, n_obs=n_obs, steps=steps, seed=seed)
    return w


def true_observations(w, mu_true):
    orc = oracle.Oracle(2, w.n_cells, w.dx, w.dt, w.gravity, w.material, w.particle_volume,
                        friction=[(2, (len(mu_true), 1), mu_true)])
    st = orc.initial_state(w.x)
    ids = w.extras["track_ids"]
    z = []
    t = 0
    for s in w.extras["obs_steps"]:
        orc.step(st, s - t)
        t = s
        z.append(st.x[ids].copy())
    return np.stack(z)


def oracle_loss_and_grad(w, mu, z):
    orc = oracle.Oracle(2, w.n_cells, w.dx, w.dt, w.gravity, w.material, w.particle_volume,
                        friction=[(2, (len(mu), 1), mu)])
    ids = w.extras["track_ids"]
    obs = {s: k for k, s in enumerate(w.extras["obs_steps"])}
    steps = max(obs)
    states = [orc.initial_state(w.x)]
    loss = 0.0
    for t in range(1, steps + 1):
        s = states[-1].copy()
        orc.step(s, 1)
        states.append(s)
        if t in obs:
            loss += float(((s.x[ids] - z[obs[t]]) ** 2).sum())
    n = w.n
    lam = [np.zeros((n, 2)), np.zeros((n, 2)), np.zeros((n, 2, 2)), np.zeros(n)]
    grad = np.zeros(len(mu))
    for t in range(steps, 0, -1):
        if t in obs:
            lam[0][ids] += 2.0 * (states[t].x[ids] - z[obs[t]])
        lam, mub = orc.step_vjp(states[t - 1], *lam)
        grad += mub[2]
    return loss, grad


def gpu_loss_and_grad(w, mu, z, precision, K, sort_every=8):
    sim = mpm.Simulation(2, w.n_cells, w.dx, w.dt, w.gravity, w.material, precision, sort_every)
    sim.load(w.x, None, w.particle_volume)
    sim.set_friction(2, (len(mu), 1), mu)
    mpm.mpm_set_observations(sim.ctx, w.extras["track_ids"], w.extras["obs_steps"], z)
    loss, grad = mpm.mpm_step_adjoint(sim.ctx, max(w.extras["obs_steps"]), K, 2, len(mu))
    x_end = sim.get("x")
    sim.close()
    return loss, grad, x_end


@pytest.fixture(scope="module")
def small():
    w = problem()
    mu_true = w.extras["mu_true"]
    z = true_observations(w, mu_true)
    mu = np.full(len(mu_true), 0.35)
    ref_loss, ref_grad = oracle_loss_and_grad(w, mu, z)
    return w, mu, z, ref_loss, ref_grad


def test_fp64_adjoint_matches_oracle_adjoint(small):
    w, mu, z, ref_loss, ref_grad = small
    loss, grad, _ = gpu_loss_and_grad(w, mu, z, mpm.MPM_FP64, K=50)
    assert np.abs(ref_grad).max() > 0
    assert loss == pytest.approx(ref_loss, rel=1e-9)
    np.testing.assert_allclose(grad, ref_grad, rtol=0, atol=1e-6 * np.abs(ref_grad).max())


def test_fp32_adjoint_close_to_oracle_adjoint(small):
    w, mu, z, ref_loss, ref_grad = small
    loss, grad, _ = gpu_loss_and_grad(w, mu, z, mpm.MPM_FP32, K=50)
    assert loss == pytest.approx(ref_loss, rel=1e-3)
    cos = grad @ ref_grad / (np.linalg.norm(grad) * np.linalg.norm(ref_grad))
    assert cos >= 0.99
    assert np.linalg.norm(grad - ref_grad) <= 5e-2 * np.linalg.norm(ref_grad)


def test_fp64_adjoint_matches_central_finite_differences(small):
    w, mu, z, _, _ = small
    _, grad, _ = gpu_loss_and_grad(w, mu, z, mpm.MPM_FP64, K=50)
    eps = 1e-3
    fd = np.zeros(len(mu))
    for s in range(len(mu)):
        mp_, mm_ = mu.copy(), mu.copy()
        mp_[s] += eps
        mm_[s] -= eps
        fd[s] = (gpu_loss_and_grad(w, mp_, z, mpm.MPM_FP64, K=50)[0] -
                 gpu_loss_and_grad(w, mm_, z, mpm.MPM_FP64, K=50)[0]) / (2 * eps)
    np.testing.assert_allclose(grad, fd, rtol=0, atol=2e-2 * np.abs(fd).max())


def test_checkpoint_interval_and_sorting_do_not_change_the_gradient(small):
    w, mu, z, _, _ = small
    ref = gpu_loss_and_grad(w, mu, z, mpm.MPM_FP64, K=50)
    for K, sort_every in ((1, 8), (7, 3), (300, 40)):
        loss, grad, _ = gpu_loss_and_grad(w, mu, z, mpm.MPM_FP64, K=K, sort_every=sort_every)
        assert loss == pytest.approx(ref[0], rel=1e-11)
        np.testing.assert_allclose(grad, ref[1], rtol=0, atol=1e-9 * np.abs(ref[1]).max())


def test_adjoint_leaves_the_end_of_horizon_state(small):
    w, mu, z, _, _ = small
    _, _, x_end = gpu_loss_and_grad(w, mu, z, mpm.MPM_FP64, K=50)
    sim = mpm.Simulation(2, w.n_cells, w.dx, w.dt, w.gravity, w.material, mpm.MPM_FP64, 8)
    sim.load(w.x, None, w.particle_volume)
    sim.set_friction(2, (len(mu), 1), mu)
    sim.step(max(w.extras["obs_steps"]))
    x_plain = sim.get("x")
    sim.close()
    np.testing.assert_allclose(x_end, x_plain, rtol=0, atol=1e-12)


def test_adjoint_argument_errors():
    w = problem()
    sim = mpm.Simulation.from_workload(w, mpm.MPM_FP64)
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_step_adjoint(sim.ctx, 10, 5, 2, 8)          # no observations yet
    assert e.value.code == mpm.MPM_ESTATE
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_set_observations(sim.ctx, np.array([0, 0]), [5], np.zeros((1, 2, 2)))   # repeated id
    assert e.value.code == mpm.MPM_EINVAL
    sim.close()


@pytest.mark.slow
def test_full_size_dam_break_inverse_fp64_vs_oracle():
    """The 32,768-particle, 128 x 128, 32-segment problem (100 steps, 10 observations)."""
    w = inputs.dam_break_inverse_2d(128, n_seg=32, n_track=64, n_obs=10, steps=100)
    z = true_observations(w, w.extras["mu_true"])
    mu = np.full(32, 0.35)
    ref_loss, ref_grad = oracle_loss_and_grad(w, mu, z)
    loss, grad, _ = gpu_loss_and_grad(w, mu, z, mpm.MPM_FP64, K=20)
    assert loss == pytest.approx(ref_loss, rel=1e-8)
    np.testing.assert_allclose(grad, ref_grad, rtol=0, atol=1e-5 * np.abs(ref_grad).max())
