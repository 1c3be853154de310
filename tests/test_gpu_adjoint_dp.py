"""The GPU adjoint of the granular (Drucker-Prager) step against the oracle's
hand-derived adjoint and central finite differences: basal friction gradient of
the tracked-particle loss (Eq. inverse_loss, Sec. 3.2) in 2D (plane strain,
floor segments) and 3D (floor patches)."""
import numpy as np
import pytest

import oracle
from paper_2507_04192_gb300 import inputs, mpm

pytestmark = pytest.mark.gpu


def column_2d(N=32, n_seg=8, steps=300, seed=0):
    dx = 1.0 / N
    x = inputs.lattice_particles((N, N), dx, 2, lambda p: (p[:, 0] < 0.25) & (p[:, 1] < 0.4), (0, 0), (0.25, 0.4),
                                 seed)
    mu = inputs.friction_field(n_seg, seed)
    ids = inputs.tracked_particles(x, 24, seed, np.array([0.0, 0.0]), np.array([0.25, 0.4]))
    return dict(dim=2, cells=(N, N), dx=dx, dt=1e-4, g=(0.0, -9.81), x=x, vol=dx * dx / 4, wall=2,
                nseg=(n_seg, 1), mu=mu, ids=ids, obs=[steps // 3, 2 * steps // 3, steps])


def column_3d(seed=0, steps=300):
    w = inputs.granular_inverse_3d((16, 16, 8), 4, 7, patches=(2, 2), n_track=16, n_obs=3, steps=steps, seed=seed,
                                   dt=2e-4, dx=1 / 16)
    return dict(dim=3, cells=w.n_cells, dx=w.dx, dt=w.dt, g=w.gravity, x=w.x, vol=w.particle_volume, wall=4,
                nseg=(2, 2), mu=w.extras["mu_true"], ids=w.extras["track_ids"], obs=w.extras["obs_steps"])


def orc_for(c, mu):
    return oracle.Oracle(c["dim"], c["cells"], c["dx"], c["dt"], c["g"], dict(inputs.SAND_DP), c["vol"],
                         friction=[(c["wall"], c["nseg"], mu)])


def truth(c):
    o = orc_for(c, c["mu"])
    st = o.initial_state(c["x"])
    z, t = [], 0
    for s in c["obs"]:
        o.step(st, s - t)
        t = s
        z.append(st.x[c["ids"]].copy())
    return np.stack(z)


def oracle_grad(c, mu, z):
    o = orc_for(c, mu)
    d, ids = c["dim"], c["ids"]
    obs = {s: k for k, s in enumerate(c["obs"])}
    states = [o.initial_state(c["x"])]
    loss = 0.0
    for t in range(1, max(obs) + 1):
        s = states[-1].copy()
        o.step(s, 1)
        states.append(s)
        if t in obs:
            loss += float(((s.x[ids] - z[obs[t]]) ** 2).sum())
    n = len(c["x"])
    lam = [np.zeros((n, d)), np.zeros((n, d)), np.zeros((n, d, d)), np.zeros(n), np.zeros((n, 3, 3))]
    grad = np.zeros(len(mu))
    for t in range(max(obs), 0, -1):
        if t in obs:
            lam[0][ids] += 2.0 * (states[t].x[ids] - z[obs[t]])
        lam, mub = o.step_vjp(states[t - 1], *lam)
        grad += mub[c["wall"]]
    return loss, grad


def gpu_grad(c, mu, z, precision=mpm.MPM_FP64, K=50, sort_every=8, keep_bytes=0):
    sim = mpm.Simulation(c["dim"], c["cells"], c["dx"], c["dt"], c["g"], dict(inputs.SAND_DP), precision, sort_every)
    sim.load(c["x"], None, c["vol"])
    mpm.mpm_set_adjoint_memory(sim.ctx, keep_bytes)
    sim.set_friction(c["wall"], c["nseg"], mu)
    mpm.mpm_set_observations(sim.ctx, c["ids"], c["obs"], z)
    loss, grad = mpm.mpm_step_adjoint(sim.ctx, max(c["obs"]), K, c["wall"], len(mu))
    sim.close()
    return loss, grad


@pytest.fixture(scope="module", params=["2d", "3d"])
def problem(request):
    c = column_2d() if request.param == "2d" else column_3d()
    z = truth(c)
    mu = np.full(len(c["mu"]), 0.35)
    ref = oracle_grad(c, mu, z)
    return c, z, mu, ref


def test_sand_fp64_adjoint_matches_oracle_adjoint(problem):
    c, z, mu, (ref_loss, ref_grad) = problem
    loss, grad = gpu_grad(c, mu, z)
    assert np.abs(ref_grad).max() > 0
    assert loss == pytest.approx(ref_loss, rel=1e-8)
    np.testing.assert_allclose(grad, ref_grad, rtol=0, atol=1e-6 * np.abs(ref_grad).max())


def test_sand_fp32_adjoint_close_to_oracle_adjoint(problem):
    c, z, mu, (ref_loss, ref_grad) = problem
    loss, grad = gpu_grad(c, mu, z, mpm.MPM_FP32)
    assert loss == pytest.approx(ref_loss, rel=2e-2)
    cos = grad @ ref_grad / (np.linalg.norm(grad) * np.linalg.norm(ref_grad))
    assert cos >= 0.99


def test_sand_fp64_adjoint_matches_central_differences(problem):
    c, z, mu, _ = problem
    _, grad = gpu_grad(c, mu, z)
    eps = 1e-3
    fd = np.zeros(len(mu))
    for k in range(len(mu)):
        mp_, mm_ = mu.copy(), mu.copy()
        mp_[k] += eps
        mm_[k] -= eps
        fd[k] = (gpu_grad(c, mp_, z)[0] - gpu_grad(c, mm_, z)[0]) / (2 * eps)
    np.testing.assert_allclose(grad, fd, rtol=0, atol=2e-2 * np.abs(fd).max())


def test_sand_checkpoint_interval_does_not_change_the_gradient(problem):
    c, z, mu, _ = problem
    ref = gpu_grad(c, mu, z, K=50)
    for K, se in ((1, 8), (13, 5)):
        loss, grad = gpu_grad(c, mu, z, K=K, sort_every=se)
        assert loss == pytest.approx(ref[0], rel=1e-11)
        np.testing.assert_allclose(grad, ref[1], rtol=0, atol=1e-9 * np.abs(ref[1]).max())


@pytest.mark.parametrize("K,se", [(50, 8), (7, 3), (1, 1)])
def test_sand_3d_fp32_adjoint_matches_fp64_on_a_short_horizon(K, se):
    # Single precision runs the v_bar scatter as a cell-ordered pass over the sort
    # tables of each kept state's generation; on a short horizon it must follow the
    # double-precision gradient to FP32 rounding, whatever the checkpoint and sort
    # intervals (which change the generations a segment holds).
    c = column_3d(steps=60)
    z = truth(c) + 2e-3                       # residuals well above FP32 position rounding
    mu = np.full(4, 0.35)
    l64, g64 = gpu_grad(c, mu, z)
    l32, g32 = gpu_grad(c, mu, z, mpm.MPM_FP32, K=K, sort_every=se)
    assert np.abs(g64).max() > 0
    assert l32 == pytest.approx(l64, rel=1e-3)
    assert np.linalg.norm(g32 - g64) <= 1e-3 * np.linalg.norm(g64)


@pytest.mark.parametrize("precision", [mpm.MPM_FP64, mpm.MPM_FP32])
def test_kept_segments_give_the_recomputed_gradient(problem, precision):
    # with memory to keep every segment of the first pass nothing is recomputed;
    # the gradient is the one of the checkpoint-and-recompute sweep
    c, z, mu, _ = problem
    ref = gpu_grad(c, mu, z, precision, K=50)
    for keep in (1 << 20, 1 << 40):                  # a few segments / all of them
        loss, grad = gpu_grad(c, mu, z, precision, K=50, keep_bytes=keep)
        tol = 1e-9 if precision == mpm.MPM_FP64 else 1e-4
        assert loss == pytest.approx(ref[0], rel=tol)
        assert np.linalg.norm(grad - ref[1]) <= tol * np.linalg.norm(ref[1])
