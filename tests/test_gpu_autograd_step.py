"""The per-step autograd Function (autograd.Stepper, backed by mpm_step_adjoint_1):
its loss gradient against the whole-horizon adjoint (mpm_step_adjoint) for
tracked positions (Eq. inverse_loss, Sec. 3.2), and against central differences
for a loss on every column of the state (x, v, C, rho and the Drucker-Prager
stress) at two times."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_04192_gb300 import autograd, inputs, mpm

pytestmark = pytest.mark.gpu


def sim_of(w, precision, v0=None):
    sim = mpm.Simulation(w.dim, w.n_cells, w.dx, w.dt, w.gravity, w.material, precision, w.sort_every)
    sim.load(w.x, v0, w.particle_volume)
    return sim


def test_tracked_position_loss_matches_the_whole_adjoint_fluid_2d():
    w = inputs.dam_break_inverse_2d(32, n_seg=8, steps=12)
    mu0 = inputs.friction_field(8, 7)
    ids = np.asarray(w.extras["track_ids"], dtype=np.int64)
    rng = np.random.default_rng(3)
    obs = [6, 12]
    z = np.stack([w.x[ids] + rng.normal(scale=2 * w.dx, size=(len(ids), 2)) for _ in obs])

    sim = sim_of(w, mpm.MPM_FP64)
    sim.set_friction(2, (8, 1), mu0)
    st = autograd.Stepper(sim, 2, (8, 1))
    mu = torch.tensor(mu0, requires_grad=True)
    s = st.reset()
    s0 = s.requires_grad_(True)
    loss = torch.zeros((), dtype=torch.float64)
    zt = torch.from_numpy(z)
    for t in range(1, 13):
        s = st.step(s, mu)
        if t in obs:
            loss = loss + ((s[ids, :2] - zt[obs.index(t)]) ** 2).sum()
    loss.backward()
    loss = loss.detach()
    sim.close()

    ref = sim_of(w, mpm.MPM_FP64)
    ref.set_friction(2, (8, 1), mu0)
    mpm.mpm_set_observations(ref.ctx, ids, obs, z)
    ref_loss, ref_grad = mpm.mpm_step_adjoint(ref.ctx, 12, 5, 2, 8)
    lam0 = {f: mpm.mpm_get_initial_adjoint(ref.ctx, f).reshape(w.n, -1) for f in ("x", "v", "C", "rho")}
    ref.close()

    assert float(loss) == pytest.approx(ref_loss, rel=1e-12)
    assert np.abs(ref_grad).max() > 0
    np.testing.assert_allclose(mu.grad.numpy(), ref_grad, rtol=0, atol=1e-9 * np.abs(ref_grad).max())
    g0 = s0.grad.numpy()
    for f, sl in (("x", slice(0, 2)), ("v", slice(2, 4)), ("C", slice(4, 8)), ("rho", slice(8, 9))):
        scale = max(float(np.abs(lam0[f]).max()), 1e-30)
        np.testing.assert_allclose(g0[:, sl], lam0[f], rtol=0, atol=1e-9 * scale, err_msg=f)


def test_state_columns_and_a_loss_on_all_of_them_sand_3d():
    # sand from a moving start (converging, downward), away from the apex of the
    # yield cone where the return mapping has a kink
    w = inputs.granular_cylinder_3d((24, 24, 24), 5, 10, dx=1 / 24, dt=2e-4, floor_mu=0.0, steps=10)
    cx, cy = w.extras["axis"]
    v0 = np.zeros_like(w.x)
    v0[:, 0] = -2.0 * (w.x[:, 0] - cx)
    v0[:, 1] = -2.0 * (w.x[:, 1] - cy)
    v0[:, 2] = -0.2
    mu0 = np.array([0.2, 0.3, 0.4, 0.5])
    sim = sim_of(w, mpm.MPM_FP64, v0)
    sim.set_friction(4, (2, 2), mu0)
    st = autograd.Stepper(sim, 4, (2, 2))
    assert st.width == 3 + 3 + 9 + 1 + 6

    # the state tensor holds the context's fields in the adjoint layout
    s = st.reset()
    for _ in range(3):
        s = st.step(s, torch.tensor(mu0))
    sg = sim.get("sigma")
    np.testing.assert_array_equal(s[:, 0:3].numpy(), sim.get("x"))
    np.testing.assert_array_equal(s[:, 3:6].numpy(), sim.get("v"))
    np.testing.assert_array_equal(s[:, 6:15].numpy(), sim.get("C").reshape(-1, 9))
    np.testing.assert_array_equal(s[:, 15].numpy(), sim.get("rho"))
    np.testing.assert_array_equal(s[:, 16:22].numpy(), np.stack([sg[:, 0, 0], sg[:, 1, 1], sg[:, 2, 2],
                                                                  sg[:, 0, 1], sg[:, 0, 2], sg[:, 1, 2]], 1))
    scale = np.maximum(np.abs(s.numpy()).mean(0), 1e-12)

    rng = np.random.default_rng(11)
    W = [torch.from_numpy(rng.normal(size=(w.n, 22)) / scale) for _ in range(2)]

    def loss_of(mu_t):
        s = st.reset()
        loss = torch.zeros((), dtype=torch.float64)
        for t in range(1, 11):
            s = st.step(s, mu_t)
            if t in (5, 10):
                loss = loss + (W[t // 5 - 1] * s).sum()
        return loss

    mu = torch.tensor(mu0, requires_grad=True)
    loss_of(mu).backward()
    g = mu.grad.numpy()
    with pytest.raises(RuntimeError):
        st.step(s, torch.tensor(mu0))                       # the context has moved on
    delta = rng.normal(size=4)
    delta /= np.linalg.norm(delta)
    eps = 1e-5
    with torch.no_grad():
        lp = float(loss_of(torch.tensor(mu0 + eps * delta)))
        lm = float(loss_of(torch.tensor(mu0 - eps * delta)))
    fd = (lp - lm) / (2 * eps)
    sim.close()
    assert abs(g @ delta) > 0
    assert g @ delta == pytest.approx(fd, rel=1e-4)
