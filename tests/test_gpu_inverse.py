"""Plain adjoint inversion of the basal friction field (Sec. 5.3) on the GPU,
the autograd wrapper, and state save/restore/export on the device."""
import numpy as np
import pytest

import oracle
from paper_2507_04192_gb300 import inputs, inverse, mpm

pytestmark = pytest.mark.gpu


def observations(w, mu):
    orc = oracle.Oracle(2, w.n_cells, w.dx, w.dt, w.gravity, w.material, w.particle_volume,
                        friction=[(2, (len(mu), 1), mu)])
    st = orc.initial_state(w.x)
    z, t = [], 0
    for s in w.extras["obs_steps"]:
        orc.step(st, s - t)
        t = s
        z.append(st.x[w.extras["track_ids"]].copy())
    return np.stack(z)


def test_autograd_function_returns_the_adjoint_gradient():
    torch = pytest.importorskip("torch")
    w = inputs.dam_break_inverse_2d(32, n_seg=8, n_track=32, n_obs=4, steps=300)
    z = observations(w, w.extras["mu_true"])
    prob = inverse.FrictionInversion(w, z, mpm.MPM_FP64, checkpoint_every=50)
    mu = torch.full((8,), 0.35, dtype=torch.float64, requires_grad=True)
    loss = inverse.friction_loss(mu, prob)
    (2.0 * loss).backward()
    L, g = prob.loss_and_grad(np.full(8, 0.35))
    assert float(loss) == pytest.approx(L, rel=1e-12)
    np.testing.assert_allclose(mu.grad.numpy(), 2.0 * g, rtol=1e-12, atol=0)
    prob.close()


def test_plain_inversion_recovers_the_constrained_segments():
    """Adam from the uniform guess 0.35 with the paper's decaying rate from 0.1."""
    w = inputs.dam_break_inverse_2d(32, n_seg=8, n_track=64, n_obs=10, steps=300, seed=1)
    mu_true = w.extras["mu_true"]
    z = observations(w, mu_true)
    prob = inverse.FrictionInversion(w, z, mpm.MPM_FP32, checkpoint_every=50)
    mu0 = np.full(8, 0.35)
    mask = inverse.constrained_segments(prob, mu0)
    assert 1 <= mask.sum() < 8
    res = inverse.invert(prob, mu0, mu_true, mask, tol=0.05, max_iters=150)
    assert res.converged and res.iterations < 150
    assert inverse.relative_error(res.mu, mu_true, mask) <= 0.05
    assert res.history[-1]["loss"] < 0.1 * res.history[0]["loss"]
    prob.close()


def test_state_slots_and_checksummed_blob():
    w = inputs.dam_break_2d(32, 0.25, 0.5)
    sim = mpm.Simulation.from_workload(w, mpm.MPM_FP64)
    sim.step(5)
    mpm.mpm_save_state(sim.ctx, 3)
    blob = mpm.mpm_export_state(sim.ctx)
    x5 = sim.get("x")
    sim.step(20)
    x25 = sim.get("x")
    mpm.mpm_restore_state(sim.ctx, 3)
    np.testing.assert_array_equal(sim.get("x"), x5)
    sim.step(20)
    np.testing.assert_allclose(sim.get("x"), x25, rtol=0, atol=1e-12)
    mpm.mpm_import_state(sim.ctx, blob)
    np.testing.assert_array_equal(sim.get("x"), x5)
    bad = bytearray(blob)
    bad[-5] ^= 0xFF
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_import_state(sim.ctx, bytes(bad))
    assert e.value.code == mpm.MPM_ECORRUPT
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_restore_state(sim.ctx, 7)
    assert e.value.code == mpm.MPM_ESTATE
    sim.close()
