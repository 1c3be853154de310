"""Device-pointer entry points: mpm_load_particles_dev and mpm_get_particles_dev
give the same state and readback as the host-buffer calls (to the rounding of
the grid's atomic sums, whose order varies from run to run), and reject what the
host calls reject."""
import numpy as np
import pytest
import torch

from paper_2507_04192_gb300 import inputs, mpm

pytestmark = pytest.mark.gpu


def _make(w, precision):
    return mpm.Simulation(w.dim, w.n_cells, w.dx, w.dt, w.gravity, w.material, precision, w.sort_every)


@pytest.mark.parametrize("precision", [mpm.MPM_FP32, mpm.MPM_FP64])
def test_device_load_and_readback_match_the_host_calls(precision):
    w = inputs.granular_cylinder_3d((32, 32, 32), 6, 12, dx=1 / 32, dt=1e-4, steps=20)
    rng = np.random.default_rng(3)
    v = rng.normal(scale=0.1, size=w.x.shape)
    a = _make(w, precision)
    a.load(w.x, v, w.particle_volume)
    a.step(20)
    ref = {f: a.get(f) for f in ("x", "v", "C", "F", "sigma")}
    a.close()
    b = _make(w, precision)
    xd = torch.tensor(w.x, dtype=torch.float64, device="cuda")
    vd = torch.tensor(v, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    mpm.mpm_load_particles_dev(b.ctx, w.n, xd.data_ptr(), vd.data_ptr(), w.particle_volume)
    del xd, vd                                   # the call has copied them
    b.step(20)
    for f, r in ref.items():
        out = torch.empty(r.size, dtype=torch.float64, device="cuda")
        mpm.mpm_get_particles_dev(b.ctx, f, out.data_ptr())
        b.synchronize()
        tol = (1e-5 if precision == mpm.MPM_FP32 else 1e-11) * max(float(np.abs(r).max()), 1e-30)
        np.testing.assert_allclose(out.cpu().numpy().reshape(r.shape), r, rtol=0, atol=tol, err_msg=f)
    b.close()


def test_device_load_rejects_what_the_host_load_rejects():
    w = inputs.dam_break_2d(16, 0.25, 0.25)
    sim = mpm.Simulation(2, w.n_cells, w.dx, w.dt, w.gravity, w.material, mpm.MPM_FP32, 8, batch=2)
    x = w.x.copy()
    x[7, 0] = -1e-3                              # outside the domain
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_load_particles_dev(sim.ctx, w.n, xd.data_ptr(), None, w.particle_volume)
    assert e.value.code == mpm.MPM_EINVAL and "outside" in str(e.value)
    xd = torch.tensor(w.x, dtype=torch.float64, device="cuda")
    sid = torch.zeros(w.n, dtype=torch.int32, device="cuda")
    sid[3] = 2                                   # batch is 2
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_load_particles_dev(sim.ctx, w.n, xd.data_ptr(), None, w.particle_volume, sid.data_ptr())
    assert e.value.code == mpm.MPM_EINVAL and "simulation id" in str(e.value)
    sid[3] = 1
    mpm.mpm_load_particles_dev(sim.ctx, w.n, xd.data_ptr(), None, w.particle_volume, sid.data_ptr())
    assert mpm.mpm_num_particles(sim.ctx) == w.n
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_get_particles_dev(sim.ctx, "x", 0)
    assert e.value.code == mpm.MPM_EINVAL
    sim.close()
