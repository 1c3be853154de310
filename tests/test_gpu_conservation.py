"""The mass gate of the explicit step on the GPU: the grid mass the
particle-to-grid transfer produces equals the particle mass, and the grid
momentum (q_i + dt f_i, Eq. semi) equals sum_p m_p v_p.

Why this holds: the quadratic B-spline weights of Sec. 2.1 form a partition of
unity (sum_i w_ip = 1), reproduce linear functions (sum_i w_ip (x_i - x_p) = 0,
so the APIC term adds no net momentum) and have gradients summing to zero
(sum_i grad w_ip = 0, so the stress force adds none); the sums therefore agree
up to rounding.  Bounds: 1e-12 relative in FP64 (the conservation target of
the explicit step) and 1e-6 in FP32 for the mass; the momentum difference is
bounded relative to sum_i |q_i + dt f_i| (the size of the terms that cancel).
The sums are taken on the device in double precision (mpm_get_diagnostics).
"""
import numpy as np
import pytest

from paper_2507_04192_gb300 import inputs, mpm

pytestmark = pytest.mark.gpu

MASS_TOL = {mpm.MPM_FP64: 1e-12, mpm.MPM_FP32: 1e-6}
MOM_TOL = {mpm.MPM_FP64: 1e-12, mpm.MPM_FP32: 1e-4}


def check(d, precision, n, mass):
    assert d["grid_nonfinite"] == 0 and d["particle_nonfinite"] == 0
    assert d["particle_mass"] == pytest.approx(n * mass, rel=1e-14)
    rel = abs(d["grid_mass"] - d["particle_mass"]) / d["particle_mass"]
    assert rel <= MASS_TOL[precision], rel
    dm = np.abs(d["grid_momentum"] - d["particle_momentum"]).max()
    assert dm <= MOM_TOL[precision] * d["grid_abs_momentum"] + 1e-300, (dm, d["grid_abs_momentum"])
    return rel


@pytest.mark.parametrize("precision", [mpm.MPM_FP64, mpm.MPM_FP32])
def test_dam_break_mass_and_momentum_every_step(precision):
    w = inputs.dam_break_2d(64)                      # 8,192 particles, 200 steps (the 2D parity workload)
    sim = mpm.Simulation.from_workload(w, precision)
    mpm.mpm_set_diagnostics(sim.ctx, True)
    mass = w.material["rho0"] * w.particle_volume
    worst = 0.0
    for s in range(200):
        sim.step(1)
        if s % 10 == 0 or s == 199:
            worst = max(worst, check(mpm.mpm_get_diagnostics(sim.ctx), precision, w.n, mass))
    v = sim.get("v")
    sim.close()
    assert np.abs(v).max() > 0.1                       # the column is collapsing: momentum is not trivially zero
    print(f"\nworst relative grid-mass error over 200 steps: {worst:.2e}")


@pytest.mark.parametrize("precision", [mpm.MPM_FP32, mpm.MPM_FP64])
def test_full_size_cylinder_mass_gate(precision):
    w = inputs.granular_cylinder_3d()                # 2,761,536 particles, 256 x 256 x 128
    sim = mpm.Simulation.from_workload(w, precision)
    mpm.mpm_set_diagnostics(sim.ctx, True)
    mass = w.material["rho0"] * w.particle_volume
    for _ in range(3):
        sim.step(1)
        check(mpm.mpm_get_diagnostics(sim.ctx), precision, w.n, mass)
    sim.close()


def test_batched_grid_mass_is_the_sum_over_simulations():
    w = inputs.dam_break_2d(32, 0.25, 0.5)
    B = 4
    sim = mpm.Simulation(2, w.n_cells, w.dx, w.dt, w.gravity, w.material, mpm.MPM_FP32, w.sort_every, batch=B)
    sim.load(np.tile(w.x, (B, 1)), None, w.particle_volume, np.repeat(np.arange(B, dtype=np.int32), w.n))
    mpm.mpm_set_diagnostics(sim.ctx, True)
    sim.step(5)
    d = mpm.mpm_get_diagnostics(sim.ctx)
    sim.close()
    check(d, mpm.MPM_FP32, B * w.n, w.material["rho0"] * w.particle_volume)


def test_diagnostics_need_a_step_and_can_be_turned_off():
    w = inputs.dam_break_2d(32, 0.25, 0.5)
    sim = mpm.Simulation.from_workload(w, mpm.MPM_FP64)
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_get_diagnostics(sim.ctx)
    assert e.value.code == mpm.MPM_ESTATE
    mpm.mpm_set_diagnostics(sim.ctx, True)
    sim.step(1)
    d1 = mpm.mpm_get_diagnostics(sim.ctx)
    mpm.mpm_set_diagnostics(sim.ctx, False)
    launches = sim.stats()["launches"]
    sim.step(1)
    assert sim.stats()["launches"] - launches == 3      # P2G, grid update, G2P: no diagnostics kernel
    d2 = mpm.mpm_get_diagnostics(sim.ctx)              # the sums of the last step that took them
    sim.close()
    assert d2["grid_mass"] == d1["grid_mass"]
