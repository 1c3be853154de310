"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle on
identical seeded inputs.

Tolerances (from the targets of the explicit step): FP64 positions within
1e-9 of the domain size and FP32 within 1e-4 after 200 steps of the 2D dam
break; the other fields scale with the same bound.  Where atomics change the
summation order, results differ by rounding only, so FP64 single-step fields
agree to ~1e-12 relative.
"""
import numpy as np
import pytest

import oracle
from paper_2507_04192_gb300 import inputs, mpm

pytestmark = pytest.mark.gpu

FIELDS = ("x", "v", "C", "F", "rho", "sigma", "eps")


def run_oracle(w, steps, dp_literal=False):
    orc = oracle.Oracle.from_workload(w, dp_literal=dp_literal)
    st = orc.initial_state(w.x, w.v)
    orc.step(st, steps)
    return dict(x=st.x, v=st.v, C=orc.affine_C(st), F=st.F, rho=st.rho, sigma=st.sigma, eps=st.eps)


def run_gpu(w, steps, precision, sort_every=None, chunked=None):
    sim = mpm.Simulation.from_workload(w, precision, sort_every)
    if chunked:
        for n in chunked:
            sim.step(n)
    else:
        sim.step(steps)
    out = {f: sim.get(f) for f in FIELDS}
    stats = sim.stats()
    sim.close()
    return out, stats


def assert_close(gpu, ref, field, atol, rtol=0.0):
    np.testing.assert_allclose(gpu[field].reshape(ref[field].shape), ref[field], rtol=rtol, atol=atol,
                               err_msg=field)


def scale(a):
    return max(float(np.abs(a).max()), 1e-30)


def test_dam_break_fp64_200_steps():
    w = inputs.dam_break_2d(64)                      # 8,192 particles, 64 x 64 cells, dt = 1e-4
    ref = run_oracle(w, 200)
    gpu, stats = run_gpu(w, 200, mpm.MPM_FP64)
    L = 1.0
    assert np.abs(gpu["x"] - ref["x"]).max() <= 1e-9 * L
    assert_close(gpu, ref, "v", 1e-7 * scale(ref["v"]))
    assert_close(gpu, ref, "C", 1e-6 * scale(ref["C"]))
    assert_close(gpu, ref, "rho", 1e-9 * 1000.0)
    assert_close(gpu, ref, "sigma", 1e-6 * scale(ref["sigma"]))
    assert_close(gpu, ref, "F", 1e-7)
    assert stats["steps"] == 200 and stats["sorts"] >= 200 // w.sort_every


def test_dam_break_fp32_200_steps():
    w = inputs.dam_break_2d(64)
    ref = run_oracle(w, 200)
    gpu, _ = run_gpu(w, 200, mpm.MPM_FP32)
    assert np.abs(gpu["x"] - ref["x"]).max() <= 1e-4 * 1.0
    assert_close(gpu, ref, "rho", 1e-3 * 1000.0)
    # every other field at the stated FP32 bounds (relative to the field's largest value;
    # F, dimensionless and near I, absolute)
    assert_close(gpu, ref, "v", 2e-3 * scale(ref["v"]))
    assert_close(gpu, ref, "C", 5e-3 * scale(ref["C"]))
    assert_close(gpu, ref, "F", 1e-4)
    K = w.material["bulk_K"]
    assert_close(gpu, ref, "sigma", 5e-3 * scale(ref["sigma"]) + 1e-6 * K)


@pytest.mark.parametrize("precision", [mpm.MPM_FP64, mpm.MPM_FP32])
def test_single_step_all_fields_2d(precision):
    rng = np.random.default_rng(3)
    w = inputs.dam_break_2d(32, 0.5, 0.5)
    w.v = rng.normal(size=w.x.shape) * 0.5
    ref = run_oracle(w, 3)
    gpu, _ = run_gpu(w, 3, precision)
    tol = 1e-12 if precision == mpm.MPM_FP64 else 2e-5
    for f in ("x", "v", "C", "F", "rho"):
        assert_close(gpu, ref, f, tol * scale(ref[f]) + (tol if f in ("x", "F") else 0.0))
    # the fluid pressure is K/gamma ((rho/rho0)^gamma - 1): its rounding error is K times the
    # relative error of rho, not a fraction of |sigma|
    K = w.material["bulk_K"]
    assert_close(gpu, ref, "sigma", tol * scale(ref["sigma"]) + (1e-6 * K if precision == mpm.MPM_FP32 else 0.0))


def small_cylinder(seed=0):
    return inputs.granular_cylinder_3d((32, 32, 32), 6, 12, seed=seed, floor_mu=0.4)


def test_granular_cylinder_3d_fp64():
    w = small_cylinder()
    ref = run_oracle(w, 60)
    gpu, _ = run_gpu(w, 60, mpm.MPM_FP64)
    L = 32 * w.dx
    assert np.abs(gpu["x"] - ref["x"]).max() <= 1e-9 * L
    assert_close(gpu, ref, "v", 1e-7 * scale(ref["v"]))
    assert_close(gpu, ref, "sigma", 1e-6 * scale(ref["sigma"]))
    assert_close(gpu, ref, "eps", 1e-6 * scale(ref["eps"]) + 1e-15)
    assert_close(gpu, ref, "F", 1e-8)


def test_granular_cylinder_3d_fp32():
    w = small_cylinder()
    ref = run_oracle(w, 60)
    gpu, _ = run_gpu(w, 60, mpm.MPM_FP32)
    L = 32 * w.dx
    assert np.abs(gpu["x"] - ref["x"]).max() <= 1e-4 * L
    assert_close(gpu, ref, "sigma", 2e-3 * scale(ref["sigma"]))


def test_basal_friction_segments_fp64():
    w = inputs.dam_break_inverse_2d(64, n_seg=32, steps=150)
    ref = run_oracle(w, 150)
    gpu, _ = run_gpu(w, 150, mpm.MPM_FP64)
    assert np.abs(gpu["x"] - ref["x"]).max() <= 1e-9
    # the friction field matters: the slip result is clearly different
    w_slip = inputs.dam_break_2d(64, steps=150)
    slip = run_oracle(w_slip, 150)
    assert np.abs(slip["x"] - ref["x"]).max() > 1e-4


def test_sort_interval_does_not_change_results_fp64():
    w = inputs.dam_break_2d(64)
    a, sa = run_gpu(w, 120, mpm.MPM_FP64, sort_every=1)
    b, sb = run_gpu(w, 120, mpm.MPM_FP64, sort_every=40, chunked=[7, 50, 63])
    assert np.abs(a["x"] - b["x"]).max() <= 1e-12
    assert sa["sorts"] == 120


def test_batched_sims_match_single_runs_fp64():
    base = inputs.dam_break_inverse_2d(32, n_seg=8, steps=80)
    mus = [inputs.friction_field(8, s) for s in (1, 2, 3)]
    B = len(mus)
    sim = mpm.Simulation(2, base.n_cells, base.dx, base.dt, base.gravity, base.material, mpm.MPM_FP64, 8, batch=B)
    x = np.concatenate([base.x] * B)
    sid = np.repeat(np.arange(B, dtype=np.int32), base.n)
    sim.load(x, None, base.particle_volume, sid)
    sim.set_friction(2, (8, 1), np.concatenate(mus))
    sim.step(80)
    xb = sim.get("x").reshape(B, base.n, 2)
    sim.close()
    for b, mu in enumerate(mus):
        w = inputs.dam_break_inverse_2d(32, n_seg=8, steps=80)
        w.friction = [(2, (8, 1), mu)]
        ref = run_oracle(w, 80)
        assert np.abs(xb[b] - ref["x"]).max() <= 1e-9


def test_edge_cases_single_and_boundary_particles():
    # one particle; particles exactly on the walls and corners; a ragged count
    w = inputs.dam_break_2d(16, 0.25, 0.25)
    extra = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0], [0.5, 0.0], [1.0, 0.37]])
    for x in (extra[:1], np.concatenate([w.x[:997], extra])):
        ww = inputs.dam_break_2d(16, 0.25, 0.25)
        ww.x = x
        ref = run_oracle(ww, 30)
        gpu, _ = run_gpu(ww, 30, mpm.MPM_FP64)
        assert np.abs(gpu["x"] - ref["x"]).max() <= 1e-10
        assert gpu["x"].min() >= 0.0 and gpu["x"].max() <= 1.0


def test_fast_particles_take_the_out_of_tile_path():
    """Sorting only every 64 steps while particles move several cells: the
    out-of-window path keeps the result exact."""
    w = inputs.dam_break_2d(64, 0.2, 0.2)
    w.x = w.x + 0.3                                 # block [0.3, 0.5]^2, far from the walls
    w.v = np.tile([4.0, 1.0], (w.n, 1))             # 1.6 cells in 64 steps at dt = 1e-4, dx = 1/64
    ref = run_oracle(w, 64)
    gpu, stats = run_gpu(w, 64, mpm.MPM_FP64, sort_every=64)
    assert stats["escaped"] > 0
    assert np.abs(gpu["x"] - ref["x"]).max() <= 1e-9


def test_fast_particles_fp32_cell_ordered_p2g_escape_path():
    """The 2D single-precision P2G sums per cell; particles that left their cell
    since the last sort (here: every particle, several cells away) are scattered
    one by one.  Both paths against the oracle."""
    w = inputs.dam_break_2d(64, 0.2, 0.2)
    w.x = w.x + 0.3
    w.v = np.tile([4.0, 1.0], (w.n, 1))
    ref = run_oracle(w, 64)
    gpu, stats = run_gpu(w, 64, mpm.MPM_FP32, sort_every=64)
    assert stats["escaped"] > 0
    assert np.abs(gpu["x"] - ref["x"]).max() <= 1e-4
    assert np.abs(gpu["v"] - ref["v"]).max() <= 1e-4 * np.abs(ref["v"]).max()


def test_batched_2d_fluid_fp32_matches_oracle_per_simulation():
    # the 2D cell-ordered P2G over several simulations of one context (per-simulation
    # grid offsets and friction), each against its own oracle run
    base = inputs.dam_break_inverse_2d(32, n_seg=8, steps=80)
    mus = [inputs.friction_field(8, s) for s in (1, 2, 3)]
    B = len(mus)
    sim = mpm.Simulation(2, base.n_cells, base.dx, base.dt, base.gravity, base.material, mpm.MPM_FP32, 8, batch=B)
    sim.load(np.concatenate([base.x] * B), None, base.particle_volume,
             np.repeat(np.arange(B, dtype=np.int32), base.n))
    sim.set_friction(2, (8, 1), np.concatenate(mus))
    sim.step(80)
    xb = sim.get("x").reshape(B, base.n, 2)
    sim.close()
    for b, mu in enumerate(mus):
        w = inputs.dam_break_inverse_2d(32, n_seg=8, steps=80)
        w.friction = [(2, (8, 1), mu)]
        ref = run_oracle(w, 80)
        assert np.abs(xb[b] - ref["x"]).max() <= 1e-4


def test_set_field_roundtrip_and_errors():
    w = inputs.dam_break_2d(32, 0.25, 0.25)
    sim = mpm.Simulation.from_workload(w, mpm.MPM_FP64)
    rng = np.random.default_rng(2)
    v = rng.normal(size=w.x.shape)
    sim.set_field("v", v)
    sim.step(3)                                      # sorted internally
    sim.set_field("v", v)
    np.testing.assert_array_equal(sim.get("v"), v)
    with pytest.raises(mpm.MPMError) as e:
        sim.set_field("sigma", np.zeros((w.n, 9)))   # fluid stress follows from rho
    assert e.value.code == mpm.MPM_EINVAL
    sim.close()


def test_nonfinite_state_is_reported_not_trapped():
    w = inputs.dam_break_2d(32, 0.25, 0.25)
    sim = mpm.Simulation.from_workload(w, mpm.MPM_FP32)
    rho = np.full(w.n, 1000.0)
    rho[5] = np.nan
    sim.set_field("rho", rho)
    sim.step(2)
    with pytest.raises(mpm.MPMError) as e:
        sim.synchronize()
    assert e.value.code == mpm.MPM_ENAN
    sim.close()


@pytest.mark.slow
@pytest.mark.parametrize("precision", [mpm.MPM_FP32, mpm.MPM_FP64])
def test_full_size_granular_cylinder_two_steps(precision):
    """The 2.76M-particle 3D collapse in the configuration the benchmark times."""
    w = inputs.granular_cylinder_3d()
    ref = run_oracle(w, 2)
    gpu, stats = run_gpu(w, 2, precision)
    L = 0.5
    tol = 1e-9 if precision == mpm.MPM_FP64 else 1e-4
    assert np.abs(gpu["x"] - ref["x"]).max() <= tol * L
    rs = scale(ref["sigma"])
    assert np.abs(gpu["sigma"].reshape(-1, 3, 3) - ref["sigma"]).max() <= (1e-8 if precision else 1e-3) * rs


def test_batched_3d_sand_fp32_matches_oracle_per_simulation():
    # several simulations in one context take the window-free P2G's per-simulation
    # grid offsets; each must follow its own oracle run
    base = inputs.granular_cylinder_3d((16, 16, 16), 4, 8, dt=2e-4, dx=1 / 16, floor_mu=0.0, steps=30)
    mus = [0.1, 0.4, 0.8]
    B = len(mus)
    sim = mpm.Simulation(3, base.n_cells, base.dx, base.dt, base.gravity, base.material, mpm.MPM_FP32, 8, batch=B)
    sim.load(np.concatenate([base.x] * B), None, base.particle_volume,
             np.repeat(np.arange(B, dtype=np.int32), base.n))
    sim.set_friction(4, (1, 1), np.array(mus))
    sim.step(30)
    xb = sim.get("x").reshape(B, base.n, 3)
    sim.close()
    for b, mu in enumerate(mus):
        w = inputs.granular_cylinder_3d((16, 16, 16), 4, 8, dt=2e-4, dx=1 / 16, floor_mu=mu, steps=30)
        ref = run_oracle(w, 30)
        assert np.abs(xb[b] - ref["x"]).max() <= 1e-4
