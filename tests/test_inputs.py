"""The synthetic workloads reproduce the sizes of the paper's scenarios and of
the configurations they stand for (particle counts, grids, geometry of the
obstacles and monitors, observation schedules); the generator is seeded and
deterministic."""
import numpy as np

from paper_2507_04192_gb300 import inputs


def test_particle_counts_of_the_configurations():
    assert inputs.dam_break_2d(64).n == 8_192                  # 16 x 32 cells x 16
    assert inputs.dam_break_inverse_2d(128).n == 32_768
    assert inputs.dam_break_2d(96).n == 18_432
    assert inputs.granular_cylinder_3d().n == 2_761_536
    assert inputs.granular_cylinder_3d((192, 192, 96), 30, 60).n == 1_356_480


def test_3d_dam_break_geometry():
    w = inputs.dam_break_3d()
    assert w.n == 1_920_000                                   # 60 x 100 x 40 cells x 8 (Sec. 4.1)
    assert w.n_cells == (200, 100, 80) and abs(w.dx - 0.005) < 1e-15
    np.testing.assert_allclose(w.domain, (1.0, 0.5, 0.4))
    assert w.x[:, 0].max() < 0.3 and w.x[:, 2].max() < 0.2
    (lo0, hi0), (lo1, hi1) = w.obstacles
    np.testing.assert_allclose(np.subtract(hi0, lo0)[:2], (0.04, 0.04))
    np.testing.assert_allclose(np.subtract(hi1, lo1)[:2], (0.06, 0.06))
    np.testing.assert_allclose((np.add(lo0, hi0) / 2)[:2], (0.5, 0.3))
    np.testing.assert_allclose((np.add(lo1, hi1) / 2)[:2], (0.6, 0.1))
    assert lo0[2] == 0.0 and hi0[2] == w.domain[2]
    assert w.material["gamma"] == 1.0 and w.material["bulk_K"] == 1000.0 * 35.0 ** 2


def test_velocity_inverse_problem():
    w = inputs.dam_break_velocity_inverse()
    assert w.n == 10_000 and w.n_cells == (150, 60)           # Table 3: 150 x 60, 10,000 particles
    steps = w.extras["obs_steps"]
    assert len(steps) == 100 and steps[-1] == 10_000 and steps[0] == 9_010
    assert np.all(np.diff(steps) == 10)
    centres = sorted(tuple(np.round((np.add(lo, hi) / 2), 12)) for lo, hi in w.extras["monitors"])
    assert centres == sorted((x, y) for x in (0.2, 0.3, 0.4) for y in (0.1, 0.2, 0.3))
    for lo, hi in w.extras["monitors"]:
        np.testing.assert_allclose(np.subtract(hi, lo), (0.02, 0.02))
    np.testing.assert_allclose(w.v[:, 0], 2.0 * (0.5 - w.x[:, 1]))
    assert inputs.dam_break_velocity_inverse(dx=0.005).n == 40_000


def test_generator_is_deterministic_and_seeded():
    a = inputs.dam_break_2d(32, seed=3)
    b = inputs.dam_break_2d(32, seed=3)
    c = inputs.dam_break_2d(32, seed=4)
    np.testing.assert_array_equal(a.x, b.x)
    assert np.abs(a.x - c.x).max() > 0
