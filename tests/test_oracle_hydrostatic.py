"""Pin of the oracle's fluid step against hydrostatic equilibrium: a column
filling the width of the box settles to p = rho0 g h (Sec. 2.3, Tait EOS)."""
import numpy as np
import pytest

import oracle
from paper_2507_04192_gb300 import inputs


@pytest.mark.slow
def test_hydrostatic_column_settles_to_rho_g_h():
    # 8 x 8 cells of water filling the width of an 8 x 16 cell box (dx = 1/32)
    dx = 1.0 / 32
    H0 = 0.25
    x0 = inputs.lattice_particles((8, 16), dx, 4, lambda p: p[:, 1] < H0, (0, 0), (0.25, H0), seed=7)
    mat = dict(inputs.FLUID_WATER)
    g = 9.81
    dt = 1e-4
    orc = oracle.Oracle(2, (8, 16), dx, dt, (0.0, -g), mat, dx * dx / 16)
    st = orc.initial_state(x0)
    y0 = x0[:, 1].copy()
    period = int(4 * H0 / np.sqrt(mat["bulk_K"] / mat["rho0"]) / dt)    # acoustic period in steps
    orc.step(st, 4 * period)
    acc = np.zeros(len(x0))
    samples = 0
    for _ in range(period // 10):
        orc.step(st, 10)
        acc += -np.trace(st.sigma, axis1=1, axis2=2) / 3.0
        samples += 1
    p = acc / samples
    # Lagrangian depth: mass above a particle per unit width is rho0 (H0 - y0)
    p_weight = mat["rho0"] * g * (H0 - y0)
    p_bottom = mat["rho0"] * g * H0
    # cell-averaged pressure (4 particle layers per cell); the first cell above the floor is the
    # boundary layer of the quadratic stencil (its particles share stencils with the wall and ghost
    # nodes, whose velocities the wall fixes), where particle pressures are not fixed by nodal
    # equilibrium alone
    cell = np.floor(y0 / dx).astype(int)
    for k in np.unique(cell):
        if k == 0:
            continue
        sel = cell == k
        assert p[sel].mean() == pytest.approx(p_weight[sel].mean(), abs=0.03 * p_bottom), f"cell {k}"
    # Tait closed form with the settled depth below the free surface
    gam, K, rho0 = mat["gamma"], mat["bulk_K"], mat["rho0"]
    top = y0 > H0 - dx / 4                      # initial top layer of particles
    surface = st.x[top, 1].mean() + 0.5 * dx / 4
    depth = surface - st.x[:, 1]
    p_tait = K / gam * ((1 + (gam - 1) * rho0 * g * depth / K) ** (gam / (gam - 1)) - 1)
    for k in np.unique(cell):
        sel = (cell == k) & (depth > 0.25 * H0)
        if k == 0 or not sel.any():
            continue
        assert p[sel].mean() == pytest.approx(p_tait[sel].mean(), abs=0.03 * p_bottom), f"cell {k}"
