"""Pins of the oracle's wall contact (Eq. coulomb_friction, Sec. 5.3) and grid
update (Sec. 2.2) against the Coulomb law, hand-worked nodes (segments, the wall
order at an edge) and a sliding-block solution, and of the position clamp of
G2P."""
import numpy as np
import pytest

import oracle
from paper_2507_04192_gb300 import inputs


def _unit(v):
    return v / np.linalg.norm(v)


def test_coulomb_law_per_node():
    rng = np.random.default_rng(0)
    for _ in range(2000):
        n = _unit(rng.normal(size=3))
        v = rng.normal(size=3)
        mu = rng.choice([0.0, rng.uniform(0.0, 1.5)])
        out = oracle.friction(v, n, mu)
        vn = v @ n
        vt = v - vn * n
        if vn <= 0.0:                                   # separating: untouched
            np.testing.assert_allclose(out, v, atol=1e-15)
            continue
        assert abs(out @ n) < 1e-12                     # normal approach removed
        ot = out - (out @ n) * n
        if mu == 0.0:
            np.testing.assert_allclose(out, vt, atol=1e-12)   # slip wall
        elif np.linalg.norm(vt) <= mu * vn:
            np.testing.assert_allclose(out, 0.0, atol=1e-12)  # sticking
        else:                                           # sliding: |v_t| reduced by mu v_n, same direction
            assert np.linalg.norm(ot) == pytest.approx(np.linalg.norm(vt) - mu * vn, rel=1e-10, abs=1e-12)
            assert ot @ vt > 0.0
            np.testing.assert_allclose(np.cross(ot, vt), 0.0, atol=1e-10)


def test_grid_update_walls_and_segments():
    """Nodes on or beyond a face get the contact correction with their segment's mu."""
    N = 8
    dx = 1.0 / N
    mu = np.array([0.0, 0.2, 0.5, 1.0])
    orc = oracle.Oracle(2, (N, N), dx, 1e-3, (0.0, 0.0), dict(inputs.FLUID_WATER), dx * dx,
                        friction=[(2, (4, 1), mu)])
    G = orc.num_nodes
    gm = np.ones(G)
    v = np.array([0.3, -0.4])                           # moving down and right
    gq = np.tile(v, (G, 1))
    gv = orc.grid_update(gm, gq, np.zeros((G, 2)))
    shape = orc.node_shape
    for idx in range(G):
        jx, jy = idx % shape[0], idx // shape[0]
        x, y = (jx - 1) * dx, (jy - 1) * dx
        out = v.copy()
        if x >= 1.0:                                    # right wall: moving outward
            out[0] = 0.0
        if y <= 0.0:                                    # floor, last
            seg = min(max(int(np.floor((jx - 1) * 4 / N)) if jx >= 1 else 0, 0), 3)
            m = mu[seg]
            vt = abs(out[0])
            vn = -out[1]
            out[1] = 0.0
            if m > 0:
                out[0] = 0.0 if vt <= m * vn else np.sign(out[0]) * (vt - m * vn)
        np.testing.assert_allclose(gv[idx], out, atol=1e-15, err_msg=f"node {jx},{jy}")


def test_floor_acts_last_at_a_3d_edge_node():
    """On the edge shared by the x- wall (slip) and the floor (friction mu) the
    walls act one after the other, the floor last.  For v = (-0.5, 0.8, -0.4)
    and mu = 0.3, by hand: the x- wall removes v_x, leaving (0, 0.8, -0.4); the
    floor then sees v_n = 0.4 and |v_t| = 0.8 > mu v_n = 0.12, so the node slides
    at 0.8 - 0.12 = 0.68.  (The floor first would leave 0.8 (1 - 0.12 / |(-0.5, 0.8)|)
    = 0.698...)."""
    N, dx = 4, 0.25
    orc = oracle.Oracle(3, (N, N, N), dx, 1e-3, (0.0, 0.0, 0.0), dict(inputs.FLUID_WATER), dx ** 3,
                        friction=[(4, (1, 1), [0.3])])
    G = orc.num_nodes
    nx, ny, _ = orc.node_shape
    gm, gq = np.zeros(G), np.zeros((G, 3))
    idx = 1 + nx * (2 + ny * 1)                         # node (x, y, z) = (0, dx, 0)
    gm[idx] = 1.0
    gq[idx] = [-0.5, 0.8, -0.4]
    # and on the edge of the x+ wall and the floor, by symmetry: (0, 0.68, 0) again
    idx2 = (N + 1) + nx * (2 + ny * 1)                  # node (x, y, z) = (L, dx, 0)
    gm[idx2] = 1.0
    gq[idx2] = [0.5, 0.8, -0.4]
    gv = orc.grid_update(gm, gq, np.zeros((G, 3)))
    np.testing.assert_allclose(gv[idx], [0.0, 0.68, 0.0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(gv[idx2], [0.0, 0.68, 0.0], rtol=0, atol=1e-15)


def test_last_segment_covers_the_floor_beyond_the_far_wall():
    """Floor nodes at and beyond x = L belong to the last segment: moving away from
    the x+ wall and into the floor with |v_t| = 0.3 <= mu_3 v_n = 1.0 x 0.4 they stick,
    while the first segment (mu 0) lets the same velocity slip."""
    N = 8
    dx = 1.0 / N
    mu = np.array([0.0, 0.2, 0.5, 1.0])
    orc = oracle.Oracle(2, (N, N), dx, 1e-3, (0.0, 0.0), dict(inputs.FLUID_WATER), dx * dx,
                        friction=[(2, (4, 1), mu)])
    G = orc.num_nodes
    nx = orc.node_shape[0]
    gv = orc.grid_update(np.ones(G), np.tile([-0.3, -0.4], (G, 1)), np.zeros((G, 2)))
    for jx in (N + 1, N + 2):                           # x = L and the ghost node beyond
        np.testing.assert_allclose(gv[jx + nx * 1], [0.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(gv[2 + nx * 1], [-0.3, 0.0], atol=1e-15)


def test_positions_are_clamped_to_the_domain():
    """Particles driven through the floor and the ceiling within one step end on
    them (x_p is clamped to [0, L] after the advection of Sec. 2.2)."""
    N = 16
    dx = 1.0 / N
    orc = oracle.Oracle(2, (N, N), dx, 2e-3, (0.0, 0.0), dict(inputs.FLUID_WATER), dx * dx / 4)
    x = np.array([[0.30, 1e-4], [0.33, 1e-4], [0.60, 1.0 - 1e-4], [0.63, 1.0 - 1e-4], [0.5, 0.5]])
    st = orc.initial_state(x, np.array([[0.2, -1.0], [0.1, -1.0], [0.0, 1.0], [0.1, 1.0], [0.0, 0.0]]))
    orc.step(st, 1)
    assert (st.x[:2, 1] == 0.0).all() and (st.x[2:4, 1] == 1.0).all()
    assert st.x[4, 1] == 0.5 and (st.x[:4, 0] > 0.25).all() and (st.x[:4, 0] < 0.75).all()


def test_mass_threshold_and_acceleration():
    N = 4
    orc = oracle.Oracle(2, (N, N), 0.25, 0.01, (0.0, -10.0), dict(inputs.FLUID_WATER), 0.01)
    G = orc.num_nodes
    gm = np.full(G, 2.0); gm[7] = 0.0
    gq = np.tile([1.0, 0.5], (G, 1))
    gf = np.tile([4.0, 2.0], (G, 1))
    gv = orc.grid_update(gm, gq, gf)
    interior = (1 + 2 * (N + 3)) + 1                    # node (2, 2)
    np.testing.assert_allclose(gv[interior], [0.5 + 0.01 * 2.0, 0.25 + 0.01 * 1.0], atol=1e-15)
    np.testing.assert_allclose(gv[7], 0.0)
    # the threshold is m_eps = 1e-10 rho0 dx^d: below it a node has no velocity, above it the update applies
    m_eps = 1e-10 * 1000.0 * 0.25 ** 2
    gm2 = np.full(G, 2.0); gm2[interior] = 0.5 * m_eps; gm2[interior + 1] = 2.0 * m_eps
    gv2 = orc.grid_update(gm2, gq, gf)
    np.testing.assert_allclose(gv2[interior], 0.0)
    np.testing.assert_allclose(gv2[interior + 1], [1.0 / (2.0 * m_eps) * (1.0 + 0.01 * 4.0),
                                                   1.0 / (2.0 * m_eps) * (0.5 + 0.01 * 2.0)], rtol=1e-12)


@pytest.mark.slow
def test_sliding_block_decelerates_at_mu_g():
    """An elastic block sliding on a floor of friction mu decelerates at mu g."""
    dx = 1.0 / 64
    mat = dict(kind=1, rho0=2000.0, E=2e6, nu=0.3, phi_deg=30.0, psi_deg=0.0, cohesion=1e6, sigma_t=1e6)
    mu = 0.3
    w = inputs.dam_break_2d(64, 0.125, 0.0625, ppc_axis=2)
    x0 = w.x + np.array([0.2, 0.0])
    dt = 2e-5
    orc = oracle.Oracle(2, (64, 64), dx, dt, (0.0, -9.81), mat, dx * dx / 4, friction=[(2, (1, 1), [mu])])
    st = orc.initial_state(x0, np.tile([1.0, 0.0], (len(x0), 1)))
    orc.step(st, 500)                                   # settle on the floor
    v1 = st.v[:, 0].mean()
    orc.step(st, 1500)
    v2 = st.v[:, 0].mean()
    decel = (v1 - v2) / (1500 * dt)
    assert decel == pytest.approx(mu * 9.81, rel=0.08)
