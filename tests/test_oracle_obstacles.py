"""Pins of the oracle's rigid-obstacle contact (Sec. 4.1, 3D dam break: the
predicted grid velocity of a node at a stationary obstacle loses its normal
component, v_i = v~_i - (v~_i . n_i) n_i, for a node moving into the body).

- the contact normals of the nodes of a small box, worked out by hand;
- a box filling the domain beyond x = M dx acts exactly as a slip wall at
  M dx: a block thrown at it evolves bit for bit as in a domain that ends there;
- the same with the box on the low side (its high face is the contact face),
  compared with the mirror image of the first run;
- fluid thrown at a free-standing column does not enter it;
- the one-step adjoint with an obstacle in contact matches central differences.
"""
import numpy as np
import pytest

import oracle
from paper_2507_04192_gb300 import inputs

WATER = dict(inputs.FLUID_WATER)


def test_contact_normals_by_hand():
    # box [2 dx, 5 dx] x [3 dx, 6 dx] in a 10 x 10 domain; oracle node j sits at (j - 1) dx
    dx = 0.1
    orc = oracle.Oracle(2, (10, 10), dx, 1e-4, (0.0, 0.0), WATER, dx * dx / 4,
                        obstacles=[((0.2, 0.3), (0.5, 0.6))])

    def nrm(c0, c1):
        n = orc.obstacle_normal(0, (c0 + 1, c1 + 1))
        return None if n is None else tuple(int(round(v)) for v in n[:2])

    assert nrm(1, 4) is None and nrm(6, 4) is None and nrm(3, 2) is None and nrm(3, 7) is None
    assert nrm(2, 4) == (-1, 0)          # on the x- face
    assert nrm(5, 4) == (1, 0)           # on the x+ face
    assert nrm(3, 3) == (0, -1)          # on the y- face, one node in from x-
    assert nrm(4, 6) == (0, 1)           # on the y+ face, one node in from x+
    assert nrm(2, 3) == (-1, 0)          # corner: x- and y- at distance 0, x- first
    assert nrm(5, 6) == (1, 0)           # corner: x+ and y+ at distance 0, x+ first
    assert nrm(3, 5) == (-1, 0)          # x- 1, x+ 2, y- 2, y+ 1: x- first
    assert nrm(4, 4) == (1, 0)           # x- 2, x+ 1, y- 1, y+ 2: x+ first


def test_contact_normal_ties_follow_face_order():
    dx = 0.1
    orc = oracle.Oracle(2, (10, 10), dx, 1e-4, (0.0, 0.0), WATER, dx * dx / 4,
                        obstacles=[((0.2, 0.3), (0.6, 0.6))])          # nodes x 2..6, y 3..6
    n = orc.obstacle_normal(0, (4 + 1, 4 + 1))                         # x- 2, x+ 2, y- 1, y+ 2
    assert tuple(np.round(n[:2]).astype(int)) == (0, -1)
    n = orc.obstacle_normal(0, (4 + 1, 5 + 1))                         # x- 2, x+ 2, y- 2, y+ 1
    assert tuple(np.round(n[:2]).astype(int)) == (0, 1)
    n = orc.obstacle_normal(0, (5 + 1, 4 + 1))                         # x- 3, x+ 1, y- 1: x+ first
    assert tuple(np.round(n[:2]).astype(int)) == (1, 0)


def test_faces_outside_the_domain_are_not_contact_faces():
    dx = 0.1
    # a full-height column: its y faces lie on the domain walls, so only x faces count
    orc = oracle.Oracle(2, (10, 10), dx, 1e-4, (0.0, 0.0), WATER, dx * dx / 4,
                        obstacles=[((0.4, 0.0), (0.6, 1.0))])
    for c1 in range(0, 11):
        assert tuple(np.round(orc.obstacle_normal(0, (4 + 1, c1 + 1))[:2]).astype(int)) == (-1, 0)
        assert tuple(np.round(orc.obstacle_normal(0, (6 + 1, c1 + 1))[:2]).astype(int)) == (1, 0)
    # a box standing on the floor: its y- face lies on the domain wall, so a node on
    # the floor inside it takes the nearest of the other faces (x- 3, x+ 3, y+ 5: x- first)
    orc = oracle.Oracle(2, (10, 10), dx, 1e-4, (0.0, 0.0), WATER, dx * dx / 4,
                        obstacles=[((0.2, 0.0), (0.8, 0.5))])
    assert tuple(np.round(orc.obstacle_normal(0, (5 + 1, 0 + 1))[:2]).astype(int)) == (-1, 0)
    assert tuple(np.round(orc.obstacle_normal(0, (5 + 1, 4 + 1))[:2]).astype(int)) == (0, 1)
    # a box covering the whole domain has no contact face
    orc = oracle.Oracle(2, (10, 10), dx, 1e-4, (0.0, 0.0), WATER, dx * dx / 4,
                        obstacles=[((-1.0, -1.0), (2.0, 2.0))])
    assert orc.obstacle_normal(0, (5, 5)) is None


def block_positions(n_cells, x0, seed=0):
    dx = 1.0 / 32
    return inputs.lattice_particles(tuple(n_cells), dx, 2,
                                    lambda p: (np.abs(p[:, 0] - x0) < 4 * dx) & (p[:, 1] < 8 * dx),
                                    (x0 - 4 * dx, 0.0), (x0 + 4 * dx, 8 * dx), seed)


def thrown_block(n_cells, x0, v0, obstacles=(), steps=30, seed=0, x=None):
    dx = 1.0 / 32
    if x is None:
        x = block_positions(n_cells, x0, seed)
    orc = oracle.Oracle(2, tuple(n_cells), dx, 2e-4, (0.0, -9.81), WATER, dx * dx / 4, obstacles=list(obstacles))
    st = orc.initial_state(x, np.tile(v0, (len(x), 1)))
    orc.step(st, steps)
    return st, dx


def test_box_beyond_a_plane_is_a_slip_wall():
    M = 16
    # the block moves at 1 m/s into the plane x = M dx from 2 cells away
    a, dx = thrown_block((24, 16), 11.5 / 32, np.array([1.0, 0.0]),
                         obstacles=[((M / 32, -1.0), (3.0, 2.0))])
    b, _ = thrown_block((M, 16), 11.5 / 32, np.array([1.0, 0.0]))
    assert a.x[:, 0].max() < M * dx                      # nobody reached the plane: no clamp differs
    assert np.abs(b.v[:, 0]).max() > 0.0
    for f in ("x", "v", "B", "F", "rho"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f), err_msg=f)


def test_low_side_box_mirrors_the_high_side_one():
    M, N = 16, 24
    dx = 1.0 / 32
    xa = block_positions((N, 16), 11.5 / 32)
    a, _ = thrown_block((N, 16), None, np.array([1.0, 0.0]), obstacles=[((M / 32, -1.0), (3.0, 2.0))], x=xa)
    # mirror image about x = N dx / 2: box [0, (N - M) dx], block thrown towards -x
    L = N * dx
    xc = xa.copy()
    xc[:, 0] = L - xc[:, 0]
    c, _ = thrown_block((N, 16), None, np.array([-1.0, 0.0]), obstacles=[((-1.0, -1.0), ((N - M) / 32, 2.0))],
                        x=xc)
    assert np.abs(a.v[:, 0]).max() > 0.1
    np.testing.assert_allclose(L - c.x[:, 0], a.x[:, 0], rtol=0, atol=1e-12)
    np.testing.assert_allclose(c.x[:, 1], a.x[:, 1], rtol=0, atol=1e-12)
    np.testing.assert_allclose(-c.v[:, 0], a.v[:, 0], rtol=0, atol=1e-9)
    np.testing.assert_allclose(c.v[:, 1], a.v[:, 1], rtol=0, atol=1e-9)


def test_fluid_does_not_enter_a_free_standing_column():
    dx = 1.0 / 32
    col = ((18 * dx, 0.0), (22 * dx, 1.0))
    st, _ = thrown_block((32, 16), 11.5 / 32, np.array([1.5, 0.0]), obstacles=[col], steps=60)
    assert st.x[:, 0].max() > 15 * dx                   # the block reached the column
    inside = (st.x[:, 0] > col[0][0] + 0.5 * dx) & (st.x[:, 0] < col[1][0] - 0.5 * dx)
    assert not inside.any()


@pytest.mark.parametrize("face", ["side", "top"])
def test_one_step_vjp_with_obstacle_contact_matches_central_differences(face):
    # fluid thrown at the box's x- face, or falling onto its top face (normal +y)
    rng = np.random.default_rng(3)
    N = 16
    dx = 1.0 / N
    if face == "side":
        x = inputs.lattice_particles((N, N), dx, 2, lambda p: (np.abs(p[:, 0] - 0.4) < 0.1) & (p[:, 1] < 0.3),
                                     (0.3, 0), (0.5, 0.3), 3)
        v = np.array([1.2, 0.3])
    else:
        x = inputs.lattice_particles((N, N), dx, 2, lambda p: (p[:, 0] > 0.55) & (p[:, 0] < 0.7),
                                     (0.55, 0.24), (0.7, 0.36), 3)
        v = np.array([0.1, -1.2])
    n = len(x)
    orc = oracle.Oracle(2, (N, N), dx, 5e-4, (0.0, -9.81), WATER, dx * dx / 4,
                        obstacles=[((0.5 + 0.5 * dx, -1.0), (0.75, 0.2 + 0.5 * dx))])
    st = orc.initial_state(x)
    st.v[:] = rng.normal(size=(n, 2)) * 0.3 + v                       # moving into the box
    st.B[:] = rng.normal(size=(n, 2, 2)) * dx * dx
    st.rho[:] = 1000.0 * rng.uniform(0.995, 1.005, n)
    for p in range(n):
        st.sigma[p] = -orc.tait_pressure(st.rho[p]) * np.eye(3)
    # the contact is active at some nodes: the step with the box differs from the one without
    free = oracle.Oracle(2, (N, N), dx, 5e-4, (0.0, -9.81), WATER, dx * dx / 4)
    s1, s2 = st.copy(), st.copy()
    orc.step(s1, 1)
    free.step(s2, 1)
    assert np.abs(s1.v - s2.v).max() > 1e-3
    lam = [rng.normal(size=(n, 2)), rng.normal(size=(n, 2)), rng.normal(size=(n, 2, 2)) / dx ** 2,
           rng.normal(size=n) * 1e-3]
    (xb, vb, Bb, rb), _ = orc.step_vjp(st, *lam)
    dirs = [rng.normal(size=(n, 2)) * dx * 0.1, rng.normal(size=(n, 2)) * 0.1, rng.normal(size=(n, 2, 2)) * dx * dx,
            rng.normal(size=n)]
    eps = 1e-6

    def J(scale):
        s = st.copy()
        s.x += scale * dirs[0]; s.v += scale * dirs[1]; s.B += scale * dirs[2]; s.rho += scale * dirs[3]
        for p in range(n):
            s.sigma[p] = -orc.tait_pressure(s.rho[p]) * np.eye(3)
        orc.step(s, 1)
        return sum(float((a * b).sum()) for a, b in zip(lam, [s.x, s.v, s.B, s.rho]))

    fd = (J(eps) - J(-eps)) / (2 * eps)
    an = sum(float((a * b).sum()) for a, b in zip([xb, vb, Bb, rb], dirs))
    assert an == pytest.approx(fd, rel=1e-5)


def test_box_beyond_a_plane_is_a_slip_wall_3d():
    # the 3D form of the pin above, with the plane normal to y and a z-column box
    dx = 1.0 / 16
    def run(n_cells, obstacles):
        x = inputs.lattice_particles(n_cells, dx, 2, lambda p: (np.abs(p[:, 1] - 5.5 * dx) < 2 * dx)
                                     & (np.abs(p[:, 0] - 4 * dx) < 2 * dx) & (p[:, 2] < 4 * dx),
                                     (2 * dx, 3.5 * dx, 0.0), (6 * dx, 7.5 * dx, 4 * dx), 0)
        orc = oracle.Oracle(3, n_cells, dx, 2e-4, (0.0, 0.0, -9.81), WATER, dx ** 3 / 8, obstacles=obstacles)
        st = orc.initial_state(x, np.tile([0.0, 1.0, 0.0], (len(x), 1)))
        orc.step(st, 25)
        return st
    a = run((8, 12, 8), [((-1.0, 8 * dx, -1.0), (2.0, 2.0, 2.0))])
    b = run((8, 8, 8), [])
    assert a.x[:, 1].max() < 8 * dx and np.abs(b.v[:, 1]).max() > 0.0
    for f in ("x", "v", "B", "F", "rho"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f), err_msg=f)
