"""Pins of the oracle's transfers (Sec. 2.2, Appendix B) against brute force,
conservation laws and exact solutions."""
import numpy as np
import pytest

import oracle
from paper_2507_04192_gb300 import inputs

from test_oracle_bspline import cardinal_bspline, cardinal_bspline_deriv

FLUID = dict(inputs.FLUID_WATER)


def make(dim, n_cells, dx, dt=1e-4, gravity=None, material=None, vol=None, friction=()):
    g = gravity if gravity is not None else (0.0,) * dim
    mat = material if material is not None else FLUID
    return oracle.Oracle(dim, n_cells, dx, dt, g, mat, vol if vol else dx ** dim / 4 ** dim, friction)


def brute_nodes(orc):
    """All node coordinates (j - 1) dx in oracle order (first axis fastest)."""
    shape = orc.node_shape
    grids = np.meshgrid(*[np.arange(s) for s in shape[::-1]], indexing="ij")
    j = np.stack([g.reshape(-1) for g in grids[::-1]], axis=1)
    return (j - 1) * orc.P.dx


def brute_weights(orc, xp, nodes):
    dx = orc.P.dx
    d = orc.dim
    phi = np.ones(len(nodes))
    f = np.zeros((len(nodes), d))
    df = np.zeros((len(nodes), d))
    for i, xi in enumerate(nodes):
        for a in range(d):
            t = (xp[a] - xi[a]) / dx + 1.5
            f[i, a] = cardinal_bspline(2, t)
            df[i, a] = cardinal_bspline_deriv(2, t) / dx
    phi = f.prod(axis=1)
    grad = np.zeros((len(nodes), d))
    for a in range(d):
        g = df[:, a].copy()
        for b in range(d):
            if b != a:
                g *= f[:, b]
        grad[:, a] = g
    return phi, grad


def random_state(orc, n, rng, lo, hi):
    d = orc.dim
    x = rng.uniform(lo, hi, (n, d))
    st = orc.initial_state(x, rng.normal(size=(n, d)))
    st.B[:] = rng.normal(size=(n, d, d)) * orc.P.dx ** 2
    st.rho[:] = orc.P.rho0 * rng.uniform(0.9, 1.1, n)
    s = rng.normal(size=(n, 3, 3)) * 100.0
    st.sigma[:] = s + s.transpose(0, 2, 1)
    return st


@pytest.mark.parametrize("dim", [2, 3])
def test_p2g_g2p_brute_force_small_grid(dim):
    """Every node's shape function evaluated directly (no stencil) on a 4^d grid."""
    rng = np.random.default_rng(10 + dim)
    dx = 0.25
    orc = make(dim, (4,) * dim, dx, dt=1e-3, gravity=(0.0,) * (dim - 1) + (-9.81,))
    st = random_state(orc, 7, rng, 0.0, 1.0)
    gm, gq, gf = orc.p2g(st)
    nodes = brute_nodes(orc)
    mp = orc.particle_mass
    bm = np.zeros(len(nodes)); bq = np.zeros((len(nodes), dim)); bf = np.zeros((len(nodes), dim))
    grav = np.array([orc.P.gravity[a] for a in range(dim)])
    for p in range(st.n):
        phi, grad = brute_weights(orc, st.x[p], nodes)
        r = nodes - st.x[p]
        D = np.einsum("i,ia,ib->ab", phi, r, r)
        M = st.B[p] @ np.linalg.inv(D)
        Vp = mp / st.rho[p]
        sig = st.sigma[p][:dim, :dim]
        bm += mp * phi
        bq += (phi * mp)[:, None] * (st.v[p] + r @ M.T)
        bf += -Vp * grad @ sig + (phi * mp)[:, None] * grav
    np.testing.assert_allclose(gm, bm, rtol=1e-13, atol=1e-13 * bm.max())
    np.testing.assert_allclose(gq, bq, rtol=1e-12, atol=1e-12 * np.abs(bq).max())
    np.testing.assert_allclose(gf, bf, rtol=1e-12, atol=1e-12 * np.abs(bf).max())

    # G2P against brute force with random nodal velocities (no walls: skip grid update)
    gv = rng.normal(size=(len(nodes), dim))
    x0 = st.x.copy()
    st2 = st.copy()
    orc.g2p(st2, gv)
    for p in range(st.n):
        phi, grad = brute_weights(orc, x0[p], nodes)
        r = nodes - x0[p]
        vp = phi @ gv
        Bp = np.einsum("i,ia,ib->ab", phi, gv, r)
        L = gv.T @ grad
        np.testing.assert_allclose(st2.v[p], vp, rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(st2.B[p], Bp, rtol=1e-12, atol=1e-13)
        xn = np.clip(x0[p] + orc.P.dt * vp, 0.0, 1.0)
        np.testing.assert_allclose(st2.x[p], xn, rtol=0, atol=1e-15)
        Fn = (np.eye(dim) + orc.P.dt * L) @ st.F[p]
        np.testing.assert_allclose(st2.F[p], Fn, rtol=1e-13, atol=1e-14)
        assert st2.rho[p] == pytest.approx(st.rho[p] / (1.0 + orc.P.dt * np.trace(L)), rel=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_p2g_conserves_mass_and_momentum(dim):
    rng = np.random.default_rng(20 + dim)
    n_cells = (16,) * dim
    dx = 1.0 / 16
    orc = make(dim, n_cells, dx)
    st = random_state(orc, 500, rng, 0.2, 0.8)
    gm, gq, gf = orc.p2g(st)
    mp = orc.particle_mass
    assert gm.sum() == pytest.approx(mp * st.n, rel=1e-13)
    np.testing.assert_allclose(gq.sum(axis=0), mp * st.v.sum(axis=0), rtol=1e-12, atol=1e-12 * mp * st.n)
    # internal forces sum to zero (sum_i grad phi_i = 0); no gravity here
    assert np.abs(gf.sum(axis=0)).max() < 1e-9 * np.abs(gf).max()


def test_free_fall_is_exact():
    """An unsupported block far from the walls: v^n = v0 + n g dt and
    x^n = x0 + n dt v0 + g dt^2 n (n + 1) / 2, to rounding."""
    w = inputs.dam_break_2d(32, 0.2, 0.2)
    x0 = w.x + 0.4                          # block [0.4, 0.6]^2
    v0 = np.array([0.3, 0.2])
    g = np.array([0.0, -9.81])
    dt = 1e-4
    orc = make(2, (32, 32), 1.0 / 32, dt, tuple(g), vol=w.particle_volume)
    st = orc.initial_state(x0, np.tile(v0, (len(x0), 1)))
    n = 60
    orc.step(st, n)
    np.testing.assert_allclose(st.v, np.tile(v0 + n * dt * g, (len(x0), 1)), rtol=0, atol=1e-12)
    xe = x0 + n * dt * v0 + g * dt * dt * n * (n + 1) / 2
    np.testing.assert_allclose(st.x, xe, rtol=0, atol=1e-13)
    np.testing.assert_allclose(st.rho, orc.P.rho0, rtol=1e-12)
    assert np.abs(st.B).max() < 1e-15


def test_free_fall_drucker_prager_3d():
    w = inputs.granular_cylinder_3d((32, 32, 32), 3, 4, seed=3)
    x0 = w.x + np.array([0.0, 0.0, 0.03])
    dt = 1e-5
    orc = make(3, (32, 32, 32), w.dx, dt, (0.0, 0.0, -9.81), dict(inputs.SAND_DP), w.particle_volume)
    # the cylinder sits at the centre of a 32^3 grid of dx = 1/256: lift it off the floor
    st = orc.initial_state(x0)
    n = 20
    orc.step(st, n)
    xe = x0.copy(); xe[:, 2] += -9.81 * dt * dt * n * (n + 1) / 2
    np.testing.assert_allclose(st.x, xe, rtol=0, atol=1e-14)
    assert np.abs(st.sigma).max() < 1e-6


def test_rigid_translation_and_affine_reproduction():
    rng = np.random.default_rng(5)
    dx = 1.0 / 32
    orc = make(2, (32, 32), dx, dt=1e-4)
    x0 = rng.uniform(0.3, 0.7, (300, 2))
    v0 = np.array([0.7, -0.4])
    st = orc.initial_state(x0, np.tile(v0, (300, 1)))
    orc.step(st, 25)
    np.testing.assert_allclose(st.x, x0 + 25 * 1e-4 * v0, rtol=0, atol=1e-14)

    # linear field v = a + B x survives P2G -> grid -> G2P: v_p exact, C_p = B, L_p = B
    a = np.array([0.2, -0.1])
    Bt = np.array([[0.3, -0.5], [0.8, -0.3]])
    st = orc.initial_state(x0, a + x0 @ Bt.T)
    st.B[:] = Bt * dx * dx / 4.0           # B_p = C_p D_p with D_p = dx^2/4 I (pinned above)
    gm, gq, gf = orc.p2g(st)
    gv = orc.grid_update(gm, gq, gf * 0.0)  # sigma = 0 at rho0 anyway; drop rounding
    xold = st.x.copy()
    orc.g2p(st, gv)
    np.testing.assert_allclose(st.v, a + xold @ Bt.T, rtol=0, atol=1e-13)
    np.testing.assert_allclose(orc.affine_C(st), np.broadcast_to(Bt, st.B.shape), rtol=0, atol=1e-11)
    L = (st.F - np.eye(2)) / orc.P.dt
    np.testing.assert_allclose(L, np.broadcast_to(Bt, L.shape), rtol=0, atol=1e-8)


def test_momentum_conserved_by_full_step_without_walls_or_gravity():
    rng = np.random.default_rng(6)
    dx = 1.0 / 32
    orc = make(2, (32, 32), dx, dt=1e-4)
    w = inputs.dam_break_2d(32, 0.25, 0.25)
    x0 = w.x + 0.35
    st = orc.initial_state(x0, rng.normal(size=x0.shape) * 0.1)
    st.rho[:] *= rng.uniform(0.99, 1.01, len(x0))     # pressure differences drive internal forces
    p0 = st.v.sum(axis=0)
    orc.step(st, 10)
    np.testing.assert_allclose(st.v.sum(axis=0), p0, rtol=0, atol=1e-9 * np.abs(st.v).sum())


def test_mirror_symmetry_of_dam_break():
    """A column centred in the box stays mirror symmetric (walls x- and x+ agree)."""
    half = inputs.dam_break_2d(32, 0.125, 0.25).x          # [0, 0.125] x [0, 0.25]
    left = half + np.array([0.375, 0.0])
    right = left.copy(); right[:, 0] = 1.0 - left[:, 0]
    x0 = np.concatenate([left, right])
    orc = make(2, (32, 32), 1.0 / 32, 1e-4, (0.0, -9.81), vol=(1 / 32) ** 2 / 16)
    st = orc.initial_state(x0)
    orc.step(st, 100)
    n = len(left)
    np.testing.assert_allclose(st.x[:n, 0], 1.0 - st.x[n:, 0], rtol=0, atol=1e-12)
    np.testing.assert_allclose(st.x[:n, 1], st.x[n:, 1], rtol=0, atol=1e-12)
    assert st.x[:, 1].min() >= 0.0
