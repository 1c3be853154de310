"""Pins of the oracle's hand-derived adjoint of one step (the reverse recursion
of Eq. dzda, Sec. 3.1) against central finite differences of the oracle's own
forward step, and of the chained adjoint of a short trajectory against
finite differences of the trajectory loss (Eq. inverse_loss, Sec. 3.2)."""
import numpy as np
import pytest

import oracle
from paper_2507_04192_gb300 import inputs


def setup(seed=0, dt=5e-4, n_seg=4):
    rng = np.random.default_rng(seed)
    N = 16
    dx = 1.0 / N
    x = inputs.lattice_particles((N, N), dx, 2, lambda p: (p[:, 0] < 0.5) & (p[:, 1] < 0.3), (0, 0), (0.5, 0.3), seed)
    n = len(x)
    mu = rng.uniform(0.1, 0.6, n_seg)
    orc = oracle.Oracle(2, (N, N), dx, dt, (0.0, -9.81), dict(inputs.FLUID_WATER), dx * dx / 4,
                        friction=[(2, (n_seg, 1), mu)])
    st = orc.initial_state(x)
    st.v[:] = rng.normal(size=(n, 2)) * 0.5 + np.array([0.8, -0.6])      # sliding into the floor
    st.B[:] = rng.normal(size=(n, 2, 2)) * dx * dx * 2.0
    st.rho[:] = 1000.0 * rng.uniform(0.995, 1.005, n)
    st.sigma[:] = 0.0
    for p in range(n):
        st.sigma[p] = -orc.tait_pressure(st.rho[p]) * np.eye(3)
    return orc, st, mu, rng


def forward(orc, st, steps=1):
    s = st.copy()
    orc.step(s, steps)
    return s


def pair(a, b):
    return sum(float((x * y).sum()) for x, y in zip(a, b))


def test_one_step_vjp_matches_central_differences_in_the_state():
    orc, st, mu, rng = setup(0)
    n = st.n
    lam = [rng.normal(size=(n, 2)), rng.normal(size=(n, 2)), rng.normal(size=(n, 2, 2)) / orc.P.dx ** 2,
           rng.normal(size=n) * 1e-3]
    (xb, vb, Bb, rb), _ = orc.step_vjp(st, *lam)
    dx = orc.P.dx
    dirs = [rng.normal(size=(n, 2)) * dx * 0.1, rng.normal(size=(n, 2)) * 0.1, rng.normal(size=(n, 2, 2)) * dx * dx,
            rng.normal(size=n) * 1.0]
    eps = 1e-5

    def J(scale):
        s = st.copy()
        s.x += scale * dirs[0]; s.v += scale * dirs[1]; s.B += scale * dirs[2]; s.rho += scale * dirs[3]
        for p in range(n):
            s.sigma[p] = -orc.tait_pressure(s.rho[p]) * np.eye(3)
        s2 = forward(orc, s)
        return pair(lam, [s2.x, s2.v, s2.B, s2.rho])

    fd = (J(eps) - J(-eps)) / (2 * eps)
    an = pair([xb, vb, Bb, rb], dirs)
    assert an == pytest.approx(fd, rel=1e-5)
    # each block on its own (a wrong sign in one block cannot cancel against another)
    for blk in range(4):
        sub = [d if k == blk else np.zeros_like(d) for k, d in enumerate(dirs)]

        def Jb(scale):
            s = st.copy()
            s.x += scale * sub[0]; s.v += scale * sub[1]; s.B += scale * sub[2]; s.rho += scale * sub[3]
            for p in range(n):
                s.sigma[p] = -orc.tait_pressure(s.rho[p]) * np.eye(3)
            s2 = forward(orc, s)
            return pair(lam, [s2.x, s2.v, s2.B, s2.rho])
        fdb = (Jb(eps) - Jb(-eps)) / (2 * eps)
        assert pair([xb, vb, Bb, rb], sub) == pytest.approx(fdb, rel=1e-5, abs=1e-9 * abs(fd)), f"block {blk}"


def test_one_step_vjp_through_the_position_clamp():
    """Particles driven through the floor and the ceiling within one step end on
    them: their new heights no longer depend on the state, and the adjoint must
    agree with central differences there as well as for the free particles."""
    N = 16
    dx = 1.0 / N
    orc = oracle.Oracle(2, (N, N), dx, 2e-3, (0.0, -9.81), dict(inputs.FLUID_WATER), dx * dx / 4)
    x = np.array([[0.30, 1e-4], [0.33, 1e-4], [0.50, 0.40], [0.52, 0.41], [0.49, 0.43],
                  [0.70, 1.0 - 1e-4], [0.73, 1.0 - 1e-4]])
    st = orc.initial_state(x, np.array([[0.2, -1.0], [0.1, -1.0], [0.3, 0.1], [-0.2, 0.0], [0.1, -0.1],
                                        [0.1, 1.0], [-0.1, 1.0]]))
    s1 = forward(orc, st)
    assert (s1.x[:2, 1] == 0.0).all() and (s1.x[5:, 1] == 1.0).all()
    rng = np.random.default_rng(9)
    n = st.n
    lam = [rng.normal(size=(n, 2)), rng.normal(size=(n, 2)), rng.normal(size=(n, 2, 2)) / dx ** 2,
           rng.normal(size=n) * 1e-3]
    (xb, vb, Bb, rb), _ = orc.step_vjp(st, *lam)
    dirs = [rng.normal(size=(n, 2)) * dx * 0.01, rng.normal(size=(n, 2)) * 0.01, rng.normal(size=(n, 2, 2)) * dx * dx,
            rng.normal(size=n) * 0.1]
    eps = 1e-5
    for blk in range(4):
        sub = [d if k == blk else np.zeros_like(d) for k, d in enumerate(dirs)]

        def J(scale):
            s = st.copy()
            s.x += scale * sub[0]; s.v += scale * sub[1]; s.B += scale * sub[2]; s.rho += scale * sub[3]
            for p in range(n):
                s.sigma[p] = -orc.tait_pressure(s.rho[p]) * np.eye(3)
            s2 = forward(orc, s)
            return pair(lam, [s2.x, s2.v, s2.B, s2.rho])
        fd = (J(eps) - J(-eps)) / (2 * eps)
        assert pair([xb, vb, Bb, rb], sub) == pytest.approx(fd, rel=1e-5, abs=1e-12), f"block {blk}"


def test_one_step_vjp_at_a_3d_edge_with_two_friction_walls():
    """Fluid driven into the edges of the floor (mu 0.4) with the x- wall (mu 0.2)
    and with the x+ wall (slip): edge nodes go through two walls in turn, so the
    adjoint must take the walls in the reverse order, each linearised about its
    own input; every state block and both friction fields against central
    differences."""
    N = 8
    dx = 1.0 / N
    rng = np.random.default_rng(11)
    x = inputs.lattice_particles((N, N, N), dx, 2, lambda p: (p[:, 0] < 2 * dx) & (p[:, 2] < 2 * dx),
                                 (0.0, 2 * dx, 0.0), (2 * dx, 5 * dx, 2 * dx), 0)
    m = len(x)
    x = np.concatenate([x, x * np.array([-1.0, 1.0, 1.0]) + np.array([1.0, 0.0, 0.0])])   # and at the x+ edge
    n = len(x)
    water = dict(inputs.FLUID_WATER)

    def make(mx, mf):
        return oracle.Oracle(3, (N, N, N), dx, 5e-4, (0.0, 0.0, -9.81), water, dx ** 3 / 8,
                             friction=[(0, (1, 1), [mx]), (4, (1, 1), [mf])])
    orc = make(0.2, 0.4)
    v0 = np.array([-0.6, 0.3, -0.5]) + 0.1 * rng.normal(size=(n, 3))
    v0[m:, 0] *= -1.0
    st = orc.initial_state(x, v0)
    st.B[:] = rng.normal(size=(n, 3, 3)) * dx * dx
    st.rho[:] = 1000.0 * rng.uniform(0.995, 1.005, n)
    for p in range(n):
        st.sigma[p] = -orc.tait_pressure(st.rho[p]) * np.eye(3)
    lam = [rng.normal(size=(n, 3)), rng.normal(size=(n, 3)), rng.normal(size=(n, 3, 3)) / dx ** 2,
           rng.normal(size=n) * 1e-3]
    (xb, vb, Bb, rb), mub = orc.step_vjp(st, *lam)
    dirs = [rng.normal(size=(n, 3)) * dx * 0.01, rng.normal(size=(n, 3)) * 0.01, rng.normal(size=(n, 3, 3)) * dx * dx,
            rng.normal(size=n) * 0.1]
    eps = 1e-5
    for blk in range(4):
        sub = [d if k == blk else np.zeros_like(d) for k, d in enumerate(dirs)]

        def J(scale):
            s = st.copy()
            s.x += scale * sub[0]; s.v += scale * sub[1]; s.B += scale * sub[2]; s.rho += scale * sub[3]
            for p in range(n):
                s.sigma[p] = -orc.tait_pressure(s.rho[p]) * np.eye(3)
            s2 = forward(orc, s)
            return pair(lam, [s2.x, s2.v, s2.B, s2.rho])
        fd = (J(eps) - J(-eps)) / (2 * eps)
        assert pair([xb, vb, Bb, rb], sub) == pytest.approx(fd, rel=1e-5, abs=1e-12), f"block {blk}"
    for w, k in ((0, 0), (4, 1)):
        h = 1e-6
        up, dn = [0.2, 0.4], [0.2, 0.4]
        up[k] += h
        dn[k] -= h
        def Jm(m):
            s2 = forward(make(*m), st)
            return pair(lam, [s2.x, s2.v, s2.B, s2.rho])
        fd = (Jm(up) - Jm(dn)) / (2 * h)
        assert abs(fd) > 0
        assert mub[w][0] == pytest.approx(fd, rel=1e-5), f"wall {w}"


def test_nodes_below_the_mass_threshold_stay_out_of_the_adjoint():
    """A particle whose stencil's outer nodes carry about 4e-13 of mass, below the
    threshold 1e-10 rho0 dx^d = 3.9e-10, so the forward gives them no velocity:
    the adjoint still agrees with central differences (such nodes weigh about
    1e-13 in the result either way)."""
    N = 16
    dx = 1.0 / N
    orc = oracle.Oracle(2, (N, N), dx, 5e-4, (0.0, -9.81), dict(inputs.FLUID_WATER), dx * dx / 4)
    base = 7
    fx = 1.5 - 1e-6                                     # w_0 = (1.5 - fx)^2 / 2 = 5e-13
    x = np.array([[(base + fx) * dx, 0.5], [0.3, 0.3], [0.32, 0.31]])
    rng = np.random.default_rng(13)
    st = orc.initial_state(x, rng.normal(size=(3, 2)) * 0.3)
    n = st.n
    lam = [rng.normal(size=(n, 2)), rng.normal(size=(n, 2)), rng.normal(size=(n, 2, 2)) / dx ** 2,
           rng.normal(size=n) * 1e-3]
    (xb, vb, Bb, rb), _ = orc.step_vjp(st, *lam)
    dirs = [rng.normal(size=(n, 2)) * dx * 0.01, rng.normal(size=(n, 2)) * 0.01, rng.normal(size=(n, 2, 2)) * dx * dx,
            rng.normal(size=n) * 0.1]
    eps = 1e-5

    def J(scale):
        s = st.copy()
        s.x += scale * dirs[0]; s.v += scale * dirs[1]; s.B += scale * dirs[2]; s.rho += scale * dirs[3]
        for p in range(n):
            s.sigma[p] = -orc.tait_pressure(s.rho[p]) * np.eye(3)
        s2 = forward(orc, s)
        return pair(lam, [s2.x, s2.v, s2.B, s2.rho])
    fd = (J(eps) - J(-eps)) / (2 * eps)
    assert pair([xb, vb, Bb, rb], dirs) == pytest.approx(fd, rel=1e-5)


def test_mu_gradient_reaches_the_last_segment_beyond_the_far_wall():
    """Fluid sliding back from the x+ wall along the floor: floor nodes at and
    beyond x = L use the last segment, whose dL/dmu must match central
    differences like the others."""
    N = 16
    dx = 1.0 / N
    rng = np.random.default_rng(12)
    x = inputs.lattice_particles((N, N), dx, 2, lambda p: (p[:, 0] > 1.0 - 3 * dx) & (p[:, 1] < 2 * dx),
                                 (1.0 - 3 * dx, 0.0), (1.0, 2 * dx), 1)
    n = len(x)
    mu = np.array([0.1, 0.2, 0.3, 0.25])

    def make(m):
        return oracle.Oracle(2, (N, N), dx, 5e-4, (0.0, -9.81), dict(inputs.FLUID_WATER), dx * dx / 4,
                             friction=[(2, (4, 1), m)])
    st = make(mu).initial_state(x, np.array([-0.8, -0.6]) + 0.1 * rng.normal(size=(n, 2)))
    lam = [rng.normal(size=(n, 2)), rng.normal(size=(n, 2)), np.zeros((n, 2, 2)), np.zeros(n)]
    _, mub = make(mu).step_vjp(st, *lam)
    assert abs(mub[2][3]) > 0
    h = 1e-6
    for k in range(4):
        up, dn = mu.copy(), mu.copy()
        up[k] += h
        dn[k] -= h
        fd = (pair(lam, [forward(make(up), st).x, forward(make(up), st).v]) -
              pair(lam, [forward(make(dn), st).x, forward(make(dn), st).v])) / (2 * h)
        assert mub[2][k] == pytest.approx(fd, rel=1e-5, abs=1e-12), f"segment {k}"


def test_one_step_vjp_matches_central_differences_in_mu():
    orc, st, mu, rng = setup(1)
    n = st.n
    lam = [rng.normal(size=(n, 2)), rng.normal(size=(n, 2)), np.zeros((n, 2, 2)), np.zeros(n)]
    _, mub = orc.step_vjp(st, *lam)
    assert np.abs(mub[2]).max() > 0
    eps = 1e-6
    for s_idx in range(len(mu)):
        def J(m):
            o2 = oracle.Oracle(2, orc.node_shape and (16, 16), orc.P.dx, orc.P.dt, (0.0, -9.81),
                               dict(inputs.FLUID_WATER), orc.P.particle_volume, friction=[(2, (len(mu), 1), m)])
            s2 = forward(o2, st)
            return pair(lam, [s2.x, s2.v])
        mp_, mm_ = mu.copy(), mu.copy()
        mp_[s_idx] += eps
        mm_[s_idx] -= eps
        fd = (J(mp_) - J(mm_)) / (2 * eps)
        assert mub[2][s_idx] == pytest.approx(fd, rel=1e-5, abs=1e-10)


def test_trajectory_loss_gradient_matches_finite_differences():
    """L = sum_t sum_l |x_l^t - z_l^t|^2 over tracked particles: chained VJPs vs FD in mu."""
    orc0, st0, mu, rng = setup(2, dt=2e-4)
    n = st0.n
    steps, obs = 6, (3, 6)
    track = rng.choice(n, 10, replace=False)
    z = {t: rng.normal(size=(10, 2)) * 0.01 + st0.x[track] for t in obs}

    def make(m):
        return oracle.Oracle(2, (16, 16), orc0.P.dx, orc0.P.dt, (0.0, -9.81), dict(inputs.FLUID_WATER),
                             orc0.P.particle_volume, friction=[(2, (len(m), 1), m)])

    def loss(m):
        o = make(m)
        s = st0.copy()
        L = 0.0
        for t in range(1, steps + 1):
            o.step(s, 1)
            if t in obs:
                L += float(((s.x[track] - z[t]) ** 2).sum())
        return L

    o = make(mu)
    states = [st0.copy()]
    for t in range(1, steps + 1):
        s = states[-1].copy()
        o.step(s, 1)
        states.append(s)
    lam = [np.zeros((n, 2)), np.zeros((n, 2)), np.zeros((n, 2, 2)), np.zeros(n)]
    grad = np.zeros(len(mu))
    for t in range(steps, 0, -1):
        if t in obs:
            lam[0][track] += 2.0 * (states[t].x[track] - z[t])
        lam, mub = o.step_vjp(states[t - 1], *lam)
        grad += mub[2]
    eps = 1e-6
    for s_idx in range(len(mu)):
        mp_, mm_ = mu.copy(), mu.copy()
        mp_[s_idx] += eps
        mm_[s_idx] -= eps
        fd = (loss(mp_) - loss(mm_)) / (2 * eps)
        assert grad[s_idx] == pytest.approx(fd, rel=1e-4, abs=1e-12)
