"""Pins of the oracle's adjoint of the Drucker-Prager update (Appendix A) and of
one granular step (state x, v, B, rho, sigma) against central finite
differences of the oracle's own forward step."""
import numpy as np
import pytest

import oracle
from paper_2507_04192_gb300 import inputs

COHESIVE = dict(inputs.SAND_DP, cohesion=2.0e3, sigma_t=500.0)
DILATANT = dict(COHESIVE, psi_deg=10.0)           # q_psi > 0: the return also moves the mean stress


def make(material, dim=2, N=16, dt=2e-4, mu=None, n_seg=4):
    dx = 1.0 / N
    cells = (N,) * dim
    g = (0.0, -9.81) if dim == 2 else (0.0, 0.0, -9.81)
    fr = [(2 * (dim - 1), (n_seg, 1) if dim == 2 else (2, 2), mu)] if mu is not None else []
    return oracle.Oracle(dim, cells, dx, dt, g, dict(material), dx ** dim / 2 ** dim, friction=fr)


def sym(a):
    return 0.5 * (a + a.T)


def dp_case(orc, zone, rng):
    """(dd, dw, sigma) well inside the given zone of the update."""
    c = orc.dp_constants()
    dd = sym(rng.normal(size=(3, 3))) * 1e-5
    dw = rng.normal(size=(3, 3)) * 1e-5
    dw = 0.5 * (dw - dw.T)
    dev = sym(rng.normal(size=(3, 3)))
    dev -= np.trace(dev) / 3 * np.eye(3)
    dev /= np.sqrt(0.5 * (dev * dev).sum())                      # tau(dev) = 1
    if zone == 1:
        sm = -2.0e4
        tau = 0.4 * (c["k_phi"] - c["q_phi"] * sm)
    elif zone == 2:
        sm = -2.0e4
        tau = 2.0 * (c["k_phi"] - c["q_phi"] * sm)
    elif zone == 3:                                             # past the tension cutoff, inside the apex cone
        sm = c["sigma_t"] + 300.0
        tau = 0.3 * c["tau_P"]
    elif zone == 4:                                             # past the cutoff and outside: the corner
        sm = c["sigma_t"] + 300.0
        tau = 3.0 * max(c["tau_P"], 100.0)
    elif zone == 5:                                             # past the cutoff, just above tau_P but under
        sm = c["sigma_t"] + 300.0                               # the zone II/III line h = 0: Zone III corner
        tau = c["tau_P"] + 0.5 * c["alpha_P"] * 300.0
    else:                                                       # 0.1 Pa past the cutoff, 1 Pa above the line
        sm = c["sigma_t"] + 0.1                                 # h = 0: Zone II, and with dilatancy the return
        tau = c["tau_P"] + 1.0                                  # lands on the cone below the cutoff
        dd, dw = dd * 1e-4, dw * 1e-4                           # increments well inside those margins
    return dd, dw, sm * np.eye(3) + tau * dev


@pytest.mark.parametrize("material,zone", [(inputs.SAND_DP, 1), (inputs.SAND_DP, 2), (inputs.SAND_DP, 4),
                                           (COHESIVE, 1), (COHESIVE, 2), (COHESIVE, 3), (COHESIVE, 4),
                                           (DILATANT, 2), (DILATANT, 4), (COHESIVE, 5), (DILATANT, 5),
                                           (DILATANT, 6)])
def test_dp_vjp_matches_central_differences(material, zone):
    rng = np.random.default_rng(zone)
    orc = make(material)
    dd, dw, s = dp_case(orc, zone, rng)
    z, _, _ = orc.dp_update(dd, dw, s)
    assert z == {1: 1, 2: 2, 3: 3, 5: 3, 6: 2}.get(zone) or (zone == 4 and z in (2, 3))
    sb1 = rng.normal(size=(3, 3))
    sb0, ddb, dwb = orc.dp_vjp(dd, dw, s, sb1)
    dirs = [rng.normal(size=(3, 3)) * 1e-6, rng.normal(size=(3, 3)) * 1e-6, rng.normal(size=(3, 3)) * 10.0]
    for blk, an in enumerate((ddb, dwb, sb0)):
        def J(h):
            a = [dd.copy(), dw.copy(), s.copy()]
            a[blk] = a[blk] + h * dirs[blk]
            return float((orc.dp_update(*a)[1] * sb1).sum())
        eps = 1e-3
        fd = (J(eps) - J(-eps)) / (2 * eps)
        assert float((an * dirs[blk]).sum()) == pytest.approx(fd, rel=1e-6, abs=1e-9), f"block {blk}"


def sand_state(orc, dim, rng, n_cells=16):
    dx = orc.P.dx
    lo, hi = (0.0,) * dim, (0.5, 0.3) if dim == 2 else (0.4, 0.4, 0.25)
    x = inputs.lattice_particles((n_cells,) * dim, dx, 2, lambda p: np.all(p < np.array(hi), axis=1), lo, hi, 0)
    st = orc.initial_state(x)
    n = st.n
    st.v[:] = rng.normal(size=(n, dim)) * 0.3
    st.v[:, 0] += 0.8
    st.v[:, -1] -= 0.4                                           # sliding into the floor
    st.B[:] = rng.normal(size=(n, dim, dim)) * dx * dx * 2.0
    st.rho[:] = 2000.0 * rng.uniform(0.99, 1.01, n)
    depth = hi[-1] - x[:, -1]
    for p in range(n):
        szz = -2000.0 * 9.81 * depth[p]
        s = np.diag([0.5 * szz, 0.5 * szz, 0.5 * szz])
        s[dim - 1, dim - 1] = szz
        d = sym(rng.normal(size=(3, 3))) * 2500.0
        st.sigma[p] = s + d
    return st


def pair(a, b):
    return sum(float((x * y).sum()) for x, y in zip(a, b))


@pytest.mark.parametrize("dim", [2, 3])
def test_sand_step_vjp_matches_central_differences(dim):
    rng = np.random.default_rng(10 + dim)
    mu = rng.uniform(0.1, 0.6, 4)
    orc = make(COHESIVE, dim, N=16 if dim == 2 else 8, mu=mu)
    st = sand_state(orc, dim, rng, 16 if dim == 2 else 8)
    n, d, dx = st.n, dim, orc.P.dx
    lam = [rng.normal(size=(n, d)), rng.normal(size=(n, d)), rng.normal(size=(n, d, d)) / dx ** 2,
           rng.normal(size=n) * 1e-3, rng.normal(size=(n, 3, 3)) * 1e-4]
    (xb, vb, Bb, rb, sb), mub = orc.step_vjp(st, *lam)
    zones = []
    dirs = [rng.normal(size=(n, d)) * dx * 0.1, rng.normal(size=(n, d)) * 0.1, rng.normal(size=(n, d, d)) * dx * dx,
            rng.normal(size=n), np.stack([sym(a) for a in rng.normal(size=(n, 3, 3))]) * 100.0]

    def run(sub, h):
        s = st.copy()
        s.x += h * sub[0]; s.v += h * sub[1]; s.B += h * sub[2]; s.rho += h * sub[3]; s.sigma += h * sub[4]
        orc.step(s, 1)
        return pair(lam, [s.x, s.v, s.B, s.rho, s.sigma])

    eps = 1e-5
    for blk in range(5):
        sub = [dd if k == blk else np.zeros_like(dd) for k, dd in enumerate(dirs)]
        fd = (run(sub, eps) - run(sub, -eps)) / (2 * eps)
        an = pair([xb, vb, Bb, rb, sb], sub)
        assert an == pytest.approx(fd, rel=1e-5, abs=1e-9 * max(1.0, abs(fd))), f"block {blk}"
    # friction
    w = 2 * (dim - 1)
    assert np.abs(mub[w]).max() > 0
    for k in range(len(mu)):
        def J(m):
            o2 = make(COHESIVE, dim, N=16 if dim == 2 else 8, mu=m)
            s = st.copy()
            o2.step(s, 1)
            return pair(lam, [s.x, s.v, s.B, s.rho, s.sigma])
        mp_, mm_ = mu.copy(), mu.copy()
        mp_[k] += 1e-6
        mm_[k] -= 1e-6
        fd = (J(mp_) - J(mm_)) / 2e-6
        assert mub[w][k] == pytest.approx(fd, rel=1e-5, abs=1e-10)


def test_sand_state_exercises_every_zone():
    """The step pins above see elastic particles, cone returns and tension cutoffs."""
    rng = np.random.default_rng(12)
    orc = make(COHESIVE, 2)
    st = sand_state(orc, 2, rng)
    s = st.copy()
    orc.step(s, 1)
    c = orc.dp_constants()
    sm = np.trace(s.sigma, axis1=1, axis2=2) / 3
    dev = s.sigma - sm[:, None, None] * np.eye(3)
    tau = np.sqrt(0.5 * (dev ** 2).sum(axis=(1, 2)))
    on_cone = np.abs(tau - (c["k_phi"] - c["q_phi"] * sm)) < 1e-9 * 1e4
    at_cutoff = np.abs(sm - c["sigma_t"]) < 1e-9 * 1e4
    inside = ~on_cone & ~at_cutoff
    assert on_cone.sum() > 0 and at_cutoff.sum() > 0 and inside.sum() > 0, (on_cone.sum(), at_cutoff.sum())
