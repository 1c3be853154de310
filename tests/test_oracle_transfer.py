"""Pins of the oracle's G2P transfer variants (Sec. 2.2 G2P transfer, Appendix B):
APIC keeps the affine matrix, TPIC the particle velocity gradient, PIC nothing.

- an affine velocity field v(x) = v0 + A x (no gravity, away from walls) is
  carried exactly through a full step by APIC and TPIC (P2G of an affine field
  with its gradient as the particle matrix reproduces it on the grid, and G2P
  returns it), while PIC loses the A x part on the grid;
- the TPIC particle matrix after a step equals the velocity gradient L_p;
- in the same affine field L_p = A at every particle, so one step gives
  F <- (I + dt A) F, rho <- rho / (1 + dt tr A) and, for a viscous fluid, the
  stress of Sec. 2.3 with the rate of deformation D = sym(A):
  -p(rho) I - (2/3) mu tr(D) I + 2 mu D;
- PIC conserves linear momentum but not angular momentum of a spinning disc,
  which APIC and TPIC conserve (linear grid interpolation of a rigid rotation).
"""
import numpy as np
import pytest

import oracle
from paper_2507_04192_gb300 import inputs


def block(transfer, N=16, seed=0):
    dx = 1.0 / N
    x = inputs.lattice_particles((N, N), dx, 2, lambda p: (np.abs(p[:, 0] - 0.5) < 0.2) & (np.abs(p[:, 1] - 0.5) < 0.2),
                                 (0.3, 0.3), (0.7, 0.7), seed)
    orc = oracle.Oracle(2, (N, N), dx, 1e-4, (0.0, 0.0), dict(inputs.FLUID_WATER, bulk_K=0.0), dx * dx / 4,
                        transfer=transfer)
    return orc, x


@pytest.mark.parametrize("transfer", [0, 1])
def test_affine_field_carried_exactly(transfer):
    orc, x = block(transfer)
    A = np.array([[0.3, -0.8], [0.5, -0.3]])
    v0 = np.array([0.2, -0.1])
    st = orc.initial_state(x, v0 + (x - 0.5) @ A.T)
    if transfer == 0:
        st.B[:] = A * orc.P.dx ** 2 / 4.0            # B = C D with D = dx^2/4 I
    else:
        st.B[:] = A
    x0 = st.x.copy()
    orc.step(st, 1)
    np.testing.assert_allclose(st.v, v0 + (x0 - 0.5) @ A.T, rtol=0, atol=1e-12)
    np.testing.assert_allclose(orc.affine_C(st), np.broadcast_to(A, st.B.shape), rtol=0, atol=1e-10)


def test_affine_field_gives_F_rho_and_the_viscous_stress():
    N = 16
    dx = 1.0 / N
    x = inputs.lattice_particles((N, N), dx, 2, lambda p: (np.abs(p[:, 0] - 0.5) < 0.2) & (np.abs(p[:, 1] - 0.5) < 0.2),
                                 (0.3, 0.3), (0.7, 0.7), 0)
    mu = 0.7
    dt = 1e-3
    orc = oracle.Oracle(2, (N, N), dx, dt, (0.0, 0.0), dict(inputs.FLUID_WATER, viscosity=mu), dx * dx / 4)
    A = np.array([[0.3, -0.8], [0.5, 0.4]])
    st = orc.initial_state(x, np.array([0.2, -0.1]) + (x - 0.5) @ A.T)
    st.B[:] = A * dx * dx / 4.0
    rng = np.random.default_rng(7)
    F0 = np.eye(2) + 0.3 * rng.normal(size=(st.n, 2, 2))
    st.F[:] = F0
    orc.step(st, 1)
    np.testing.assert_allclose(st.F, np.einsum("ab,pbc->pac", np.eye(2) + dt * A, F0), rtol=0, atol=1e-12)
    rho1 = 1000.0 / (1.0 + dt * np.trace(A))
    np.testing.assert_allclose(st.rho, rho1, rtol=1e-13)
    D = np.zeros((3, 3))
    D[:2, :2] = 0.5 * (A + A.T)
    sig = -orc.tait_pressure(rho1) * np.eye(3) - 2.0 / 3.0 * mu * np.trace(D) * np.eye(3) + 2.0 * mu * D
    np.testing.assert_allclose(st.sigma, np.broadcast_to(sig, st.sigma.shape), rtol=0, atol=1e-9 * np.abs(sig).max())


def test_pic_loses_the_affine_part():
    orc, x = block(2)
    A = np.array([[0.0, -0.8], [0.8, 0.0]])
    st = orc.initial_state(x, (x - 0.5) @ A.T)
    v_in = st.v.copy()
    orc.step(st, 1)
    assert np.abs(st.B).max() == 0.0
    assert np.abs(st.v - v_in).max() > 1e-3


def angular_momentum(x, v):
    r = x - 0.5
    return float((r[:, 0] * v[:, 1] - r[:, 1] * v[:, 0]).sum())


@pytest.mark.parametrize("transfer,conserved", [(0, True), (1, True), (2, False)])
def test_rigid_rotation_angular_momentum(transfer, conserved):
    orc, x = block(transfer)
    omega = 2.0
    A = np.array([[0.0, -omega], [omega, 0.0]])
    st = orc.initial_state(x, (x - 0.5) @ A.T)
    if transfer == 0:
        st.B[:] = A * orc.P.dx ** 2 / 4.0
    elif transfer == 1:
        st.B[:] = A
    L0 = angular_momentum(st.x, st.v)
    P0 = st.v.sum(axis=0)
    orc.step(st, 5)
    L1 = angular_momentum(st.x, st.v)
    np.testing.assert_allclose(st.v.sum(axis=0), P0, rtol=0, atol=1e-10 * len(x))
    if conserved:
        assert L1 == pytest.approx(L0, rel=1e-3)
    else:
        assert abs(L1 - L0) > 1e-2 * abs(L0)


def test_flip_adds_the_grid_velocity_increment():
    """FLIP (alpha = 1) with gravity only: the grid velocity changes by g dt
    everywhere, so every particle's velocity, however scattered, changes by
    exactly g dt (partition of unity); PIC would smooth the scatter away."""
    orc, x = block(3)
    orc.P.gravity[1] = -9.8
    rng = np.random.default_rng(3)
    v0 = rng.normal(size=x.shape) * 0.3
    st = orc.initial_state(x, v0)
    orc.step(st, 1)
    np.testing.assert_allclose(st.v, v0 + np.array([0.0, -9.8]) * orc.P.dt, rtol=0, atol=1e-12)
    assert np.abs(st.B).max() == 0.0


def test_flip_with_alpha_zero_is_pic():
    rng = np.random.default_rng(4)
    res = []
    for transfer, alpha in ((3, 0.0), (2, 1.0)):
        orc, x = block(transfer)
        orc.P.flip_alpha = alpha
        orc.P.gravity[1] = -9.8
        st = orc.initial_state(x, rng.normal(size=x.shape) * 0.0 + 0.1)
        orc.step(st, 3)
        res.append((st.x.copy(), st.v.copy()))
    np.testing.assert_allclose(res[0][0], res[1][0], rtol=0, atol=1e-14)
    np.testing.assert_allclose(res[0][1], res[1][1], rtol=0, atol=1e-14)
