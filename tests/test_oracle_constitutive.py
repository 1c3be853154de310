"""Pins of the oracle's constitutive updates (Sec. 2.3, Appendix A) against
textbook elasticity, objectivity and the yield-surface geometry."""
import numpy as np
import pytest

import oracle
from paper_2507_04192_gb300 import inputs


def dp_oracle(**over):
    mat = dict(inputs.SAND_DP)
    mat.update(over)
    lit = mat.pop("dp_literal", False)
    return oracle.Oracle(3, (8, 8, 8), 0.1, 1e-4, (0, 0, 0), mat, 1e-3, dp_literal=lit)


def invariants(s):
    sm = np.trace(s) / 3.0
    dev = s - sm * np.eye(3)
    return sm, np.sqrt(0.5 * (dev * dev).sum()), dev


def test_tait_gamma_one_is_linear_eos():
    mat = dict(inputs.FLUID_WATER, gamma=1.0)
    orc = oracle.Oracle(2, (4, 4), 0.25, 1e-4, (0, 0), mat, 0.01)
    c2 = mat["bulk_K"] / mat["rho0"]
    for rho in (950.0, 1000.0, 1003.7, 1100.0):
        assert orc.tait_pressure(rho) == pytest.approx(c2 * (rho - mat["rho0"]), rel=1e-14, abs=1e-9)


def test_tait_gamma_seven():
    orc = oracle.Oracle(2, (4, 4), 0.25, 1e-4, (0, 0), dict(inputs.FLUID_WATER), 0.01)
    assert orc.tait_pressure(1010.0) == pytest.approx(2e5 / 7 * (1.01 ** 7 - 1), rel=1e-14)


def test_dp_constants_at_30_degrees():
    c = dp_oracle().dp_constants()
    assert c["K"] == pytest.approx(1e6 / 1.2)
    assert c["G"] == pytest.approx(1e6 / 2.6)
    assert c["q_phi"] == pytest.approx(3.0 / (np.sqrt(3.0) * 3.5), rel=1e-14)
    assert c["k_phi"] == 0.0 and c["sigma_t"] == 0.0 and c["tau_P"] == 0.0
    assert c["alpha_P"] == pytest.approx(np.sqrt(1 + c["q_phi"] ** 2) - c["q_phi"])


def test_dp_constants_with_cohesion_and_a_tension_cutoff():
    # phi = 30 deg: sin = 1/2 and cos = sqrt(3)/2, so q_phi = 2 sqrt(3)/7 and k_phi = 6 c / 7;
    # the cone's apex sits at the mean stress k_phi / q_phi = sqrt(3) c
    q = 2.0 * np.sqrt(3.0) / 7.0
    c = dp_oracle(cohesion=700.0, sigma_t=100.0).dp_constants()
    assert c["q_phi"] == pytest.approx(q, rel=1e-14)
    assert c["k_phi"] == pytest.approx(600.0, rel=1e-14)
    assert c["sigma_t"] == 100.0
    assert c["tau_P"] == pytest.approx(600.0 - 100.0 * q, rel=1e-14)
    assert c["alpha_P"] == pytest.approx(np.sqrt(1.0 + q * q) - q, rel=1e-14)
    # dilatancy: q_psi follows the same form in psi (psi = 90 deg: 6 / (4 sqrt(3)))
    assert dp_oracle(psi_deg=90.0).dp_constants()["q_psi"] == pytest.approx(1.5 / np.sqrt(3.0), rel=1e-14)
    # a tension cutoff beyond the apex is brought back to it, where tau_P vanishes
    c = dp_oracle(cohesion=700.0, sigma_t=5000.0).dp_constants()
    assert c["sigma_t"] == pytest.approx(np.sqrt(3.0) * 700.0, rel=1e-14)
    assert abs(c["tau_P"]) < 1e-10


def test_dp_elastic_oedometric_step():
    """Uniaxial strain increment under confinement: textbook oedometric response."""
    orc = dp_oracle()
    c = orc.dp_constants()
    s0 = -5e4 * np.eye(3)
    e = 1e-5
    dd = np.diag([-e, 0.0, 0.0])
    zone, s, eps = orc.dp_update(dd, np.zeros((3, 3)), s0)
    assert zone == 1 and eps == 0.0
    assert s[0, 0] == pytest.approx(-5e4 - (c["K"] + 4 * c["G"] / 3) * e, rel=1e-14)
    assert s[1, 1] == pytest.approx(-5e4 - (c["K"] - 2 * c["G"] / 3) * e, rel=1e-14)
    assert s[2, 2] == pytest.approx(s[1, 1], rel=1e-14)
    assert abs(s[0, 1]) < 1e-12


def test_dp_jaumann_rotation_is_objective():
    """A pure spin increment rotates the stress: sigma^R = R sigma R^T + O(theta^2)."""
    orc = dp_oracle()
    rng = np.random.default_rng(3)
    a = rng.normal(size=(3, 3)) * 1e3
    s0 = -1e5 * np.eye(3) + 0.5 * (a + a.T)
    for axis in np.eye(3):
        th = 1e-4
        W = th * np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
        # Rodrigues: R = exp(W)
        K = W / th
        R = np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K
        zone, s, _ = orc.dp_update(np.zeros((3, 3)), W, s0)
        assert zone == 1
        exact = R @ s0 @ R.T
        change = np.abs(exact - s0).max()
        assert np.abs(s - exact).max() < 1e-3 * change


def test_dp_zone2_returns_to_the_cone():
    orc = dp_oracle(cohesion=2e3, psi_deg=10.0)
    c = orc.dp_constants()
    rng = np.random.default_rng(4)
    hits = 0
    for _ in range(200):
        a = rng.normal(size=(3, 3)) * 4e4
        s0 = -2e4 * np.eye(3) + 0.5 * (a + a.T)
        zone, s, eps = orc.dp_update(np.zeros((3, 3)), np.zeros((3, 3)), s0)
        sm0, tau0, dev0 = invariants(s0)
        if zone != 2 or sm0 >= c["sigma_t"]:
            continue
        hits += 1
        sm, tau, dev = invariants(s)
        assert tau - c["k_phi"] + c["q_phi"] * sm == pytest.approx(0.0, abs=1e-9 * abs(sm0))
        np.testing.assert_allclose(dev / tau, dev0 / tau0, atol=1e-12)     # radial return
        dl = (tau0 - c["k_phi"] + c["q_phi"] * sm0) / (c["G"] + c["K"] * c["q_phi"] * c["q_psi"])
        assert sm == pytest.approx(sm0 - c["K"] * c["q_psi"] * dl, rel=1e-12)
        assert eps == pytest.approx(dl * np.sqrt(1 / 3 + 2 / 9 * c["q_psi"] ** 2), rel=1e-12)
    assert hits > 20


def test_dp_zone3_caps_mean_stress():
    orc = dp_oracle(cohesion=5e3, sigma_t=1e3, dp_literal=True)
    c = orc.dp_constants()
    s0 = np.diag([3e3, 2.5e3, 2.8e3])
    zone, s, eps = orc.dp_update(np.zeros((3, 3)), np.zeros((3, 3)), s0)
    sm0, tau0, dev0 = invariants(s0)
    assert zone == 3
    sm, tau, dev = invariants(s)
    assert sm == pytest.approx(c["sigma_t"], rel=1e-14)
    np.testing.assert_allclose(dev, dev0, atol=1e-9)
    assert eps == pytest.approx(np.sqrt(2) / 3 * (sm0 - c["sigma_t"]) / c["K"], rel=1e-12)


def test_dp_zone3_corner_of_a_cohesive_material():
    # past the cutoff, with tau between tau_P and the zone II/III line h = 0: Zone III, and
    # the deviator beyond tau_P takes it to the corner, sigma_m = sigma_t and tau = tau_P
    orc = dp_oracle(cohesion=5e3, sigma_t=1e3)
    c = orc.dp_constants()
    dev = np.diag([1.0, -0.5, -0.5]) / np.sqrt(0.75)          # tau(dev) = 1
    s0 = (c["sigma_t"] + 500.0) * np.eye(3) + (c["tau_P"] + 0.5 * c["alpha_P"] * 500.0) * dev
    zone, s, _ = orc.dp_update(np.zeros((3, 3)), np.zeros((3, 3)), s0)
    sm, tau, d = invariants(s)
    assert zone == 3 and c["sigma_t"] > 0 and c["tau_P"] > 0
    assert sm == pytest.approx(c["sigma_t"], rel=1e-14)
    assert tau == pytest.approx(c["tau_P"], rel=1e-12)
    np.testing.assert_allclose(d / tau, dev, atol=1e-12)


def test_dp_cohesionless_tension_is_stress_free():
    """c = 0: any trial state with positive mean stress returns to the apex (zero stress)."""
    orc = dp_oracle()
    rng = np.random.default_rng(5)
    for _ in range(100):
        a = rng.normal(size=(3, 3)) * 1e3
        s0 = 2e3 * np.eye(3) + 0.5 * (a + a.T)
        zone, s, _ = orc.dp_update(np.zeros((3, 3)), np.zeros((3, 3)), s0)
        assert zone in (2, 3)
        np.testing.assert_allclose(s, 0.0, atol=1e-9)


def test_dp_zone_classification_is_exhaustive():
    orc = dp_oracle(cohesion=3e3, sigma_t=2e3, dp_literal=True)
    c = orc.dp_constants()
    dev_dir = np.diag([1.0, -1.0, 0.0]) / np.sqrt(1.0)   # tau(dev_dir) = 1
    counts = {1: 0, 2: 0, 3: 0}
    for sm in np.linspace(-2e4, 1e4, 61) + 0.37:
        for tau in np.linspace(0.0, 2e4, 41) + 0.11:
            s0 = sm * np.eye(3) + tau * dev_dir
            zone, s, _ = orc.dp_update(np.zeros((3, 3)), np.zeros((3, 3)), s0)
            fs = tau - c["k_phi"] + c["q_phi"] * sm
            ft = sm - c["sigma_t"]
            h = tau - c["tau_P"] - c["alpha_P"] * (sm - c["sigma_t"])
            conds = {1: fs <= 0 and ft < 0, 2: (fs > 0 and ft < 0) or (h > 0 and ft >= 0),
                     3: h <= 0 and ft >= 0}
            assert sum(conds.values()) == 1
            assert conds[zone]
            counts[zone] += 1
    assert min(counts.values()) > 0
