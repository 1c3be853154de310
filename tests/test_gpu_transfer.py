"""The G2P transfer variants (Sec. 2.2 G2P transfer, Appendix B: APIC, TPIC,
PIC, FLIP / PIC blend) on the GPU against the oracle: 2D dam break, FP64,
positions within 1e-9 of the domain size after 100 steps; the particle matrix
field against the oracle's (C for APIC, the velocity gradient for TPIC, zero for
PIC and FLIP)."""
import numpy as np
import pytest

import oracle
from paper_2507_04192_gb300 import inputs, mpm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("transfer", [mpm.MPM_TRANSFER_TPIC, mpm.MPM_TRANSFER_PIC, mpm.MPM_TRANSFER_FLIP])
def test_transfer_variant_matches_oracle_fp64(transfer):
    w = inputs.dam_break_2d(32)
    orc = oracle.Oracle.from_workload(w, transfer=transfer, flip_alpha=0.95)
    st = orc.initial_state(w.x)
    orc.step(st, 100)
    sim = mpm.Simulation.from_workload(w, mpm.MPM_FP64, transfer=transfer, flip_alpha=0.95)
    sim.step(100)
    x, v, Cm = sim.get("x"), sim.get("v"), sim.get("C")
    sim.close()
    L = 32 * w.dx
    assert np.abs(x - st.x).max() <= 1e-9 * L
    assert np.abs(v - st.v).max() <= 1e-7 * max(np.abs(st.v).max(), 1e-12)
    ref_C = orc.affine_C(st)
    np.testing.assert_allclose(Cm.reshape(ref_C.shape), ref_C, rtol=0, atol=1e-6 * max(np.abs(ref_C).max(), 1.0))
    if transfer in (mpm.MPM_TRANSFER_PIC, mpm.MPM_TRANSFER_FLIP):
        assert np.abs(Cm).max() == 0.0


def test_flip_fp32_and_3d_sand():
    """FLIP / PIC blend in FP32 (2D fluid) and for Drucker-Prager sand in 3D, against the oracle."""
    w = inputs.dam_break_2d(32)
    orc = oracle.Oracle.from_workload(w, transfer=3, flip_alpha=0.9)
    st = orc.initial_state(w.x)
    orc.step(st, 100)
    sim = mpm.Simulation.from_workload(w, mpm.MPM_FP32, transfer=3, flip_alpha=0.9)
    sim.step(100)
    assert np.abs(sim.get("x") - st.x).max() <= 1e-4 * 32 * w.dx
    sim.close()
    w3 = inputs.granular_cylinder_3d((16, 16, 16), 4, 8, dt=2e-4, dx=1 / 16)
    orc = oracle.Oracle.from_workload(w3, transfer=3, flip_alpha=0.9)
    st = orc.initial_state(w3.x)
    orc.step(st, 40)
    sim = mpm.Simulation.from_workload(w3, mpm.MPM_FP64, transfer=3, flip_alpha=0.9)
    sim.step(40)
    assert np.abs(sim.get("x") - st.x).max() <= 1e-9 * 16 * w3.dx
    np.testing.assert_allclose(sim.get("sigma").reshape(st.sigma.shape), st.sigma, rtol=0,
                               atol=1e-6 * np.abs(st.sigma).max())
    sim.close()


def test_transfer_variants_differ_and_adjoint_rejects_them():
    w = inputs.dam_break_2d(32)
    xs = []
    for tr in (mpm.MPM_TRANSFER_APIC, mpm.MPM_TRANSFER_TPIC, mpm.MPM_TRANSFER_PIC, mpm.MPM_TRANSFER_FLIP):
        sim = mpm.Simulation.from_workload(w, mpm.MPM_FP64, transfer=tr)
        sim.step(50)
        xs.append(sim.get("x"))
        if tr != mpm.MPM_TRANSFER_APIC:
            mpm.mpm_set_friction_field(sim.ctx, 2, (4, 1), np.full(4, 0.3))
            mpm.mpm_set_observations(sim.ctx, np.array([0]), [5], np.zeros((1, 1, 2)))
            with pytest.raises(mpm.MPMError) as e:
                mpm.mpm_step_adjoint(sim.ctx, 5, 5, 2, 4)
            assert e.value.code == mpm.MPM_EINVAL
        sim.close()
    assert np.abs(xs[0] - xs[1]).max() > 1e-9 and np.abs(xs[0] - xs[2]).max() > 1e-9
    with pytest.raises(mpm.MPMError):
        mpm.Simulation(2, (8, 8), 1 / 8, 1e-4, (0, -9.8), dict(inputs.FLUID_WATER), transfer=4)
    with pytest.raises(mpm.MPMError):
        mpm.Simulation(2, (8, 8), 1 / 8, 1e-4, (0, -9.8), dict(inputs.FLUID_WATER), transfer=3, flip_alpha=1.5)
