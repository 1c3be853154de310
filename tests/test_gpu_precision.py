"""FP32 error of every result field against the FP64 oracle (the per-result
precision statement for single-precision runs): 2D dam break (Tait fluid) and
3D granular cylinder (Drucker-Prager), 200 steps each, no FP64 arithmetic in
the FP32 path.  Error of a field = max |gpu - oracle| / max |oracle| (positions:
/ domain size).  The bounds written here are the stated FP32 tolerances."""
import numpy as np
import pytest

import oracle
from paper_2507_04192_gb300 import inputs, mpm

pytestmark = pytest.mark.gpu

FIELDS = ("x", "v", "C", "F", "rho", "sigma", "eps")
BOUNDS = {"x": 1e-4, "v": 2e-3, "C": 5e-3, "F": 1e-4, "rho": 1e-5, "sigma": 5e-3, "eps": 2e-2}


def errors(w, steps):
    orc = oracle.Oracle.from_workload(w)
    st = orc.initial_state(w.x, w.v)
    orc.step(st, steps)
    ref = dict(x=st.x, v=st.v, C=orc.affine_C(st), F=st.F, rho=st.rho, sigma=st.sigma, eps=st.eps)
    sim = mpm.Simulation.from_workload(w, mpm.MPM_FP32)
    sim.step(steps)
    gpu = {f: sim.get(f) for f in FIELDS}
    sim.close()
    L = max(w.n_cells) * w.dx
    out = {}
    for f in FIELDS:
        r = np.asarray(ref[f], dtype=np.float64)
        g = np.asarray(gpu[f], dtype=np.float64).reshape(r.shape)
        den = L if f == "x" else max(float(np.abs(r).max()), 1e-30)
        out[f] = float(np.abs(g - r).max()) / den if np.abs(r).max() > 0 else float(np.abs(g).max())
    return out


@pytest.mark.parametrize("case", ["dam_break_2d_64", "granular_cylinder_3d_32"])
def test_fp32_error_per_result(case):
    if case == "dam_break_2d_64":
        w = inputs.dam_break_2d(64)
    else:
        w = inputs.granular_cylinder_3d((32, 32, 16), 6, 12, dt=8e-5, dx=1 / 32)
    err = errors(w, 200)
    print(f"\n{case} FP32 vs FP64 oracle, 200 steps: " + ", ".join(f"{f} {e:.2e}" for f, e in err.items()))
    for f, e in err.items():
        if case == "dam_break_2d_64" and f in ("sigma", "eps"):
            continue                      # fluid: sigma is -p I (checked via rho), eps unused
        assert e <= BOUNDS[f], (f, e)
