"""Long 3D run: runout and deposit height of the granular collapse, FP32 within
1 % of FP64 (the parity gate for runs the oracle cannot reach)."""
import numpy as np
import pytest

from paper_2507_04192_gb300 import inputs, longrun

pytestmark = pytest.mark.gpu


def test_collapse_to_rest_fp32_within_one_percent_of_fp64():
    # the 2.76M-particle column at a quarter of the resolution (dx = 1/64 m, same
    # physical size), 1 s of physical time, on a floor 1.5 m wide (96 x 96 x 32
    # cells) so that the deposit stays clear of the side walls and the walls do
    # not bound the runout statistic
    w = inputs.granular_cylinder_3d((96, 96, 32), 9.5, 19, dt=4e-5, dx=1 / 64)
    out = longrun.compare(w, 25_000)
    assert out["fp32"]["finite"] and out["fp64"]["finite"]
    # the column collapsed and spread, and the deposit ends short of the side walls
    assert out["fp64"]["H_f"] < 0.8 * out["initial"]["H"]
    assert out["fp64"]["R_f"] > 1.3 * out["initial"]["R"]
    half_width = 0.5 * 96 / 64
    assert out["fp64"]["max_r"] < half_width - 2 / 64 and out["fp32"]["max_r"] < half_width - 2 / 64, out
    assert out["rel_diff"]["R_f"] <= 0.01, out
    assert out["rel_diff"]["H_f"] <= 0.01, out
