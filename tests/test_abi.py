"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares; struct layouts agree between C and the binding.  No
compute calls (these run without a GPU)."""
import ctypes as C
import glob
import os
import re
import subprocess

import pytest

from paper_2507_04192_gb300 import mpm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:int|void|int64_t)\s+\**\s*(mpm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("mpm_create", "mpm_load_particles", "mpm_step", "mpm_set_friction_field", "mpm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = mpm.load_library()
    out = subprocess.run(["nm", "-D", "--defined-only", mpm.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mpm_\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "mpm.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(mpm_grid_desc), offsetof(mpm_grid_desc, batch),"
        " offsetof(mpm_grid_desc, gravity), sizeof(mpm_material), offsetof(mpm_material, dp_literal),"
        " offsetof(mpm_material, sigma_t)); return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals == [C.sizeof(mpm.GridDesc), mpm.GridDesc.batch.offset, mpm.GridDesc.gravity.offset,
                    C.sizeof(mpm.Material), mpm.Material.dp_literal.offset, mpm.Material.sigma_t.offset]


def test_invalid_descriptors_rejected_before_device_use():
    g = mpm.grid_struct(4, (8, 8, 8), 0.1, 1e-4, (0, 0, 0))
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_create(g, mpm.material_struct(dict(kind=0, rho0=1000, bulk_K=1e5, gamma=7)))
    assert e.value.code == mpm.MPM_EINVAL
    g = mpm.grid_struct(2, (8, 8), -0.1, 1e-4, (0, 0))
    with pytest.raises(mpm.MPMError):
        mpm.mpm_create(g, mpm.material_struct(dict(kind=0, rho0=1000, bulk_K=1e5, gamma=7)))
    g = mpm.grid_struct(2, (8, 8), 0.1, 1e-4, (0, 0))
    with pytest.raises(mpm.MPMError) as e:       # viscous fluid is not supported
        mpm.mpm_create(g, mpm.material_struct(dict(kind=0, rho0=1000, bulk_K=1e5, gamma=7, viscosity=1e-3)))
    assert e.value.code == mpm.MPM_EINVAL


def test_non_finite_and_unphysical_parameters_rejected_before_device_use():
    fluid = dict(kind=0, rho0=1000, bulk_K=1e5, gamma=7)
    sand = dict(kind=1, rho0=2000, E=1e6, nu=0.3, phi_deg=30, psi_deg=0, cohesion=0, sigma_t=0)
    good = dict(dim=2, n_cells=(8, 8), dx=0.1, dt=1e-4, gravity=(0, -9.81))
    cases = [(dict(good, dx=float("inf")), fluid), (dict(good, dt=float("nan")), fluid),
             (dict(good, gravity=(0, float("nan"))), fluid), (good, dict(fluid, bulk_K=float("inf"))),
             (good, dict(sand, phi_deg=90.0)), (good, dict(sand, phi_deg=-5.0)), (good, dict(sand, psi_deg=95.0)),
             (good, dict(sand, cohesion=-1.0)), (good, dict(sand, sigma_t=-1.0)),
             (good, dict(sand, sigma_t=float("inf"))), (good, dict(sand, nu=0.5)), (good, dict(sand, E=float("nan")))]
    for gd, mat in cases:
        g = mpm.grid_struct(gd["dim"], gd["n_cells"], gd["dx"], gd["dt"], gd["gravity"])
        with pytest.raises(mpm.MPMError) as e:
            mpm.mpm_create(g, mpm.material_struct(mat))
        assert e.value.code == mpm.MPM_EINVAL, (gd, mat)
    # the allocation-free step applies the same checks before it touches its buffers
    ptrs = mpm.StatePtrs()
    for gd, mat in cases[:4] + cases[-2:]:
        g = mpm.grid_struct(gd["dim"], gd["n_cells"], gd["dx"], gd["dt"], gd["gravity"], precision=mpm.MPM_FP64)
        with pytest.raises(mpm.MPMError) as e:
            mpm.mpm_step_noalloc(g, mpm.material_struct(mat), 10, 1e-4, ptrs, ptrs)
        assert e.value.code == mpm.MPM_EINVAL, (gd, mat)
        assert "missing state buffer" not in str(e.value), (gd, mat)      # rejected by the parameter checks
