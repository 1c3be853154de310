"""The no-allocation step (mpm_step_noalloc) against the regular step.

Callers that cannot allocate device memory (plugins in an application that
owns all device memory, real-time loops that must not enter the allocator) use
mpm_step_noalloc with their own device buffers; its grid scratch is a static
device array.  This checks, through the C-ABI, that two calls in a row give the
same particle state as two steps of mpm_step, with separate input and output
buffers and with one buffer updated in place.  The test allocates its device
buffers with torch (the entry point itself allocates nothing).  Kept in its own
file so that it is collected last.
"""
import numpy as np
import pytest

from paper_2507_04192_gb300 import inputs, mpm

pytestmark = pytest.mark.gpu

FIELDS = ("x", "v", "C", "F", "rho", "sigma", "eps")


def _device_state(torch, fields, n, dim):
    shapes = {"x": (n, dim), "v": (n, dim), "C": (n, dim, dim), "F": (n, dim, dim), "rho": (n,),
              "sigma": (n, 9), "eps": (n,)}
    t = {k: torch.tensor(np.ascontiguousarray(fields[k]).reshape(shapes[k]), dtype=torch.float64, device="cuda")
         for k in FIELDS}
    ptrs = mpm.StatePtrs(**{k: t[k].data_ptr() for k in FIELDS})
    return t, ptrs


@pytest.mark.parametrize("case", ["fluid2d", "sand3d"])
def test_noalloc_matches_regular_step_two_calls(case):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    if case == "fluid2d":
        w = inputs.dam_break_2d(32, 0.25, 0.5)
        rng = np.random.default_rng(1)
        w.v = rng.normal(size=w.x.shape) * 0.2
    else:
        w = inputs.granular_cylinder_3d((32, 32, 32), 6, 12, floor_mu=0.0)
    sim = mpm.Simulation.from_workload(w, mpm.MPM_FP64)
    s0 = {f: sim.get(f) for f in FIELDS}
    sim.step(1)
    s1 = {f: sim.get(f) for f in FIELDS}
    sim.step(1)
    s2 = {f: sim.get(f) for f in FIELDS}
    sim.close()

    n, d = w.n, w.dim
    g = mpm.grid_struct(d, w.n_cells, w.dx, w.dt, w.gravity, mpm.MPM_FP64, 1, 1)
    m = mpm.material_struct(w.material)
    t_in, p_in = _device_state(torch, s0, n, d)
    t_mid, p_mid = _device_state(torch, {k: np.zeros_like(s0[k]) for k in FIELDS}, n, d)
    stream = torch.cuda.current_stream().cuda_stream
    mpm.mpm_step_noalloc(g, m, n, w.particle_volume, p_in, p_mid, stream)
    mpm.mpm_step_noalloc(g, m, n, w.particle_volume, p_mid, p_in, stream)     # second call, into the first buffer
    torch.cuda.synchronize()
    for ref, t in ((s1, t_mid), (s2, t_in)):
        _compare(ref, t, case)
    # in place: the same buffers as input and output, two calls
    t_ip, p_ip = _device_state(torch, s0, n, d)
    mpm.mpm_step_noalloc(g, m, n, w.particle_volume, p_ip, p_ip, stream)
    mpm.mpm_step_noalloc(g, m, n, w.particle_volume, p_ip, p_ip, stream)
    torch.cuda.synchronize()
    _compare(s2, t_ip, case)


def _compare(ref, t, case):
    for f in ("x", "v", "C", "F", "rho") + (("sigma", "eps") if case == "sand3d" else ()):
        got = t[f].cpu().numpy().reshape(ref[f].shape)
        scale = max(1.0, float(np.abs(ref[f]).max()))
        np.testing.assert_allclose(got, ref[f], rtol=0, atol=1e-10 * scale, err_msg=f)


def test_noalloc_rejects_a_grid_beyond_its_static_scratch():
    torch = pytest.importorskip("torch")
    w = inputs.dam_break_2d(32, 0.25, 0.5)
    g = mpm.grid_struct(2, (512, 512), w.dx, w.dt, w.gravity, mpm.MPM_FP64, 1, 1)
    m = mpm.material_struct(w.material)
    fields = {"x": w.x, "v": np.zeros_like(w.x), "C": np.zeros((w.n, 2, 2)), "F": np.tile(np.eye(2), (w.n, 1, 1)),
              "rho": np.full(w.n, 1000.0), "sigma": np.zeros((w.n, 9)), "eps": np.zeros(w.n)}
    _, p = _device_state(torch, fields, w.n, 2)
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_step_noalloc(g, m, w.n, w.particle_volume, p, p)
    assert e.value.code == mpm.MPM_EINVAL and "maximum" in str(e.value)
