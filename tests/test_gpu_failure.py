"""Error paths of the library on the GPU, caused on the host or by a wait that
is made to run out -- never by faulting the GPU.

* Allocation failure: MPM_FAIL_ALLOC=1 in the environment makes every device
  allocation of the library fail before it calls cudaMalloc; mpm_create and the
  first mpm_step_adjoint (which allocates its checkpoints) report MPM_ENOMEM
  and the context stays usable.
* Bounded device wait: with MPM_DEBUG_WITHHOLD_WINDOW_COPY the grid-to-particle
  kernel arms no copy for its grid window, so its wait (bounded at about one
  second by the device timer) runs out with nothing in flight; the next
  synchronising call reports MPM_ETIMEOUT, and the GPU goes on working.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2507_04192_gb300 import inputs, mpm

pytestmark = pytest.mark.gpu


def test_forced_allocation_failure_in_create(monkeypatch):
    w = inputs.dam_break_2d(32, 0.25, 0.5)
    monkeypatch.setenv("MPM_FAIL_ALLOC", "1")
    with pytest.raises(mpm.MPMError) as e:
        mpm.Simulation.from_workload(w, mpm.MPM_FP32)
    assert e.value.code == mpm.MPM_ENOMEM


def test_forced_allocation_failure_in_adjoint(monkeypatch):
    w = inputs.dam_break_inverse_2d(32, n_seg=8, n_track=4, n_obs=2, steps=20)
    sim = mpm.Simulation.from_workload(w, mpm.MPM_FP32)
    z = np.zeros((len(w.extras["obs_steps"]), len(w.extras["track_ids"]), 2))
    mpm.mpm_set_observations(sim.ctx, w.extras["track_ids"], w.extras["obs_steps"], z)
    monkeypatch.setenv("MPM_FAIL_ALLOC", "1")
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_step_adjoint(sim.ctx, 20, 10, 2, 8)
    assert e.value.code == mpm.MPM_ENOMEM
    monkeypatch.delenv("MPM_FAIL_ALLOC")
    loss, g = mpm.mpm_step_adjoint(sim.ctx, 20, 10, 2, 8)   # the same context, now with memory
    sim.close()
    assert np.isfinite(loss) and np.isfinite(g).all() and loss > 0


def test_device_wait_runs_out_and_reports_timeout():
    w = inputs.dam_break_2d(32, 0.25, 0.5, steps=10)
    sim = mpm.Simulation.from_workload(w, mpm.MPM_FP32)
    sim.step(1)
    mpm.mpm_synchronize(sim.ctx)
    mpm.mpm_set_debug(sim.ctx, mpm.MPM_DEBUG_WITHHOLD_WINDOW_COPY)
    t0 = time.perf_counter()
    sim.step(1)
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_synchronize(sim.ctx)
    elapsed = time.perf_counter() - t0
    sim.close()
    assert e.value.code == mpm.MPM_ETIMEOUT
    assert elapsed < 60.0
    # the GPU and the CUDA context are still usable: a fresh run matches the oracle
    orc = oracle.Oracle.from_workload(w)
    st = orc.initial_state(w.x)
    orc.step(st, w.steps)
    sim = mpm.Simulation.from_workload(w, mpm.MPM_FP64)
    sim.step(w.steps)
    x = sim.get("x")
    sim.close()
    assert np.abs(x - st.x).max() <= 1e-9


def test_debug_flags_are_checked():
    w = inputs.dam_break_2d(32, 0.25, 0.5)
    sim = mpm.Simulation.from_workload(w, mpm.MPM_FP32)
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_set_debug(sim.ctx, 1 << 5)
    sim.close()
    assert e.value.code == mpm.MPM_EINVAL
