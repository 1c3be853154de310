"""Benchmark of the explicit MPM step on the 2.76M-particle 3D granular
cylinder collapse (256 x 256 x 128 cells, Drucker-Prager sand, frictional
floor), the workload of the paper's cylinder-collapse timing (Sec. 4.2.3).

One bench step is one MPM time step (sort every k steps, P2G, grid update,
G2P) of the whole particle set.  Prints one JSON line on rank 0.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle as it stands on the host cores
(bounded samples of the same workload).  With N > 1 (torchrun) every rank runs
an independent replica of the simulation (the step does not shard), and the
value is all ranks' particle-steps divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (2.7M 3D collapse, FP32 vs FP64 plain); adjoint/forward ratio"
WORKLOAD = "granular_cylinder_3d_256x256x128"
FORWARD_KERNELS = ("sort", "p2g", "grid", "g2p")      # kernel classes of a forward step


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(v: float, device=None) -> float:
    """The largest value over the ranks of the default process group (the value
    itself without one).  Replicas only: this and the barriers are the whole
    multi-GPU protocol; no data crosses between ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(v)
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank: int, world: int, seconds_max: float) -> float:
    """Whole-job throughput of N replicas: the units all ranks processed over the
    slowest rank's time."""
    return world * units_per_rank / seconds_max


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.gpu = gpu_index
        if shutil.which("nvidia-smi") is None:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.fh = open(self.path, "w")
        self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.QUERY}",
                                      "--format=csv,noheader,nounits", "-lms", "200"],
                                     stdout=self.fh, stderr=subprocess.DEVNULL)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


REJECTING_REASONS = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}


def clocks_rejected(clocks) -> bool:
    """A timed region whose clock record shows a hardware or thermal slowdown, or an
    SM clock well below its maximum with no reason given (a leftover clock lock),
    does not give a valid number.  sw_power_cap is kept (noted in the record)."""
    if not clocks:
        return False
    if REJECTING_REASONS & set(clocks.get("reasons", [])):
        return True
    sm, mx = clocks.get("sm_mhz"), clocks.get("sm_max_mhz")
    return bool(sm and mx and sm < 0.8 * mx and not clocks.get("reasons"))


def load_peaks_bf16() -> float:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p)).get("bf16_tflops", 1900.0))
    return 1900.0


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def algorithmic_bytes_per_particle(kernel: str, dim: int, material: int, rsz: int) -> int:
    """Compulsory particle bytes of one launch per particle (the state each kernel must
    read and write once; grid traffic excluded)."""
    d = dim
    x, v, C, F, rho = d, d, d * d, d * d, 1
    sig, eps = (6, 1) if material == 1 else (0, 0)
    if kernel == "p2g":            # reads x, v, C, rho (and sigma)
        words = x + v + C + rho + sig
    elif kernel == "g2p":          # reads x, F, rho, sigma, eps; writes the whole state
        words = (x + F + rho + sig + eps) + (x + v + C + F + rho + sig + eps)
    else:
        return 0
    return words * rsz


def oracle_sample(n_particles: int):
    """A bounded sample of the 3D collapse for the CPU oracle: the first
    n_particles of the cylinder in load order (its bottom layers), on a grid
    cropped around them."""
    from paper_2507_04192_gb300 import inputs
    w = inputs.granular_cylinder_3d()
    x = w.x[:n_particles].copy()
    lo = np.floor(x.min(axis=0) / w.dx) - 2
    lo[2] = 0.0
    x -= lo * w.dx
    n_cells = tuple(int(np.ceil(x[:, a].max() / w.dx)) + 3 for a in range(3))
    return w, x, n_cells


def run_oracle_steps(n_particles: int, steps: int, warmup: int = 0):
    import oracle
    w, x, n_cells = oracle_sample(n_particles)
    orc = oracle.Oracle(3, n_cells, w.dx, w.dt, w.gravity, w.material, w.particle_volume, w.friction)
    st = orc.initial_state(x)
    if warmup:
        orc.step(st, warmup)
    t0 = time.perf_counter()
    orc.step(st, steps)
    return time.perf_counter() - t0


def host_cpu() -> dict:
    """The host's logical CPU count and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None and os.path.exists("/proc/cpuinfo"):
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


def cpu_baseline_full_step():
    """The oracle on one full step of the whole 2.76M-particle workload: the serial
    build as it stands, and its OpenMP build on every host core."""
    import oracle
    from paper_2507_04192_gb300 import inputs
    w = inputs.granular_cylinder_3d()
    orc = oracle.Oracle.from_workload(w)
    st = orc.initial_state(w.x)
    t0 = time.perf_counter()
    orc.step(st, 1)
    dt = time.perf_counter() - t0
    host = host_cpu()
    out = {"value": w.n / dt, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
           "sample": f"1 full step of all {w.n} particles on the 256x256x128 grid, FP64, single thread, "
                     f"{dt:.1f} s", "host": host}
    try:
        threads = os.cpu_count() or 1
        os.environ.setdefault("OMP_NUM_THREADS", str(threads))
        st = orc.initial_state(w.x)
        t0 = time.perf_counter()
        orc.step(st, 1, omp=True)
        dto = time.perf_counter() - t0
        out["openmp"] = {"value": w.n / dto, "unit": "particle-steps/s", "cores": int(os.environ["OMP_NUM_THREADS"]),
                         "sample": f"the same step, OpenMP build of the oracle (particle-parallel transfers with "
                                   f"atomic grid sums, node-parallel grid update), {dto:.2f} s"}
    except Exception as e:          # no OpenMP runtime on the host: the serial figure stands alone
        out["openmp"] = {"unavailable": str(e).splitlines()[0][:200]}
    return out


def workload_config(world: int) -> dict:
    """The headline workload (the same object on both arms)."""
    return {"workload": WORKLOAD, "particles": 2761536, "grid": "256x256x128", "precision": "fp32",
            "material": "drucker_prager", "sort_every": 32, "parallelism": f"replicas{world}",
            "l2": "inputs larger than L2 (353 MB particle state per step)",
            "sort": "the timed window starts with a sort (keys, radix passes, tiles, state permutation), "
                    "so every window holds at least one"}


def bench_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    # calibrate: per-step sample sized so that warmup + steps fit in ~120 s
    probe_n = 20000
    t = run_oracle_steps(probe_n, 1)
    per_particle = t / probe_n
    budget = 120.0
    n = int(max(2000, min(200000, budget / max(1, args.steps + args.warmup) / per_particle)))
    dt = run_oracle_steps(n, args.steps, args.warmup)
    value = n * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(world),
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step: the first {n} particles of the 2.76M-particle cylinder "
                                       f"(bottom layers) on a grid cropped around them, FP64, single thread",
                             "host": host_cpu()},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


STATE_BYTES_FP32_3D_DP = 128          # x3 v3 C9 F9 rho1 sigma6 eps1 = 32 words
PAPER_FP32_PARTICLE_STEPS = 1.22e8    # 2,712,960 particles x 1000 steps in 22.3 s (Sec. 5, timing table)


def count_active_nodes(x: np.ndarray, dx: float, n_cells) -> int:
    """Grid nodes inside the quadratic B-spline stencils of particles at x."""
    d = x.shape[1]
    G = [int(c) + 4 for c in n_cells]
    base = np.floor(x / dx - 0.5).astype(np.int64) + 1          # first stencil node, shifted to >= 0
    mark = np.zeros(int(np.prod(G)), dtype=bool)
    for off in np.ndindex(*(3,) * d):
        idx = np.zeros(len(x), dtype=np.int64)
        for a in reversed(range(d)):
            idx = idx * G[a] + np.clip(base[:, a] + off[a], 0, G[a] - 1)
        mark[idx] = True
    return int(mark.sum())


def read_traffic(kernel: str):
    """DRAM bytes (read + write) per launch of ``kernel`` from the ncu summary
    table in profiles/traffic.txt (lines: kernel bytes), or None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if len(f) >= 2 and not line.startswith("#") and f[0] == f"k_{kernel}":
            return float(f[1])
    return None


def _event_ms(stream, fn):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def secondary_measurements(stream, dev):
    """The other hot-path rows, each on its own workload: the checkpointed
    adjoint of the 128 x 128 dam-break inverse (FP32, 500 steps, checkpoint 50)
    and of the 3D granular inverse (1.36M particles, 600 steps, checkpoint 60),
    a batch of 256 independent 96 x 96 dam breaks (FP32, 300 steps), the 3D dam
    break with two rigid columns (1.92M particles, FP32), and the 640-256-256-32
    network's training step and inference at batch 256."""
    from paper_2507_04192_gb300 import inputs, mpm

    out = {}
    # adjoint / forward
    w = inputs.dam_break_inverse_2d(128)
    mu = w.extras["mu_true"]
    z = np.zeros((len(w.extras["obs_steps"]), len(w.extras["track_ids"]), 2))
    steps = max(w.extras["obs_steps"])
    sim = mpm.Simulation(2, w.n_cells, w.dx, w.dt, w.gravity, w.material, mpm.MPM_FP32, w.sort_every,
                         stream=stream.cuda_stream)
    sim.load(w.x, None, w.particle_volume)
    sim.set_friction(2, (len(mu), 1), mu)
    mpm.mpm_save_state(sim.ctx, 0)
    mpm.mpm_set_observations(sim.ctx, w.extras["track_ids"], w.extras["obs_steps"], z)
    sim.step(20)
    mpm.mpm_restore_state(sim.ctx, 0)
    fwd = min(_event_ms(stream, lambda: (mpm.mpm_restore_state(sim.ctx, 0), sim.step(steps))) for _ in range(3))
    adj = min(_event_ms(stream, lambda: (mpm.mpm_restore_state(sim.ctx, 0),
                                         mpm.mpm_step_adjoint(sim.ctx, steps, 50, 2, len(mu)))) for _ in range(3))
    sim.close()
    out["adjoint"] = {"workload": f"dam_break_inverse_2d_128 ({w.n} particles, {steps} steps, checkpoint 50, fp32)",
                      "forward_ms": fwd, "adjoint_ms": adj, "adjoint_over_forward": (adj - fwd) / fwd,
                      "total_over_forward": adj / fwd,
                      "note": "adjoint_ms = checkpointed forward + per-segment recompute + reverse sweep; "
                              "adjoint_over_forward counts the recompute and reverse sweep only"}
    # adjoint / forward of the 3D granular inverse problem (1.36M particles, 600 steps, checkpoint 60)
    w3 = inputs.granular_inverse_3d()
    mu3 = w3.extras["mu_true"]
    z3 = np.zeros((len(w3.extras["obs_steps"]), len(w3.extras["track_ids"]), 3))
    steps3 = max(w3.extras["obs_steps"])
    sim = mpm.Simulation.from_workload(w3, mpm.MPM_FP32, stream=stream.cuda_stream)
    mpm.mpm_save_state(sim.ctx, 0)
    mpm.mpm_set_observations(sim.ctx, w3.extras["track_ids"], w3.extras["obs_steps"], z3)
    fwd3 = min(_event_ms(stream, lambda: (mpm.mpm_restore_state(sim.ctx, 0), sim.step(steps3))) for _ in range(2))
    adj3 = min(_event_ms(stream, lambda: (mpm.mpm_restore_state(sim.ctx, 0),
                                          mpm.mpm_step_adjoint(sim.ctx, steps3, 60, 4, len(mu3)))) for _ in range(2))
    # time per kernel class inside the default sweep (CUDA events around each launch
    # group; there the reverse steps of a segment overlap the recompute of the one
    # before it, so they share the GPU)
    mpm.mpm_set_timing(sim.ctx, True)
    mpm.mpm_reset_timing(sim.ctx)
    mpm.mpm_restore_state(sim.ctx, 0)
    mpm.mpm_step_adjoint(sim.ctx, steps3, 60, 4, len(mu3))
    kt3 = {k: mpm.mpm_get_timing(sim.ctx, k) for k in mpm.KERNELS}
    # one forward step and one reverse step on their own: a plain forward run, and
    # the sweep that keeps every segment (no recompute runs beside its reverse steps)
    mpm.mpm_reset_timing(sim.ctx)
    mpm.mpm_restore_state(sim.ctx, 0)
    sim.step(steps3)
    kf3 = {k: mpm.mpm_get_timing(sim.ctx, k) for k in FORWARD_KERNELS}
    mpm.mpm_set_adjoint_memory(sim.ctx, 1 << 38)
    mpm.mpm_reset_timing(sim.ctx)
    mpm.mpm_restore_state(sim.ctx, 0)
    mpm.mpm_step_adjoint(sim.ctx, steps3, 60, 4, len(mu3))
    kr3 = mpm.mpm_get_timing(sim.ctx, "reverse")
    mpm.mpm_set_timing(sim.ctx, False)
    fwd_step3 = sum(kf3[k][0] for k in FORWARD_KERNELS) / steps3
    rev_step3 = kr3[0] / max(1, kr3[1])
    # the same sweep keeping every segment of the first pass in HBM (no recomputation)
    adj3k = min(_event_ms(stream, lambda: (mpm.mpm_restore_state(sim.ctx, 0),
                                           mpm.mpm_step_adjoint(sim.ctx, steps3, 60, 4, len(mu3)))) for _ in range(2))
    sim.close()
    out["adjoint_3d"] = {"workload": f"granular_inverse_3d_192x192x96 ({w3.n} particles, {steps3} steps, "
                                     f"checkpoint 60, 16x16 floor patches, fp32)",
                         "forward_ms": fwd3, "adjoint_ms": adj3, "adjoint_over_forward": (adj3 - fwd3) / fwd3,
                         "total_over_forward": adj3 / fwd3,
                         "reverse_step_ms": rev_step3, "forward_step_ms": fwd_step3,
                         "reverse_step_over_forward_step": rev_step3 / fwd_step3,
                         "step_note": "one reverse step timed in the sweep that keeps every segment (nothing runs "
                                      "beside it), one forward step in a plain forward run",
                         "sweep_ms_by_class": {k: v[0] for k, v in kt3.items()},
                         "sweep_launches_by_class": {k: v[1] for k, v in kt3.items()},
                         "kept_segments": {"adjoint_ms": adj3k, "adjoint_over_forward": (adj3k - fwd3) / fwd3,
                                           "total_over_forward": adj3k / fwd3,
                                           "note": "mpm_set_adjoint_memory: all ten 60-step segments of the "
                                                   "first pass kept in HBM (about 150 GB), none recomputed"}}
    # batched forward (training data)
    wb = inputs.dam_break_2d(96)
    B, nb, bsteps = 256, wb.n, 300
    sim = mpm.Simulation(2, wb.n_cells, wb.dx, wb.dt, wb.gravity, wb.material, mpm.MPM_FP32, wb.sort_every,
                         batch=B, stream=stream.cuda_stream)
    sim.load(np.tile(wb.x, (B, 1)), None, wb.particle_volume, np.repeat(np.arange(B, dtype=np.int32), nb))
    sim.set_friction(2, (32, 1), np.stack([inputs.friction_field(32, 1_000_000 + i) for i in range(B)]).reshape(-1))
    sim.step(5)
    ms = _event_ms(stream, lambda: sim.step(bsteps))
    xb = sim.get("x").reshape(B, nb, 2)
    sim.close()
    # compulsory traffic: the 13-word fluid state read and written once per particle,
    # 32 B per active node of each simulation's grid (counted on a sample of 16)
    bnodes = int(round(np.mean([count_active_nodes(xb[i], wb.dx, wb.n_cells) for i in range(0, B, B // 16)]) * B))
    bbytes = B * nb * 2 * 13 * 4 + bnodes * 32
    peak, _ = load_peaks()
    out["batched_forward"] = {"workload": f"{B} x dam_break_2d_96 ({B * nb} particles, {bsteps} steps, fp32)",
                              "value": B * nb * bsteps / (ms * 1e-3), "unit": "particle-steps/s",
                              "ms_per_step": ms / bsteps,
                              "step_roofline": {"bytes_per_step": bbytes, "active_nodes": bnodes,
                                                "achieved": bbytes / (ms / bsteps * 1e-3) / 1e9, "peak": peak,
                                                "frac": bbytes / (ms / bsteps * 1e-3) / 1e9 / peak, "unit": "GB/s"}}
    # the 3D dam break with two rigid columns (1.92M fluid particles, FP32)
    wd = inputs.dam_break_3d()
    sim = mpm.Simulation.from_workload(wd, mpm.MPM_FP32, stream=stream.cuda_stream)
    sim.step(20)
    dsteps = 200
    mpm.mpm_set_timing(sim.ctx, True)
    mpm.mpm_reset_timing(sim.ctx)
    ms = _event_ms(stream, lambda: sim.step(dsteps))
    kt = {k: mpm.mpm_get_timing(sim.ctx, k)[0] / dsteps for k in FORWARD_KERNELS}
    xd = sim.get("x")
    sim.close()
    dnodes = count_active_nodes(xd, wd.dx, wd.n_cells)
    dbytes = wd.n * 2 * 25 * 4 + dnodes * 32          # fluid state x v C F rho: 25 words read + written
    peak, _ = load_peaks()
    out["dam_break_3d"] = {"workload": f"dam_break_3d_200x100x80 ({wd.n} particles, two rigid columns, "
                                       f"{dsteps} steps after 20, fp32)",
                           "value": wd.n * dsteps / (ms * 1e-3), "unit": "particle-steps/s",
                           "ms_per_step": ms / dsteps, "kernels_ms_per_step": kt,
                           "step_roofline": {"bytes_per_step": dbytes, "active_nodes": dnodes,
                                             "achieved": dbytes / (ms / dsteps * 1e-3) / 1e9, "peak": peak,
                                             "frac": dbytes / (ms / dsteps * 1e-3) / 1e9 / peak, "unit": "GB/s"},
                           "paper_context": {"value": 1.92e6 * 1000 / 8.2, "unit": "particle-steps/s",
                                             "note": "paper's FP32 figure for this workload (1000 steps in "
                                                     "8.2 s, Table 3): context, other GPU"}}
    # network
    W = [640, 256, 256, 32]
    net = mpm.MLP(W, 256, stream=stream.cuda_stream)
    rng = np.random.default_rng(0)
    net.set_params((rng.standard_normal(net.num_params) * 0.03).astype(np.float32))
    xs = rng.standard_normal((256, 640)).astype(np.float32)
    ts = rng.uniform(0.1, 0.6, (256, 32)).astype(np.float32)
    for _ in range(5):
        net.train_step(xs, ts, 1e-3)
    reps = 50
    tr = _event_ms(stream, lambda: [net.train_step(xs, ts, 1e-3) for _ in range(reps)]) / reps
    inf = _event_ms(stream, lambda: [net.infer(xs) for _ in range(reps)]) / reps
    # device-only: inputs resident, no host copies and no synchronisation inside the timed region
    import torch
    dx_, dt_ = torch.tensor(xs, device=dev), torch.tensor(ts, device=dev)
    dl_ = torch.zeros(1, dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    for _ in range(5):
        net.train_step_async(256, dx_.data_ptr(), dt_.data_ptr(), 1e-3, dl_.data_ptr())
    tr_dev = _event_ms(stream, lambda: [net.train_step_async(256, dx_.data_ptr(), dt_.data_ptr(), 1e-3,
                                                             dl_.data_ptr()) for _ in range(reps)]) / reps
    net.close()
    fl_fwd = 2 * 256 * sum(W[i] * W[i + 1] for i in range(3))
    out["mlp"] = {"widths": W, "batch": 256, "train_step_ms": tr, "infer_ms": inf,
                  "train_tflops": 3 * fl_fwd / (tr * 1e-3) / 1e12,
                  "note": "host-synchronous calls incl. host<->device copies of x, targets and loss",
                  "device_train_step_ms": tr_dev, "device_train_tflops": 3 * fl_fwd / (tr_dev * 1e-3) / 1e12,
                  "device_note": "mpm_mlp_train_step_async on resident device buffers: forward, backward, Adam "
                                 "(about 30 launches per step at this size; launch- and latency-bound)",
                  "gemm": gemm_measurement(stream),
                  "gemm_network_shape": gemm_measurement(stream, shape=(256, 256, 640), reps=200)}
    return out


def mlp_device_measurement(reps=20):
    """The 640-256-256-32 network's training step on resident device buffers at batch 256."""
    import torch

    from paper_2507_04192_gb300 import mpm
    stream = torch.cuda.Stream()
    W = [640, 256, 256, 32]
    net = mpm.MLP(W, 256, stream=stream.cuda_stream)
    rng = np.random.default_rng(0)
    net.set_params((rng.standard_normal(net.num_params) * 0.03).astype(np.float32))
    dx_ = torch.tensor(rng.standard_normal((256, 640)).astype(np.float32), device="cuda")
    dt_ = torch.tensor(rng.uniform(0.1, 0.6, (256, 32)).astype(np.float32), device="cuda")
    dl_ = torch.zeros(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    step = lambda: net.train_step_async(256, dx_.data_ptr(), dt_.data_ptr(), 1e-3, dl_.data_ptr())
    for _ in range(3):
        step()
    ms = _event_ms(stream, lambda: [step() for _ in range(reps)]) / reps
    net.close()
    return {"widths": W, "batch": 256, "train_step_ms": ms}


def gemm_measurement(stream, shape=(8192, 2048, 2048), reps=10):
    """The tensor-core GEMM itself (C = A B^T, bf16 in, fp32 out) on a shape large
    enough to fill the GPU, against the measured cuBLAS bf16 burst peak."""
    import torch

    from paper_2507_04192_gb300 import mpm

    gM, gN, gK = shape
    ga = torch.randn(gM, gK, device="cuda").to(torch.bfloat16)
    gb = torch.randn(gN, gK, device="cuda").to(torch.bfloat16)
    gc = torch.empty(gM, gN, device="cuda")
    gst = torch.zeros(1, dtype=torch.int32, device="cuda")
    run = lambda: mpm.mpm_gemm_bf16(gM, gN, gK, ga.data_ptr(), gK, gb.data_ptr(), gK, gc.data_ptr(), gN,
                                    gst.data_ptr(), stream.cuda_stream)
    for _ in range(3):
        run()
    gms = _event_ms(stream, lambda: [run() for _ in range(reps)]) / reps
    assert int(gst.item()) == 0
    peak_tf = load_peaks_bf16()
    gemm_tf = 2.0 * gM * gN * gK / (gms * 1e-3) / 1e12
    return {"shape": [gM, gN, gK], "ms": gms, "tflops": gemm_tf, "peak": peak_tf, "frac": gemm_tf / peak_tf,
            "peak_source": "measured bf16_tflops (cuBLAS burst)"}


def bench_ours(args):
    import torch

    from paper_2507_04192_gb300 import inputs, mpm

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)          # a real stream handle: the library and the events share it

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    w = inputs.granular_cylinder_3d()
    n = w.n
    assert n == workload_config(world)["particles"] and w.sort_every == workload_config(world)["sort_every"]

    def timed_run(precision, steps, warmup, timing=False):
        sim = mpm.Simulation.from_workload(w, precision, stream=stream.cuda_stream)
        sim.step(warmup)
        sim.synchronize()
        if timing:
            mpm.mpm_set_timing(sim.ctx, True)
            mpm.mpm_reset_timing(sim.ctx)
        barrier()
        torch.cuda.synchronize(dev)
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        st0 = sim.stats()
        # the window starts with a sort: whatever --steps is, one sort (the full state
        # permutation included) is amortised over the timed steps, at least its share
        # 1/sort_every of a long run
        mpm.mpm_request_sort(sim.ctx)
        start.record(stream)
        sim.step(steps)
        end.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        ms = start.elapsed_time(end)
        sim.synchronize()
        st1 = sim.stats()
        launches = st1["launches"] - st0["launches"]
        sorts = st1["sorts"] - st0["sorts"]
        ktimes = {k: mpm.mpm_get_timing(sim.ctx, k) for k in FORWARD_KERNELS} if timing else None
        sim.close()
        return ms, launches, ktimes, sorts

    # FP32 headline (clean timed region), with clocks sampled during it
    sampler = ClockSampler(local)
    ms32, launches, _, sorts = timed_run(mpm.MPM_FP32, args.steps, args.warmup)
    clocks = sampler.stop()
    # a throttled or clock-locked region is measured once more (every rank takes the same decision)
    if max_over_ranks(1.0 if clocks_rejected(clocks) else 0.0, dev) > 0.0:
        sampler = ClockSampler(local)
        ms32, launches, _, sorts = timed_run(mpm.MPM_FP32, args.steps, args.warmup)
        clocks = sampler.stop()
        if clocks is not None:
            clocks["remeasured"] = True
    # per-kernel device times (library CUDA events on the launch stream), same workload
    _, _, kt, _ = timed_run(mpm.MPM_FP32, args.steps, 3, timing=True)
    # FP64 mode, fewer steps
    steps64 = max(1, min(args.steps, 200))
    ms64 = timed_run(mpm.MPM_FP64, steps64, 3)[0] if not args.no_fp64 else float("nan")

    def reduce_max(v):
        return max_over_ranks(v, dev)

    ms32 = reduce_max(ms32)
    ms64 = reduce_max(ms64)
    value = replica_value(n * args.steps, world, ms32 * 1e-3)
    value64 = replica_value(n * steps64, world, ms64 * 1e-3)

    # end to end through the C-ABI with host buffers: load (h2d), steps, read back (d2h)
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    sim = mpm.Simulation.from_workload(w, mpm.MPM_FP32, stream=stream.cuda_stream, load=False)
    sim.load(w.x, None, w.particle_volume)
    for wall, nseg, mu in w.friction:
        sim.set_friction(wall, nseg, mu)
    sim.step(args.steps)
    xout = sim.get("x")
    e2e_s = time.perf_counter() - t0
    sim.close()
    e2e_s = reduce_max(e2e_s)
    assert np.isfinite(xout).all()

    # whole-step roofline: compulsory particle state (read once, written once) plus
    # the active grid nodes (m and q written once and read once)
    active_nodes = count_active_nodes(xout, w.dx, w.n_cells)
    step_bytes = n * 2 * STATE_BYTES_FP32_3D_DP + active_nodes * 32

    # roofline of the dominant kernel
    peak, peak_kind = load_peaks()
    dom = max(("p2g", "g2p"), key=lambda k: kt[k][0])
    dom_ms, dom_n = kt[dom]
    per_launch_ms = dom_ms / max(1, dom_n)
    bpp = algorithmic_bytes_per_particle(dom, 3, 1, 4)
    achieved = bpp * n / (per_launch_ms * 1e-3) / 1e9
    traffic = read_traffic(dom)

    extra = secondary_measurements(stream, dev) if (rank == 0 and not args.headline_only) else {}

    if rank == 0:
        cpu = cpu_baseline_full_step() if (world == 1 and not args.no_cpu) else None
        line = {
            "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms32 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": workload_config(world),
            "fp64": ({"value": value64, "unit": "particle-steps/s", "steps": steps64,
                      "ms_per_step": ms64 / steps64,
                      "bound": "fp64 alu",
                      "ceiling_note": "ncu: the FP64 P2G and G2P keep the FP64 pipe busy on 81-87 % of their "
                                      "active cycles (profiles/k_p2g_k_g2p_fp64_granular_cylinder_3d_128x128x64.md): "
                                      "at most about 1.2x faster with the same FP64 instruction count"}
                     if not args.no_fp64 else None),
            "kernels_ms_per_step": {k: kt[k][0] / max(1, args.steps) for k in kt},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"{peak_kind} hbm_gbs", "bytes_per_particle": bpp},
            "step_roofline": {"bound": "hbm", "bytes_per_step": step_bytes,
                              "achieved": step_bytes / (ms32 / args.steps * 1e-3) / 1e9, "peak": peak,
                              "unit": "GB/s", "frac": step_bytes / (ms32 / args.steps * 1e-3) / 1e9 / peak,
                              "active_nodes": active_nodes,
                              "note": "128 B state read + 128 B written per particle, 32 B per active node"},
            "paper_context": {"value": PAPER_FP32_PARTICLE_STEPS, "unit": "particle-steps/s",
                              "note": "paper's FP32 figure for its 2.71M-particle collapse on an A100 "
                                      "(400x400x100 grid): context, not the same workload"},
            "cpu_baseline": cpu,
            "e2e": {"value": world * n * args.steps / e2e_s, "unit": "particle-steps/s",
                    "h2d_bytes_per_step": n * 3 * 8 / args.steps, "d2h_bytes_per_step": n * 3 * 8 / args.steps,
                    "note": "one mpm_load_particles from host, K steps, one mpm_get_particles to host"},
            "gpu_launches": launches,
            "sorts_in_window": sorts,
            "clocks": clocks,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def profile_run(what: str, steps: int):
    """A short run of one workload for ncu (no timing): ``forward`` steps the
    2.76M-particle collapse in FP32, ``fp64`` the 345,648-particle collapse
    (128 x 128 x 64 cells) in FP64, ``batched`` the 256 batched 96^2 dam breaks,
    ``adjoint`` runs one 120-step adjoint of the 1.36M-particle inverse problem
    (checkpoint 60), ``adjoint-small`` the same on its 96 x 96 x 48 counterpart
    (169,680 particles, a few GB on the device).  Prints one JSON line with the
    sizes."""
    from paper_2507_04192_gb300 import inputs, mpm
    if what == "forward":
        w = inputs.granular_cylinder_3d()
        sim = mpm.Simulation.from_workload(w, mpm.MPM_FP32)
        sim.step(steps)
        out = {"particles": w.n}
    elif what == "fp64":
        w = inputs.granular_cylinder_3d((128, 128, 64), 19, 38, dx=1 / 128.0, dt=2e-5)
        sim = mpm.Simulation.from_workload(w, mpm.MPM_FP64)
        sim.step(steps)
        out = {"particles": w.n}
    elif what == "batched":
        wb = inputs.dam_break_2d(96)
        B = 256
        sim = mpm.Simulation(2, wb.n_cells, wb.dx, wb.dt, wb.gravity, wb.material, mpm.MPM_FP32, wb.sort_every,
                             batch=B)
        sim.load(np.tile(wb.x, (B, 1)), None, wb.particle_volume, np.repeat(np.arange(B, dtype=np.int32), wb.n))
        sim.set_friction(2, (32, 1), np.stack([inputs.friction_field(32, 1_000_000 + i) for i in range(B)]).reshape(-1))
        sim.step(steps)
        out = {"particles": B * wb.n}
    else:
        w3 = (inputs.granular_inverse_3d() if what == "adjoint" else
              inputs.granular_inverse_3d((96, 96, 48), 15, 30, steps=120, checkpoint_every=60))
        obs = [s for s in w3.extras["obs_steps"] if s <= 120]
        sim = mpm.Simulation.from_workload(w3, mpm.MPM_FP32)
        mpm.mpm_set_observations(sim.ctx, w3.extras["track_ids"], obs,
                                 np.zeros((len(obs), len(w3.extras["track_ids"]), 3)))
        loss, _ = mpm.mpm_step_adjoint(sim.ctx, 120, 60, 4, len(w3.extras["mu_true"]))
        out = {"particles": w3.n, "loss": loss}
    sim.synchronize()
    sim.close()
    print(json.dumps({"profile": what, "steps": steps, **out}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--headline-only", action="store_true", help="skip the adjoint, batched and network lines")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 line")
    ap.add_argument("--gemm-only", action="store_true", help="only the tensor-core GEMM line (profiling)")
    ap.add_argument("--mlp-only", action="store_true",
                    help="only the network's device-side training step at batch 256 (profiling)")
    ap.add_argument("--profile", choices=["forward", "fp64", "batched", "adjoint", "adjoint-small"],
                    help="a short untimed run of one workload for ncu (--steps sets its length)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        bench_reference(args)
    elif args.profile:
        profile_run(args.profile, args.steps)
    elif args.mlp_only:
        print(json.dumps({"mlp_device": mlp_device_measurement()}), flush=True)
    elif args.gemm_only:
        import torch
        stream = torch.cuda.Stream()
        print(json.dumps({"mlp_gemm": gemm_measurement(stream)}), flush=True)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
