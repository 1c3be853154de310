"""Deposit statistics of a granular column collapse run to rest.

Runout R_f: the 99.9th percentile of the particles' distance from the column
axis; deposit height H_f: the 99.9th percentile of their height.  The largest
distance is reported too: on a floor too narrow for the deposit, the side walls
and not the flow would bound the runout.  The FP32 run
is compared with the FP64 run of the same inputs (the oracle cannot run 1e5
steps of millions of particles; the FP64 GPU path is itself oracle-checked on
short runs).
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import inputs, mpm


def deposit_stats(x: np.ndarray, axis) -> tuple:
    r = np.hypot(x[:, 0] - axis[0], x[:, 1] - axis[1])
    return float(np.percentile(r, 99.9)), float(np.percentile(x[:, 2], 99.9))


def run(w, precision, steps: int, chunk: int = 5000):
    sim = mpm.Simulation.from_workload(w, precision)
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        k = min(chunk, steps - done)
        sim.step(k)
        done += k
    sim.synchronize()
    x = sim.get("x")
    sim.close()
    return x, time.perf_counter() - t0


def compare(w, steps: int):
    """FP32 vs FP64: (R_f, H_f) of each and their relative differences."""
    out = {"workload": w.name, "particles": int(w.x.shape[0]), "steps": steps, "t_end_s": steps * w.dt}
    r0, h0 = deposit_stats(w.x, w.extras["axis"])
    out["initial"] = {"R": r0, "H": h0}
    for prec, name in ((mpm.MPM_FP64, "fp64"), (mpm.MPM_FP32, "fp32")):
        x, secs = run(w, prec, steps)
        R, H = deposit_stats(x, w.extras["axis"])
        max_r = float(np.hypot(x[:, 0] - w.extras["axis"][0], x[:, 1] - w.extras["axis"][1]).max())
        out[name] = {"R_f": R, "H_f": H, "max_r": max_r, "seconds": secs, "finite": bool(np.isfinite(x).all())}
    out["rel_diff"] = {"R_f": abs(out["fp32"]["R_f"] - out["fp64"]["R_f"]) / out["fp64"]["R_f"],
                       "H_f": abs(out["fp32"]["H_f"] - out["fp64"]["H_f"]) / out["fp64"]["H_f"]}
    return out


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="FP32 vs FP64 deposit of the 3D granular collapse")
    ap.add_argument("--steps", type=int, default=100_000)
    ap.add_argument("--scale", type=int, default=1, help="1: 256x256x128 (2.76M particles); 4: 64x64x32")
    ap.add_argument("--wide", action="store_true",
                    help="a floor 1.5 m wide (384x384x128 at scale 1) so the deposit stays clear of the side walls")
    args = ap.parse_args(argv)
    s = args.scale
    nxy = (384 if args.wide else 256) // s
    w = inputs.granular_cylinder_3d((nxy, nxy, 128 // s), 38 / s, 76 / s, dt=1e-5 * s, dx=s / 256.0)
    print(json.dumps(compare(w, args.steps)))


if __name__ == "__main__":
    main()
