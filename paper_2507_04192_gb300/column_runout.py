"""Influence of the aspect ratio on the runout of a 3D granular column (Sec.
4.2.2): columns of aspect ratio a = H0 / L0 = 0.5, 1, 2 and 3 collapse for 2 s
(200,000 steps of 1e-5 s); the normalised runout is d_n = (L_f - L0) / L0,
with L_f the final front position (the 99.9th percentile of the particles' x).
The paper prints d_n = 2.05, 3.97, 7.76 and 10.65 and a trend from linear to
sublinear in a.  The column geometry per aspect ratio is not given in the
paper; the reading here is a fixed base length L0 = 0.05 m on the
400 x 32 x 200 grid of its timing table (see inputs.granular_column_3d).

    python -m paper_2507_04192_gb300.column_runout [--steps N] [--precision fp32|fp64]
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import inputs, mpm

ASPECTS = (0.5, 1.0, 2.0, 3.0)
PAPER_DN = {0.5: 2.05, 1.0: 3.97, 2.0: 7.76, 3.0: 10.65}


def front(x: np.ndarray) -> float:
    """Runout front: the 99.9th percentile of the particles' x."""
    return float(np.percentile(x[:, 0], 99.9))


def runout(aspect: float, steps: int = 200_000, precision=mpm.MPM_FP32, chunk: int = 20_000, **kw) -> dict:
    w = inputs.granular_column_3d(aspect, steps=steps, **kw)
    sim = mpm.Simulation.from_workload(w, precision)
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        k = min(chunk, steps - done)
        sim.step(k)
        done += k
    x = sim.get("x")
    v = sim.get("v")
    sim.close()
    secs = time.perf_counter() - t0
    L0 = w.extras["L0"]
    Lf = front(x)
    return {"aspect": aspect, "particles": w.n, "L0": L0, "H0": w.extras["H0"], "steps": steps, "L_f": Lf,
            "d_n": (Lf - L0) / L0, "H_f": float(np.percentile(x[:, 2], 99.9)),
            "max_speed_end": float(np.linalg.norm(v, axis=1).max()), "seconds": secs,
            "finite": bool(np.isfinite(x).all()), "paper_d_n": PAPER_DN.get(aspect)}


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="normalised runout of 3D granular columns against the aspect ratio")
    ap.add_argument("--steps", type=int, default=200_000)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    args = ap.parse_args(argv)
    prec = mpm.MPM_FP32 if args.precision == "fp32" else mpm.MPM_FP64
    for a in ASPECTS:
        print(json.dumps(runout(a, args.steps, prec)), flush=True)


if __name__ == "__main__":
    main()
