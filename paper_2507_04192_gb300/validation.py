"""Physical validation: the shallow-water dam break of Sec. 5.1 against the
shallow-water surface of Eq. shallow.

Shallow-water theory places the water surface of height y at
x(y, t) = L0 + (2 sqrt(g H0) - 3 sqrt(g y)) t (the tip, y -> 0, moves at
2 sqrt(g H0)); the paper reports close agreement once the flow is shallow
(t >= 0.3 s), with finite-depth effects earlier.  The simulated x(y, t) is the
largest x among the particles above height y.
"""
from __future__ import annotations

import json

import numpy as np

from . import inputs, mpm


def surface_x(x: np.ndarray, heights) -> np.ndarray:
    """x position of the water surface at each height (the largest x among the particles above it)."""
    return np.array([float(x[x[:, 1] > y, 0].max()) if np.any(x[:, 1] > y) else np.nan for y in heights])


def shallow_water_x(heights, t, length=1.0, height=0.1, g=9.8):
    return length + (2.0 * np.sqrt(g * height) - 3.0 * np.sqrt(g * np.asarray(heights))) * t


def dam_break_surface(heights, times, dx: float = 0.004, precision=mpm.MPM_FP32):
    """Simulated x(y, t) (len(times) x len(heights)) of the shallow dam break."""
    w = inputs.shallow_dam_break_2d(dx=dx)
    sim = mpm.Simulation.from_workload(w, precision)
    out, steps = [], 0
    for t in times:
        n = int(round(t / w.dt)) - steps
        sim.step(n)
        steps += n
        out.append(surface_x(sim.get("x"), heights))
    sim.close()
    return np.array(out), w


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--dx", type=float, default=0.004)
    args = ap.parse_args(argv)
    heights = [0.002, 0.005, 0.01, 0.02, 0.03, 0.05]
    times = [0.1, 0.2, 0.3, 0.4, 0.5]
    xs, w = dam_break_surface(heights, times, args.dx)
    ref = np.array([shallow_water_x(heights, t) for t in times])
    print(json.dumps({"particles": int(w.x.shape[0]), "dx": args.dx, "heights": heights, "times": times,
                      "x": xs.tolist(), "shallow_water": ref.tolist()}))


if __name__ == "__main__":
    main()
