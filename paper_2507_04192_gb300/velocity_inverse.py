"""Initial-velocity inversion on libmpm (the inverse problems of Sec. 5.2).

Two parametrisations of the unknown initial horizontal velocity of a dam
break:

* a constant alpha in v_x0 = alpha (H0 - y) (Sec. 5.2, "initial velocity
  constant"), recovered from tracked particle positions (all particles, or a
  sparse subset) or from nine Eulerian velocity monitors;
* a field v_x0(y) = N_theta(y / H0) given by a coordinate network with three
  hidden layers of 30 ReLU units (Sec. 5.2, "initial velocity field"),
  recovered from sparse tracked positions.

The loss and dL/dv0 come from the library's checkpointed adjoint
(mpm_step_adjoint with no friction parameter, then mpm_get_initial_adjoint);
dL/dalpha and dL/dtheta follow by the chain rule on the host (the network has
2,911 weights and is evaluated once per iteration on the particles' initial
heights).  Adam (beta 0.9 / 0.999, eps 1e-8) with lr = lr0 * decay^k.

    python -m paper_2507_04192_gb300.velocity_inverse [--case tracked|sparse|monitors|field] [--dx 0.01]
"""
from __future__ import annotations

import argparse
import json
import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import inputs, mpm


class VelocityInversion:
    """One problem: particles, observations (tracked positions and/or monitors)."""

    def __init__(self, w, zx: Optional[np.ndarray] = None, zv: Optional[np.ndarray] = None,
                 precision: int = mpm.MPM_FP32, stream: int = 0):
        self.w = w
        self.steps = int(max(w.extras["obs_steps"]))
        self.K = int(w.extras.get("checkpoint_every", 100))
        self.sim = mpm.Simulation(w.dim, w.n_cells, w.dx, w.dt, w.gravity, w.material, precision, w.sort_every,
                                  stream=stream)
        self.sim.load(w.x, w.v, w.particle_volume)
        mpm.mpm_save_state(self.sim.ctx, 0)             # the initial state; each run replaces its velocity
        if zx is not None:
            mpm.mpm_set_observations(self.sim.ctx, w.extras["track_ids"], w.extras["obs_steps"], zx)
        if zv is not None:
            mpm.mpm_set_velocity_monitors(self.sim.ctx, w.extras["monitors"], w.extras["obs_steps"], zv)
        self.evaluations = 0

    def loss_and_grad_v0(self, v0: np.ndarray):
        """Loss and dL/dv0 (n x dim, load order) of the run from initial velocities v0."""
        mpm.mpm_restore_state(self.sim.ctx, 0)
        self.sim.set_field("v", v0)
        self.evaluations += 1
        loss, _ = mpm.mpm_step_adjoint(self.sim.ctx, self.steps, self.K, -1, 0)
        return loss, mpm.mpm_get_initial_adjoint(self.sim.ctx, "v")

    def close(self):
        self.sim.close()


def record_observations(w, v0: np.ndarray, precision: int = mpm.MPM_FP32, stream: int = 0):
    """Tracked positions (n_obs x n_track x dim) and monitor means (n_obs x 9 x dim)
    of the run from v0, simulated by the library."""
    sim = mpm.Simulation(w.dim, w.n_cells, w.dx, w.dt, w.gravity, w.material, precision, w.sort_every,
                         stream=stream)
    sim.load(w.x, v0, w.particle_volume)
    ids = w.extras["track_ids"]
    zx, zv = [], []
    t = 0
    for s in w.extras["obs_steps"]:
        sim.step(s - t)
        t = s
        zx.append(sim.get("x")[ids].copy())
        zv.append(mpm.mpm_monitor_means(sim.ctx, w.extras["monitors"])[0])
    sim.close()
    return np.stack(zx), np.stack(zv)


class Adam:
    """Adam on a flat parameter vector with lr = lr0 * decay^k."""

    def __init__(self, n: int, lr0: float = 0.1, decay: float = 0.97, b1: float = 0.9, b2: float = 0.999,
                 eps: float = 1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.k = 0
        self.lr0, self.decay, self.b1, self.b2, self.eps = lr0, decay, b1, b2, eps

    def step(self, p: np.ndarray, g: np.ndarray) -> np.ndarray:
        self.k += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.k)
        vh = self.v / (1 - self.b2 ** self.k)
        lr = self.lr0 * self.decay ** (self.k - 1)
        return p - lr * mh / (np.sqrt(vh) + self.eps)


@dataclass
class Result:
    params: np.ndarray
    iterations: int
    converged: bool
    history: List[dict] = field(default_factory=list)


def invert_alpha(problem: VelocityInversion, alpha0: float = 0.1, alpha_true: Optional[float] = None,
                 tol: float = 0.01, max_iters: int = 100, lr0: float = 0.1, decay: float = 0.97) -> Result:
    """Recover alpha of v_x0 = alpha (H0 - y); stops at |alpha - alpha_true| <= tol alpha_true."""
    w = problem.w
    H0 = w.extras["H0"]
    dv = H0 - w.x[:, 1]                              # d v_x0 / d alpha per particle
    a = np.array([alpha0], dtype=np.float64)
    opt = Adam(1, lr0, decay)
    hist = []
    for k in range(max_iters + 1):
        err = abs(a[0] - alpha_true) / abs(alpha_true) if alpha_true is not None else None
        if err is not None and err <= tol:
            return Result(a.copy(), k, True, hist)
        if k == max_iters:
            break
        loss, g0 = problem.loss_and_grad_v0(inputs.velocity_profile_linear(w.x, a[0], H0))
        g = np.array([float((g0[:, 0] * dv).sum())])
        hist.append({"iter": k, "alpha": float(a[0]), "loss": loss, "grad": float(g[0]), "error": err})
        a = opt.step(a, g)
    return Result(a.copy(), max_iters, False, hist)


class CoordinateMLP:
    """v_x0 = N(y / H0): 1 -> 30 -> 30 -> 30 -> 1 with ReLU, weights He-normal by seed."""

    def __init__(self, widths=(1, 30, 30, 30, 1), seed: int = 0):
        rng = np.random.default_rng(seed)
        self.W = [rng.normal(0.0, np.sqrt(2.0 / widths[i]), (widths[i + 1], widths[i]))
                  for i in range(len(widths) - 1)]
        self.b = [np.zeros(widths[i + 1]) for i in range(len(widths) - 1)]

    @property
    def n_params(self) -> int:
        return sum(W.size + b.size for W, b in zip(self.W, self.b))

    def flat(self) -> np.ndarray:
        return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in zip(self.W, self.b)])

    def set_flat(self, p: np.ndarray):
        o = 0
        for i, (W, b) in enumerate(zip(self.W, self.b)):
            self.W[i] = p[o:o + W.size].reshape(W.shape)
            o += W.size
            self.b[i] = p[o:o + b.size].copy()
            o += b.size

    def forward(self, s: np.ndarray):
        h = [s.reshape(-1, 1)]
        for i, (W, b) in enumerate(zip(self.W, self.b)):
            z = h[-1] @ W.T + b
            h.append(np.maximum(z, 0.0) if i < len(self.W) - 1 else z)
        return h[-1][:, 0], h

    def backward(self, h, gout: np.ndarray) -> np.ndarray:
        """Gradient of sum(gout * N(s)) with respect to the flat parameters."""
        g = gout.reshape(-1, 1)
        grads = []
        for i in range(len(self.W) - 1, -1, -1):
            gW = g.T @ h[i]
            gb = g.sum(axis=0)
            grads.append((gW, gb))
            if i > 0:
                g = (g @ self.W[i]) * (h[i] > 0.0)
        grads.reverse()
        return np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])


def field_error(net: CoordinateMLP, w) -> float:
    """Relative L2 error of N(y / H0) against the reference field over the column's particles."""
    H0 = w.extras["H0"]
    y = w.x[:, 1]
    pred = net.forward(y / H0)[0]
    ref = inputs.velocity_profile_field(y, H0)
    return float(np.linalg.norm(pred - ref) / np.linalg.norm(ref))


def invert_field(problem: VelocityInversion, epochs: int = 400, lr0: float = 1e-2, decay: float = 0.995,
                 seed: int = 0) -> Result:
    w = problem.w
    H0 = w.extras["H0"]
    net = CoordinateMLP(seed=seed)
    opt = Adam(net.n_params, lr0, decay)
    hist = []
    s = w.x[:, 1] / H0
    for k in range(epochs):
        vx, h = net.forward(s)
        v0 = np.zeros_like(w.x)
        v0[:, 0] = vx
        loss, g0 = problem.loss_and_grad_v0(v0)
        g = net.backward(h, g0[:, 0])
        hist.append({"epoch": k, "loss": loss, "error": field_error(net, w)})
        net.set_flat(opt.step(net.flat(), g))
    return Result(net.flat(), epochs, True, hist)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--case", default="monitors", choices=["tracked", "sparse", "monitors", "field"])
    ap.add_argument("--dx", type=float, default=0.01)
    ap.add_argument("--n-track", type=int, default=100, help="tracked particles (case sparse / field)")
    ap.add_argument("--iters", type=int, default=100)
    ap.add_argument("--epochs", type=int, default=400)
    args = ap.parse_args(argv)
    n_track = 0 if args.case == "tracked" else args.n_track
    w = inputs.dam_break_velocity_inverse(dx=args.dx, n_track=n_track)
    H0 = w.extras["H0"]
    if args.case == "field":
        v_true = np.zeros_like(w.x)
        v_true[:, 0] = inputs.velocity_profile_field(w.x[:, 1], H0)
    else:
        v_true = inputs.velocity_profile_linear(w.x, w.extras["alpha_true"], H0)
    t0 = time.perf_counter()
    zx, zv = record_observations(w, v_true)
    prob = VelocityInversion(w, zx=None if args.case == "monitors" else zx, zv=zv if args.case == "monitors" else None)
    if args.case == "field":
        res = invert_field(prob, args.epochs)
        out = {"case": args.case, "particles": w.n, "n_track": len(w.extras["track_ids"]), "epochs": res.iterations,
               "field_error": res.history[-1]["error"], "loss_first": res.history[0]["loss"],
               "loss_last": res.history[-1]["loss"]}
    else:
        res = invert_alpha(prob, alpha_true=w.extras["alpha_true"], max_iters=args.iters)
        out = {"case": args.case, "particles": w.n, "iterations_to_1pct": res.iterations if res.converged else None,
               "alpha": float(res.params[0]), "alpha_true": w.extras["alpha_true"]}
    out["seconds"] = time.perf_counter() - t0
    prob.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
