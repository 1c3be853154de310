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
dL/dalpha follows by the chain rule on the host; dL/dtheta by back-propagating
dL/dv0 through the network on the tensor cores (mpm_mlp_backward; the network
has 1,951 weights, as in the paper's Table 3, and is evaluated once per iteration on the particles' initial
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


class CoordinateNet:
    """v_x0 = N(y / H0): the coordinate network 1 -> 30 -> 30 -> 30 -> 1 with ReLU
    (Eq. nn_apprx, Sec. 5.2) on the library's tensor-core network (mpm_mlp_*).
    The tensor-core GEMMs take widths that are multiples of 8, so the network is
    held as 8 -> 32 -> 32 -> 32 -> 8 with the extra inputs, units and outputs
    zero: a unit whose weights in and out are zero stays zero under ReLU and gets
    zero gradients, so the padding never changes (the network is exactly the
    30-unit one).  Weights He-normal by seed, biases zero; forward and backward in
    BF16 operands with FP32 accumulation, Adam on FP32 master weights."""

    TRUE = (1, 30, 30, 30, 1)
    PADDED = (8, 32, 32, 32, 8)

    def __init__(self, max_batch: int, seed: int = 0, stream: int = 0):
        self.max_batch = (int(max_batch) + 7) // 8 * 8
        self.net = mpm.MLP(list(self.PADDED), self.max_batch, stream=stream, hidden=mpm.MPM_ACT_RELU,
                           output=mpm.MPM_OUT_LINEAR)
        rng = np.random.default_rng(seed)
        flat = []
        for i in range(len(self.TRUE) - 1):
            W = np.zeros((self.PADDED[i + 1], self.PADDED[i]))
            W[:self.TRUE[i + 1], :self.TRUE[i]] = rng.normal(0.0, np.sqrt(2.0 / self.TRUE[i]),
                                                             (self.TRUE[i + 1], self.TRUE[i]))
            flat += [W.ravel(), np.zeros(self.PADDED[i + 1])]
        self.net.set_params(np.concatenate(flat).astype(np.float32))

    def _inputs(self, s: np.ndarray) -> np.ndarray:
        x = np.zeros((self.max_batch, self.PADDED[0]), dtype=np.float32)
        x[:len(s), 0] = s
        return x

    def forward(self, s: np.ndarray) -> np.ndarray:
        return self.net.infer(self._inputs(s))[:len(s), 0].astype(np.float64)

    def step(self, s: np.ndarray, gout: np.ndarray, lr: float):
        """Back-propagate dL/dN(s) = gout and take one Adam step with rate lr (rows
        beyond len(s) are padding with zero gradient)."""
        dy = np.zeros((self.max_batch, self.PADDED[-1]), dtype=np.float32)
        dy[:len(s), 0] = gout
        self.net.backward(self._inputs(s), dy, lr=lr, update=True)

    def close(self):
        self.net.close()


def field_error(net: CoordinateNet, w) -> float:
    """Relative L2 error of N(y / H0) against the reference field over the column's particles."""
    H0 = w.extras["H0"]
    y = w.x[:, 1]
    pred = net.forward(y / H0)
    ref = inputs.velocity_profile_field(y, H0)
    return float(np.linalg.norm(pred - ref) / np.linalg.norm(ref))


def invert_field(problem: VelocityInversion, epochs: int = 400, lr0: float = 1e-2, decay: float = 0.995,
                 seed: int = 0) -> Result:
    """Adam (beta 0.9 / 0.999, eps 1e-8, lr0 decay^k) on the coordinate network's
    weights; each epoch one checkpointed adjoint of the whole horizon gives
    dL/dv0, the network back-propagates its x component."""
    w = problem.w
    H0 = w.extras["H0"]
    net = CoordinateNet(w.n, seed=seed)
    hist = []
    s = w.x[:, 1] / H0
    try:
        for k in range(epochs):
            v0 = np.zeros_like(w.x)
            v0[:, 0] = net.forward(s)
            loss, g0 = problem.loss_and_grad_v0(v0)
            hist.append({"epoch": k, "loss": loss, "error": field_error(net, w)})
            net.step(s, g0[:, 0], lr0 * decay ** k)
        hist.append({"epoch": epochs, "loss": None, "error": field_error(net, w)})
        params = net.net.get_params(0)
    finally:
        net.close()
    return Result(params, epochs, True, hist)


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
               "loss_last": res.history[-2]["loss"], "network": "tensor-core mpm_mlp (BF16 operands, FP32 accumulate)"}
    else:
        res = invert_alpha(prob, alpha_true=w.extras["alpha_true"], max_iters=args.iters)
        out = {"case": args.case, "particles": w.n, "iterations_to_1pct": res.iterations if res.converged else None,
               "alpha": float(res.params[0]), "alpha_true": w.extras["alpha_true"]}
    out["seconds"] = time.perf_counter() - t0
    prob.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
