"""Learned warm start of the basal-friction inversion.

The solver's own batched forward runs (many independent dam breaks sharing one
grid shape, each with its own random 32-segment friction field) give pairs
(observations, friction field); a small network on the tensor cores
(mpm_mlp_*) learns the map from the tracked particles' horizontal
displacements to the field, and its prediction replaces the uniform first
guess of the adjoint inversion (Sec. 5.3).  The paper parameterises a field
with a coordinate network (Eq. nn_apprx, Sec. 3.2); this one is an amortised
observations-to-parameters map of the same kind of component.

Features: one scalar per (observation time, track), (x_t - x_0) / scale along
the floor, time-major; targets: the per-segment friction coefficients.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from . import inputs, mpm

MU_LO, MU_HI = 0.1, 0.6
UNIFORM_GUESS = 0.35
TRAIN_SEED_BASE = 1_000_000          # friction seeds of training runs; held-out problems use small seeds


@dataclass
class Setup:
    """Geometry, tracks and horizon shared by every run of one training set."""
    n_cells: int = 96
    n_seg: int = 32
    n_track: int = 64
    n_obs: int = 10
    steps: int = 300
    checkpoint_every: int = 50
    geometry_seed: int = 0

    def workload(self, mu_seed: Optional[int] = None):
        w = inputs.dam_break_inverse_2d(self.n_cells, n_seg=self.n_seg, n_track=self.n_track, n_obs=self.n_obs,
                                        steps=self.steps, seed=self.geometry_seed,
                                        checkpoint_every=self.checkpoint_every)
        if mu_seed is not None:
            mu = inputs.friction_field(self.n_seg, mu_seed, MU_LO, MU_HI)
            w.extras["mu_true"] = mu
            w.friction = [(2, (self.n_seg, 1), mu)]
        return w

    feature_axes = (0,)                      # displacement along the floor

    @property
    def n_features(self):
        return self.n_obs * self.n_track * len(self.feature_axes)

    def scale(self, w):
        return float(w.extras["body_hi"][0] - w.extras["body_lo"][0])


@dataclass
class Setup3D:
    """The 3D granular counterpart: a Drucker-Prager cylinder on a floor whose
    friction is piecewise constant over patches x patches (Sec. 5.3 carried to
    3D); features are the tracks' displacements along both floor axes."""
    n_cells: tuple = (64, 64, 32)
    dx: float = 1.0 / 64.0
    radius_cells: float = 10.0
    height_cells: float = 20.0
    patches: int = 4
    n_track: int = 64
    n_obs: int = 10
    steps: int = 1500
    dt: float = 4.0e-5
    checkpoint_every: int = 100
    geometry_seed: int = 0
    feature_axes = (0, 1)

    @property
    def n_seg(self):
        return self.patches * self.patches

    def workload(self, mu_seed: Optional[int] = None):
        w = inputs.granular_inverse_3d(tuple(self.n_cells), self.radius_cells, self.height_cells,
                                       patches=(self.patches, self.patches), n_track=self.n_track, n_obs=self.n_obs,
                                       steps=self.steps, seed=self.geometry_seed,
                                       checkpoint_every=self.checkpoint_every, dt=self.dt, dx=self.dx)
        if mu_seed is not None:
            mu = inputs.friction_field(self.n_seg, mu_seed, MU_LO, MU_HI)
            w.extras["mu_true"] = mu
            w.friction = [(4, (self.patches, self.patches), mu)]
        return w

    @property
    def n_features(self):
        return self.n_obs * self.n_track * len(self.feature_axes)

    def scale(self, w):
        return float(w.extras["body_hi"][0] - w.extras["body_lo"][0])


def setup_3d_full() -> Setup3D:
    """The inverse problem at scale: the 1.36M-particle collapse (radius 30 dx,
    height 60 dx, 192 x 192 x 96 cells, dx = 1/256 m), floor friction over 16 x 16
    patches, 128 tracks observed 10 times over a 600-step horizon (checkpoint 60).
    The time step is 2.5e-5 s (15 ms of flow; a Courant number of 0.17 for the
    P-wave speed of this sand), so that the base of the column has begun to slide
    by the last observation."""
    return Setup3D(n_cells=(192, 192, 96), dx=1.0 / 256.0, radius_cells=30.0, height_cells=60.0, patches=16,
                   n_track=128, n_obs=10, steps=600, dt=2.5e-5, checkpoint_every=60)


def observe_batch(w, mus: np.ndarray, precision=mpm.MPM_FP32, stream: int = 0) -> np.ndarray:
    """Tracked positions (B, n_obs, n_track, dim) of B independent runs of workload
    ``w`` that differ only in their floor friction ``mus`` (B, n_seg); one batched
    context steps them together."""
    mus = np.atleast_2d(np.asarray(mus, dtype=np.float64))
    B, n_seg = mus.shape
    n = w.x.shape[0]
    wall, shape = (w.friction[0][0], tuple(w.friction[0][1])) if w.friction else (2 * (w.dim - 1), (n_seg, 1))
    sim = mpm.Simulation(w.dim, w.n_cells, w.dx, w.dt, w.gravity, w.material, precision, w.sort_every, batch=B,
                         stream=stream)
    try:
        sim.load(np.tile(w.x, (B, 1)), None, w.particle_volume, np.repeat(np.arange(B, dtype=np.int32), n))
        sim.set_friction(wall, shape, mus.reshape(-1))
        ids = (np.arange(B)[:, None] * n + np.asarray(w.extras["track_ids"])[None, :])
        out, t = [], 0
        for s in w.extras["obs_steps"]:
            sim.step(s - t)
            t = s
            out.append(sim.get("x")[ids])
        return np.stack(out, axis=1)
    finally:
        sim.close()


def features(setup: Setup, w, z_obs: np.ndarray) -> np.ndarray:
    """Network input from observations z_obs (n_obs, n_track, dim) or a batch of them."""
    z = np.asarray(z_obs, dtype=np.float64)
    x0 = w.x[np.asarray(w.extras["track_ids"])]
    ax = list(setup.feature_axes)
    d = (z[..., ax] - x0[:, ax]) / setup.scale(w)            # (..., n_obs, n_track, n_axes)
    return d.reshape(d.shape[:-3] + (-1,)).astype(np.float32)


def generate(setup: Setup, n_runs: int, batch: int = 256, first_seed: int = TRAIN_SEED_BASE,
             precision=mpm.MPM_FP32):
    """n_runs (features, friction field) pairs from batched forward runs."""
    w = setup.workload()
    X, Y = [], []
    for b0 in range(0, n_runs, batch):
        B = min(batch, n_runs - b0)
        mus = np.stack([inputs.friction_field(setup.n_seg, first_seed + b0 + i, MU_LO, MU_HI) for i in range(B)])
        X.append(features(setup, w, observe_batch(w, mus, precision)))
        Y.append(mus.astype(np.float32))
    return np.concatenate(X), np.concatenate(Y)


class WarmStartNet:
    """n_features -> hidden -> hidden -> n_seg network, output in [MU_LO, MU_HI]."""

    def __init__(self, n_in: int, n_out: int, hidden=(256, 256), max_batch: int = 256, seed: int = 0):
        self.widths = [n_in, *hidden, n_out]
        self.max_batch = max_batch
        self.net = mpm.MLP(self.widths, max_batch, MU_LO, MU_HI)
        rng = np.random.default_rng(seed)
        p = []
        for l in range(len(self.widths) - 1):
            fan_in = self.widths[l]
            p.append(rng.standard_normal(self.widths[l + 1] * fan_in) * np.sqrt(2.0 / fan_in))
            p.append(np.zeros(self.widths[l + 1]))
        self.net.set_params(np.concatenate(p).astype(np.float32))
        self.x_mean = np.zeros(n_in)
        self.x_scale = np.ones(n_in)
        self.val_rmse, self.val_rmse_seg = None, None

    def _standardise(self, X):
        return ((np.asarray(X, dtype=np.float64) - self.x_mean) / self.x_scale).astype(np.float32)

    def fit(self, X, Y, epochs: int = 40, lr: float = 1e-3, seed: int = 0) -> List[float]:
        """Adam on the mean squared error over shuffled mini-batches of max_batch.
        Inputs are standardised per feature with the training set's mean and
        spread (the displacements friction changes differ by orders of magnitude
        between tracks near the front and inside the column)."""
        X = np.asarray(X, dtype=np.float64)
        Y = np.asarray(Y, dtype=np.float32)
        # the last 1/16 of the runs (at least one batch) is held back to measure the
        # network's error: the spread a warm start carries, which sets the step of
        # the adjoint refinement that follows it (see refine_rate)
        n_val = max(self.max_batch, len(X) // 16) if len(X) >= 2 * self.max_batch else 0
        Xv, Yv = X[len(X) - n_val:], Y[len(Y) - n_val:]
        X, Y = X[:len(X) - n_val], Y[:len(Y) - n_val]
        self.x_mean = X.mean(axis=0)
        sd = X.std(axis=0)
        self.x_scale = np.where(sd > 1e-9, sd, 1.0)          # tracks friction never reaches stay ~0
        Xs = self._standardise(X)
        rng = np.random.default_rng(seed)
        B = self.max_batch
        n = (len(X) // B) * B
        hist = []
        for _ in range(epochs):
            order = rng.permutation(len(X))[:n]
            losses = [self.net.train_step(Xs[order[i:i + B]], Y[order[i:i + B]], lr) for i in range(0, n, B)]
            hist.append(float(np.mean(losses)))
        if n_val:
            err = self.predict(Xv) - Yv
            self.val_rmse = float(np.sqrt(np.mean(err ** 2)))
            self.val_rmse_seg = np.sqrt(np.mean(err ** 2, axis=0))
        else:
            self.val_rmse, self.val_rmse_seg = None, None
        return hist

    def refine_rate(self, default: float = 0.1):
        """First Adam step of the adjoint refinement that starts from this network's
        prediction, per segment: Adam moves every coefficient by about its rate in
        the first steps, so each segment's rate is the network's held-out RMS error
        on that segment (at most the uniform guess's 0.1, at least 2e-3).  Segments
        the observations pin down are predicted well and refined with small steps;
        segments they do not reach keep the large step (a single rate for all would
        either throw a good warm start away or freeze the rest)."""
        if self.val_rmse_seg is None:
            return default
        return np.clip(self.val_rmse_seg, 2e-3, default)

    def predict(self, X) -> np.ndarray:
        X = self._standardise(np.atleast_2d(X))
        out = [self.net.infer(X[i:i + self.max_batch]) for i in range(0, len(X), self.max_batch)]
        return np.concatenate(out).astype(np.float64)

    def close(self):
        self.net.close()


def held_out_problem(setup: Setup, mu_seed: int, precision=mpm.MPM_FP32):
    """Workload and observations of one inversion problem (friction from ``mu_seed``)."""
    w = setup.workload(mu_seed)
    z = observe_batch(w, w.extras["mu_true"][None, :], precision)[0]
    return w, z


def compare(setup: Setup, net: WarmStartNet, mu_seeds, tol: float = 0.05, max_iters: int = 300,
            precision=mpm.MPM_FP32, mask_rel: float = 1e-2):
    """Adjoint inversion from the uniform guess and from the network's prediction,
    per held-out problem: first-guess error and iterations to ``tol`` relative L2
    error over the segments the observations constrain (gradient test at the
    true field, see inverse.sensitive_segments)."""
    from . import inverse
    rows = []
    for s in mu_seeds:
        w, z = held_out_problem(setup, s, precision)
        mu_true = w.extras["mu_true"]
        prob = inverse.FrictionInversion(w, z, precision, checkpoint_every=setup.checkpoint_every)
        try:
            mask = inverse.sensitive_segments(prob, mu_true, z, mask_rel)
            mu_warm = np.clip(net.predict(features(setup, w, z)[None, :])[0], 0.0, 1.0)
            mu_unif = np.full(setup.n_seg, UNIFORM_GUESS)
            res_u = inverse.invert(prob, mu_unif, mu_true, mask, tol, max_iters)
            res_w = inverse.invert(prob, mu_warm, mu_true, mask, tol, max_iters, lr0=net.refine_rate())
        finally:
            prob.close()
        rows.append(dict(seed=int(s), constrained=int(mask.sum()),
                         err0_uniform=inverse.relative_error(mu_unif, mu_true, mask),
                         err0_warm=inverse.relative_error(mu_warm, mu_true, mask),
                         iters_uniform=res_u.iterations, converged_uniform=res_u.converged,
                         iters_warm=res_w.iterations, converged_warm=res_w.converged,
                         err_uniform=inverse.relative_error(res_u.mu, mu_true, mask),
                         err_warm=inverse.relative_error(res_w.mu, mu_true, mask),
                         full_err_uniform=inverse.relative_error(res_u.mu, mu_true),
                         full_err_warm=inverse.relative_error(res_w.mu, mu_true)))
    return rows


def main(argv=None):
    """Warm start vs uniform guess on held-out problems; prints one JSON line."""
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--runs", type=int, default=8192)
    ap.add_argument("--held-out", type=int, default=16)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--max-iters", type=int, default=300)
    ap.add_argument("--setup", choices=["2d", "3d", "3d-full"], default="2d",
                    help="2d: 96^2 dam breaks, 32 floor segments; 3d: 64x64x32 granular collapses, 4x4 floor "
                         "patches; 3d-full: the 1.36M-particle collapse, 16x16 floor patches")
    ap.add_argument("--batch", type=int, default=256)
    args = ap.parse_args(argv)
    setup = {"2d": Setup, "3d": Setup3D, "3d-full": setup_3d_full}[args.setup]()
    t0 = time.perf_counter()
    X, Y = generate(setup, args.runs, batch=args.batch)
    t1 = time.perf_counter()
    net = WarmStartNet(setup.n_features, setup.n_seg)
    hist = net.fit(X, Y, epochs=args.epochs)
    t2 = time.perf_counter()
    rows = compare(setup, net, range(1, args.held_out + 1), max_iters=args.max_iters)
    summary = {
        "setup": {k: v for k, v in setup.__dict__.items()}, "runs": args.runs, "generate_s": t1 - t0, "train_s": t2 - t1,
        "train_loss": [hist[0], hist[-1]], "val_rmse": net.val_rmse,
        "warm_refine_lr0": {"min": float(np.min(net.refine_rate())), "median": float(np.median(net.refine_rate())),
                            "max": float(np.max(net.refine_rate()))},
        "uniform": {"converged": sum(r["converged_uniform"] for r in rows),
                    "median_iters": float(np.median([r["iters_uniform"] for r in rows])),
                    "mean_err0": float(np.mean([r["err0_uniform"] for r in rows]))},
        "warm": {"converged": sum(r["converged_warm"] for r in rows),
                 "median_iters": float(np.median([r["iters_warm"] for r in rows])),
                 "mean_err0": float(np.mean([r["err0_warm"] for r in rows]))},
        "rows": rows,
    }
    net.close()
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
