"""Basal-friction inversion on libmpm (the inverse problem of Sec. 5.3).

The parameter field is the friction coefficient of each floor segment
(Eq. coulomb_friction); the loss is Eq. inverse_loss of Sec. 3.2 with
Lagrangian observations (tracked particle positions).  Loss and gradient come
from the library's checkpointed adjoint (mpm_step_adjoint); torch serves as
the optimiser (Adam with a decaying learning rate from 0.1, the paper's
setting) and for the autograd wrapper.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

from . import mpm


class FrictionInversion:
    """One inversion problem: initial particles, observations, friction wall."""

    def __init__(self, workload, z_obs: np.ndarray, precision: int = mpm.MPM_FP32, checkpoint_every: int = 50,
                 wall: Optional[int] = None, n_seg: Optional[int] = None, stream: int = 0):
        w = workload
        self.w = w
        # the friction wall and its segment layout: from the workload's friction field
        # (floor segments in 2D, floor patches in 3D) unless given
        fw, shape = (w.friction[0][0], tuple(w.friction[0][1])) if w.friction else (2 * (w.dim - 1), None)
        self.wall = fw if wall is None else wall
        self.n_seg = int(n_seg if n_seg is not None else len(w.extras["mu_true"]))
        self.seg_shape = shape if shape is not None and shape[0] * shape[1] == self.n_seg else (self.n_seg, 1)
        self.steps = int(max(w.extras["obs_steps"]))
        self.K = int(checkpoint_every)
        self.sim = mpm.Simulation(w.dim, w.n_cells, w.dx, w.dt, w.gravity, w.material, precision, w.sort_every,
                                  stream=stream)
        self.sim.load(w.x, w.v, w.particle_volume)
        mpm.mpm_save_state(self.sim.ctx, 0)
        mpm.mpm_set_observations(self.sim.ctx, w.extras["track_ids"], w.extras["obs_steps"], z_obs)
        self.z_obs = np.asarray(z_obs, dtype=np.float64)
        self.evaluations = 0

    def loss_and_grad(self, mu: np.ndarray):
        mu = np.clip(np.asarray(mu, dtype=np.float64).reshape(-1), 0.0, None)
        mpm.mpm_restore_state(self.sim.ctx, 0)
        self.sim.set_friction(self.wall, self.seg_shape, mu)
        self.evaluations += 1
        return mpm.mpm_step_adjoint(self.sim.ctx, self.steps, self.K, self.wall, self.n_seg)

    def close(self):
        self.sim.close()


def _torch():
    import torch
    return torch


def friction_loss(mu, problem: FrictionInversion):
    """Loss of the friction field ``mu`` (a torch tensor) with the library's adjoint as its gradient."""
    torch = _torch()

    class FrictionLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, m):
            loss, grad = problem.loss_and_grad(m.detach().cpu().double().numpy())
            ctx.save_for_backward(torch.as_tensor(grad, dtype=m.dtype, device=m.device))
            return torch.tensor(loss, dtype=m.dtype, device=m.device)

        @staticmethod
        def backward(ctx, g):
            (grad,) = ctx.saved_tensors
            return g * grad

    return FrictionLoss.apply(mu)


def relative_error(mu, mu_true, mask=None) -> float:
    mu = np.asarray(mu, dtype=np.float64)
    mu_true = np.asarray(mu_true, dtype=np.float64)
    if mask is None:
        mask = np.ones_like(mu_true, dtype=bool)
    return float(np.linalg.norm((mu - mu_true)[mask]) / np.linalg.norm(mu_true[mask]))


@dataclass
class InversionResult:
    mu: np.ndarray
    iterations: int
    converged: bool
    history: List[dict] = field(default_factory=list)


def invert(problem: FrictionInversion, mu0, mu_true=None, mask=None, tol: float = 0.05, max_iters: int = 300,
           lr0=0.1, decay: float = 0.97, callback: Optional[Callable[[dict], None]] = None
           ) -> InversionResult:
    """Adam (beta 0.9 / 0.999, eps 1e-8) with lr = lr0 * decay^k, mu clamped to [0, 1].
    ``lr0`` is one rate, or one per segment (an array): Adam's update is taken
    element by element, so a per-segment rate scales each segment's steps.

    Stops when the relative L2 error of mu on ``mask`` (the segments the
    observations constrain) falls to ``tol``, or after ``max_iters`` updates.
    """
    torch = _torch()
    mu = torch.tensor(np.asarray(mu0, dtype=np.float64), requires_grad=True)
    per_segment = np.ndim(lr0) > 0
    if per_segment:
        lr_vec = torch.tensor(np.broadcast_to(np.asarray(lr0, dtype=np.float64), mu.shape).copy())
        b1, b2, eps = 0.9, 0.999, 1e-8
        m1 = torch.zeros_like(mu, requires_grad=False)
        m2 = torch.zeros_like(mu, requires_grad=False)
    else:
        opt = torch.optim.Adam([mu], lr=lr0, betas=(0.9, 0.999), eps=1e-8)
        sched = torch.optim.lr_scheduler.ExponentialLR(opt, gamma=decay)
    history = []
    for k in range(max_iters + 1):
        err = relative_error(mu.detach().numpy(), mu_true, mask) if mu_true is not None else None
        if err is not None and err <= tol:
            return InversionResult(mu.detach().numpy().copy(), k, True, history)
        if k == max_iters:
            break
        if mu.grad is not None:
            mu.grad = None
        loss = friction_loss(mu, problem)
        loss.backward()
        lr_now = float((lr_vec * decay ** k).max()) if per_segment else opt.param_groups[0]["lr"]
        rec = {"iter": k, "loss": float(loss.detach()), "error": err, "lr": lr_now}
        history.append(rec)
        if callback:
            callback(rec)
        if per_segment:                  # the update of torch.optim.Adam, with an elementwise rate
            with torch.no_grad():
                g = mu.grad
                m1.mul_(b1).add_(g, alpha=1.0 - b1)
                m2.mul_(b2).addcmul_(g, g, value=1.0 - b2)
                t = k + 1
                denom = (m2.sqrt() / np.sqrt(1.0 - b2 ** t)).add_(eps)
                mu.sub_(lr_vec * decay ** k / (1.0 - b1 ** t) * m1 / denom)
        else:
            opt.step()
            sched.step()
        with torch.no_grad():
            mu.clamp_(0.0, 1.0)
    return InversionResult(mu.detach().numpy().copy(), max_iters, False, history)


def sensitive_segments(problem: FrictionInversion, mu_true: np.ndarray, z_obs: np.ndarray, rel: float = 1e-2,
                       shift: float = 1e-3) -> np.ndarray:
    """Segments whose friction moves the tracked particles along the floor at the
    true field: with the observations shifted by ``shift`` (in units of dx) along
    the first axis the loss gradient at ``mu_true`` is -2 shift dx times the
    summed sensitivities of the tracks' first coordinates (the residuals vanish
    there), which is zero for segments without sliding contact."""
    w = problem.w
    z = np.array(z_obs, dtype=np.float64, copy=True)
    z[..., 0] += shift * w.dx
    mpm.mpm_set_observations(problem.sim.ctx, w.extras["track_ids"], w.extras["obs_steps"], z)
    try:
        _, g = problem.loss_and_grad(mu_true)
    finally:
        mpm.mpm_set_observations(problem.sim.ctx, w.extras["track_ids"], w.extras["obs_steps"], z_obs)
    return np.abs(g) > rel * np.abs(g).max()


def constrained_segments(problem: FrictionInversion, mu: np.ndarray, rel: float = 1e-2) -> np.ndarray:
    """Segments the observations constrain: loss gradient at ``mu`` at least ``rel``
    times its largest entry (segments the flow never reaches have zero gradient;
    barely touched ones have gradients orders of magnitude below the rest)."""
    _, g = problem.loss_and_grad(mu)
    return np.abs(g) > rel * np.abs(g).max()
