"""Per-step differentiable simulation for torch.autograd.

``Stepper.step(state, mu)`` advances the context by one explicit step (Sec. 2)
and returns the new particle state as a tensor; torch's backward pass calls
``mpm_step_adjoint_1`` once per step, the vector-Jacobian product of one step
(Eq. dzda for a single step, Sec. 3.1), so that any loss written in torch on
the states of a trajectory, and on the friction field of one wall (Eq.
coulomb_friction), is differentiated through the library's adjoint.  This is
the per-step counterpart of ``inverse.friction_loss``, whose backward is the
whole checkpointed sweep (Sec. 3.3.2).

A state tensor is (n, mpm_adjoint_width) doubles on the host in load order:
x (dim), v (dim), C (dim^2, row-major), rho (1) and, for Drucker-Prager, sigma
(6: xx yy zz xy xz yz), the adjoint layout of ``mpm_step_adjoint_1``.  The
context holds the state a tensor describes; the tensor is a copy for the loss,
and gradients flow to it, not from it: a state is advanced only from the
tensor the last step (or ``reset``) returned.  Each step keeps the state it
started from on the host (``mpm_export_state``) for its backward.
"""
from __future__ import annotations

import numpy as np

from . import mpm


def _torch():
    import torch
    return torch


class Stepper:
    """One context, the wall whose friction field ``step`` takes, its segment layout."""

    def __init__(self, sim: mpm.Simulation, wall: int = -1, seg_shape=(1, 1)):
        self.sim = sim
        self.wall = int(wall)
        self.seg_shape = tuple(int(s) for s in seg_shape)
        self.n_seg = self.seg_shape[0] * self.seg_shape[1] if self.wall >= 0 else 0
        self.width = mpm.mpm_adjoint_width(sim.ctx)
        self._start = mpm.mpm_export_state(sim.ctx)
        self._tag = None

    # -- the context's state as a tensor ------------------------------------------
    def _gather(self):
        torch = _torch()
        s, d = self.sim, self.sim.dim
        cols = [s.get("x").reshape(-1, d), s.get("v").reshape(-1, d), s.get("C").reshape(-1, d * d),
                s.get("rho").reshape(-1, 1)]
        if self.width > 2 * d + d * d + 1:             # Drucker-Prager: sigma as xx yy zz xy xz yz
            sg = s.get("sigma")
            cols.append(np.stack([sg[:, 0, 0], sg[:, 1, 1], sg[:, 2, 2], sg[:, 0, 1], sg[:, 0, 2], sg[:, 1, 2]], 1))
        out = torch.from_numpy(np.ascontiguousarray(np.concatenate(cols, 1), dtype=np.float64))
        assert out.shape[1] == self.width
        return out

    def _mark(self, t):
        """Mark t as the tensor of the context's current state."""
        self._tag = object()
        t._mpm_tag = self._tag
        return t

    def reset(self):
        """Back to the state the context held when the stepper was made; returns it."""
        mpm.mpm_import_state(self.sim.ctx, self._start)
        return self._mark(self._gather())

    def state(self):
        """The context's current state (a new tensor, outside any graph)."""
        return self._mark(self._gather())

    def step(self, state, mu=None):
        """S^{t+1} from S^t = ``state`` (the tensor the last step or ``reset``
        returned) under the friction field ``mu`` (a tensor of the wall's
        n_seg values; None: the context's field, and no gradient for it)."""
        torch = _torch()
        if getattr(state, "_mpm_tag", None) is not self._tag:
            raise RuntimeError("Stepper.step: the context is not at this state (advance the last state returned)")
        if self.wall >= 0 and mu is not None:
            m = mu
        else:
            m = torch.zeros(0, dtype=torch.float64)
        return self._mark(_Step.apply(state, m, self))


def _make_step():
    torch = _torch()

    class Step(torch.autograd.Function):
        @staticmethod
        def forward(ctx, state, mu, st: Stepper):
            ctx.st = st
            ctx.blob = mpm.mpm_export_state(st.sim.ctx)          # S^t, for the backward pass
            ctx.mu = None
            if mu.numel() > 0:
                ctx.mu = mu.detach().cpu().double().numpy().reshape(-1).copy()
                st.sim.set_friction(st.wall, st.seg_shape, ctx.mu)
            ctx.mu_shape, ctx.mu_dtype = mu.shape, mu.dtype
            st.sim.step(1)
            return st._gather()

        @staticmethod
        def backward(ctx, g):
            st = ctx.st
            mpm.mpm_import_state(st.sim.ctx, ctx.blob)
            if ctx.mu is not None:
                st.sim.set_friction(st.wall, st.seg_shape, ctx.mu)
            lam_next = np.ascontiguousarray(g.detach().cpu().double().numpy())
            lam_prev, gmu = mpm.mpm_step_adjoint_1(st.sim.ctx, st.wall if ctx.mu is not None else -1, lam_next,
                                                  st.n_seg)
            st._tag = None                                       # the context moved: no forward from here
            gm = None
            if ctx.mu is not None and ctx.needs_input_grad[1]:
                gm = torch.from_numpy(gmu).to(ctx.mu_dtype).reshape(ctx.mu_shape)
            return torch.from_numpy(lam_prev).to(g.dtype), gm, None

    return Step


class _LazyStep:
    """The autograd Function, built on first use (torch is imported lazily)."""
    _fn = None

    @classmethod
    def apply(cls, *args):
        if cls._fn is None:
            cls._fn = _make_step()
        return cls._fn.apply(*args)


_Step = _LazyStep
