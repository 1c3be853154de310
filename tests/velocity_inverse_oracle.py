"""Oracle loss and initial-state adjoint for the initial-velocity inverse
problems of Sec. 5.2 (tracked particle positions and velocity monitors), by the
reverse recursion of Eq. dzda over the oracle's one-step adjoint.  Test helper:
imports only the oracle."""
import numpy as np

import oracle


def small_problem(inputs, steps=240, frames=6, frame_every=10, n_track=24, dx=0.05):
    """The Sec. 5.2 dam break at a coarse resolution and a short horizon."""
    return inputs.dam_break_velocity_inverse(dx=dx, steps=steps, n_frames=frames, frame_every=frame_every,
                                             n_track=n_track, checkpoint_every=50)


def make_oracle(w):
    return oracle.Oracle(w.dim, w.n_cells, w.dx, w.dt, w.gravity, w.material, w.particle_volume)


def observe(w, v0, tracked=True, monitors=True):
    """Observations of the run from initial velocities v0: positions of the tracked
    particles and monitor means at every observation step."""
    orc = make_oracle(w)
    st = orc.initial_state(w.x, v0)
    ids = w.extras["track_ids"]
    zx, zv = [], []
    t = 0
    for s in w.extras["obs_steps"]:
        orc.step(st, s - t)
        t = s
        zx.append(st.x[ids].copy())
        zv.append(oracle.monitor_means(st.x, st.v, w.extras["monitors"])[0])
    return np.stack(zx), np.stack(zv)


def loss_and_v0_adjoint(w, v0, zx=None, zv=None):
    """Loss (tracked positions when zx is given, monitors when zv is given) and
    dL/dv0 (n x dim)."""
    orc = make_oracle(w)
    ids = w.extras["track_ids"]
    boxes = w.extras["monitors"]
    obs = {s: k for k, s in enumerate(w.extras["obs_steps"])}
    steps = max(obs)
    states = [orc.initial_state(w.x, v0)]
    for t in range(1, steps + 1):
        s = states[-1].copy()
        orc.step(s, 1)
        states.append(s)
    n, d = w.n, w.dim
    lam = [np.zeros((n, d)), np.zeros((n, d)), np.zeros((n, d, d)), np.zeros(n)]
    loss = 0.0
    for t in range(steps, -1, -1):
        if t in obs:
            st = states[t]
            if zx is not None:
                e = st.x[ids] - zx[obs[t]]
                loss += float((e * e).sum())
                lam[0][ids] += 2.0 * e
            if zv is not None:
                lm, g = oracle.monitor_loss_and_seed(st.x, st.v, boxes, zv[obs[t]])
                loss += lm
                lam[1] += g
        if t > 0:
            lam, _ = orc.step_vjp(states[t - 1], *lam)
    return loss, lam[1]
