"""Host logic of the per-step autograd Function (autograd.Stepper) on a fake
context: a linear step S' = S M^T + N mu whose vector-Jacobian product stands
in for mpm_step_adjoint_1.  Checks the state tensor's columns, the routing of
the adjoint through a chain of steps (loss terms at two times, the friction
field used at every step) against torch's own autograd of the same linear
map, and the refusal to advance a state the context no longer holds."""
import pickle

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_04192_gb300 import autograd, mpm

N_P, D, W, N_SEG = 6, 2, 9, 3          # particles, dim, adjoint width (fluid 2D), segments


class FakeSim:
    def __init__(self, rng):
        self.ctx = object()
        self.dim = D
        self.S = rng.normal(size=(N_P, W))
        self.M = rng.normal(size=(W, W)) / 3.0
        self.N = rng.normal(size=(N_P, W, N_SEG))
        self.mu = np.zeros(N_SEG)
        self.steps = 0

    def get(self, field):
        s = self.S
        return {"x": s[:, 0:2].copy(), "v": s[:, 2:4].copy(), "C": s[:, 4:8].reshape(-1, 2, 2).copy(),
                "rho": s[:, 8].copy()}[field]

    def set_friction(self, wall, shape, mu):
        assert wall == 2 and tuple(shape) == (N_SEG, 1)
        self.mu = np.asarray(mu, dtype=np.float64).copy()

    def step(self, n=1):
        for _ in range(n):
            self.S = self.S @ self.M.T + np.einsum("pwk,k->pw", self.N, self.mu)
            self.steps += 1


@pytest.fixture
def fake(monkeypatch):
    sim = FakeSim(np.random.default_rng(0))
    calls = []

    def vjp(ctx, wall, lam_next, n_seg):
        assert ctx is sim.ctx and lam_next.shape == (N_P, W) and lam_next.dtype == np.float64
        calls.append(wall)
        sim.step(1)                                         # the real call runs the step too
        g = np.einsum("pwk,pw->k", sim.N, lam_next) if wall >= 0 else np.zeros(n_seg)
        return lam_next @ sim.M, g[:n_seg]

    monkeypatch.setattr(mpm, "mpm_adjoint_width", lambda ctx: W)
    monkeypatch.setattr(mpm, "mpm_export_state", lambda ctx: pickle.dumps(sim.S.copy()))
    monkeypatch.setattr(mpm, "mpm_import_state", lambda ctx, blob: setattr(sim, "S", pickle.loads(blob)))
    monkeypatch.setattr(mpm, "mpm_step_adjoint_1", vjp)
    return sim, calls


def reference(sim, S0, mu, Wts):
    """The same chain in plain torch: the loss and its gradients."""
    M, N = torch.from_numpy(sim.M), torch.from_numpy(sim.N)
    S = S0
    loss = torch.zeros((), dtype=torch.float64)
    for t in range(1, 5):
        S = S @ M.T + torch.einsum("pwk,k->pw", N, mu)
        if t in (2, 4):
            loss = loss + (Wts[t] * S).sum()
    return loss


def test_chain_gradients_match_torch_autograd_of_the_same_map(fake):
    sim, calls = fake
    rng = np.random.default_rng(1)
    Wts = {t: torch.from_numpy(rng.normal(size=(N_P, W))) for t in (2, 4)}
    mu0 = np.array([0.2, 0.4, 0.3])
    S_start = sim.S.copy()

    st = autograd.Stepper(sim, 2, (N_SEG, 1))
    s = st.reset()
    np.testing.assert_array_equal(s.numpy(), S_start)      # x, v, C row-major, rho: the adjoint layout
    s0 = s.requires_grad_(True)
    mu = torch.tensor(mu0, requires_grad=True)
    loss = torch.zeros((), dtype=torch.float64)
    for t in range(1, 5):
        s = st.step(s, mu)
        if t in (2, 4):
            loss = loss + (Wts[t] * s).sum()
    loss.backward()
    assert calls == [2, 2, 2, 2]

    S0r = torch.from_numpy(S_start).requires_grad_(True)
    mur = torch.tensor(mu0, requires_grad=True)
    lr = reference(sim, S0r, mur, Wts)
    lr.backward()
    assert float(loss.detach()) == pytest.approx(float(lr.detach()), rel=1e-12)
    np.testing.assert_allclose(mu.grad.numpy(), mur.grad.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(s0.grad.numpy(), S0r.grad.numpy(), rtol=1e-12, atol=1e-12)


def test_without_a_friction_field_no_mu_gradient(fake):
    sim, calls = fake
    st = autograd.Stepper(sim)                             # wall -1
    s = st.reset().requires_grad_(True)
    s1 = st.step(s)
    s1.sum().backward()
    assert calls == [-1]
    np.testing.assert_allclose(s.grad.numpy(), np.ones((N_P, W)) @ sim.M)


def test_only_the_latest_state_can_be_advanced(fake):
    sim, _ = fake
    st = autograd.Stepper(sim, 2, (N_SEG, 1))
    mu = torch.tensor([0.1, 0.2, 0.3], requires_grad=True)
    s0 = st.reset()
    s1 = st.step(s0, mu)
    with pytest.raises(RuntimeError):
        st.step(s0, mu)                                     # the context holds s1
    with pytest.raises(RuntimeError):
        st.step(torch.zeros(N_P, W), mu)                    # not a state of this context
    s2 = st.step(s1, mu)
    s2.sum().backward()
    with pytest.raises(RuntimeError):
        st.step(s2, mu)                                     # the backward pass moved the context
    s = st.reset()                                          # a reset starts a new chain
    st.step(s, mu)
