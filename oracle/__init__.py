"""CPU FP64 oracle of the explicit MPM step (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package.  The product path (the CUDA library and its Python
binding) never imports, calls or loads it.

The arithmetic lives in ``mpm_oracle.c`` (plain loops, FP64, compiled with
``-ffp-contract=off`` so that the result does not depend on the host's FMA
contraction).  This module only builds it with gcc and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmpm_oracle.so")
_LIB_OMP = os.path.join(_BUILD, "libmpm_oracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

MAX_WALLS = 6
MAX_OBSTACLES = 8


class Params(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("n_cells", C.c_int * 3),
        ("dx", C.c_double),
        ("dt", C.c_double),
        ("gravity", C.c_double * 3),
        ("material", C.c_int),
        ("dp_literal", C.c_int),
        ("rho0", C.c_double),
        ("bulk_K", C.c_double),
        ("gamma", C.c_double),
        ("viscosity", C.c_double),
        ("E", C.c_double),
        ("nu", C.c_double),
        ("phi_deg", C.c_double),
        ("psi_deg", C.c_double),
        ("cohesion", C.c_double),
        ("sigma_t", C.c_double),
        ("particle_volume", C.c_double),
        ("n_seg", (C.c_int * 2) * MAX_WALLS),
        ("mu", C.c_void_p * MAX_WALLS),
        ("transfer", C.c_int),
        ("flip_alpha", C.c_double),
        ("flip_grid", C.c_void_p),
        ("n_obstacles", C.c_int),
        ("obstacle", ((C.c_double * 3) * 2) * MAX_OBSTACLES),
    ]


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build`` (idempotent).

    omp=True builds the OpenMP variant of the same source (particle-parallel
    transfers with atomic grid sums, node-parallel grid update): a timing
    baseline only, whose sums vary in rounding with the thread schedule.  The
    checks use the serial build."""
    out = _LIB_OMP if omp else _LIB
    with _lock:
        if (not force and os.path.exists(out)
                and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
            return out
        os.makedirs(_BUILD, exist_ok=True)
        tmp = out + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               *(["-fopenmp"] if omp else []), _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
        return out


def lib(omp: bool = False):
    global _lib, _lib_omp
    if omp:
        if _lib_omp is None:
            _lib_omp = C.CDLL(build(omp=True))
            _declare(_lib_omp)
        return _lib_omp
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


def _declare(lib_):
    d, p, i, l = C.c_double, C.c_void_p, C.c_int, C.c_long
    P = C.POINTER(Params)
    sig = {
        "orc_phi_bar": (d, [d]),
        "orc_dphi_bar": (d, [d]),
        "orc_num_nodes": (l, [P]),
        "orc_particle_mass": (d, [P]),
        "orc_p2g": (None, [P, l, p, p, p, p, p, p, p, p]),
        "orc_grid_update": (None, [P, p, p, p, p]),
        "orc_g2p": (None, [P, l, p, p, p, p, p, p, p, p]),
        "orc_step": (i, [P, l, p, p, p, p, p, p, p, i]),
        "orc_friction": (None, [p, p, d, p]),
        "orc_dp_update": (i, [P, p, p, p, p]),
        "orc_dp_constants": (None, [P, p]),
        "orc_tait_pressure": (d, [P, d]),
        "orc_affine_C": (None, [P, l, p, p, p]),
        "orc_step_vjp": (i, [P, l] + [p] * 16),
        "orc_dp_vjp": (None, [P, p, p, p, p, p, p, p]),
        "orc_obstacle_normal": (i, [P, i, p, p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib_, name)
        f.restype = res
        f.argtypes = args


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous float64"
    return a.ctypes.data_as(C.c_void_p)


class Oracle:
    """Parameters of one scenario plus the numpy arrays kept alive for ctypes."""

    def __init__(self, dim, n_cells, dx, dt, gravity, material, particle_volume,
                 friction=(), dp_literal=False, transfer=0, flip_alpha=1.0, obstacles=()):
        P = Params()
        P.dim = dim
        for a in range(3):
            P.n_cells[a] = int(n_cells[a]) if a < dim else 1
            P.gravity[a] = float(gravity[a]) if a < dim else 0.0
        P.dx, P.dt = float(dx), float(dt)
        P.material = int(material.get("kind", 0))
        P.dp_literal = int(bool(dp_literal))
        P.transfer = int(transfer)
        P.flip_alpha = float(flip_alpha)
        for k in ("rho0", "bulk_K", "gamma", "viscosity", "E", "nu", "phi_deg", "psi_deg",
                  "cohesion", "sigma_t"):
            setattr(P, k, float(material.get(k, 0.0)))
        P.particle_volume = float(particle_volume)
        self._mu = []
        for wall, nseg, mu in friction:
            arr = np.ascontiguousarray(np.asarray(mu, dtype=np.float64).reshape(-1))
            assert arr.size == nseg[0] * nseg[1]
            self._mu.append(arr)
            P.n_seg[wall][0], P.n_seg[wall][1] = int(nseg[0]), int(nseg[1])
            P.mu[wall] = arr.ctypes.data
        assert len(obstacles) <= MAX_OBSTACLES
        P.n_obstacles = len(obstacles)
        for o, (lo, hi) in enumerate(obstacles):          # stationary boxes (Sec. 4.1)
            for a in range(dim):
                P.obstacle[o][0][a] = float(lo[a])
                P.obstacle[o][1][a] = float(hi[a])
        self.P = P
        self.dim = dim

    @classmethod
    def from_workload(cls, w, dp_literal=False, dt=None, transfer=0, flip_alpha=1.0):
        return cls(w.dim, w.n_cells, w.dx, w.dt if dt is None else dt, w.gravity, w.material,
                   w.particle_volume, w.friction, dp_literal, transfer, flip_alpha,
                   getattr(w, "obstacles", ()))

    # -- state ------------------------------------------------------------------
    def initial_state(self, x: np.ndarray, v: Optional[np.ndarray] = None) -> "State":
        n, d = x.shape
        st = State(
            x=np.ascontiguousarray(x, dtype=np.float64).copy(),
            v=np.zeros((n, d)) if v is None else np.ascontiguousarray(v, dtype=np.float64).copy(),
            B=np.zeros((n, d, d)),
            F=np.tile(np.eye(d), (n, 1, 1)),
            rho=np.full(n, self.P.rho0),
            sigma=np.zeros((n, 3, 3)),
            eps=np.zeros(n),
        )
        return st

    @property
    def num_nodes(self) -> int:
        return int(lib().orc_num_nodes(C.byref(self.P)))

    @property
    def node_shape(self):
        return tuple(self.P.n_cells[a] + 3 for a in range(self.dim))

    @property
    def particle_mass(self) -> float:
        return float(lib().orc_particle_mass(C.byref(self.P)))

    # -- transfers ---------------------------------------------------------------
    def p2g(self, st: "State"):
        G, d = self.num_nodes, self.dim
        gm, gq, gf = np.zeros(G), np.zeros((G, d)), np.zeros((G, d))
        lib().orc_p2g(C.byref(self.P), st.n, _ptr(st.x), _ptr(st.v), _ptr(st.B), _ptr(st.rho),
                      _ptr(st.sigma), _ptr(gm), _ptr(gq), _ptr(gf))
        return gm, gq, gf

    def obstacle_normal(self, o: int, j) -> Optional[np.ndarray]:
        """Contact normal of oracle node index j with obstacle o (None outside it)."""
        jj = np.zeros(3, dtype=np.int32)
        jj[:len(j)] = j
        nrm = np.zeros(3)
        hit = lib().orc_obstacle_normal(C.byref(self.P), int(o), jj.ctypes.data_as(C.c_void_p), _ptr(nrm))
        return nrm if hit else None

    def grid_update(self, gm, gq, gf):
        gv = np.zeros((self.num_nodes, self.dim))
        lib().orc_grid_update(C.byref(self.P), _ptr(gm), _ptr(gq), _ptr(gf), _ptr(gv))
        return gv

    def g2p(self, st: "State", gv):
        lib().orc_g2p(C.byref(self.P), st.n, _ptr(gv), _ptr(st.x), _ptr(st.v), _ptr(st.B), _ptr(st.F),
                      _ptr(st.rho), _ptr(st.sigma), _ptr(st.eps))

    def step(self, st: "State", n_steps: int = 1, omp: bool = False):
        rc = lib(omp).orc_step(C.byref(self.P), st.n, _ptr(st.x), _ptr(st.v), _ptr(st.B), _ptr(st.F),
                            _ptr(st.rho), _ptr(st.sigma), _ptr(st.eps), int(n_steps))
        if rc != 0:
            raise MemoryError("oracle grid allocation failed")

    def affine_C(self, st: "State") -> np.ndarray:
        Cm = np.zeros_like(st.B)
        lib().orc_affine_C(C.byref(self.P), st.n, _ptr(st.x), _ptr(st.B), _ptr(Cm))
        return Cm

    def step_vjp(self, st: "State", xb, vb, Bb, rhob, sigb=None):
        """Adjoint of one step: given the adjoint of S^{t+1} = (x, v, B, rho) and,
        for Drucker-Prager, of sigma (n x 3 x 3, entries independent), return the
        adjoint of S^t (same layout) and dL/dmu per wall with a friction field."""
        n, d = st.n, self.dim
        sand = self.P.material == 1
        out = [np.zeros((n, d)), np.zeros((n, d)), np.zeros((n, d, d)), np.zeros(n)]
        ins = [np.ascontiguousarray(a, dtype=np.float64) for a in (xb, vb, Bb, rhob)]
        sig = np.ascontiguousarray(st.sigma, dtype=np.float64).reshape(n, 3, 3) if sand else None
        sigb1 = np.ascontiguousarray(sigb, dtype=np.float64).reshape(n, 3, 3) if sand else None
        sigb0 = np.zeros((n, 3, 3)) if sand else None
        mub = {}
        ptrs = (C.c_void_p * MAX_WALLS)()
        for w in range(MAX_WALLS):
            if self.P.mu[w]:
                mub[w] = np.zeros(self.P.n_seg[w][0] * self.P.n_seg[w][1])
                ptrs[w] = mub[w].ctypes.data
        opt = lambda a: None if a is None else _ptr(a)
        rc = lib().orc_step_vjp(C.byref(self.P), n, _ptr(st.x), _ptr(st.v), _ptr(st.B), _ptr(st.rho), opt(sig),
                                *[_ptr(a) for a in ins], opt(sigb1), *[_ptr(a) for a in out], opt(sigb0), ptrs)
        if rc != 0:
            raise RuntimeError(f"orc_step_vjp failed ({rc})")
        if sand:
            out.append(sigb0)
        return out, mub

    def dp_vjp(self, dd, dw, sigma, sigb1):
        """Adjoint of dp_update: (sigma_bar, dd_bar, dw_bar) for the output adjoint sigb1."""
        a = [np.ascontiguousarray(x, dtype=np.float64).reshape(3, 3) for x in (dd, dw, sigma, sigb1)]
        sb0, ddb, dwb = np.zeros((3, 3)), np.zeros((3, 3)), np.zeros((3, 3))
        lib().orc_dp_vjp(C.byref(self.P), *[_ptr(x) for x in a], _ptr(sb0), _ptr(ddb), _ptr(dwb))
        return sb0, ddb, dwb

    # -- constitutive pieces ------------------------------------------------------
    def tait_pressure(self, rho: float) -> float:
        return float(lib().orc_tait_pressure(C.byref(self.P), float(rho)))

    def dp_constants(self) -> dict:
        out = np.zeros(8)
        lib().orc_dp_constants(C.byref(self.P), _ptr(out))
        return dict(zip(("K", "G", "q_phi", "k_phi", "q_psi", "sigma_t", "tau_P", "alpha_P"), out))

    def dp_update(self, dd, dw, sigma, eps=0.0):
        dd = np.ascontiguousarray(dd, dtype=np.float64).reshape(3, 3)
        dw = np.ascontiguousarray(dw, dtype=np.float64).reshape(3, 3)
        s = np.ascontiguousarray(sigma, dtype=np.float64).reshape(3, 3).copy()
        e = np.array([eps], dtype=np.float64)
        zone = lib().orc_dp_update(C.byref(self.P), _ptr(dd), _ptr(dw), _ptr(s), _ptr(e))
        return zone, s, float(e[0])


@dataclass
class State:
    x: np.ndarray
    v: np.ndarray
    B: np.ndarray
    F: np.ndarray
    rho: np.ndarray
    sigma: np.ndarray
    eps: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def copy(self) -> "State":
        return State(*(getattr(self, k).copy() for k in ("x", "v", "B", "F", "rho", "sigma", "eps")))


def phi_bar(xi: float) -> float:
    return float(lib().orc_phi_bar(float(xi)))


def dphi_bar(xi: float) -> float:
    return float(lib().orc_dphi_bar(float(xi)))


def friction(v, n, mu):
    v3 = np.zeros(3); v3[: len(v)] = v
    n3 = np.zeros(3); n3[: len(n)] = n
    out = np.zeros(3)
    lib().orc_friction(_ptr(v3), _ptr(n3), float(mu), _ptr(out))
    return out[: len(v)]


def monitor_means(x: np.ndarray, v: np.ndarray, boxes):
    """Eulerian velocity monitors (Sec. 5.2, Case 3): per closed box [lo, hi] the
    mean velocity of the particles whose position lies inside, and their count
    (mean 0 for an empty monitor)."""
    Q = np.zeros((len(boxes), v.shape[1]))
    cnt = np.zeros(len(boxes), dtype=np.int64)
    for l, (lo, hi) in enumerate(boxes):
        inside = np.all((x >= np.asarray(lo, dtype=np.float64)) & (x <= np.asarray(hi, dtype=np.float64)), axis=1)
        cnt[l] = int(inside.sum())
        if cnt[l] > 0:
            Q[l] = v[inside].sum(axis=0) / cnt[l]
    return Q, cnt


def monitor_loss_and_seed(x: np.ndarray, v: np.ndarray, boxes, z: np.ndarray):
    """sum_l |Q_l - z_l|^2 over the non-empty monitors, and its gradient with
    respect to the particle velocities at fixed positions (the membership is a
    step function of x: its derivative is zero almost everywhere)."""
    Q, cnt = monitor_means(x, v, boxes)
    loss = 0.0
    g = np.zeros_like(v)
    for l, (lo, hi) in enumerate(boxes):
        if cnt[l] == 0:
            continue
        e = Q[l] - z[l]
        loss += float((e * e).sum())
        inside = np.all((x >= np.asarray(lo, dtype=np.float64)) & (x <= np.asarray(hi, dtype=np.float64)), axis=1)
        g[inside] += 2.0 * e / cnt[l]
    return loss, g
