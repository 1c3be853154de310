"""Thin ctypes binding of libmpm (include/mpm.h).

Argument marshalling only: every step of the MPM path runs in the CUDA
kernels of ``libmpm.so``.  There is no CPU fallback: if the library is
missing or cannot be built, loading fails with an error.

The module-level functions carry the C names (``mpm_create``, ``mpm_step``,
...); :class:`Simulation` is a small convenience wrapper over them.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Sequence

import numpy as np

from . import build as _build

MPM_OK, MPM_EINVAL, MPM_ENOMEM, MPM_ECUDA, MPM_ENAN = 0, -1, -2, -3, -4
MPM_EDOMAIN, MPM_ETIMEOUT, MPM_ECORRUPT, MPM_ESTATE = -5, -6, -7, -8
STATUS_NAMES = {0: "MPM_OK", -1: "MPM_EINVAL", -2: "MPM_ENOMEM", -3: "MPM_ECUDA", -4: "MPM_ENAN",
                -5: "MPM_EDOMAIN", -6: "MPM_ETIMEOUT", -7: "MPM_ECORRUPT", -8: "MPM_ESTATE"}
MPM_FP32, MPM_FP64 = 0, 1
MPM_FLUID, MPM_DRUCKER_PRAGER = 0, 1
FIELDS = {"x": 0, "v": 1, "C": 2, "F": 3, "rho": 4, "sigma": 5, "eps": 6}
KERNELS = {"sort": 0, "p2g": 1, "grid": 2, "g2p": 3, "reverse": 4}


class GridDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_cells", C.c_int * 3), ("dx", C.c_double), ("dt", C.c_double),
                ("gravity", C.c_double * 3), ("precision", C.c_int), ("sort_every", C.c_int),
                ("batch", C.c_int), ("transfer", C.c_int), ("flip_alpha", C.c_double)]


class Material(C.Structure):
    _fields_ = [("kind", C.c_int), ("rho0", C.c_double), ("bulk_K", C.c_double), ("gamma", C.c_double),
                ("viscosity", C.c_double), ("E", C.c_double), ("nu", C.c_double), ("phi_deg", C.c_double),
                ("psi_deg", C.c_double), ("cohesion", C.c_double), ("sigma_t", C.c_double),
                ("dp_literal", C.c_int)]


class StatePtrs(C.Structure):
    """Device pointers of one particle state (mpm_state_ptrs)."""
    _fields_ = [(k, C.c_void_p) for k in ("x", "v", "C", "F", "rho", "sigma", "eps")]


class MPMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libmpm.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libmpm is not built ({path}); run paper_2507_04192_gb300/build.py")
        lib = C.CDLL(path)
        P, I, L, D = C.c_void_p, C.c_int, C.c_int64, C.c_double
        sigs = {
            "mpm_create": (I, [C.POINTER(GridDesc), C.POINTER(Material), P, C.POINTER(P)]),
            "mpm_destroy": (None, [P]),
            "mpm_load_particles": (I, [P, L, P, P, D, P]),
            "mpm_load_particles_dev": (I, [P, L, P, P, D, P]),
            "mpm_set_particle_field": (I, [P, I, P]),
            "mpm_set_friction_field": (I, [P, I, P, P]),
            "mpm_set_obstacles": (I, [P, I, P]),
            "mpm_set_velocity_monitors": (I, [P, I, P, I, P, P]),
            "mpm_get_initial_adjoint": (I, [P, I, P]),
            "mpm_monitor_means": (I, [P, I, P, P]),
            "mpm_set_adjoint_memory": (I, [P, C.c_int64]),
            "mpm_step": (I, [P, I]),
            "mpm_request_sort": (I, [P]),
            "mpm_set_diagnostics": (I, [P, I]),
            "mpm_get_diagnostics": (I, [P, P, I]),
            "mpm_set_debug": (I, [P, I]),
            "mpm_synchronize": (I, [P]),
            "mpm_get_particles": (I, [P, I, P]),
            "mpm_get_particles_dev": (I, [P, I, P]),
            "mpm_field_width": (I, [P, I]),
            "mpm_num_particles": (L, [P]),
            "mpm_last_error": (I, [P, C.c_char_p, I]),
            "mpm_set_timing": (I, [P, I]),
            "mpm_get_timing": (I, [P, I, C.POINTER(D), C.POINTER(L)]),
            "mpm_reset_timing": (I, [P]),
            "mpm_get_stats": (I, [P, C.POINTER(L), I]),
            "mpm_step_noalloc": (I, [C.POINTER(GridDesc), C.POINTER(Material), P, L, D, StatePtrs, StatePtrs,
                                     C.c_char_p, I]),
            "mpm_set_observations": (I, [P, I, P, I, P, P]),
            "mpm_gemm_bf16": (I, [I, I, I, P, I, P, I, P, I, P, P]),
            "mpm_mlp_create": (I, [I, P, I, D, D, P, C.POINTER(P)]),
            "mpm_mlp_destroy": (None, [P]),
            "mpm_mlp_num_params": (L, [P]),
            "mpm_mlp_set_params": (I, [P, P]),
            "mpm_mlp_get_params": (I, [P, P, I]),
            "mpm_mlp_infer": (I, [P, I, P, P, I]),
            "mpm_mlp_train_step": (I, [P, I, P, P, D, I, C.POINTER(D), I]),
            "mpm_mlp_last_error": (I, [P, C.c_char_p, I]),
            "mpm_mlp_train_step_async": (I, [P, I, P, P, D, P]),
            "mpm_mlp_set_activations": (I, [P, I, I]),
            "mpm_mlp_backward": (I, [P, I, P, P, D, I, I]),
            "mpm_save_state": (I, [P, I]),
            "mpm_restore_state": (I, [P, I]),
            "mpm_state_blob_size": (L, [P]),
            "mpm_export_state": (I, [P, P, L]),
            "mpm_import_state": (I, [P, P, L]),
            "mpm_step_adjoint": (I, [P, I, I, I, C.POINTER(D), P]),
            "mpm_step_adjoint_1": (I, [P, I, P, P, P]),
            "mpm_adjoint_width": (I, [P]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _check(ctx, rc: int):
    if rc != MPM_OK:
        buf = C.create_string_buffer(512)
        if ctx:
            load_library().mpm_last_error(ctx, buf, 512)
        raise MPMError(rc, buf.value.decode(errors="replace"))


# ---------------------------------------------------------------- C-named wrappers

def mpm_create(grid: GridDesc, material: Material, stream: int = 0):
    h = C.c_void_p()
    _check(None, load_library().mpm_create(C.byref(grid), C.byref(material), C.c_void_p(stream), C.byref(h)))
    return h


def mpm_destroy(ctx):
    load_library().mpm_destroy(ctx)


def mpm_load_particles(ctx, x: np.ndarray, v: Optional[np.ndarray], particle_volume: float,
                       sim_id: Optional[np.ndarray] = None):
    x = np.ascontiguousarray(x, dtype=np.float64)
    vv = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    sid = None if sim_id is None else np.ascontiguousarray(sim_id, dtype=np.int32)
    _check(ctx, load_library().mpm_load_particles(ctx, x.shape[0], _dptr(x), None if vv is None else _dptr(vv),
                                                  float(particle_volume), None if sid is None else _dptr(sid)))


def mpm_load_particles_dev(ctx, n: int, x_ptr: int, v_ptr: Optional[int], particle_volume: float,
                           sim_id_ptr: Optional[int] = None):
    """mpm_load_particles from device pointers (e.g. tensor.data_ptr() of float64 and
    int32 CUDA tensors) read on the context's stream."""
    _check(ctx, load_library().mpm_load_particles_dev(ctx, int(n), C.c_void_p(x_ptr),
                                                      None if v_ptr is None else C.c_void_p(v_ptr),
                                                      float(particle_volume),
                                                      None if sim_id_ptr is None else C.c_void_p(sim_id_ptr)))


def mpm_set_particle_field(ctx, field: str, values: np.ndarray):
    a = np.ascontiguousarray(values, dtype=np.float64)
    _check(ctx, load_library().mpm_set_particle_field(ctx, FIELDS[field], _dptr(a)))


def mpm_set_friction_field(ctx, wall: int, n_seg: Sequence[int], mu: np.ndarray):
    ns = (C.c_int * 2)(int(n_seg[0]), int(n_seg[1]) if len(n_seg) > 1 else 1)
    m = np.ascontiguousarray(mu, dtype=np.float64)
    _check(ctx, load_library().mpm_set_friction_field(ctx, int(wall), ns, _dptr(m)))


def mpm_set_obstacles(ctx, boxes):
    """Stationary rigid boxes [(lo, hi), ...] with frictionless contact."""
    b = np.ascontiguousarray(np.asarray([list(lo) + list(hi) for lo, hi in boxes], dtype=np.float64).reshape(-1))
    _check(ctx, load_library().mpm_set_obstacles(ctx, len(boxes), _dptr(b) if len(boxes) else None))


def mpm_step(ctx, n_steps: int):
    _check(ctx, load_library().mpm_step(ctx, int(n_steps)))


def mpm_request_sort(ctx):
    _check(ctx, load_library().mpm_request_sort(ctx))


MPM_DIAG_COUNT = 11
MPM_DEBUG_WITHHOLD_WINDOW_COPY = 1


def mpm_set_diagnostics(ctx, enable: bool):
    _check(ctx, load_library().mpm_set_diagnostics(ctx, int(bool(enable))))


def mpm_get_diagnostics(ctx) -> dict:
    """Conservation sums of the last step run with the diagnostics enabled."""
    out = np.zeros(MPM_DIAG_COUNT, dtype=np.float64)
    _check(ctx, load_library().mpm_get_diagnostics(ctx, _dptr(out), MPM_DIAG_COUNT))
    return {"grid_mass": out[0], "grid_momentum": out[1:4].copy(), "particle_mass": out[4],
            "particle_momentum": out[5:8].copy(), "grid_nonfinite": int(out[8]), "particle_nonfinite": int(out[9]),
            "grid_abs_momentum": out[10]}


def mpm_set_debug(ctx, flags: int):
    _check(ctx, load_library().mpm_set_debug(ctx, int(flags)))


def mpm_synchronize(ctx):
    _check(ctx, load_library().mpm_synchronize(ctx))


def mpm_field_width(ctx, field: str) -> int:
    return int(load_library().mpm_field_width(ctx, FIELDS[field]))


def mpm_num_particles(ctx) -> int:
    return int(load_library().mpm_num_particles(ctx))


def mpm_get_particles(ctx, field: str, out: Optional[np.ndarray] = None) -> np.ndarray:
    n = mpm_num_particles(ctx)
    w = mpm_field_width(ctx, field)
    if out is None:
        out = np.empty((n, w), dtype=np.float64)
    assert out.dtype == np.float64 and out.flags["C_CONTIGUOUS"] and out.size == n * w
    _check(ctx, load_library().mpm_get_particles(ctx, FIELDS[field], _dptr(out)))
    return out


def mpm_get_particles_dev(ctx, field: str, out_ptr: int):
    """mpm_get_particles into a device pointer (n x width float64, load order),
    queued on the context's stream without waiting."""
    _check(ctx, load_library().mpm_get_particles_dev(ctx, FIELDS[field], C.c_void_p(out_ptr)))


def mpm_set_timing(ctx, enable: bool):
    _check(ctx, load_library().mpm_set_timing(ctx, int(bool(enable))))


def mpm_get_timing(ctx, kernel: str):
    ms, n = C.c_double(), C.c_int64()
    _check(ctx, load_library().mpm_get_timing(ctx, KERNELS[kernel], C.byref(ms), C.byref(n)))
    return ms.value, n.value


def mpm_reset_timing(ctx):
    _check(ctx, load_library().mpm_reset_timing(ctx))


def mpm_get_stats(ctx) -> dict:
    out = (C.c_int64 * 6)()
    _check(ctx, load_library().mpm_get_stats(ctx, out, 6))
    keys = ("active_tiles", "chunks", "escaped", "sorts", "steps", "launches")
    return dict(zip(keys, list(out)))


def mpm_save_state(ctx, slot: int):
    _check(ctx, load_library().mpm_save_state(ctx, int(slot)))


def mpm_restore_state(ctx, slot: int):
    _check(ctx, load_library().mpm_restore_state(ctx, int(slot)))


def mpm_export_state(ctx) -> bytes:
    size = int(load_library().mpm_state_blob_size(ctx))
    if size < 0:
        _check(ctx, size)
    buf = (C.c_ubyte * size)()
    _check(ctx, load_library().mpm_export_state(ctx, buf, size))
    return bytes(buf)


def mpm_import_state(ctx, blob: bytes):
    buf = (C.c_ubyte * len(blob)).from_buffer_copy(blob)
    _check(ctx, load_library().mpm_import_state(ctx, buf, len(blob)))


def mpm_set_observations(ctx, ids: np.ndarray, steps: Sequence[int], z_obs: np.ndarray):
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    st = np.ascontiguousarray(steps, dtype=np.int32)
    z = np.ascontiguousarray(z_obs, dtype=np.float64)
    assert z.size == len(st) * len(ids) * (z.shape[-1] if z.ndim else 1)
    _check(ctx, load_library().mpm_set_observations(ctx, len(ids), _dptr(ids), len(st), _dptr(st), _dptr(z)))


def mpm_clear_observations(ctx):
    _check(ctx, load_library().mpm_set_observations(ctx, 0, None, 0, None, None))


def mpm_set_velocity_monitors(ctx, boxes, steps: Sequence[int], v_obs: np.ndarray):
    """Eulerian velocity monitors: boxes [(lo, hi), ...], observation steps and the
    observed mean velocities (n_obs x n_mon x dim)."""
    b = np.ascontiguousarray(np.asarray([list(lo) + list(hi) for lo, hi in boxes], dtype=np.float64).reshape(-1))
    st = np.ascontiguousarray(steps, dtype=np.int32)
    z = np.ascontiguousarray(v_obs, dtype=np.float64)
    assert z.shape[:2] == (len(st), len(boxes))
    _check(ctx, load_library().mpm_set_velocity_monitors(ctx, len(boxes), _dptr(b), len(st), _dptr(st), _dptr(z)))


def mpm_monitor_means(ctx, boxes):
    """Mean velocity (n_mon x dim) and particle count (n_mon) of each monitor box on the current state."""
    b = np.ascontiguousarray(np.asarray([list(lo) + list(hi) for lo, hi in boxes], dtype=np.float64).reshape(-1))
    dim = len(boxes[0][0])
    out = np.zeros((len(boxes), dim + 1), dtype=np.float64)
    _check(ctx, load_library().mpm_monitor_means(ctx, len(boxes), _dptr(b), _dptr(out)))
    return out[:, :dim].copy(), out[:, dim].astype(np.int64)


def mpm_clear_velocity_monitors(ctx):
    _check(ctx, load_library().mpm_set_velocity_monitors(ctx, 0, None, 0, None, None))


def mpm_step_adjoint(ctx, n_steps: int, checkpoint_every: int, wall: int, n_mu: int):
    """Loss and dL/dmu of one wall (wall = -1: no friction gradient, returns an empty array)."""
    loss = C.c_double()
    g = np.zeros(max(n_mu, 0), dtype=np.float64)
    _check(ctx, load_library().mpm_step_adjoint(ctx, int(n_steps), int(checkpoint_every), int(wall),
                                                C.byref(loss), _dptr(g) if wall >= 0 else None))
    return loss.value, g


def mpm_adjoint_width(ctx) -> int:
    return int(load_library().mpm_adjoint_width(ctx))


def mpm_step_adjoint_1(ctx, wall: int, lam_next: np.ndarray, n_seg: int = 0):
    """One step and its vector-Jacobian product: returns (lam_prev, dL/dmu of this
    step) for lam_next = dL/dS^{t+1} (n x mpm_adjoint_width doubles, load order)."""
    lam_next = np.ascontiguousarray(lam_next, dtype=np.float64)
    lam_prev = np.empty_like(lam_next)
    g = np.zeros(max(int(n_seg), 1), dtype=np.float64)
    _check(ctx, load_library().mpm_step_adjoint_1(ctx, int(wall), _dptr(lam_next), _dptr(lam_prev),
                                                  _dptr(g) if wall >= 0 else None))
    return lam_prev, g[:n_seg]


def mpm_set_adjoint_memory(ctx, nbytes: int):
    """Device bytes the adjoint may spend keeping more first-pass segments (0: recompute all but the last)."""
    _check(ctx, load_library().mpm_set_adjoint_memory(ctx, int(nbytes)))


def mpm_get_initial_adjoint(ctx, field: str) -> np.ndarray:
    """dL/d(field of the initial state) of the last adjoint, load order, (n, width)."""
    n = mpm_num_particles(ctx)
    w = {"x": None, "v": None, "C": None, "rho": 1}[field]
    dim = mpm_field_width(ctx, "x")
    w = w if w is not None else (dim * dim if field == "C" else dim)
    out = np.zeros((n, w), dtype=np.float64)
    _check(ctx, load_library().mpm_get_initial_adjoint(ctx, FIELDS[field], _dptr(out)))
    return out


def mpm_step_noalloc(grid: GridDesc, material: Material, n: int, particle_volume: float, state_in: StatePtrs,
                     state_out: StatePtrs, stream: int = 0):
    """One step with caller-owned device buffers and no allocation (see include/mpm.h)."""
    buf = C.create_string_buffer(256)
    rc = load_library().mpm_step_noalloc(C.byref(grid), C.byref(material), C.c_void_p(stream), int(n),
                                         float(particle_volume), state_in, state_out, buf, 256)
    if rc != MPM_OK:
        raise MPMError(rc, buf.value.decode(errors="replace"))


def mpm_gemm_bf16(M, N, K, A_ptr, lda, B_ptr, ldb, C_ptr, ldc, status_ptr, stream=0):
    rc = load_library().mpm_gemm_bf16(M, N, K, C.c_void_p(A_ptr), lda, C.c_void_p(B_ptr), ldb, C.c_void_p(C_ptr),
                                      ldc, C.c_void_p(status_ptr), C.c_void_p(stream))
    if rc != MPM_OK:
        raise MPMError(rc, "mpm_gemm_bf16")


MPM_ACT_GELU, MPM_ACT_RELU = 0, 1
MPM_OUT_SIGMOID, MPM_OUT_LINEAR = 0, 1


class MLP:
    """Binding of mpm_mlp_* (argument marshalling only)."""

    def __init__(self, widths, max_batch, out_lo=0.1, out_hi=0.6, stream=0, hidden=MPM_ACT_GELU,
                 output=MPM_OUT_SIGMOID):
        lib = load_library()
        self.widths = list(widths)
        w = (C.c_int * len(widths))(*widths)
        h = C.c_void_p()
        rc = lib.mpm_mlp_create(len(widths) - 1, w, int(max_batch), float(out_lo), float(out_hi),
                                C.c_void_p(stream), C.byref(h))
        if rc != MPM_OK:
            raise MPMError(rc, "mpm_mlp_create")
        self.h = h
        if hidden != MPM_ACT_GELU or output != MPM_OUT_SIGMOID:
            self._check(lib.mpm_mlp_set_activations(self.h, int(hidden), int(output)))

    def _check(self, rc):
        if rc != MPM_OK:
            buf = C.create_string_buffer(256)
            load_library().mpm_mlp_last_error(self.h, buf, 256)
            raise MPMError(rc, buf.value.decode(errors="replace"))

    @property
    def num_params(self):
        return int(load_library().mpm_mlp_num_params(self.h))

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.num_params
        self._check(load_library().mpm_mlp_set_params(self.h, _dptr(p)))

    def get_params(self, which=0):
        p = np.empty(self.num_params, dtype=np.float32)
        self._check(load_library().mpm_mlp_get_params(self.h, _dptr(p), int(which)))
        return p

    def infer(self, x):
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.empty((x.shape[0], self.widths[-1]), dtype=np.float32)
        self._check(load_library().mpm_mlp_infer(self.h, x.shape[0], _dptr(x), _dptr(y), 0))
        return y

    def train_step(self, x, target, lr, update=True):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(target, dtype=np.float32)
        loss = C.c_double()
        self._check(load_library().mpm_mlp_train_step(self.h, x.shape[0], _dptr(x), _dptr(t), float(lr),
                                                      int(bool(update)), C.byref(loss), 0))
        return loss.value

    def train_step_async(self, batch, x_ptr, target_ptr, lr, loss_ptr=0):
        """Device pointers, no synchronisation (mpm_mlp_train_step_async)."""
        self._check(load_library().mpm_mlp_train_step_async(self.h, int(batch), C.c_void_p(x_ptr),
                                                            C.c_void_p(target_ptr), float(lr),
                                                            C.c_void_p(loss_ptr) if loss_ptr else None))

    def backward(self, x, dy, lr=0.0, update=False):
        """Back-propagate a given dL/dy (host arrays); with update, one Adam step."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        g = np.ascontiguousarray(dy, dtype=np.float32)
        self._check(load_library().mpm_mlp_backward(self.h, x.shape[0], _dptr(x), _dptr(g), float(lr),
                                                    int(bool(update)), 0))

    def close(self):
        if self.h:
            load_library().mpm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- convenience wrapper

def material_struct(mat: dict, dp_literal: bool = False) -> Material:
    m = Material()
    m.kind = int(mat.get("kind", 0))
    for k in ("rho0", "bulk_K", "gamma", "viscosity", "E", "nu", "phi_deg", "psi_deg", "cohesion", "sigma_t"):
        setattr(m, k, float(mat.get(k, 0.0)))
    m.dp_literal = int(bool(dp_literal or mat.get("dp_literal", False)))
    return m


MPM_TRANSFER_APIC, MPM_TRANSFER_TPIC, MPM_TRANSFER_PIC, MPM_TRANSFER_FLIP = 0, 1, 2, 3


def grid_struct(dim, n_cells, dx, dt, gravity, precision=MPM_FP32, sort_every=8, batch=1,
                transfer=MPM_TRANSFER_APIC, flip_alpha=1.0) -> GridDesc:
    g = GridDesc()
    g.dim = int(dim)
    for a in range(3):
        g.n_cells[a] = int(n_cells[a]) if a < dim else 1
        g.gravity[a] = float(gravity[a]) if a < dim else 0.0
    g.dx, g.dt = float(dx), float(dt)
    g.precision = int(precision)
    g.sort_every = int(sort_every)
    g.batch = int(batch)
    g.transfer = int(transfer)
    g.flip_alpha = float(flip_alpha)
    return g


class Simulation:
    """One libmpm context: a grid, a material and a set of particles."""

    def __init__(self, dim, n_cells, dx, dt, gravity, material: dict, precision=MPM_FP32, sort_every=8,
                 batch=1, stream: int = 0, dp_literal=False, transfer=MPM_TRANSFER_APIC, flip_alpha=1.0):
        self.dim = dim
        self._grid = grid_struct(dim, n_cells, dx, dt, gravity, precision, sort_every, batch, transfer, flip_alpha)
        self._mat = material_struct(material, dp_literal)
        self.ctx = mpm_create(self._grid, self._mat, stream)

    @classmethod
    def from_workload(cls, w, precision=MPM_FP32, sort_every=None, batch=1, stream=0, load=True, dt=None,
                      transfer=MPM_TRANSFER_APIC, flip_alpha=1.0):
        sim = cls(w.dim, w.n_cells, w.dx, w.dt if dt is None else dt, w.gravity, w.material, precision,
                  w.sort_every if sort_every is None else sort_every, batch, stream, transfer=transfer,
                  flip_alpha=flip_alpha)
        if load:
            sim.load(w.x, w.v, w.particle_volume)
            for wall, nseg, mu in w.friction:
                sim.set_friction(wall, nseg, np.tile(np.asarray(mu, dtype=np.float64).reshape(-1), batch))
            if getattr(w, "obstacles", None):
                sim.set_obstacles(w.obstacles)
        return sim

    def close(self):
        if self.ctx:
            mpm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, x, v=None, particle_volume=1.0, sim_id=None):
        mpm_load_particles(self.ctx, x, v, particle_volume, sim_id)

    def set_field(self, field, values):
        mpm_set_particle_field(self.ctx, field, values)

    def set_friction(self, wall, n_seg, mu):
        mpm_set_friction_field(self.ctx, wall, n_seg, mu)

    def set_obstacles(self, boxes):
        mpm_set_obstacles(self.ctx, boxes)

    def step(self, n=1):
        mpm_step(self.ctx, n)

    def synchronize(self):
        mpm_synchronize(self.ctx)

    def get(self, field):
        a = mpm_get_particles(self.ctx, field)
        d = self.dim
        if field in ("C", "F"):
            return a.reshape(-1, d, d)
        if field == "sigma":
            return a.reshape(-1, 3, 3)
        if field in ("rho", "eps"):
            return a.reshape(-1)
        return a

    @property
    def n(self):
        return mpm_num_particles(self.ctx)

    def stats(self):
        return mpm_get_stats(self.ctx)
