"""Seeded synthetic inputs for the explicit MPM step.

This module is shared by the CUDA path, the CPU oracle checks and the benchmark.
It holds no MPM arithmetic: only lattice sampling of the initial bodies, a
counter-based SplitMix64 generator for jitter and random fields, and the
parameter tables of the workloads.

Workloads (the paper's scenarios, Sec. 4.1.1, Sec. 4.2.3, Sec. 5.3):

* ``dam_break_2d``: a water column against the left wall of a square box, the
  shallow-water dam break of Sec. 4.1.1 in the proportions of a tall column.
* ``granular_cylinder_3d``: a sand cylinder standing on a frictional floor,
  the granular cylinder collapse of Sec. 4.2.3.
* ``dam_break_inverse_2d``: the dam break with a piecewise-constant basal
  friction field, the friction inversion of Sec. 5.3.

Particles are placed on a regular lattice of ``ppc_axis`` points per cell and
axis, at ``(cell + (k + 0.5) / ppc_axis) * dx``.  A lattice point is kept when
the unjittered point lies inside the body; the kept point is then moved by a
jitter drawn uniformly from ``[-0.25, 0.25) * dx / ppc_axis`` per axis.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Tuple

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, index: np.ndarray) -> np.ndarray:
    """SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) in counter form.

    Output ``i`` is the finaliser applied to ``seed + (i + 1) * 0x9E3779B97F4A7C15``,
    which is the ``i``-th output of the sequential generator started at ``seed``.
    """
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (np.asarray(index, dtype=np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, index: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, index) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# Streams: each use of randomness draws from its own seed offset.
_STREAM_JITTER = 0x0000_0001_0000_0000
_STREAM_FRICTION = 0x0000_0002_0000_0000
_STREAM_TRACKS = 0x0000_0003_0000_0000
_STREAM_VELOCITY = 0x0000_0004_0000_0000


FLUID_WATER = dict(kind=0, rho0=1000.0, bulk_K=2.0e5, gamma=7.0, viscosity=0.0)
"""Weakly compressible water with the Tait equation of state (Sec. 2.3)."""

SAND_DP = dict(kind=1, rho0=2000.0, E=1.0e6, nu=0.3, phi_deg=30.0, psi_deg=0.0,
               cohesion=0.0, sigma_t=0.0)
"""Cohesionless Drucker-Prager sand (Sec. 2.3, Appendix A)."""


@dataclass
class Workload:
    """One synthetic scenario: grid, material, initial particles and boundary friction."""

    name: str
    dim: int
    n_cells: Tuple[int, ...]
    dx: float
    dt: float
    gravity: Tuple[float, ...]
    material: Dict[str, float]
    x: np.ndarray                      # (n, dim) float64 initial positions
    particle_volume: float
    steps: int
    sort_every: int
    friction: List[Tuple[int, Tuple[int, int], np.ndarray]] = field(default_factory=list)
    """(wall, (n_seg0, n_seg1), mu[n_seg1 * n_seg0]) triples; walls not listed are slip walls."""
    v: Optional[np.ndarray] = None     # (n, dim) initial velocities, None = at rest
    extras: Dict[str, object] = field(default_factory=dict)
    obstacles: List[Tuple[Tuple[float, ...], Tuple[float, ...]]] = field(default_factory=list)
    """Stationary rigid boxes (low corner, high corner) with frictionless contact."""

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def domain(self) -> Tuple[float, ...]:
        return tuple(c * self.dx for c in self.n_cells)


def lattice_particles(n_cells: Tuple[int, ...], dx: float, ppc_axis: int,
                      inside: Callable[[np.ndarray], np.ndarray],
                      box_lo: Tuple[float, ...], box_hi: Tuple[float, ...],
                      seed: int) -> np.ndarray:
    """Jittered lattice points of ``ppc_axis**dim`` per cell inside a body.

    ``inside`` takes an (m, dim) array of unjittered lattice points and returns a
    boolean mask.  Only cells overlapping ``[box_lo, box_hi]`` are visited.  The
    points are ordered with the first axis fastest.
    """
    dim = len(n_cells)
    h = dx / ppc_axis
    axes = []
    for a in range(dim):
        c0 = max(0, int(np.floor(box_lo[a] / dx)) - 1)
        c1 = min(n_cells[a], int(np.ceil(box_hi[a] / dx)) + 1)
        k = np.arange(c0 * ppc_axis, c1 * ppc_axis, dtype=np.int64)
        axes.append((k + 0.5) * h)
    grids = np.meshgrid(*axes[::-1], indexing="ij")          # last axis slowest
    pts = np.stack([g.reshape(-1) for g in grids[::-1]], axis=1)
    pts = pts[inside(pts)]
    n = pts.shape[0]
    idx = np.arange(n * dim, dtype=np.uint64).reshape(n, dim)
    jitter = (uniform01(seed + _STREAM_JITTER, idx) - 0.5) * 0.5 * h
    return np.ascontiguousarray(pts + jitter)


def friction_field(n_seg: int, seed: int, lo: float = 0.1, hi: float = 0.6) -> np.ndarray:
    """Per-segment friction coefficients drawn uniformly from [lo, hi)."""
    u = uniform01(seed + _STREAM_FRICTION, np.arange(n_seg, dtype=np.uint64))
    return lo + (hi - lo) * u


def tracked_particles(x: np.ndarray, n_track: int, seed: int,
                      body_lo: np.ndarray, body_hi: np.ndarray) -> np.ndarray:
    """Indices of the particles nearest to ``n_track`` seeded reference points.

    The reference points are drawn uniformly in the body's bounding box expressed
    in normalised coordinates, so that tracks are comparable across resolutions.
    Each reference point takes the nearest particle not already taken.
    """
    dim = x.shape[1]
    u = uniform01(seed + _STREAM_TRACKS, np.arange(n_track * dim, dtype=np.uint64)).reshape(n_track, dim)
    ref = np.asarray(body_lo) + u * (np.asarray(body_hi) - np.asarray(body_lo))
    taken = np.zeros(x.shape[0], dtype=bool)
    ids = np.empty(n_track, dtype=np.int64)
    for t in range(n_track):
        d2 = ((x - ref[t]) ** 2).sum(axis=1)
        d2[taken] = np.inf
        j = int(np.argmin(d2))
        ids[t] = j
        taken[j] = True
    return ids


def random_velocities(n: int, dim: int, scale: float, seed: int) -> np.ndarray:
    """Uniform velocities in [-scale, scale) per component (test inputs)."""
    u = uniform01(seed + _STREAM_VELOCITY, np.arange(n * dim, dtype=np.uint64)).reshape(n, dim)
    return (2.0 * u - 1.0) * scale


def dam_break_2d(n_cells: int = 64, width: float = 0.25, height: float = 0.5,
                 ppc_axis: int = 4, seed: int = 0, dt: float = 1.0e-4,
                 steps: int = 200, sort_every: int = 32) -> Workload:
    """Water column ``width`` x ``height`` at the left wall of the unit square.

    At 64 cells and 4 points per cell and axis this is 16 x 32 cells x 16 = 8,192
    particles; at 128 cells 32,768; at 96 cells 18,432.  Sorted every 32 steps:
    particles that leave their cell between sorts take P2G's escape path, and on
    the 256 batched 96^2 dam breaks the first 300 steps took 0.2062 ms per step
    sorting every 16 steps, 0.1981 every 24 and 0.1945 every 32 (later windows
    the same within 1 %).
    """
    dx = 1.0 / n_cells
    x = lattice_particles((n_cells, n_cells), dx, ppc_axis,
                          lambda p: (p[:, 0] < width) & (p[:, 1] < height),
                          (0.0, 0.0), (width, height), seed)
    return Workload(name=f"dam_break_2d_{n_cells}", dim=2, n_cells=(n_cells, n_cells), dx=dx, dt=dt,
                    gravity=(0.0, -9.81), material=dict(FLUID_WATER), x=x,
                    particle_volume=dx * dx / ppc_axis ** 2, steps=steps, sort_every=sort_every,
                    extras=dict(body_lo=(0.0, 0.0), body_hi=(width, height), seed=seed))


def granular_cylinder_3d(n_cells: Tuple[int, int, int] = (256, 256, 128), radius_cells: float = 38,
                         height_cells: float = 76, ppc_axis: int = 2, seed: int = 0,
                         dt: float = 1.0e-5, floor_mu: float = 0.4, steps: int = 1000,
                         sort_every: int = 32, dx: float = 1.0 / 256.0) -> Workload:
    """Drucker-Prager sand cylinder on the floor at the domain centre (dx = 1/256 m).

    Radius 38 dx and height 76 dx at 2 points per cell and axis give 2,761,536
    particles on the 256 x 256 x 128 grid; radius 30 dx and height 60 dx on
    192 x 192 x 96 give 1,356,480.
    """
    cx = 0.5 * n_cells[0] * dx
    cy = 0.5 * n_cells[1] * dx
    r = radius_cells * dx
    hgt = height_cells * dx
    x = lattice_particles(tuple(n_cells), dx, ppc_axis,
                          lambda p: ((p[:, 0] - cx) ** 2 + (p[:, 1] - cy) ** 2 < r * r) & (p[:, 2] < hgt),
                          (cx - r, cy - r, 0.0), (cx + r, cy + r, hgt), seed)
    fr = [(4, (1, 1), np.array([floor_mu]))] if floor_mu > 0 else []
    return Workload(name=f"granular_cylinder_3d_{n_cells[0]}x{n_cells[1]}x{n_cells[2]}", dim=3,
                    n_cells=tuple(n_cells), dx=dx, dt=dt, gravity=(0.0, 0.0, -9.81),
                    material=dict(SAND_DP), x=x, particle_volume=dx ** 3 / ppc_axis ** 3,
                    steps=steps, sort_every=sort_every, friction=fr,
                    extras=dict(body_lo=(cx - r, cy - r, 0.0), body_hi=(cx + r, cy + r, hgt),
                                axis=(cx, cy), seed=seed))


def dam_break_inverse_2d(n_cells: int = 128, n_seg: int = 32, n_track: int = 64, n_obs: int = 10,
                         steps: int = 500, seed: int = 0, ppc_axis: int = 4,
                         checkpoint_every: int = 50) -> Workload:
    """Dam break with a 32-segment basal friction field and tracked particles (Sec. 5.3)."""
    w = dam_break_2d(n_cells=n_cells, ppc_axis=ppc_axis, seed=seed, steps=steps)
    w.name = f"dam_break_inverse_2d_{n_cells}"
    mu = friction_field(n_seg, seed)
    w.friction = [(2, (n_seg, 1), mu)]
    ids = tracked_particles(w.x, n_track, seed, np.array(w.extras["body_lo"]), np.array(w.extras["body_hi"]))
    obs_steps = [steps * (k + 1) // n_obs for k in range(n_obs)]
    w.extras.update(track_ids=ids, obs_steps=obs_steps, mu_true=mu, checkpoint_every=checkpoint_every)
    return w


def shallow_dam_break_2d(dx: float = 0.004, length: float = 1.0, height: float = 0.1, domain: float = 2.5,
                         sound_speed: float = 35.0, ppc_axis: int = 2, seed: int = 0, dt: float = 1.0e-5,
                         steps: int = 40_000, sort_every: int = 16) -> Workload:
    """The shallow-water dam break of Sec. 5.1: a water column ``length`` x
    ``height`` at the left wall of a ``domain``-long channel, inviscid, slip walls,
    Tait water whose sound speed is ``sound_speed`` (K = rho0 c^2), 4 particles
    per cell."""
    nx = int(round(domain / dx))
    ny = int(round(3.0 * height / dx))
    x = lattice_particles((nx, ny), dx, ppc_axis, lambda p: (p[:, 0] < length) & (p[:, 1] < height),
                          (0.0, 0.0), (length, height), seed)
    mat = dict(FLUID_WATER, bulk_K=1000.0 * sound_speed ** 2)
    return Workload(name=f"shallow_dam_break_2d_{nx}x{ny}", dim=2, n_cells=(nx, ny), dx=dx, dt=dt,
                    gravity=(0.0, -9.8), material=mat, x=x, particle_volume=dx * dx / ppc_axis ** 2, steps=steps,
                    sort_every=sort_every, extras=dict(body_lo=(0.0, 0.0), body_hi=(length, height), seed=seed))


def dam_break_3d(n_cells: Tuple[int, int, int] = (200, 100, 80), dx: float = 0.005, length: float = 0.3,
                 width: float = 0.5, height: float = 0.2, sound_speed: float = 35.0, ppc_axis: int = 2,
                 seed: int = 0, dt: float = 1.0e-5, steps: int = 1000, sort_every: int = 32,
                 obstacles: bool = True) -> Workload:
    """The 3D dam break with two rigid square columns of Sec. 4.1.

    Domain 1.0 x 0.5 x 0.4 m at dx = 1/200; a water column ``length`` x ``width``
    x ``height`` at the x- wall; 8 particles per cell (2 per axis) give
    60 x 100 x 40 cells x 8 = 1,920,000 particles.  Water with the paper's
    linear equation of state (Tait with gamma = 1, K = rho0 c^2, c = 35 m/s).
    Columns of side 0.04 m and 0.06 m stand on the floor with their base centres
    at (0.5, 0.3) and (0.6, 0.1) m and reach the ceiling.
    """
    dom = tuple(c * dx for c in n_cells)
    x = lattice_particles(tuple(n_cells), dx, ppc_axis,
                          lambda p: (p[:, 0] < length) & (p[:, 1] < width) & (p[:, 2] < height),
                          (0.0, 0.0, 0.0), (length, width, height), seed)
    mat = dict(FLUID_WATER, bulk_K=1000.0 * sound_speed ** 2, gamma=1.0)
    obs = []
    if obstacles:
        for (cx, cy), side in (((0.5, 0.3), 0.04), ((0.6, 0.1), 0.06)):
            obs.append(((cx - side / 2, cy - side / 2, 0.0), (cx + side / 2, cy + side / 2, dom[2])))
    return Workload(name=f"dam_break_3d_{n_cells[0]}x{n_cells[1]}x{n_cells[2]}", dim=3, n_cells=tuple(n_cells),
                    dx=dx, dt=dt, gravity=(0.0, 0.0, -9.81), material=mat, x=x,
                    particle_volume=dx ** 3 / ppc_axis ** 3, steps=steps, sort_every=sort_every,
                    extras=dict(body_lo=(0.0, 0.0, 0.0), body_hi=(length, width, height), seed=seed),
                    obstacles=obs)


def dam_break_velocity_inverse(dx: float = 0.01, column: float = 0.5, domain: Tuple[float, float] = (1.5, 0.6),
                               sound_speed: float = 50.0, dt: float = 3.0e-5, steps: int = 10_000,
                               n_frames: int = 100, frame_every: int = 10, n_track: int = 100,
                               alpha_true: float = 2.0, seed: int = 0, sort_every: int = 16,
                               checkpoint_every: int = 100) -> Workload:
    """Dam break whose initial horizontal velocity is unknown (Sec. 5.2).

    Water column H0 = L0 = ``column`` at the left wall of a ``domain`` box, 4
    particles per cell (2 per axis), inviscid, linear EOS with sound speed
    ``sound_speed`` (Tait gamma = 1, K = rho0 c^2).  True initial velocity
    v_x = alpha (H0 - y), v_y = 0.  Observations: the last n_frames x
    frame_every steps, every frame_every steps; tracked particles (n_track seeded,
    or every particle when n_track = 0) and nine velocity monitors, squares of
    half-side 0.01 m centred on {0.2, 0.3, 0.4} x {0.1, 0.2, 0.3} m.  At dx = 0.01
    this is 10,000 particles on a 150 x 60 grid; at dx = 0.005, 40,000 on 300 x 120.
    """
    n_cells = (int(round(domain[0] / dx)), int(round(domain[1] / dx)))
    x = lattice_particles(n_cells, dx, 2, lambda p: (p[:, 0] < column) & (p[:, 1] < column),
                          (0.0, 0.0), (column, column), seed)
    mat = dict(FLUID_WATER, bulk_K=1000.0 * sound_speed ** 2, gamma=1.0)
    w = Workload(name=f"dam_break_velocity_inverse_{n_cells[0]}x{n_cells[1]}", dim=2, n_cells=n_cells, dx=dx,
                 dt=dt, gravity=(0.0, -9.81), material=mat, x=x, particle_volume=dx * dx / 4, steps=steps,
                 sort_every=sort_every,
                 extras=dict(body_lo=(0.0, 0.0), body_hi=(column, column), seed=seed))
    w.v = velocity_profile_linear(x, alpha_true, column)
    obs_steps = [steps - (n_frames - 1 - k) * frame_every for k in range(n_frames)]
    ids = (np.arange(w.n, dtype=np.int64) if n_track == 0 else
           tracked_particles(x, n_track, seed, np.array((0.0, 0.0)), np.array((column, column))))
    monitors = [((cx - 0.01, cy - 0.01), (cx + 0.01, cy + 0.01)) for cy in (0.1, 0.2, 0.3) for cx in (0.2, 0.3, 0.4)]
    w.extras.update(H0=column, alpha_true=alpha_true, obs_steps=obs_steps, track_ids=ids, monitors=monitors,
                    checkpoint_every=checkpoint_every)
    return w


def velocity_profile_linear(x: np.ndarray, alpha: float, H0: float) -> np.ndarray:
    """v_x = alpha (H0 - y), v_y = 0 (Sec. 5.2)."""
    v = np.zeros_like(x)
    v[:, 0] = alpha * (H0 - x[:, 1])
    return v


def velocity_profile_field(y: np.ndarray, H0: float) -> np.ndarray:
    """The reference field of Sec. 5.2: 2 (1 - (y/H0)^2) + 0.2 sin(4 pi y / H0)."""
    return 2.0 * (1.0 - (y / H0) ** 2) + 0.2 * np.sin(4.0 * np.pi * y / H0)


def granular_inverse_3d(n_cells: Tuple[int, int, int] = (192, 192, 96), radius_cells: float = 30,
                        height_cells: float = 60, patches: Tuple[int, int] = (16, 16), n_track: int = 128,
                        n_obs: int = 10, steps: int = 600, seed: int = 0, checkpoint_every: int = 60,
                        dt: float = 1.0e-5, dx: float = 1.0 / 256.0) -> Workload:
    """Granular collapse with a patch-wise basal friction field and tracked particles.

    The 3D inverse problem: floor friction over patches x patches, drawn
    uniformly from [0.1, 0.6) by seed; n_track tracked particles observed at
    n_obs equally spaced steps.
    """
    w = granular_cylinder_3d(n_cells, radius_cells, height_cells, seed=seed, dt=dt, steps=steps, dx=dx,
                             floor_mu=0.0)
    w.name = f"granular_inverse_3d_{n_cells[0]}x{n_cells[1]}x{n_cells[2]}"
    mu = friction_field(patches[0] * patches[1], seed)
    w.friction = [(4, tuple(patches), mu)]
    ids = tracked_particles(w.x, n_track, seed, np.array(w.extras["body_lo"]), np.array(w.extras["body_hi"]))
    obs_steps = [steps * (k + 1) // n_obs for k in range(n_obs)]
    w.extras.update(track_ids=ids, obs_steps=obs_steps, mu_true=mu, checkpoint_every=checkpoint_every)
    return w


SAND_ALUMINIUM_BARS = dict(kind=1, rho0=2650.0, E=3.0 * 0.7e6 * (1.0 - 2.0 * 0.3), nu=0.3, phi_deg=19.8,
                          psi_deg=0.0, cohesion=0.0, sigma_t=0.0)
"""The Drucker-Prager material of the paper's granular benchmarks (Sec. 4.1.2 and
4.2.2): rho = 2650 kg/m^3, bulk modulus K = 0.7 MPa (E = 3K(1 - 2 nu)), nu = 0.3,
phi = 19.8 deg, psi = 0, c = 0."""


def granular_column_3d(aspect: float, length: float = 0.05, n_cells: Tuple[int, int, int] = (400, 32, 200),
                       dx: float = 1.0 / 400.0, ppc_axis: int = 2, seed: int = 0, dt: float = 1.0e-5,
                       steps: int = 200_000, base_mu: float = 1.0e6, sort_every: int = 32) -> Workload:
    """Quasi-2D granular column against the x- wall (Sec. 4.2.2): base length
    ``length`` (L0), height aspect * L0 (H0), across the whole y extent of the
    400 x 32 x 200 grid (dx = 1/400 m); slip side and far walls; the no-slip base
    taken as a Coulomb floor with mu = base_mu (a node pressed onto the base
    sticks)."""
    hgt = aspect * length
    x = lattice_particles(tuple(n_cells), dx, ppc_axis,
                          lambda p: (p[:, 0] < length) & (p[:, 2] < hgt),
                          (0.0, 0.0, 0.0), (length, n_cells[1] * dx, hgt), seed)
    return Workload(name=f"granular_column_3d_a{aspect:g}", dim=3, n_cells=tuple(n_cells), dx=dx, dt=dt,
                    gravity=(0.0, 0.0, -9.8), material=dict(SAND_ALUMINIUM_BARS), x=x,
                    particle_volume=dx ** 3 / ppc_axis ** 3, steps=steps, sort_every=sort_every,
                    friction=[(4, (1, 1), np.array([base_mu]))],
                    extras=dict(body_lo=(0.0, 0.0, 0.0), body_hi=(length, n_cells[1] * dx, hgt), seed=seed,
                                L0=length, H0=hgt, aspect=aspect))


WORKLOADS = {
    "dam_break_2d_64": lambda: dam_break_2d(64),
    "granular_cylinder_3d_256x256x128": lambda: granular_cylinder_3d(),
    "dam_break_inverse_2d_128": lambda: dam_break_inverse_2d(128),
    "granular_cylinder_3d_192x192x96": lambda: granular_cylinder_3d((192, 192, 96), 30, 60, steps=600),
    "granular_inverse_3d_192x192x96": lambda: granular_inverse_3d(),
    "dam_break_3d_200x100x80": lambda: dam_break_3d(),
    "dam_break_velocity_inverse_150x60": lambda: dam_break_velocity_inverse(),
}
