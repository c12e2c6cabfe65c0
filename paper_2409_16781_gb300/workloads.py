"""Seeded synthetic inputs for the D3Q19 lattice workloads.

This module builds the inputs that both the CUDA library and the CPU oracle
are run on: flag fields (uint8 per cell, x fastest), initial density and
velocity fields, and the request stream of the serving workload.  It holds
none of the lattice-Boltzmann arithmetic itself (no velocity set, no
equilibrium, no collision), so the two implementations under comparison share
only their inputs.

Arrays use the layout of the library: a scalar field is (nz, ny, nx), a vector
field is (3, nz, ny, nx), cell index x + nx*(y + ny*z).  Flag values: 0 fluid,
1 wall (no-slip bounce-back), 2 lid (bounce-back from a wall moving at u_lid),
3 far field (the free stream moving at u_lid: inflow / outflow planes).

The workloads stand in for the paper's use cases (arXiv 2409.16781 Sec. 3.3:
lid-driven cavity, Taylor-Green vortex, flow past an obstacle), extended to 3D.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FLUID, WALL, LID, FARFIELD = 0, 1, 2, 3
_MASK64 = (1 << 64) - 1


# --------------------------------------------------------------------------
# SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
# generators", OOPSLA 2014): a counter-based 64-bit generator, used so that the
# porous geometry is defined by a published stream rather than by a library's
# internal generator.
# --------------------------------------------------------------------------
class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform real in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


# --------------------------------------------------------------------------
# Flag fields
# --------------------------------------------------------------------------
def all_fluid(nx: int, ny: int, nz: int) -> np.ndarray:
    return np.zeros((nz, ny, nx), dtype=np.uint8)


def cavity_flags(nx: int, ny: int, nz: int) -> np.ndarray:
    """Lid-driven cavity: the outer layer of cells is solid; every cell of the
    top plane z = nz-1 (edges and corners included) is LID, every other
    boundary cell is WALL.  Interior (nx-2)(ny-2)(nz-2) cells are fluid."""
    f = np.zeros((nz, ny, nx), dtype=np.uint8)
    f[0, :, :] = WALL
    f[:, 0, :] = WALL
    f[:, ny - 1, :] = WALL
    f[:, :, 0] = WALL
    f[:, :, nx - 1] = WALL
    f[nz - 1, :, :] = LID
    return f


def channel_flags(nx: int, ny: int, nz: int, walls=("y",)) -> np.ndarray:
    """Periodic channel: bounce-back walls on both faces of the listed axes."""
    f = np.zeros((nz, ny, nx), dtype=np.uint8)
    if "x" in walls:
        f[:, :, 0] = WALL
        f[:, :, nx - 1] = WALL
    if "y" in walls:
        f[:, 0, :] = WALL
        f[:, ny - 1, :] = WALL
    if "z" in walls:
        f[0, :, :] = WALL
        f[nz - 1, :, :] = WALL
    return f


def cylinder_flags(nx: int, ny: int, nz: int, diameter: float, cx: float, cy: float) -> np.ndarray:
    """Flow past a cylinder (the paper's von Karman street use case, in 3D):
    a cylinder along z of the given diameter centred at (cx, cy) -- cell
    (x, y, z) solid when (x - cx)^2 + (y - cy)^2 <= (diameter/2)^2 -- with
    FARFIELD planes at x = 0 and x = nx-1 (inflow and outflow held at the
    free stream) and periodic y and z (an unconfined cylinder, repeated
    every ny cells)."""
    f = np.zeros((nz, ny, nx), dtype=np.uint8)
    yy, xx = np.mgrid[0:ny, 0:nx]
    r = 0.5 * diameter
    f[:, (xx - cx) ** 2 + (yy - cy) ** 2 <= r * r] = WALL
    f[:, :, 0] = FARFIELD
    f[:, :, nx - 1] = FARFIELD
    return f


@dataclass
class Sphere:
    cx: float
    cy: float
    cz: float
    r: float


def porous_spheres(nx: int, ny: int, nz: int, n_spheres: int = 400,
                   r_min: float = 8.0, r_max: float = 24.0, seed: int = 2409):
    """Sphere centres uniform in [0,n) per axis and radii uniform in
    [r_min, r_max], drawn in the order (cx, cy, cz, r) per sphere from one
    SplitMix64 stream seeded with ``seed``."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(n_spheres):
        cx = rng.uniform() * nx
        cy = rng.uniform() * ny
        cz = rng.uniform() * nz
        r = r_min + (r_max - r_min) * rng.uniform()
        out.append(Sphere(cx, cy, cz, r))
    return out


def porous_flags(nx: int, ny: int, nz: int, n_spheres: int = 400,
                 r_min: float = 8.0, r_max: float = 24.0, seed: int = 2409) -> np.ndarray:
    """Porous channel: periodic in x, WALL planes at y = 0, ny-1 and
    z = 0, nz-1, and cell (x,y,z) solid when (x-cx)^2+(y-cy)^2+(z-cz)^2 <= r^2
    for some sphere (cell centres at integer coordinates, no wrap; spheres
    clip at the domain edge)."""
    f = channel_flags(nx, ny, nz, walls=("y", "z"))
    for s in porous_spheres(nx, ny, nz, n_spheres, r_min, r_max, seed):
        x0, x1 = max(0, math.ceil(s.cx - s.r)), min(nx - 1, math.floor(s.cx + s.r))
        y0, y1 = max(0, math.ceil(s.cy - s.r)), min(ny - 1, math.floor(s.cy + s.r))
        z0, z1 = max(0, math.ceil(s.cz - s.r)), min(nz - 1, math.floor(s.cz + s.r))
        if x0 > x1 or y0 > y1 or z0 > z1:
            continue
        zz, yy, xx = np.meshgrid(np.arange(z0, z1 + 1), np.arange(y0, y1 + 1),
                                 np.arange(x0, x1 + 1), indexing="ij")
        inside = (xx - s.cx) ** 2 + (yy - s.cy) ** 2 + (zz - s.cz) ** 2 <= s.r * s.r
        sub = f[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1]
        sub[inside] = WALL
    return f


def random_flags(nx: int, ny: int, nz: int, seed: int, p_wall: float = 0.2,
                 p_lid: float = 0.1) -> np.ndarray:
    """Independent random flags per cell (for small parity grids)."""
    rng = np.random.default_rng(seed)
    r = rng.random((nz, ny, nx))
    f = np.zeros((nz, ny, nx), dtype=np.uint8)
    f[r < p_wall + p_lid] = LID
    f[r < p_wall] = WALL
    return f


# --------------------------------------------------------------------------
# Initial fields
# --------------------------------------------------------------------------
def taylor_green_fields(nx: int, ny: int, nz: int, u0: float = 0.05):
    """3D Taylor-Green vortex, wavenumber 2*pi/n on each axis:
    u = u0 ( sin kx cos ky cos kz, -cos kx sin ky cos kz, 0 ), rho = 1."""
    kx, ky, kz = 2 * math.pi / nx, 2 * math.pi / ny, 2 * math.pi / nz
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny)[None, :, None]
    z = np.arange(nz)[:, None, None]
    u = np.zeros((3, nz, ny, nx))
    u[0] = u0 * np.sin(kx * x) * np.cos(ky * y) * np.cos(kz * z)
    u[1] = -u0 * np.cos(kx * x) * np.sin(ky * y) * np.cos(kz * z)
    rho = np.ones((nz, ny, nx))
    return rho, u


def random_fields(nx: int, ny: int, nz: int, seed: int, du: float = 0.05,
                  drho: float = 0.02):
    """Small random density and velocity perturbations (parity inputs)."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + drho * (rng.random((nz, ny, nx)) - 0.5)
    u = du * (rng.random((3, nz, ny, nx)) - 0.5)
    return rho, u


def random_populations(nx: int, ny: int, nz: int, seed: int, w=None, amp: float = 0.01):
    """A random post-collision state (19, nz, ny, nx): w_i + amp*noise.  The
    weights are passed in by the caller (this module holds no velocity set);
    with w=None the base is a flat 1/19."""
    rng = np.random.default_rng(seed)
    base = np.full(19, 1.0 / 19) if w is None else np.asarray(w, dtype=np.float64)
    return base[:, None, None, None] + amp * (rng.random((19, nz, ny, nx)) - 0.5)


# --------------------------------------------------------------------------
# Serving workload: a seeded Poisson stream of simulation requests
# --------------------------------------------------------------------------
@dataclass
class Request:
    rid: int
    arrival_s: float
    nx: int
    ny: int
    nz: int
    tau: float
    steps: int
    kind: str          # "cavity" or "channel"
    storage: str       # "f32" or "f16s"
    u_lid: tuple = (0.05, 0.0, 0.0)
    force: tuple = (0.0, 0.0, 0.0)
    extra: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def flags(self) -> np.ndarray:
        """The request's geometry (built once, then kept with the request)."""
        f = self.extra.get("flags")
        if f is None:
            if self.kind == "cavity":
                f = cavity_flags(self.nx, self.ny, self.nz)
            else:
                f = channel_flags(self.nx, self.ny, self.nz, walls=("y", "z"))
            self.extra["flags"] = f
        return f


def request_stream(n: int = 2000, rate_hz: float = 10.0, seed: int = 16781,
                   min_cells: int = 16 ** 3, max_cells: int = 192 ** 3,
                   max_aspect: float = 4.0, tau_range=(0.52, 1.0),
                   steps_range=(200, 5000)):
    """Seeded stream of cavity/channel requests: Poisson arrivals at rate_hz,
    cell counts log-uniform in [min_cells, max_cells], aspect ratio: two
    log-factors uniform in [-ln 4, ln 4], redrawn until max/min edge <= 4,
    tau uniform, steps uniform integers, kind and storage 50/50."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    lo, hi = math.log(min_cells), math.log(max_cells)
    for rid in range(n):
        t += rng.exponential(1.0 / rate_hz)
        cells = math.exp(rng.uniform(lo, hi))
        while True:
            a = rng.uniform(-math.log(max_aspect), math.log(max_aspect))
            b = rng.uniform(-math.log(max_aspect), math.log(max_aspect))
            # edges proportional to (e^a, e^b, 1) scaled to the cell count
            s = (cells / math.exp(a + b)) ** (1.0 / 3.0)
            dims = [max(4, round(s * math.exp(a))), max(4, round(s * math.exp(b))),
                    max(4, round(s))]
            if max(dims) / min(dims) <= max_aspect:
                break
        tau = rng.uniform(*tau_range)
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        kind = "cavity" if rng.random() < 0.5 else "channel"
        storage = "f32" if rng.random() < 0.5 else "f16s"
        force = (0.0, 0.0, 0.0) if kind == "cavity" else (1e-6, 0.0, 0.0)
        u_lid = (0.05, 0.0, 0.0) if kind == "cavity" else (0.0, 0.0, 0.0)
        out.append(Request(rid, t, dims[0], dims[1], dims[2], tau, steps, kind,
                           storage, u_lid, force))
    return out
