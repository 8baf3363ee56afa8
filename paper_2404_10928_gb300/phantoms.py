"""Seeded synthetic inputs: imaging geometries, phantoms and noise draws.

This module only *describes* problems.  It holds none of the reconstruction
arithmetic (no time of flight, no interpolation, no operator), so both the
CUDA path and the FP64 oracle can take their inputs from it without sharing
any of the method's code.

Conventions (shared by every consumer):

* The image is a point-sampled field on a regular grid.  Pixel (i, j, l) sits
  at ``origin + (i*dx, j*dy, l*dz)``; ``origin`` is the centre of pixel
  (0, 0, 0) and the generators centre the grid on the coordinate origin, i.e.
  ``origin = -(n-1)/2 * spacing`` per axis.
* Images are stored row-major as ``[nz][ny][nx]`` (x fastest); 2D problems
  have ``nz == 1``.
* Sensors are ``[S][dim]`` float64 positions in metres.
* Traces are ``[S][K]`` with sample k at time ``t0 + k/fs``.

The paper's murine-vascular frames (Sec. 4.1, 166 frames of 127x127 pixels) are
not available; the disk, vessel and vessel-tree phantoms below stand in for
them with the shapes of the workloads the paper's method is run on.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

SOUND_SPEED = 1500.0  # m/s, speed of sound in soft tissue (the "c" of Eq. 1)
SAMPLE_RATE = 40e6  # Hz


@dataclass
class Problem:
    """One imaging problem: grid, sensors, acquisition and a phantom."""

    dim: int
    shape: tuple  # (nx, ny, nz)
    spacing: tuple  # (dx, dy, dz) metres
    origin: tuple  # centre of pixel (0,0,0), metres, length 3
    sensors: np.ndarray  # [S][dim] float64
    c: float
    fs: float
    n_samples: int
    t0: float = 0.0
    amp_scale: float = 1.0
    x_true: Optional[np.ndarray] = None  # flat float64, length nx*ny*nz
    noise_unit: Optional[np.ndarray] = None  # [S][K] standard normal draws
    noise_level: float = 0.0
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n_pixels(self) -> int:
        nx, ny, nz = self.shape
        return nx * ny * nz

    @property
    def n_sensors(self) -> int:
        return int(self.sensors.shape[0])

    @property
    def pairs(self) -> int:
        """Pixel-sensor pairs evaluated by one application of A or its adjoint."""
        return self.n_pixels * self.n_sensors

    def pixel_axes(self):
        """Coordinates of pixel centres along x, y, z (float64 arrays)."""
        nx, ny, nz = self.shape
        dx, dy, dz = self.spacing
        ox, oy, oz = self.origin
        return (ox + dx * np.arange(nx), oy + dy * np.arange(ny), oz + dz * np.arange(nz))


def centred_origin(shape, spacing):
    return tuple(-(n - 1) / 2.0 * d for n, d in zip(shape, spacing))


# ----------------------------------------------------------------------------
# sensor geometries
# ----------------------------------------------------------------------------

def ring_sensors(n_sensors: int, radius: float) -> np.ndarray:
    """Full-view ring: sensor s at angle 2*pi*s/S on a circle about the origin."""
    th = 2.0 * np.pi * np.arange(n_sensors) / n_sensors
    return np.stack([radius * np.cos(th), radius * np.sin(th)], axis=1)


def linear_array(n_sensors: int, pitch: float, y: float) -> np.ndarray:
    """Linear array along x, centred laterally, at height y."""
    xs = (np.arange(n_sensors) - (n_sensors - 1) / 2.0) * pitch
    return np.stack([xs, np.full(n_sensors, y)], axis=1)


def planar_array(nx: int, ny: int, pitch: float, z: float) -> np.ndarray:
    """nx x ny planar array in the plane at height z, centred on the z axis."""
    xs = (np.arange(nx) - (nx - 1) / 2.0) * pitch
    ys = (np.arange(ny) - (ny - 1) / 2.0) * pitch
    gy, gx = np.meshgrid(ys, xs, indexing="ij")
    return np.stack([gx.ravel(), gy.ravel(), np.full(nx * ny, z)], axis=1)


def ring_radius_for(n: int, spacing: float) -> float:
    """Ring radius that keeps every sensor 2 mm outside the grid's corners."""
    return 0.5 * n * spacing * np.sqrt(2.0) + 2e-3


# ----------------------------------------------------------------------------
# phantoms
# ----------------------------------------------------------------------------

def _grid_points_2d(shape, spacing, origin):
    nx, ny, _ = shape
    xs = origin[0] + spacing[0] * np.arange(nx)
    ys = origin[1] + spacing[1] * np.arange(ny)
    gy, gx = np.meshgrid(ys, xs, indexing="ij")
    return gx, gy


def disk_phantom(shape, spacing, origin, rng, n_disks=5, r_range=(0.2e-3, 0.8e-3),
                 amp_range=(0.5, 1.0), inner=0.8) -> np.ndarray:
    """Disks with centres uniform over the inner 80% of the grid; overlaps take the max."""
    gx, gy = _grid_points_2d(shape, spacing, origin)
    half_x = 0.5 * inner * (shape[0] - 1) * spacing[0]
    half_y = 0.5 * inner * (shape[1] - 1) * spacing[1]
    img = np.zeros(gx.shape)
    for _ in range(n_disks):
        cx = rng.uniform(-half_x, half_x)
        cy = rng.uniform(-half_y, half_y)
        r = rng.uniform(*r_range)
        a = rng.uniform(*amp_range)
        inside = (gx - cx) ** 2 + (gy - cy) ** 2 <= r * r
        img = np.where(inside, np.maximum(img, a), img)
    return img.ravel()


def _bezier(ctrl: np.ndarray, n: int) -> np.ndarray:
    t = np.linspace(0.0, 1.0, n)[:, None]
    b0 = (1 - t) ** 3
    b1 = 3 * (1 - t) ** 2 * t
    b2 = 3 * (1 - t) * t ** 2
    b3 = t ** 3
    return b0 * ctrl[0] + b1 * ctrl[1] + b2 * ctrl[2] + b3 * ctrl[3]


def vessel_phantom(shape, spacing, origin, rng, n_tubes=12, width_range=(0.1e-3, 0.5e-3),
                   amp_range=(0.5, 1.0), samples=4096) -> np.ndarray:
    """Cubic Bezier tubes; control points uniform over the grid; overlaps take the max."""
    from scipy.spatial import cKDTree

    gx, gy = _grid_points_2d(shape, spacing, origin)
    pts = np.stack([gx.ravel(), gy.ravel()], axis=1)
    lo = np.array([origin[0], origin[1]])
    hi = lo + np.array([(shape[0] - 1) * spacing[0], (shape[1] - 1) * spacing[1]])
    img = np.zeros(pts.shape[0])
    for _ in range(n_tubes):
        ctrl = rng.uniform(lo, hi, size=(4, 2))
        w = rng.uniform(*width_range)
        a = rng.uniform(*amp_range)
        curve = _bezier(ctrl, samples)
        dist, _ = cKDTree(curve).query(pts, distance_upper_bound=w)
        inside = dist <= 0.5 * w
        img = np.where(inside, np.maximum(img, a), img)
    return img


def vessel_tree_phantom(shape, spacing, origin, rng, depth=5, r0=0.6e-3, r_min=0.2e-3,
                        shrink=0.8, amp_range=(0.5, 1.0)) -> np.ndarray:
    """3D branching tree of cylinders with radii shrinking from r0 towards r_min."""
    nx, ny, nz = shape
    dx, dy, dz = spacing
    ext = np.array([(nx - 1) * dx, (ny - 1) * dy, (nz - 1) * dz])
    lo = np.array(origin)
    img = np.zeros((nz, ny, nx))
    segs = []

    def grow(p, direction, radius, level):
        length = rng.uniform(0.15, 0.3) * ext.min()
        q = p + direction * length
        q = np.clip(q, lo, lo + ext)
        segs.append((p.copy(), q.copy(), radius, rng.uniform(*amp_range)))
        if level + 1 >= depth:
            return
        for _ in range(2):
            nd = direction + rng.normal(scale=0.6, size=3)
            nd /= np.linalg.norm(nd)
            grow(q, nd, max(r_min, radius * shrink), level + 1)

    start = lo + ext * np.array([rng.uniform(0.3, 0.7), rng.uniform(0.3, 0.7), 0.05])
    d0 = np.array([rng.normal(scale=0.2), rng.normal(scale=0.2), 1.0])
    grow(start, d0 / np.linalg.norm(d0), r0, 0)

    for p, q, r, a in segs:
        bmin = np.minimum(p, q) - r
        bmax = np.maximum(p, q) + r
        i0 = np.clip(np.floor((bmin - lo) / spacing).astype(int), 0, [nx - 1, ny - 1, nz - 1])
        i1 = np.clip(np.ceil((bmax - lo) / spacing).astype(int), 0, [nx - 1, ny - 1, nz - 1])
        xs = lo[0] + dx * np.arange(i0[0], i1[0] + 1)
        ys = lo[1] + dy * np.arange(i0[1], i1[1] + 1)
        zs = lo[2] + dz * np.arange(i0[2], i1[2] + 1)
        gz, gy, gx = np.meshgrid(zs, ys, xs, indexing="ij")
        v = q - p
        vv = max(float(v @ v), 1e-30)
        t = ((gx - p[0]) * v[0] + (gy - p[1]) * v[1] + (gz - p[2]) * v[2]) / vv
        t = np.clip(t, 0.0, 1.0)
        ddx = gx - (p[0] + t * v[0])
        ddy = gy - (p[1] + t * v[1])
        ddz = gz - (p[2] + t * v[2])
        inside = ddx * ddx + ddy * ddy + ddz * ddz <= r * r
        sub = img[i0[2]:i1[2] + 1, i0[1]:i1[1] + 1, i0[0]:i1[0] + 1]
        sub[...] = np.where(inside, np.maximum(sub, a), sub)
    return img.ravel()


def add_noise(p_clean: np.ndarray, noise_unit: np.ndarray, level: float) -> np.ndarray:
    """Gaussian noise with sigma = level * max|p_clean|, i.i.d. per sample."""
    return p_clean + level * np.max(np.abs(p_clean)) * noise_unit


def power_start(n_pixels: int, seed: int = 7) -> np.ndarray:
    """Start vector of the power iteration (seeded standard normal)."""
    return np.random.default_rng(seed).standard_normal(n_pixels)


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

def linear_array_disks(seed: int = 1001) -> Problem:
    """2D 64x64, 0.1 mm pixels; 64-element linear array (0.2 mm pitch) 2 mm above
    the grid's outer edge; 512 samples at 40 MHz; five random disks."""
    rng = np.random.default_rng(seed)
    shape, spacing = (64, 64, 1), (1e-4, 1e-4, 1e-4)
    origin = centred_origin(shape, spacing)
    edge = 0.5 * shape[1] * spacing[1]
    sensors = linear_array(64, 0.2e-3, edge + 2e-3)
    x = disk_phantom(shape, spacing, origin, rng)
    return Problem(2, shape, spacing, origin, sensors, SOUND_SPEED, SAMPLE_RATE, 512,
                   x_true=x, name="2d-64x64-linear64-k512-disks",
                   extra={"method": "landweber", "n_iter": 10})


def ring_vessels(seed: int = 1002) -> Problem:
    """2D 256x256, 0.1 mm pixels; 256-element full-view ring of radius 20 mm;
    2048 samples at 40 MHz; Bezier vessel phantom; 1% Gaussian noise on traces."""
    rng = np.random.default_rng(seed)
    shape, spacing = (256, 256, 1), (1e-4, 1e-4, 1e-4)
    origin = centred_origin(shape, spacing)
    sensors = ring_sensors(256, 20e-3)
    x = vessel_phantom(shape, spacing, origin, rng)
    noise = np.random.default_rng(seed + 1).standard_normal((256, 2048))
    return Problem(2, shape, spacing, origin, sensors, SOUND_SPEED, SAMPLE_RATE, 2048,
                   x_true=x, noise_unit=noise, noise_level=0.01,
                   name="2d-256x256-ring256-k2048-vessels", extra={"method": "cgls", "n_iter": 50})


def ring_vessels_batch(seed: int = 1003, batch: int = 8) -> List[Problem]:
    """Batch of 2D 256x256 vessel images seen by a 128-element ring, 2048 samples;
    the traces are generated with c = 1540 m/s and the fit starts from 1500 m/s."""
    rng = np.random.default_rng(seed)
    shape, spacing = (256, 256, 1), (1e-4, 1e-4, 1e-4)
    origin = centred_origin(shape, spacing)
    sensors = ring_sensors(128, ring_radius_for(256, 1e-4))
    out = []
    for b in range(batch):
        x = vessel_phantom(shape, spacing, origin, rng)
        out.append(Problem(2, shape, spacing, origin, sensors, SOUND_SPEED, SAMPLE_RATE, 2048,
                           x_true=x, name=f"2d-256x256-ring128-k2048-vessels[{b}]",
                           extra={"c_true": 1540.0, "c_init": 1500.0, "n_iter": 10}))
    return out


def ragged_time_series(seed: int = 1004, n_frames: int = 64) -> List[Problem]:
    """Frames of uneven size: grid from {128,192,256,384,512}^2, 128-512 ring sensors,
    1024-4096 samples at 40 MHz; the measured traces are stored as FP16."""
    rng = np.random.default_rng(seed)
    sizes = [128, 192, 256, 384, 512]
    out = []
    for f in range(n_frames):
        n = int(rng.choice(sizes))
        s = int(rng.integers(128, 513))
        k = int(rng.integers(1024, 4097))
        shape, spacing = (n, n, 1), (1e-4, 1e-4, 1e-4)
        origin = centred_origin(shape, spacing)
        sensors = ring_sensors(s, ring_radius_for(n, 1e-4))
        x = vessel_phantom(shape, spacing, origin, rng, samples=2048)
        out.append(Problem(2, shape, spacing, origin, sensors, SOUND_SPEED, SAMPLE_RATE, k,
                           x_true=x, name=f"2d-{n}x{n}-ring{s}-k{k}[{f}]",
                           extra={"method": "landweber", "n_iter": 20, "y_dtype": "f16"}))
    return out


def planar_vessel_tree(seed: int = 1005, n: int = 128) -> Problem:
    """3D n^3 voxels at 0.2 mm; 32x32 planar array at 0.8 mm pitch 5 mm from the
    volume's top face; 1024 samples at 40 MHz; seeded 3D vessel tree."""
    rng = np.random.default_rng(seed)
    shape, spacing = (n, n, n), (2e-4, 2e-4, 2e-4)
    origin = centred_origin(shape, spacing)
    face = 0.5 * n * spacing[2]
    sensors = planar_array(32, 32, 0.8e-3, face + 5e-3)
    x = vessel_tree_phantom(shape, spacing, origin, rng)
    return Problem(3, shape, spacing, origin, sensors, SOUND_SPEED, SAMPLE_RATE, 1024,
                   x_true=x, name=f"3d-{n}^3-planar32x32-k1024-tree",
                   extra={"method": "cgls", "n_iter": 30})


def dense_paper_size(seed: int = 1006) -> Problem:
    """The size of the paper's dense measurement matrix (Sec. 4, Table 4:
    6144 x 16384): a 128x128 frame at 0.1 mm and 6144 = 48 sensors x 128
    samples -- a 48-element ring of radius 10 mm sampled at 10 MHz (the paper
    does not give the split); Bezier vessel phantom."""
    rng = np.random.default_rng(seed)
    shape, spacing = (128, 128, 1), (1e-4, 1e-4, 1e-4)
    origin = centred_origin(shape, spacing)
    sensors = ring_sensors(48, 10e-3)
    x = vessel_phantom(shape, spacing, origin, rng)
    return Problem(2, shape, spacing, origin, sensors, SOUND_SPEED, 10e6, 128, x_true=x,
                   name="2d-128x128-ring48-k128-10MHz-dense")


def custom(dim: int, shape: Sequence[int], spacing: Sequence[float], sensors: np.ndarray,
           n_samples: int, seed: int, c: float = SOUND_SPEED, fs: float = SAMPLE_RATE,
           density: float = 0.3, t0: float = 0.0, amp_scale: float = 1.0) -> Problem:
    """Small problem with a seeded random non-negative image (for edge-case tests)."""
    rng = np.random.default_rng(seed)
    shape = tuple(shape) + (1,) * (3 - len(shape))
    spacing = tuple(spacing) + (spacing[-1],) * (3 - len(spacing))
    origin = centred_origin(shape, spacing)
    n = shape[0] * shape[1] * shape[2]
    x = rng.uniform(0.0, 1.0, n) * (rng.uniform(0.0, 1.0, n) < density)
    return Problem(dim, shape, spacing, origin, np.asarray(sensors, dtype=np.float64), c, fs,
                   n_samples, t0=t0, amp_scale=amp_scale, x_true=x, name=f"custom-{dim}d-{shape}")
