"""Seeded synthetic inputs shared by the CUDA path's tests/benchmarks and the oracle's tests.

This module holds no operator arithmetic: only geometry (grids, sensor caps), phantoms
(spheres, vessel trees, blobs, free Gaussians), measurement noise and a band-limiting filter
applied to measured signals.  Every generator takes an explicit seed.

The workloads stand in for the paper's simulation and in-vivo data, which are not available:
a 3-D vascular network imaged by hemispherical / limited-view arrays of 64-1024 point
sensors (Results, "Validation on synthetic vascular data" and "in vivo" sections), with
the reconstruction grid 256 x 256 x 128 and 1024 detectors of the in-vivo studies.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SOUND_SPEED = 1500.0   # m/s
FS = 40e6              # Hz


@dataclass
class Grid:
    """Regular grid of Gaussian centres: centre of node (ix, iy, iz) is o + (idx + 1/2) h,
    x fastest.  sigma is the shared Gaussian width (Methods: sigma equals the grid size)."""
    nx: int
    ny: int
    nz: int
    h: float
    sigma: float
    ox: float = 0.0
    oy: float = 0.0
    oz: float = 0.0

    @property
    def M(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape_zyx(self):
        return (self.nz, self.ny, self.nx)

    def centres(self) -> np.ndarray:
        """(M, 3) float64 node centres in x-fastest order."""
        iz, iy, ix = np.meshgrid(np.arange(self.nz), np.arange(self.ny), np.arange(self.nx), indexing="ij")
        f = lambda q: float(np.float32(q))
        return np.stack([f(self.ox) + (ix.ravel() + 0.5) * f(self.h),
                         f(self.oy) + (iy.ravel() + 0.5) * f(self.h),
                         f(self.oz) + (iz.ravel() + 0.5) * f(self.h)], axis=1)


def centred_grid(nx, ny, nz, h, sigma=None, centre=(0.0, 0.0, 0.0)) -> Grid:
    """Grid whose bounding box is centred on `centre` (the array's centre of curvature)."""
    return Grid(nx, ny, nz, float(h), float(sigma if sigma is not None else h),
                ox=centre[0] - nx * h / 2, oy=centre[1] - ny * h / 2, oz=centre[2] - nz * h / 2)


def cap_sensors(n: int, radius: float, opening_deg: float, centre=(0.0, 0.0, 0.0)) -> np.ndarray:
    """n point sensors evenly spread over a spherical cap of the given radius and full opening
    angle, centred on `centre` and facing -z (the cap lies below the volume).  Area-uniform
    golden-angle spiral: cos(theta_i) uniform in [cos(opening/2), 1].  Returns (n, 3) float32."""
    th_max = math.radians(opening_deg) / 2.0
    i = np.arange(n, dtype=np.float64)
    cos_t = 1.0 - (1.0 - math.cos(th_max)) * (i + 0.5) / n
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t ** 2))
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    xyz = np.stack([radius * sin_t * np.cos(phi), radius * sin_t * np.sin(phi), -radius * cos_t], 1)
    return (xyz + np.asarray(centre, dtype=np.float64)).astype(np.float32)


def spheres_phantom(grid: Grid, n_spheres: int, r_range, v_range, seed: int) -> np.ndarray:
    """Amplitudes (M,) float32: union of n random balls (radius U[r_range], value U[v_range]);
    overlapping balls keep the larger value."""
    rng = np.random.default_rng(seed)
    c = grid.centres()
    lo, hi = c.min(0), c.max(0)
    A = np.zeros(grid.M)
    for _ in range(n_spheres):
        r = rng.uniform(*r_range)
        val = rng.uniform(*v_range)
        ctr = rng.uniform(lo + 0.25 * (hi - lo), hi - 0.25 * (hi - lo))
        inside = np.sum((c - ctr) ** 2, axis=1) <= r * r
        A[inside] = np.maximum(A[inside], val)
    return A.astype(np.float32)


def _rasterise_capsule(A, grid: Grid, p0, p1, radius, val):
    h = grid.h
    org = np.array([grid.ox, grid.oy, grid.oz])
    lo = np.floor((np.minimum(p0, p1) - radius - org) / h - 0.5).astype(int)
    hi = np.ceil((np.maximum(p0, p1) + radius - org) / h - 0.5).astype(int)
    dims = np.array([grid.nx, grid.ny, grid.nz])
    lo = np.clip(lo, 0, dims - 1)
    hi = np.clip(hi, 0, dims - 1)
    if np.any(hi < lo):
        return
    ix = np.arange(lo[0], hi[0] + 1)
    iy = np.arange(lo[1], hi[1] + 1)
    iz = np.arange(lo[2], hi[2] + 1)
    Z, Y, X = np.meshgrid(iz, iy, ix, indexing="ij")
    P = np.stack([org[0] + (X + 0.5) * h, org[1] + (Y + 0.5) * h, org[2] + (Z + 0.5) * h], -1)
    seg = p1 - p0
    L2 = float(seg @ seg) or 1e-30
    tpar = np.clip(((P - p0) @ seg) / L2, 0.0, 1.0)
    dist2 = np.sum((P - (p0 + tpar[..., None] * seg)) ** 2, -1)
    mask = dist2 <= radius * radius
    flat = (Z * grid.ny + Y) * grid.nx + X
    idx = flat[mask]
    A[idx] = np.maximum(A[idx], val)


def vessel_tree_phantom(grid: Grid, seed: int, r_range=(50e-6, 300e-6), n_roots=3,
                        max_segments=400, blob_count=0, blob_r=(100e-6, 300e-6)) -> np.ndarray:
    """Amplitudes (M,) float32 of a random branching vessel tree: cylinders (capsules) with
    radius shrinking from r_range[1] towards r_range[0] at each branching, each segment with
    a log-normal intensity (median 1, shape 0.4), plus `blob_count` sparse balls."""
    rng = np.random.default_rng(seed)
    A = np.zeros(grid.M)
    ext = np.array([grid.nx, grid.ny, grid.nz]) * grid.h
    org = np.array([grid.ox, grid.oy, grid.oz])
    seg_len = 0.12 * float(np.min(ext[:2]))
    stack = []
    for _ in range(n_roots):
        p = org + ext * rng.uniform([0.1, 0.1, 0.3], [0.9, 0.9, 0.7])
        d = rng.normal(size=3)
        d[2] *= 0.3
        d /= np.linalg.norm(d)
        stack.append((p, d, r_range[1]))
    n = 0
    while stack and n < max_segments:
        p, d, r = stack.pop(0)
        L = seg_len * rng.uniform(0.6, 1.4)
        q = p + d * L
        q = np.clip(q, org + 0.02 * ext, org + 0.98 * ext)
        val = float(np.exp(rng.normal(0.0, 0.4)))
        _rasterise_capsule(A, grid, p, q, max(r, r_range[0]), val)
        n += 1
        if r <= r_range[0] * 1.05:
            continue
        nb = 2 if rng.uniform() < 0.6 else 1
        for _ in range(nb):
            nd = d + rng.normal(scale=0.6, size=3)
            nd[2] *= 0.5
            nd /= np.linalg.norm(nd)
            stack.append((q, nd, max(r_range[0], r * rng.uniform(0.6, 0.85))))
    for _ in range(blob_count):
        ctr = org + ext * rng.uniform(0.05, 0.95, size=3)
        _rasterise_capsule(A, grid, ctr, ctr, rng.uniform(*blob_r), float(np.exp(rng.normal(0.0, 0.4))))
    return A.astype(np.float32)


def free_gaussians(grid: Grid, seed: int, jitter=0.05e-3, sigma_range=(0.05e-3, 0.2e-3), A=None):
    """Free Gaussians on a jittered grid: centres = node centre + U[-jitter, jitter] per axis,
    sigma log-uniform in sigma_range.  Returns float32 (cx, cy, cz, sigma, A)."""
    rng = np.random.default_rng(seed)
    c = grid.centres() + rng.uniform(-jitter, jitter, size=(grid.M, 3))
    sig = np.exp(rng.uniform(math.log(sigma_range[0]), math.log(sigma_range[1]), size=grid.M))
    if A is None:
        A = rng.uniform(0.0, 1.0, size=grid.M)
    f = lambda q: np.ascontiguousarray(q, dtype=np.float32)
    return f(c[:, 0]), f(c[:, 1]), f(c[:, 2]), f(sig), f(A)


def add_noise(y: np.ndarray, snr_db: float, seed: int) -> np.ndarray:
    """White Gaussian noise at a global SNR: noise variance = mean(y^2) / 10^(snr/10)."""
    rng = np.random.default_rng(seed)
    var = float(np.mean(np.asarray(y, dtype=np.float64) ** 2)) / (10.0 ** (snr_db / 10.0))
    return (y + rng.normal(scale=math.sqrt(var), size=y.shape)).astype(np.float32)


def bandlimit(y: np.ndarray, fs: float, f_lo: float, f_hi: float, order: int = 4) -> np.ndarray:
    """Zero-phase band-pass of each row: magnitude of an order-n Butterworth high-pass at f_lo
    times a low-pass at f_hi, applied through the real FFT."""
    y = np.asarray(y, dtype=np.float64)
    n = y.shape[-1]
    f = np.fft.rfftfreq(n, 1.0 / fs)
    hp = np.where(f > 0, (f / f_lo) ** order / np.sqrt(1.0 + (f / f_lo) ** (2 * order)), 0.0)
    lp = 1.0 / np.sqrt(1.0 + (f / f_hi) ** (2 * order))
    return np.fft.irfft(np.fft.rfft(y, axis=-1) * (hp * lp), n=n, axis=-1).astype(np.float32)


@dataclass
class Workload:
    """One seeded synthetic workload: Gaussian set, sensor array and acquisition."""
    name: str
    grid: Grid
    sensors: np.ndarray             # (Nd, 3) float32
    Nt: int
    A: np.ndarray | None = None     # (M,) float32 amplitudes (grid mode)
    free: tuple | None = None       # (cx, cy, cz, sigma, A) float32 (free-centre mode)
    v: float = SOUND_SPEED
    fs: float = FS
    t0: float = 0.0
    k: float = 3.0
    meta: dict = field(default_factory=dict)

    @property
    def Nd(self) -> int:
        return int(self.sensors.shape[0])

    @property
    def M(self) -> int:
        return self.grid.M


def tiny(seed: int = 1) -> Workload:
    """16^3 Gaussians on a 0.2 mm grid, sigma 0.2 mm, 3 random balls (r 0.5-1 mm, U[0.5, 1]);
    128 sensors on a hemispherical cap of radius 20 mm; 1024 samples at 40 MHz."""
    g = centred_grid(16, 16, 16, 0.2e-3)
    A = spheres_phantom(g, 3, (0.5e-3, 1.0e-3), (0.5, 1.0), seed)
    return Workload("tiny-16^3-128x1024", g, cap_sensors(128, 20e-3, 180.0), 1024, A=A)


def mid(seed: int = 2) -> Workload:
    """128x128x64 Gaussians on a 0.1 mm grid, vessel tree; 1024 sensors on a 120-degree cap of
    radius 60 mm; 4096 samples."""
    g = centred_grid(128, 128, 64, 0.1e-3)
    A = vessel_tree_phantom(g, seed, n_roots=6, max_segments=1200)
    return Workload("mid-128x128x64-1024x4096", g, cap_sensors(1024, 60e-3, 120.0), 4096, A=A,
                    meta={"bandlimit": (0.5e6, 10e6)})


def paper_scale(seed: int = 3) -> Workload:
    """256x256x128 = 8.4M Gaussians on a 0.1 mm grid, vessel tree plus sparse blobs; 1024
    sensors on a 140-degree cap of radius 80 mm; 4096 samples (the in-vivo grid and array size
    of the paper's Table 2)."""
    g = centred_grid(256, 256, 128, 0.1e-3)
    A = vessel_tree_phantom(g, seed, n_roots=10, max_segments=2500, blob_count=200)
    return Workload("paper-256x256x128-1024x4096", g, cap_sensors(1024, 80e-3, 140.0), 4096, A=A)


def differentiable(seed: int = 4) -> Workload:
    """262,144 free Gaussians (64^3 jittered by U[-0.05, 0.05] mm, sigma log-U[0.05, 0.2] mm);
    512 sensors on a hemispherical cap of radius 40 mm; 2048 samples."""
    g = centred_grid(64, 64, 64, 0.1e-3)
    phantom = vessel_tree_phantom(g, seed + 1, n_roots=2, max_segments=120)
    free = free_gaussians(g, seed, A=phantom)
    return Workload("diff-64^3-free-512x2048", g, cap_sensors(512, 40e-3, 180.0), 2048, free=free)


def subset_workload(w: Workload, sensors_idx) -> Workload:
    """Same Gaussians and acquisition with a subset of the sensors."""
    return Workload(w.name + f"-sub{len(sensors_idx)}", w.grid, np.ascontiguousarray(w.sensors[sensors_idx]),
                    w.Nt, A=w.A, free=w.free, v=w.v, fs=w.fs, t0=w.t0, k=w.k, meta=dict(w.meta))
