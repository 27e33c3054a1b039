"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generation only -- no k-means arithmetic -- so both
the CUDA path and the FP64 oracle can be fed the same arrays.  The paper's
own datasets (T-drive, Porto, Argo-AVL trajectories; Argo-PC, 3D-RD,
ShapeNet point clouds; Section VI, Table "datasets") are not available, so
these recipes stand in for them:

  geo2d-blobs   2D mixture of isotropic Gaussians (small parity gate)
  geo2d-roads   2D points jittered along random polylines plus uniform noise
                (road-network-like GPS points, coordinates up to 1e5)
  lidar3d       3D ground plane plus the surfaces of random boxes / spheres
                (LiDAR-like point cloud)
  batched3d     many uneven 3D Gaussian-mixture clouds
  soft3d        equal-size 3D Gaussian-mixture clouds for the
                differentiable loss

All coordinates are drawn in FP64 and rounded to float32 once.  Every
generator is a pure function of (sizes, seed): numpy PCG64.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Workload:
    name: str
    points: np.ndarray            # (n, d) float32
    init: np.ndarray              # (k, d) float32, rows of points
    k: int
    max_iter: int
    early_stop: bool
    seed: int
    recipe: str
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.points.shape[0])

    @property
    def d(self) -> int:
        return int(self.points.shape[1])


def init_from_permutation(points: np.ndarray, k: int, rng: np.random.Generator) -> np.ndarray:
    """Initial centroids = the first k points of a seeded permutation."""
    idx = rng.permutation(points.shape[0])[:k]
    return np.ascontiguousarray(points[idx].astype(np.float32))


def gaussian_blobs_2d(n: int, n_blobs: int, rng: np.random.Generator,
                      lo: float = 0.0, hi: float = 1000.0,
                      sigma_lo: float = 5.0, sigma_hi: float = 20.0) -> np.ndarray:
    centres = rng.uniform(lo, hi, size=(n_blobs, 2))
    sig = rng.uniform(sigma_lo, sigma_hi, size=n_blobs)
    which = rng.integers(0, n_blobs, size=n)           # equal mixture weights
    pts = centres[which] + rng.standard_normal((n, 2)) * sig[which, None]
    return np.ascontiguousarray(pts.astype(np.float32))


def polylines_2d(n: int, n_lines: int, rng: np.random.Generator, extent: float = 1.0e5,
                 jitter: float = 15.0, noise_frac: float = 0.05,
                 seg_lo: int = 5, seg_hi: int = 20,
                 len_lo: float = 1.0e3, len_hi: float = 1.0e4) -> np.ndarray:
    """Road-network-like GPS points: jittered samples along random polylines."""
    segs_a, segs_b = [], []
    for _ in range(n_lines):
        m = int(rng.integers(seg_lo, seg_hi + 1))
        p = rng.uniform(0.0, extent, size=2)
        for _s in range(m):
            ang = rng.uniform(0.0, 2.0 * np.pi)
            ln = rng.uniform(len_lo, len_hi)
            q = np.clip(p + ln * np.array([np.cos(ang), np.sin(ang)]), 0.0, extent)
            segs_a.append(p)
            segs_b.append(q)
            p = q
    A = np.asarray(segs_a)
    B = np.asarray(segs_b)
    L = np.linalg.norm(B - A, axis=1) + 1e-9
    n_noise = int(round(noise_frac * n))
    n_line = n - n_noise
    which = rng.choice(A.shape[0], size=n_line, p=L / L.sum())   # points per length
    t = rng.uniform(0.0, 1.0, size=n_line)[:, None]
    on = A[which] + t * (B[which] - A[which]) + rng.standard_normal((n_line, 2)) * jitter
    noise = rng.uniform(0.0, extent, size=(n_noise, 2))
    pts = np.concatenate([on, noise], axis=0)
    pts = pts[rng.permutation(n)]
    return np.ascontiguousarray(pts.astype(np.float32))


def lidar_3d(n: int, n_objects: int, rng: np.random.Generator, half: float = 100.0,
             ground_frac: float = 0.6, ground_sigma: float = 0.05,
             size_lo: float = 0.5, size_hi: float = 10.0) -> np.ndarray:
    """Ground plane z~N(0, sigma) over [-half, half]^2 plus points sampled
    area-uniformly on the surfaces of random boxes and spheres resting on z=0."""
    n_ground = int(round(ground_frac * n))
    n_obj = n - n_ground
    g = np.empty((n_ground, 3))
    g[:, 0:2] = rng.uniform(-half, half, size=(n_ground, 2))
    g[:, 2] = rng.standard_normal(n_ground) * ground_sigma
    is_box = rng.uniform(size=n_objects) < 0.5
    ctr = rng.uniform(-half, half, size=(n_objects, 2))
    size = rng.uniform(size_lo, size_hi, size=(n_objects, 3))
    radius = 0.5 * size[:, 0]
    area = np.where(is_box,
                    2.0 * (size[:, 0] * size[:, 1] + size[:, 0] * size[:, 2]
                           + size[:, 1] * size[:, 2]),
                    4.0 * np.pi * radius ** 2)
    which = rng.choice(n_objects, size=n_obj, p=area / area.sum())
    o = np.empty((n_obj, 3))
    # spheres: uniform direction on the unit sphere, centre at height r
    sph = ~is_box[which]
    ns = int(sph.sum())
    v = rng.standard_normal((ns, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    ws = which[sph]
    o[sph, 0:2] = ctr[ws] + radius[ws, None] * v[:, 0:2]
    o[sph, 2] = radius[ws] + radius[ws] * v[:, 2]
    # boxes: pick a face by area, then a uniform point on it
    bx = ~sph
    wb = which[bx]
    sx, sy, sz = size[wb, 0], size[wb, 1], size[wb, 2]
    fa = np.stack([sx * sy, sx * sy, sx * sz, sx * sz, sy * sz, sy * sz], axis=1)
    cum = np.cumsum(fa, axis=1)
    r = rng.uniform(size=wb.shape[0]) * cum[:, -1]
    face = (r[:, None] > cum).sum(axis=1)
    u = rng.uniform(size=(wb.shape[0], 3))
    local = u * np.stack([sx, sy, sz], axis=1)              # inside the box
    axis = face // 2                                        # 0: z faces, 1: y faces, 2: x faces
    side = face % 2
    fix_axis = np.array([2, 1, 0])[axis]
    dims = np.stack([sx, sy, sz], axis=1)
    rows = np.arange(wb.shape[0])
    local[rows, fix_axis] = side * dims[rows, fix_axis]
    o[bx, 0] = ctr[wb, 0] - 0.5 * sx + local[:, 0]
    o[bx, 1] = ctr[wb, 1] - 0.5 * sy + local[:, 1]
    o[bx, 2] = local[:, 2]
    pts = np.concatenate([g, o], axis=0)
    pts = pts[rng.permutation(n)]
    return np.ascontiguousarray(pts.astype(np.float32))


def gaussian_mixture_3d(n: int, n_blobs: int, rng: np.random.Generator,
                        sigma_lo: float = 0.01, sigma_hi: float = 0.05) -> np.ndarray:
    """Gaussian mixture of n_blobs isotropic blobs with centres in the unit cube."""
    centres = rng.uniform(0.0, 1.0, size=(n_blobs, 3))
    sig = rng.uniform(sigma_lo, sigma_hi, size=n_blobs)
    which = rng.integers(0, n_blobs, size=n)
    pts = centres[which] + rng.standard_normal((n, 3)) * sig[which, None]
    return np.ascontiguousarray(pts.astype(np.float32))


# ---------------------------------------------------------------------------
# The five workloads.  ``scale`` < 1 shrinks n (and k with it) while keeping
# the geometry; scaled-down versions are the parity-test cases.
# ---------------------------------------------------------------------------

def geo2d_blobs(seed: int = 1, n: int = 100_000, k: int = 100, max_iter: int = 20) -> Workload:
    rng = np.random.default_rng(seed)
    pts = gaussian_blobs_2d(n, 50, rng)
    init = init_from_permutation(pts, k, rng)
    return Workload("geo2d-blobs", pts, init, k, max_iter, True, seed,
                    "2D, 50 isotropic Gaussians, centres U[0,1000]^2, sigma U[5,20], "
                    "equal weights; init = first k of a seeded permutation; early stop")


def geo2d_roads(seed: int = 2, n: int = 1_000_000, k: int = 1000, max_iter: int = 50,
                n_lines: int = 2000) -> Workload:
    rng = np.random.default_rng(seed)
    pts = polylines_2d(n, n_lines, rng)
    init = init_from_permutation(pts, k, rng)
    return Workload("geo2d-roads", pts, init, k, max_iter, False, seed,
                    "2D, points along 2000 random polylines (5-20 segments, angle U[0,2pi), "
                    "length U[1e3,1e4], clipped to [0,1e5]^2), jitter sigma=15, "
                    "5% uniform noise; seeded-permutation init; fixed iterations",
                    meta=dict(n_lines=n_lines))


def lidar3d(seed: int = 3, n: int = 10_000_000, k: int = 10_000, max_iter: int = 30,
            n_objects: int = 3000) -> Workload:
    rng = np.random.default_rng(seed)
    pts = lidar_3d(n, n_objects, rng)
    init = init_from_permutation(pts, k, rng)
    return Workload("lidar3d", pts, init, k, max_iter, False, seed,
                    "3D, 60% ground plane U[-100,100]^2 x N(0,0.05), 40% area-uniform on "
                    "3000 boxes/spheres (50/50, sizes U[0.5,10] m) resting on z=0; "
                    "seeded-permutation init; fixed iterations",
                    meta=dict(n_objects=n_objects))


def batched3d(seed: int = 4, n_clouds: int = 512, log2_lo: float = 10.0, log2_hi: float = 17.0,
              max_iter: int = 25) -> List[Workload]:
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_clouds):
        n_i = int(round(2.0 ** rng.uniform(log2_lo, log2_hi)))
        blobs = int(rng.integers(4, 65))
        pts = gaussian_mixture_3d(n_i, blobs, rng)
        k_i = max(8, n_i // 100)
        init = init_from_permutation(pts, k_i, rng)
        out.append(Workload(f"batched3d[{c}]", pts, init, k_i, max_iter, False, seed,
                            "3D Gaussian mixture of 4-64 blobs in the unit cube, sigma U[0.01,0.05]; "
                            "n_i = round(2^U[10,17]); k_i = max(8, n_i // 100)"))
    return out


def soft3d(seed: int = 5, n_clouds: int = 64, n: int = 16_384, k: int = 256) -> List[Workload]:
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_clouds):
        pts = gaussian_mixture_3d(n, 32, rng)
        init = init_from_permutation(pts, k, rng)
        out.append(Workload(f"soft3d[{c}]", pts, init, k, 10, False, seed,
                            "3D Gaussian mixture of 32 blobs in the unit cube, sigma U[0.01,0.05]"))
    return out


def by_name(name: str, seed: Optional[int] = None, scale: float = 1.0) -> Workload:
    """One of the single-cloud workloads, optionally shrunk by ``scale``."""
    def sc(v: int, lo: int) -> int:
        return max(lo, int(round(v * scale)))
    if name == "geo2d-blobs":
        return geo2d_blobs(seed if seed is not None else 1, n=sc(100_000, 64), k=sc(100, 2))
    if name == "geo2d-roads":
        return geo2d_roads(seed if seed is not None else 2, n=sc(1_000_000, 64), k=sc(1000, 2),
                           n_lines=sc(2000, 4))
    if name == "lidar3d":
        return lidar3d(seed if seed is not None else 3, n=sc(10_000_000, 64), k=sc(10_000, 2),
                       n_objects=sc(3000, 4))
    raise KeyError(name)
