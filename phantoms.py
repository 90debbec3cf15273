"""Seeded synthetic inputs for the semi-Lagrangian Metamorphosis workloads.

This module only synthesises images, targets and initial momenta. It holds none
of the registration method's arithmetic (no RKHS blur, no shooting, no cost):
phantoms are smoothed and warped with scipy.ndimage, a different code path from
both the oracle and the CUDA library, and both sides receive exactly the arrays
produced here.

The paper's own images (a 'C' shape and a small disk, Sec. 3, Fig. 1-2) are not
available; these phantoms stand in for them:

* ``disk_pair_64``   - 64x64 disk -> ellipse plus a bright blob that the
  source lacks (the topology change Metamorphosis is meant to model, Fig. 2).
* ``ellipse_pairs``  - batches of random smooth 2-D phantoms (3-6 blurred
  ellipses) whose targets are jittered copies plus one blob.
* ``head_pair_3d``   - nested-ellipsoid "brain" volume, target warped by a
  random smooth displacement plus a blob, optional Rician-like noise.
* ``c_pair_64``      - a disk and a 'C' (an annulus with a gap), the stand-in for
  the 'C' picture of the scheme comparison (Fig. 1).

All arrays are float32, C-contiguous, axis 0 first, values clipped to [0, 1].
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence, Tuple

import numpy as np
from scipy import ndimage


@dataclasses.dataclass
class Workload:
    """One batch of registration problems that share shape, T and sigma."""

    name: str
    ndim: int
    dims: Tuple[int, ...]
    T: int
    sigma: float
    I0: np.ndarray          # [B, *dims] float32 source images
    J: np.ndarray           # [B, *dims] float32 targets
    p0: np.ndarray          # [B, *dims] float32 initial momenta
    mu: np.ndarray          # [B] float32
    rho: np.ndarray         # [B] float32
    lam: np.ndarray         # [B] float32

    @property
    def batch(self) -> int:
        return int(self.I0.shape[0])

    @property
    def voxels(self) -> int:
        return int(np.prod(self.dims))


def _grid(dims: Sequence[int]) -> List[np.ndarray]:
    return list(np.meshgrid(*[np.arange(n, dtype=np.float64) for n in dims], indexing="ij"))


def _smooth(img: np.ndarray, s: float) -> np.ndarray:
    return ndimage.gaussian_filter(img, s, mode="constant", truncate=4.0)


def _blob(dims: Sequence[int], centre: Sequence[float], radius: float) -> np.ndarray:
    """exp(-|x-c|^2 / (2 (R/2)^2)): a bright blob of nominal radius R."""
    X = _grid(dims)
    d2 = sum((x - c) ** 2 for x, c in zip(X, centre))
    return np.exp(-d2 / (2.0 * (radius / 2.0) ** 2))


def _ellipse(dims, centre, semi_axes, angle) -> np.ndarray:
    """Indicator of a 2-D ellipse; semi_axes = (axis-0 extent, axis-1 extent)."""
    Y, X = _grid(dims)
    dy, dx = Y - centre[0], X - centre[1]
    c, s = np.cos(angle), np.sin(angle)
    a0 = c * dy + s * dx
    a1 = -s * dy + c * dx
    return ((a0 / semi_axes[0]) ** 2 + (a1 / semi_axes[1]) ** 2 <= 1.0).astype(np.float64)


def _ellipsoid(dims, centre, semi_axes) -> np.ndarray:
    X = _grid(dims)
    q = sum(((x - c) / a) ** 2 for x, c, a in zip(X, centre, semi_axes))
    return (q <= 1.0).astype(np.float64)


def _f32(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.clip(a, 0.0, 1.0), dtype=np.float32)


def disk_pair_64(seed: int = 1001, random_p0: bool = True, p0_std: float = 0.01) -> Workload:
    """64x64 disk (radius 18) -> ellipse (semi-axes 14 x 22) + blob of radius 8.

    The blob sits outside the ellipse, like the small disk of Fig. 2 that LDDMM
    cannot create and Metamorphosis can.  T=10, sigma=3, mu=0.1, rho=1,
    lambda=1e-3.  p0 is N(0, p0_std^2) when random_p0 else exactly zero.
    """
    dims = (64, 64)
    Y, X = _grid(dims)
    S = ((Y - 32.0) ** 2 + (X - 32.0) ** 2 <= 18.0 ** 2).astype(np.float64)
    S = _smooth(S, 1.0)
    J = _smooth(_ellipse(dims, (32.0, 32.0), (14.0, 22.0), 0.0), 1.0)
    J = np.maximum(J, _blob(dims, (52.0, 32.0), 8.0))
    rng = np.random.default_rng(seed)
    p0 = rng.normal(0.0, p0_std, size=dims) if random_p0 else np.zeros(dims)
    return Workload("disk64", 2, dims, 10, 3.0, _f32(S)[None], _f32(J)[None],
                    np.ascontiguousarray(p0, dtype=np.float32)[None],
                    np.array([0.1], np.float32), np.array([1.0], np.float32),
                    np.array([1e-3], np.float32))


def c_pair_64(size: int = 64) -> Workload:
    """Disk (radius 0.28 size) -> a 'C': an annulus (radii 0.17 and 0.36 size) with a
    gap of 0.24 size on the axis-1 positive side, both blurred with sigma 1.  The
    stand-in for the 'C' picture of the stability comparison (Fig. 1).  T=20, sigma=3,
    mu=0 (LDDMM), rho=1, lambda=1e-3, p0 = 0."""
    dims = (size, size)
    Y, X = _grid(dims)
    c = (size - 1) / 2.0
    r2 = (Y - c) ** 2 + (X - c) ** 2
    S = _smooth((r2 <= (0.28 * size) ** 2).astype(np.float64), 1.0)
    ring = (r2 <= (0.36 * size) ** 2) & (r2 >= (0.17 * size) ** 2)
    gap = (np.abs(Y - c) <= 0.12 * size) & (X > c)
    J = _smooth((ring & ~gap).astype(np.float64), 1.0)
    return Workload("c64", 2, dims, 20, 3.0, _f32(S)[None], _f32(J)[None],
                    np.zeros((1,) + dims, np.float32), np.array([0.0], np.float32),
                    np.array([1.0], np.float32), np.array([1e-3], np.float32))


def _random_ellipse_image(rng, dims, ellipses) -> np.ndarray:
    img = np.zeros(dims)
    for (cy, cx, ay, ax, ang, val) in ellipses:
        img = np.maximum(img, val * _ellipse(dims, (cy, cx), (ay, ax), ang))
    return _smooth(img, 1.0)


def ellipse_pairs(batch: int = 16, size: Tuple[int, int] = (256, 256), T: int = 20,
                  sigma: float = 6.0, mus: Sequence[float] = (0.0, 0.05, 0.2),
                  lam: float = 1e-3, seed: int = 1002, p0_std: float = 0.0) -> Workload:
    """`batch` independent 2-D pairs of random smooth phantoms.

    Each source holds 3-6 blurred ellipses (centres in the central 60 %,
    semi-axes U[0.08, 0.3] of the size, random angle, intensity U[0.2, 1]);
    its target holds the same ellipses jittered by U[-4, 4] px with axes
    scaled by U[0.9, 1.1], plus one blob of radius U[5, 20] px.  Instance i
    uses mu = mus[i % len(mus)], rho = 1.
    """
    rng = np.random.default_rng(seed)
    H, W = size
    I0 = np.empty((batch, H, W), np.float32)
    J = np.empty((batch, H, W), np.float32)
    for b in range(batch):
        n_ell = int(rng.integers(3, 7))
        src, tgt = [], []
        for _ in range(n_ell):
            cy, cx = rng.uniform(0.2, 0.8) * H, rng.uniform(0.2, 0.8) * W
            ay, ax = rng.uniform(0.08, 0.3) * H, rng.uniform(0.08, 0.3) * W
            ang, val = rng.uniform(0, np.pi), rng.uniform(0.2, 1.0)
            src.append((cy, cx, ay, ax, ang, val))
            jy, jx = rng.uniform(-4, 4, size=2)
            sy, sx = rng.uniform(0.9, 1.1, size=2)
            tgt.append((cy + jy, cx + jx, ay * sy, ax * sx, ang, val))
        I0[b] = _f32(_random_ellipse_image(rng, (H, W), src))
        t = _random_ellipse_image(rng, (H, W), tgt)
        br = rng.uniform(5, 20)
        bc = (rng.uniform(0.2, 0.8) * H, rng.uniform(0.2, 0.8) * W)
        J[b] = _f32(np.maximum(t, _blob((H, W), bc, br)))
    p0 = (rng.normal(0.0, p0_std, size=(batch, H, W)) if p0_std > 0
          else np.zeros((batch, H, W))).astype(np.float32)
    mu = np.array([mus[i % len(mus)] for i in range(batch)], np.float32)
    return Workload("ellipses%dx%dx%d" % (batch, H, W), 2, (H, W), T, sigma, I0, J, p0, mu,
                    np.ones(batch, np.float32), np.full(batch, lam, np.float32))


def head_phantom(dims: Tuple[int, int, int]) -> np.ndarray:
    """Nested ellipsoids 0.5 / 0.9 / 0.1 (semi-axes (0.42,0.38,0.34)*n, x0.7, x0.3)."""
    c = [n / 2.0 - 0.5 for n in dims]
    outer = [f * n for f, n in zip((0.42, 0.38, 0.34), dims)]
    img = 0.5 * _ellipsoid(dims, c, outer)
    img = np.where(_ellipsoid(dims, c, [0.7 * a for a in outer]) > 0, 0.9, img)
    img = np.where(_ellipsoid(dims, c, [0.3 * a for a in outer]) > 0, 0.1, img)
    return _smooth(img, 1.0)


def _smooth_displacement(rng, dims, amplitude: float, smooth: float) -> List[np.ndarray]:
    comps = [_smooth(rng.normal(0.0, 1.0, size=dims), smooth) for _ in dims]
    norm = np.sqrt(sum(c ** 2 for c in comps)).max()
    return [c * (amplitude / norm) for c in comps]


def head_pair_3d(dims: Tuple[int, int, int] = (128, 128, 128), T: int = 20, sigma: float = 5.0,
                 mu: float = 0.1, lam: float = 1e-3, blob_radius: Optional[float] = 12.0,
                 noise: float = 0.0, seed: int = 1003, p0_std: float = 0.0) -> Workload:
    """3-D head phantom; target = S o (Id + u) plus a blob inside the head.

    u is white noise smoothed with a sigma=16 Gaussian, scaled to max |u| = 4
    voxels.  blob_radius=None draws it from U[10, 25].  With noise > 0 both
    images get Rician-like noise sqrt((I + n1)^2 + n2^2), n ~ N(0, noise^2).
    """
    rng = np.random.default_rng(seed)
    S = head_phantom(dims)
    u = _smooth_displacement(rng, dims, 4.0, 16.0)
    X = _grid(dims)
    J = ndimage.map_coordinates(S, [x + ui for x, ui in zip(X, u)], order=1, mode="nearest")
    R = float(rng.uniform(10, 25)) if blob_radius is None else float(blob_radius)
    c = [n / 2.0 + rng.uniform(-0.12, 0.12) * n for n in dims]
    J = np.maximum(J, _blob(dims, c, R))
    if noise > 0:
        S = np.sqrt((S + rng.normal(0, noise, dims)) ** 2 + rng.normal(0, noise, dims) ** 2)
        J = np.sqrt((J + rng.normal(0, noise, dims)) ** 2 + rng.normal(0, noise, dims) ** 2)
    p0 = (rng.normal(0.0, p0_std, size=dims) if p0_std > 0 else np.zeros(dims))
    return Workload("head%dx%dx%d" % dims, 3, tuple(dims), T, sigma, _f32(S)[None], _f32(J)[None],
                    np.ascontiguousarray(p0, dtype=np.float32)[None],
                    np.array([mu], np.float32), np.array([1.0], np.float32),
                    np.array([lam], np.float32))


def mri_pair_3d(seed: int = 1005) -> Workload:
    """160x192x160 head phantom with Rician-like noise (sigma 0.02), blob R~U[10,25]."""
    return head_pair_3d(dims=(160, 192, 160), T=20, sigma=6.0, mu=0.05, lam=1e-4,
                        blob_radius=None, noise=0.02, seed=seed)


def block_average(vol: np.ndarray, f: int = 2) -> np.ndarray:
    """f-times block-averaged copy of a [B, *dims] batch (dims divisible by f)."""
    B = vol.shape[0]
    dims = vol.shape[1:]
    shp = [B]
    for n in dims:
        shp += [n // f, f]
    v = vol.reshape(shp)
    return np.ascontiguousarray(v.mean(axis=tuple(range(2, 2 + 2 * len(dims), 2))), dtype=np.float32)


def random_fields(seed: int, batch: int, dims: Sequence[int], p_std: float = 0.05,
                  smooth: float = 2.0) -> Tuple[np.ndarray, np.ndarray]:
    """Generic smooth random (I, p) pairs for kernel tests on ragged shapes.

    I has a smooth ramp added so that its gradient vanishes nowhere, which keeps
    the backtracked feet off the grid lines in tests that compare gradients.
    """
    rng = np.random.default_rng(seed)
    dims = tuple(dims)
    I = np.empty((batch,) + dims, np.float32)
    p = np.empty((batch,) + dims, np.float32)
    X = _grid(dims)
    ramp = sum((k + 1) * 0.03 * x / max(n - 1, 1) for k, (x, n) in enumerate(zip(X, dims)))
    for b in range(batch):
        img = ndimage.gaussian_filter(rng.uniform(0, 1, dims), smooth, mode="nearest")
        img = (img - img.min()) / max(img.max() - img.min(), 1e-12)
        I[b] = np.clip(0.8 * img + ramp, 0.0, 1.0)
        p[b] = rng.normal(0.0, p_std, dims)
    return I, p


def mixed_pairs(n: int = 64, seed: int = 1004) -> List[Workload]:
    """`n` single-pair workloads of uneven size and dimension: sizes drawn from
    {96^2, 160^2, 224^2, 64^3, 96^3}, T from {10, 15, 20}, sigma_K ~ U[2, 6],
    mu ~ U[0, 0.2], rho = 1, lambda = 1e-3; 2-D pairs as ellipse_pairs, 3-D as
    head_pair_3d (blob radius ~ U[10, 25] scaled to the volume)."""
    rng = np.random.default_rng(seed)
    sizes = [(96, 96), (160, 160), (224, 224), (64, 64, 64), (96, 96, 96)]
    out = []
    for i in range(n):
        dims = sizes[int(rng.integers(0, len(sizes)))]
        T = int(rng.choice([10, 15, 20]))
        sigma = float(rng.uniform(2.0, 6.0))
        mu = float(rng.uniform(0.0, 0.2))
        sub = int(rng.integers(0, 2 ** 31))
        if len(dims) == 2:
            w = ellipse_pairs(batch=1, size=dims, T=T, sigma=sigma, mus=(mu,), seed=sub)
        else:
            w = head_pair_3d(dims=dims, T=T, sigma=sigma, mu=mu,
                             blob_radius=float(rng.uniform(10, 25)) * dims[0] / 160.0, seed=sub)
        w.name = "mix%d" % i
        out.append(w)
    return out
