"""Seeded synthetic inputs shared by the CUDA path, the tests and the FP64 oracle.

This module holds random draws and phantom geometry only: no step of the rendering method
(signal equation, activations, rendering, slice profile, optimiser) is computed here, so
that the CUDA path and the oracle each apply the method to the same draws independently.
It imports neither the CUDA binding nor the oracle.

Workloads (all coordinates in world units, mm; grids are 1 mm isotropic unless stated):
  * ``gaussian_cloud``: means uniform in the volume, per-axis scales log-uniform in
    [0.5, 3] voxels, rotations from random-normal quaternions, PD ~ U[0, 1],
    T1 ~ U[300, 2000] ms, T2 ~ U[30, 200] ms (tissue ranges of the paper's MRI setting).
  * ``phantom_draws``: a 3D tissue phantom of 12 random ellipsoids (later ones overwrite
    earlier ones), each with PD/T1/T2 drawn as above, plus Rician noise draws for the LR
    scan. It stands in for the MSD / FeTA brain volumes of Sec. 4.1, which are not used.
  * ``gmm_cloud``: clustered, strongly anisotropic clouds (Gaussian-mixture blobs; one axis
    scale log-uniform in [4, 8] voxels, the others in [0.5, 1.5]).
  * ``serving_draws``: a stream of fitting and re-rendering requests for the serving runtime
    (Poisson arrivals, scan sizes, slice factors, output grids).
"""
from __future__ import annotations

import numpy as np

# Tissue parameter ranges (ms) and the acquisition used to map them through Eq. 2.
T1_RANGE = (300.0, 2000.0)
T2_RANGE = (30.0, 200.0)
TR_MS = 2000.0
TE_MS = 100.0


def assemble_params(mu, log_s, q, a, t) -> np.ndarray:
    """Stack per-Gaussian columns into the raw ``[N, 12]`` float32 parameter layout
    ``[mu(3), log_s(3), q_wxyz(4), a, t]`` (pure data arrangement)."""
    n = np.asarray(mu).shape[0]
    out = np.empty((n, 12), np.float32)
    out[:, 0:3] = mu
    out[:, 3:6] = log_s
    out[:, 6:10] = q
    out[:, 10] = a
    out[:, 11] = t
    return out


def gaussian_cloud(seed: int, n: int, shape_zyx, h=(1.0, 1.0, 1.0),
                   scale_range=(0.5, 3.0)) -> dict:
    """Random Gaussian cloud: returns draws dict(mu, log_s, q, pd, t1, t2).

    ``log_s`` is the log of a scale drawn log-uniformly in ``scale_range`` voxels, converted
    to world units per axis; ``q`` is an unnormalised random-normal quaternion (w, x, y, z).
    """
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape_zyx
    ext = np.array([nx * h[0], ny * h[1], nz * h[2]])
    mu = rng.uniform(0.0, 1.0, size=(n, 3)) * ext[None, :]
    lo, hi = np.log(scale_range[0]), np.log(scale_range[1])
    log_s = rng.uniform(lo, hi, size=(n, 3)) + np.log(np.array(h))[None, :]
    q = rng.standard_normal(size=(n, 4))
    pd = rng.uniform(0.0, 1.0, size=n)
    t1 = rng.uniform(*T1_RANGE, size=n)
    t2 = rng.uniform(*T2_RANGE, size=n)
    return dict(mu=mu.astype(np.float32), log_s=log_s.astype(np.float32),
                q=q.astype(np.float32), pd=pd, t1=t1, t2=t2)


def gmm_cloud(seed: int, n: int, shape_zyx, n_blobs: int = 20, blob_std: float = 24.0,
              long_range=(4.0, 8.0), short_range=(0.5, 1.5)) -> dict:
    """Clustered anisotropic cloud: means from ``n_blobs`` equal-weight isotropic Gaussian
    blobs (centres uniform in the volume, std ``blob_std`` voxels, clipped to the volume);
    one random axis has a scale log-uniform in ``long_range``, the other two in
    ``short_range`` (voxels); random rotations; tissue draws as ``gaussian_cloud``."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape_zyx
    ext = np.array([nx, ny, nz], np.float64)
    centres = rng.uniform(0.0, 1.0, size=(n_blobs, 3)) * ext[None, :]
    which = rng.integers(0, n_blobs, size=n)
    mu = centres[which] + rng.standard_normal(size=(n, 3)) * blob_std
    mu = np.clip(mu, 0.0, ext[None, :] - 1e-3)
    log_s = rng.uniform(np.log(short_range[0]), np.log(short_range[1]), size=(n, 3))
    axis = rng.integers(0, 3, size=n)
    log_s[np.arange(n), axis] = rng.uniform(np.log(long_range[0]), np.log(long_range[1]),
                                            size=n)
    q = rng.standard_normal(size=(n, 4))
    pd = rng.uniform(0.0, 1.0, size=n)
    t1 = rng.uniform(*T1_RANGE, size=n)
    t2 = rng.uniform(*T2_RANGE, size=n)
    return dict(mu=mu.astype(np.float32), log_s=log_s.astype(np.float32),
                q=q.astype(np.float32), pd=pd, t1=t1, t2=t2)


def _random_rotations(rng, n):
    """Uniform random rotation matrices (scipy's implementation of Shoemake's method)."""
    from scipy.spatial.transform import Rotation
    return Rotation.random(n, random_state=rng).as_matrix()


def phantom_draws(seed: int, shape_zyx, n_ell: int = 12, s: int = 4,
                  semi_axes=(10.0, 80.0), noise_sigma: float = 0.02, lr_shape=None) -> dict:
    """Ellipsoid tissue phantom draws.

    Returns dict(label [nz, ny, nx] uint8 (0 background, e + 1 for ellipsoid e; later
    ellipsoids overwrite earlier ones), pd, t1, t2 [n_ell], n1, n2 of shape ``lr_shape``
    (default [nz // s, ny, nx]: independent N(0, noise_sigma^2) draws for the real and
    imaginary noise channels of the LR scan).
    Semi-axes are drawn uniformly in ``semi_axes`` voxels, capped at 45 % of the volume's
    extent along the ellipsoid's longest box axis so that every ellipsoid stays visible.
    """
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape_zyx
    ext = np.array([nx, ny, nz], np.float64)
    label = np.zeros(shape_zyx, np.uint8)
    centres = rng.uniform(0.2, 0.8, size=(n_ell, 3)) * ext[None, :]
    axes = rng.uniform(semi_axes[0], semi_axes[1], size=(n_ell, 3))
    axes = np.minimum(axes, 0.45 * ext.max())
    rots = _random_rotations(rng, n_ell)
    pd = rng.uniform(0.0, 1.0, size=n_ell)
    t1 = rng.uniform(*T1_RANGE, size=n_ell)
    t2 = rng.uniform(*T2_RANGE, size=n_ell)
    zs = np.arange(nz) + 0.5
    ys = np.arange(ny) + 0.5
    xs = np.arange(nx) + 0.5
    for e in range(n_ell):
        c, a, R = centres[e], axes[e], rots[e]
        # voxel centres p inside when sum_k ((R^T (p - c))_k / a_k)^2 <= 1 (box-limited)
        r = a.max()
        z0, z1 = int(max(0, np.floor(c[2] - r))), int(min(nz, np.ceil(c[2] + r) + 1))
        y0, y1 = int(max(0, np.floor(c[1] - r))), int(min(ny, np.ceil(c[1] + r) + 1))
        x0, x1 = int(max(0, np.floor(c[0] - r))), int(min(nx, np.ceil(c[0] + r) + 1))
        if z0 >= z1 or y0 >= y1 or x0 >= x1:
            continue
        Z, Y, X = np.meshgrid(zs[z0:z1] - c[2], ys[y0:y1] - c[1], xs[x0:x1] - c[0],
                              indexing="ij")
        u = (R[0, 0] * X + R[1, 0] * Y + R[2, 0] * Z) / a[0]
        v = (R[0, 1] * X + R[1, 1] * Y + R[2, 1] * Z) / a[1]
        w = (R[0, 2] * X + R[1, 2] * Y + R[2, 2] * Z) / a[2]
        inside = (u * u + v * v + w * w) <= 1.0
        sub = label[z0:z1, y0:y1, x0:x1]
        sub[inside] = e + 1
    lshape = tuple(lr_shape) if lr_shape is not None else (nz // s, ny, nx)
    n1 = rng.standard_normal(size=lshape).astype(np.float32) * np.float32(noise_sigma)
    n2 = rng.standard_normal(size=lshape).astype(np.float32) * np.float32(noise_sigma)
    return dict(label=label, pd=pd, t1=t1, t2=t2, n1=n1, n2=n2, s=s)


def crop_dI(seed: int, crop_shape_zyx) -> np.ndarray:
    """Random upstream gradient dL/dI on a crop (standard normal, float32)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=crop_shape_zyx).astype(np.float32)


# Scan sizes (nz, ny, nx) of the serving stream: 128^3, 192 x 192 x 128 and 256 x 256 x
# 160 / 192 (brain-MRI-like fields of view at 1 mm).
SERVE_SHAPES = ((128, 128, 128), (128, 192, 192), (160, 256, 256), (192, 256, 256))
SERVE_RENDER_SPACINGS = (0.8, 1.0, 1.25)


def serve_n_gauss(shape_zyx) -> int:
    """Cloud size of a scan: 1M Gaussians for 256 x 256 x 192 voxels, in proportion to the
    voxel count, at least 100k."""
    v = int(np.prod(shape_zyx))
    return max(100_000, int(round(1e6 * v / (256 * 256 * 192))))


def serving_draws(seed: int = 0, n: int = 32, rate_hz: float = 2.0, fit_frac: float = 0.75,
                  iters: int = 500) -> list:
    """Request stream: arrivals of a Poisson process of `rate_hz` (the first at t = 0); each
    request fits a new scan (probability fit_frac; shape from SERVE_SHAPES, slice factor in
    {2, 3, 4}, `iters` steps) or re-renders the cloud of an earlier fit request on the same
    field of view at isotropic spacing from SERVE_RENDER_SPACINGS. The first request is a fit.
    Each entry: dict(kind 'fit' | 'render', arrival_s, shape (nz, ny, nx), s, iters, n_gauss,
    seed) for a fit; dict(kind, arrival_s, source (index of the fit), spacing, shape) for a
    render (shape = the source's field of view / spacing, rounded)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=n)
    arrivals = np.concatenate([[0.0], np.cumsum(gaps[1:])])
    out = []
    fits = []
    for i in range(n):
        u_kind = rng.uniform()
        i_shape = int(rng.integers(len(SERVE_SHAPES)))
        s = int(rng.integers(2, 5))
        i_src = rng.uniform()
        i_sp = int(rng.integers(len(SERVE_RENDER_SPACINGS)))
        if not fits or u_kind < fit_frac:
            shape = SERVE_SHAPES[i_shape]
            out.append(dict(kind="fit", arrival_s=float(arrivals[i]), shape=shape, s=s,
                            iters=iters, n_gauss=serve_n_gauss(shape), seed=1000 + i))
            fits.append(i)
        else:
            src = fits[int(i_src * len(fits))]
            h = SERVE_RENDER_SPACINGS[i_sp]
            shape = tuple(int(round(d / h)) for d in out[src]["shape"])
            out.append(dict(kind="render", arrival_s=float(arrivals[i]), source=src,
                            spacing=h, shape=shape))
    return out
