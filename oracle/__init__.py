"""FP64 CPU oracle for physics-grounded Gaussian volume rendering (test infrastructure).

Only the test suite, the smoke check and the benchmark's CPU-baseline / reference leg may
import this package. It shares no code with the CUDA library in ``paper_2603_09621_gb300``
and never imports it; inputs reach both sides from ``paper_2603_09621_gb300.inputs``, which
holds random draws and phantom geometry only.

Each function cites the passage of the paper ("Physics-Driven 3D Gaussian Rendering for
Zero-Shot MRI Super-Resolution") it follows. Where the paper is silent the reading is stated
in the docstring.

Parameter layout of one Gaussian (12 raw values, Sec. 3.1: position 3, covariance 7,
amplitude 1, relaxation proxy 1): ``[mu_x, mu_y, mu_z, log_s_x, log_s_y, log_s_z,
q_w, q_x, q_y, q_z, a, t]``.

Volumes are ``[nz, ny, nx]`` arrays (x fastest); voxel (i, j, k) has centre
``origin + (i + 1/2, j + 1/2, k + 1/2) * h``.

Parity status: every function here is pinned by ``tests/test_oracle_*.py`` against closed
forms, invariants, brute force or library routines. ``ssim3d`` is a stated reading of the
paper's evaluation metric whose window the paper does not give (Gaussian, std 1.5 voxels);
it is pinned to that reading by closed forms (constant volumes; an impulse against zero).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgs_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (FP64, OpenMP, no floating-point contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, f64, f32, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_float, ctypes.c_int
        _lib.og_render.restype = i64
        _lib.og_render.argtypes = [P, i64, P, P, P, P, f64, f64, i32, i32, i32, f64, i32,
                                   P, P, P, P, P, P, P, P, P, P, P, P, P]
        _lib.og_render_grad.restype = i64
        _lib.og_render_grad.argtypes = [P, i64, P, P, P, P, f64, f64, i32, i32, i32, f64, i32,
                                        P, P, P, P, P, P]
        _lib.og_bins_fp32.restype = None
        _lib.og_bins_fp32.argtypes = [P, i64, P, P, P, P, f32, P]
        _lib.og_signal_proxy.restype = None
        _lib.og_signal_proxy.argtypes = [P, P, i64, f64, f64, P]
        _lib.og_exp_cw_public.restype = f32
        _lib.og_exp_cw_public.argtypes = [f32]
        _lib.og_num_threads.restype = i32
        _lib.og_set_num_threads.argtypes = [i32]
    return _lib


def num_threads() -> int:
    return int(lib().og_num_threads())


def set_num_threads(n: int) -> None:
    lib().og_set_num_threads(int(n))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Grid:
    """Voxel grid: dims (nx, ny, nz), spacing h and origin (world units, mm)."""
    nx: int
    ny: int
    nz: int
    h: tuple = (1.0, 1.0, 1.0)
    origin: tuple = (0.0, 0.0, 0.0)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


@dataclass
class Config:
    """Rendering options. Defaults follow the readings stated in the module docstring."""
    trunc_sigma: float = 3.0     # Sec. 3.3: 3-sigma Mahalanobis ellipsoids
    eps: float = 1e-12           # W floor (the paper gives none)
    signal_mode: int = 0         # 0: v = A, r = T ; 1: v = A T, r = 1
    a_act: int = 0               # 0 identity, 1 sigmoid
    t_act: int = 0               # 0 identity, 1 sigmoid
    brick: tuple = (8, 8, 8)     # brick shape (x, y, z); the paper uses 8 x 8 x 4


def _grid_arrays(grid: Grid):
    dims = np.array([grid.nx, grid.ny, grid.nz], dtype=np.int32)
    h = np.array(grid.h, dtype=np.float64)
    o = np.array(grid.origin, dtype=np.float64)
    return dims, h, o


def _crop_array(grid: Grid, crop):
    if crop is None:
        return None, (grid.nz, grid.ny, grid.nx)
    x0, x1, y0, y1, z0, z1 = [int(v) for v in crop]
    assert 0 <= x0 <= x1 <= grid.nx and 0 <= y0 <= y1 <= grid.ny and 0 <= z0 <= z1 <= grid.nz
    return np.array([x0, x1, y0, y1, z0, z1], dtype=np.int32), (z1 - z0, y1 - y0, x1 - x0)


# --------------------------------------------------------------------------- Eq. 2

def signal_proxy(T1, T2, TR: float, TE: float) -> np.ndarray:
    """Eq. 2 (Sec. 3.1): relaxation proxy T = (1 - exp(-TR/T1)) exp(-TE/T2), FP64."""
    T1 = np.ascontiguousarray(T1, dtype=np.float64).ravel()
    T2 = np.ascontiguousarray(T2, dtype=np.float64).ravel()
    out = np.empty_like(T1)
    lib().og_signal_proxy(_ptr(T1), _ptr(T2), T1.size, float(TR), float(TE), _ptr(out))
    return out


# --------------------------------------------------------------------- Eq. 3-4

# Ambiguous pairs recorded per voxel by render(..., want_amb=True) (og_render's slots).
AMB_SLOTS = 8

# Default half-width of the ambiguity band around the truncation boundary, relative to
# sum_ab |C_ab d_a d_b| (the rounding scale of the quadratic form): a pair with
# |d^2 - sigma_t^2| <= AMB_TOL sum_ab |C_ab d_a d_b| may be decided either way by a rounded
# FP32 evaluation. The value is derived from the FP32 operation sequence of a renderer that
# builds its per-Gaussian coefficients and evaluates the form in single precision (about
# 335 units of 2^-24).
AMB_TOL = 2e-5


def render(params, grid: Grid, cfg: Config = Config(), crop=None, amb_tol=None, prune=True,
           want_amb=False):
    """Eq. 3-4 with the Sec. 3.3 truncation, brute force in FP64.

    Returns dict(I, W, S, amb, npair, n_invalid), each volume crop-shaped ``[z, y, x]``.
    ``amb`` counts, per voxel, the pairs with |d^2 - sigma_t^2| <= amb_tol sum_ab
    |C_ab d_a d_b| (default ``AMB_TOL``): a rounded FP32 evaluation of d^2 may put them on
    either side of the truncation boundary, so either decision is a valid result.
    ``npair`` counts the contributing pairs per voxel.

    With ``want_amb`` the dict also holds, for validating a result that took its own
    decisions on the ambiguous pairs: ``S_sure``, ``W_sure`` (sums over the contributing pairs
    that are not ambiguous); per voxel and slot k < ``AMB_SLOTS`` (the first ambiguous pairs in
    Gaussian order) ``amb_id`` (the Gaussian, -1 for an unused slot), ``amb_vw`` (v w),
    ``amb_w`` (w = exp(-d^2/2) r whichever side of the boundary), ``amb_rel``
    ((d^2 - sigma_t^2) / sum_ab |C_ab d_a d_b|; <= 0 means the FP64 decision includes it);
    ``cond_w`` (sum over contributing pairs of w sum_ab |C_ab d_a d_b|) and ``cond_i`` (the
    same sum with each term also weighted by |v - I|, the sensitivity of I to that weight).
    """
    p = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 12)
    dims, h, o = _grid_arrays(grid)
    carr, shape = _crop_array(grid, crop)
    if amb_tol is None:
        amb_tol = AMB_TOL
    I = np.zeros(shape, np.float64)
    W = np.zeros(shape, np.float64)
    S = np.zeros(shape, np.float64)
    amb = np.zeros(shape, np.int32)
    npair = np.zeros(shape, np.int32)
    extra = {}
    if want_amb:
        extra = dict(S_sure=np.zeros(shape, np.float64), W_sure=np.zeros(shape, np.float64),
                     amb_id=np.full(shape + (AMB_SLOTS,), -1, np.int32),
                     amb_vw=np.zeros(shape + (AMB_SLOTS,), np.float64),
                     amb_w=np.zeros(shape + (AMB_SLOTS,), np.float64),
                     amb_rel=np.zeros(shape + (AMB_SLOTS,), np.float64),
                     cond_w=np.zeros(shape, np.float64), cond_i=np.zeros(shape, np.float64))
    ep = (lambda k: _ptr(extra[k]) if want_amb else None)
    n_bad = lib().og_render(_ptr(p), p.shape[0], _ptr(dims), _ptr(h), _ptr(o),
                            None if carr is None else _ptr(carr), cfg.trunc_sigma, cfg.eps,
                            cfg.signal_mode, cfg.a_act, cfg.t_act, float(amb_tol),
                            1 if prune else 0, _ptr(I), _ptr(W), _ptr(S), _ptr(amb),
                            _ptr(npair), ep("S_sure"), ep("W_sure"), ep("amb_id"),
                            ep("amb_vw"), ep("amb_w"), ep("amb_rel"), ep("cond_w"),
                            ep("cond_i"))
    if n_bad < 0:
        raise MemoryError("oracle render: allocation failed")
    out = dict(I=I, W=W, S=S, amb=amb, npair=npair, n_invalid=int(n_bad))
    out.update(extra)
    return out


def render_grad(params, grid: Grid, dI, cfg: Config = Config(), crop=None, prune=True,
                want_geo=False, want_box=False, amb_tol=None):
    """Eq. 5-6 (Sec. 3.3) and the chain to the raw parameters, FP64.

    ``dI`` is dL/dI on the crop (crop-shaped); voxels outside the crop have dL/dI = 0.
    Returns dL/d(raw params) ``[N, 12]`` and, with ``want_geo``, dL/d(mu, c_xx, c_yy, c_zz,
    c_xy, c_xz, c_yz, v, r) ``[N, 11]``.

    With ``want_box`` it returns a dict(grad, lo, hi, n_unenum) instead: ``lo`` and ``hi``
    bound, per Gaussian and parameter, the gradient of every renderer that decides each pair
    of the ambiguity band (``amb_tol``, default ``AMB_TOL``; see ``render``) either way,
    voxel by voxel (all include/exclude subsets of a voxel's ambiguous pairs, up to
    ``AMB_SLOTS`` of them). ``n_unenum`` counts voxels with dI != 0 and more ambiguous pairs
    than that (not covered by the bounds). ``grad`` is the FP64 decision's gradient.
    """
    p = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 12)
    dims, h, o = _grid_arrays(grid)
    carr, shape = _crop_array(grid, crop)
    dI = np.ascontiguousarray(dI, dtype=np.float64)
    assert dI.shape == shape, (dI.shape, shape)
    if amb_tol is None:
        amb_tol = AMB_TOL
    out = np.zeros((p.shape[0], 12), np.float64)
    geo = np.zeros((p.shape[0], 11), np.float64) if want_geo else None
    lo = np.zeros((p.shape[0], 12), np.float64) if want_box else None
    hi = np.zeros((p.shape[0], 12), np.float64) if want_box else None
    nun = np.zeros(1, np.int64)
    n_bad = lib().og_render_grad(_ptr(p), p.shape[0], _ptr(dims), _ptr(h), _ptr(o),
                                 None if carr is None else _ptr(carr), cfg.trunc_sigma,
                                 cfg.eps, cfg.signal_mode, cfg.a_act, cfg.t_act,
                                 float(amb_tol) if want_box else 0.0, 1 if prune else 0,
                                 _ptr(dI), _ptr(out), None if geo is None else _ptr(geo),
                                 None if lo is None else _ptr(lo),
                                 None if hi is None else _ptr(hi), _ptr(nun))
    if n_bad < 0:
        raise MemoryError("oracle render_grad: allocation failed")
    if want_box:
        res = dict(grad=out, lo=lo, hi=hi, n_unenum=int(nun[0]))
        if want_geo:
            res["geo"] = geo
        return res
    return (out, geo) if want_geo else out


# ------------------------------------------------------------ brick binning (FP32)

def exp_cw(x: float) -> float:
    """The FP32 exponential of the binning specification (Cody-Waite, see gs_oracle.c)."""
    return float(lib().og_exp_cw_public(float(x)))


def brick_ranges_fp32(params, grid: Grid, cfg: Config = Config()) -> np.ndarray:
    """Per-Gaussian brick range ``[N, 7]`` (lo xyz, hi xyz, meets-grid flag), decided in FP32.

    Sec. 3.3 bins each Gaussian by its 3-sigma extent; the axis-aligned bounding box of the
    ellipsoid {d^2 <= sigma_t^2} has half-extent sigma_t sqrt(Sigma_kk). The decision is an
    integer made by floating point, so it is taken in the kernel's precision (FP32) with the
    operation order documented in gs_oracle.c.
    """
    p = np.ascontiguousarray(params, dtype=np.float32).reshape(-1, 12)
    dims = np.array([grid.nx, grid.ny, grid.nz], dtype=np.int32)
    h = np.array(grid.h, dtype=np.float32)
    o = np.array(grid.origin, dtype=np.float32)
    b = np.array(cfg.brick, dtype=np.int32)
    out = np.zeros((p.shape[0], 7), np.int32)
    lib().og_bins_fp32(_ptr(p), p.shape[0], _ptr(dims), _ptr(h), _ptr(o), _ptr(b),
                       float(cfg.trunc_sigma), _ptr(out))
    return out


def brick_grid(grid: Grid, cfg: Config = Config()):
    """Number of bricks along x, y, z (partial bricks at the far edges count)."""
    bx, by, bz = cfg.brick
    return (-(-grid.nx // bx), -(-grid.ny // by), -(-grid.nz // bz))


def brick_lists(params, grid: Grid, cfg: Config = Config()):
    """Per-brick Gaussian lists (Sec. 3.3: 'for each brick b we identify intersecting
    Gaussians'), brick-major, ascending Gaussian id inside each brick.

    Returns dict(brick_off [nb+1], pair_gid [P], gm_off [N+1], gm_brick [P]) where the
    Gaussian-major list enumerates, for each Gaussian in ascending order, its bricks in
    ascending linear brick index (x fastest).
    """
    rng = brick_ranges_fp32(params, grid, cfg)
    nbx, nby, nbz = brick_grid(grid, cfg)
    nb = nbx * nby * nbz
    lo = rng[:, :3].astype(np.int64)
    ok = rng[:, 6] == 1
    ext = np.where(ok[:, None], rng[:, 3:6].astype(np.int64) - lo + 1, 0)
    counts = ext.prod(axis=1)
    gm_off = np.zeros(rng.shape[0] + 1, np.int64)
    gm_off[1:] = np.cumsum(counts)
    gm_gid = np.repeat(np.arange(rng.shape[0]), counts)
    # Local index t of each pair inside its Gaussian's brick box, x fastest, so that the
    # bricks of one Gaussian come in ascending linear brick index.
    t = np.arange(gm_off[-1], dtype=np.int64) - gm_off[gm_gid]
    ex, ey = ext[gm_gid, 0], ext[gm_gid, 1]
    bx = lo[gm_gid, 0] + t % ex
    by = lo[gm_gid, 1] + (t // ex) % ey
    bz = lo[gm_gid, 2] + t // (ex * ey)
    gm_brick = (bz * nby + by) * nbx + bx
    order = np.argsort(gm_brick, kind="stable")
    pair_gid = gm_gid[order]
    per_brick = np.bincount(gm_brick, minlength=nb) if gm_brick.size else np.zeros(nb, np.int64)
    brick_off = np.zeros(nb + 1, np.int64)
    brick_off[1:] = np.cumsum(per_brick)
    return dict(brick_off=brick_off, pair_gid=pair_gid, gm_off=gm_off, gm_brick=gm_brick,
                ranges=rng)


# ------------------------------------------------------- slice-profile forward model

def downsample(hr, s: int) -> np.ndarray:
    """Box slice profile along z: LR[k] = (1/s) sum_{j<s} HR[s k + j], k < floor(nz/s).

    The paper does not give its training forward model (it builds LR data by trilinear
    downsampling, Sec. 4.1); the z box profile is the stated reading used for fitting.
    """
    hr = np.asarray(hr, dtype=np.float64)
    nz = hr.shape[0]
    nl = nz // s
    out = np.zeros((nl,) + hr.shape[1:], np.float64)
    for k in range(nl):
        acc = np.zeros(hr.shape[1:], np.float64)
        for j in range(s):
            acc += hr[s * k + j]
        out[k] = acc / s
    return out


def downsample_adjoint(dlr, nz: int, s: int) -> np.ndarray:
    """Adjoint of ``downsample``: dHR[z] = dLR[z // s] / s for z < s floor(nz/s), else 0."""
    dlr = np.asarray(dlr, dtype=np.float64)
    out = np.zeros((nz,) + dlr.shape[1:], np.float64)
    for z in range(s * (nz // s)):
        out[z] = dlr[z // s] / s
    return out


def resample_map(n_src: int, n_dst: int):
    """One axis of the trilinear resize that makes the LR inputs (Sec. 4.1: volumes are
    "downsampled via trilinear interpolation"; the sampling convention is not given).

    Reading: half-pixel centres, i.e. destination sample j sits at the source continuous
    index c_j = (n_src / n_dst)(j + 1/2) - 1/2, raised to 0 where it is negative; it reads
    source samples i0 = floor(c_j) and i1 = min(i0 + 1, n_src - 1) with weights 1 - w and
    w = c_j - i0. The position c_j decides the integers i0, so it is taken in FP32, one
    rounding per operation, as the CUDA kernels take it; the weights are then FP64.
    Returns (i0, i1, w) arrays of length n_dst.
    """
    scale = np.float32(n_src) / np.float32(n_dst)
    j = np.arange(n_dst, dtype=np.float32)
    c = scale * (j + np.float32(0.5)) - np.float32(0.5)
    c = np.maximum(c, np.float32(0.0))
    i0 = np.floor(c).astype(np.int64)
    i1 = np.minimum(i0 + 1, n_src - 1)
    w = c.astype(np.float64) - i0
    return i0, i1, w


def resample(vol, out_shape) -> np.ndarray:
    """Trilinear resize of a [z, y, x] volume to ``out_shape``: every output voxel is the sum
    over the 8 corners of its source cell of w_z w_y w_x times the corner value
    (``resample_map`` along each axis)."""
    vol = np.asarray(vol, np.float64)
    maps = [resample_map(vol.shape[a], out_shape[a]) for a in range(3)]
    out = np.zeros(tuple(out_shape), np.float64)
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                iz = maps[0][1] if cz else maps[0][0]
                iy = maps[1][1] if cy else maps[1][0]
                ix = maps[2][1] if cx else maps[2][0]
                wz = maps[0][2] if cz else 1.0 - maps[0][2]
                wy = maps[1][2] if cy else 1.0 - maps[1][2]
                wx = maps[2][2] if cx else 1.0 - maps[2][2]
                w = wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
                out += w * vol[np.ix_(iz, iy, ix)]
    return out


def resample_adjoint(dout, in_shape) -> np.ndarray:
    """Adjoint (transpose) of ``resample``: each output voxel's value is added back to its 8
    source corners with the same weights."""
    dout = np.asarray(dout, np.float64)
    maps = [resample_map(in_shape[a], dout.shape[a]) for a in range(3)]
    din = np.zeros(tuple(in_shape), np.float64)
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                iz = maps[0][1] if cz else maps[0][0]
                iy = maps[1][1] if cy else maps[1][0]
                ix = maps[2][1] if cx else maps[2][0]
                wz = maps[0][2] if cz else 1.0 - maps[0][2]
                wy = maps[1][2] if cy else 1.0 - maps[1][2]
                wx = maps[2][2] if cx else 1.0 - maps[2][2]
                w = wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
                Z, Y, X = np.meshgrid(iz, iy, ix, indexing="ij")
                np.add.at(din, (Z, Y, X), w * dout)
    return din


def resample_grid(grid_hr: Grid, lr_shape) -> Grid:
    """The LR grid of a trilinear resize: same field of view and origin as the HR grid,
    spacing L_a / n_a (destination sample j of ``resample_map`` is the centre of LR voxel j)."""
    nz, ny, nx = lr_shape
    n_hr = (grid_hr.nx, grid_hr.ny, grid_hr.nz)
    n_lr = (nx, ny, nz)
    h = tuple(grid_hr.h[a] * n_hr[a] / n_lr[a] for a in range(3))
    return Grid(nx, ny, nz, h, grid_hr.origin)


def l1_loss(pred, target):
    """Mean absolute error and its gradient sign(pred - target) / n (sign(0) = 0)."""
    pred = np.asarray(pred, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    diff = pred - target
    n = diff.size
    return float(np.abs(diff).sum() / n), np.sign(diff) / n


# ------------------------------------------------------------------------- Adam

@dataclass
class AdamConfig:
    """Adam with per-group learning rates (the paper gives no optimiser; these follow the
    fitting configuration: 1e-3 on means, 5e-3 on scales and tissue parameters)."""
    lr_mu: float = 1e-3
    lr_scale: float = 5e-3
    lr_rot: float = 5e-3
    lr_a: float = 5e-3
    lr_t: float = 5e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8

    def lr_vector(self):
        return np.array([self.lr_mu] * 3 + [self.lr_scale] * 3 + [self.lr_rot] * 4
                        + [self.lr_a, self.lr_t], dtype=np.float64)


def adam_step(params, grad, m, v, step: int, acfg: AdamConfig = AdamConfig()):
    """One Adam update (Kingma & Ba 2015, bias-corrected); ``step`` counts from 1."""
    params = np.asarray(params, np.float64).copy()
    g = np.asarray(grad, np.float64)
    m = acfg.beta1 * np.asarray(m, np.float64) + (1 - acfg.beta1) * g
    v = acfg.beta2 * np.asarray(v, np.float64) + (1 - acfg.beta2) * g * g
    mhat = m / (1 - acfg.beta1 ** step)
    vhat = v / (1 - acfg.beta2 ** step)
    lr = acfg.lr_vector()[None, :]
    params -= lr * mhat / (np.sqrt(vhat) + acfg.eps)
    return params, m, v


# ------------------------------------------------------------------ initialisation

def lattice_dims(grid: Grid, n_target: int):
    """Lattice of about n_target points over the volume with isotropic spacing
    l = (V / n_target)^(1/3): n_a = max(1, round(L_a / l)) points along axis a."""
    L = np.array([grid.nx * grid.h[0], grid.ny * grid.h[1], grid.nz * grid.h[2]])
    ell = (L.prod() / n_target) ** (1.0 / 3.0)
    n = [max(1, int(round(L[a] / ell))) for a in range(3)]
    return n, L


def trilinear(vol, grid_lr: Grid, pts) -> np.ndarray:
    """Trilinear sample of ``vol`` ([z, y, x] on ``grid_lr``) at world points ``pts`` [M, 3],
    with edge clamping (the continuous index is clamped to [0, n-1])."""
    vol = np.asarray(vol, np.float64)
    out = np.empty(pts.shape[0], np.float64)
    n = (grid_lr.nx, grid_lr.ny, grid_lr.nz)
    u = np.empty_like(pts, dtype=np.float64)
    for a in range(3):
        u[:, a] = (pts[:, a] - grid_lr.origin[a]) / grid_lr.h[a] - 0.5
        u[:, a] = np.clip(u[:, a], 0.0, n[a] - 1)
    i0 = np.floor(u).astype(np.int64)
    i1 = np.minimum(i0 + 1, np.array(n) - 1)
    f = u - i0
    out[:] = 0.0
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                wx = f[:, 0] if cx else 1.0 - f[:, 0]
                wy = f[:, 1] if cy else 1.0 - f[:, 1]
                wz = f[:, 2] if cz else 1.0 - f[:, 2]
                xi = i1[:, 0] if cx else i0[:, 0]
                yi = i1[:, 1] if cy else i0[:, 1]
                zi = i1[:, 2] if cz else i0[:, 2]
                out += wx * wy * wz * vol[zi, yi, xi]
    return out


def init_lattice(lr_vol, grid_hr: Grid, s: int, n_target: int, t_act: int = 1,
                 t_init: float = 0.5):
    """Initial Gaussians from the LR volume ("3D Gaussians are initialized solely from the
    coordinates of the low-resolution volume", Fig. 1 caption; details are not given).

    Reading: an axis lattice (``lattice_dims``) with centres at the cell centres, amplitude
    = trilinear sample of the LR volume at the centre, T = t_init, isotropic-per-axis scale
    s_a = l_a / 2 (l_a = L_a / n_a), identity rotation. The LR grid has spacing (h_x, h_y,
    s h_z) and the HR origin. Returns float32 ``[N, 12]`` raw parameters.
    """
    grid_lr = Grid(grid_hr.nx, grid_hr.ny, grid_hr.nz // s,
                   (grid_hr.h[0], grid_hr.h[1], grid_hr.h[2] * s), grid_hr.origin)
    return init_lattice_on(lr_vol, grid_lr, grid_hr, n_target, t_act, t_init)


def init_lattice_lr(lr_vol, grid_hr: Grid, n_target: int, t_act: int = 1,
                    t_init: float = 0.5):
    """``init_lattice`` for an LR volume made by the trilinear resize: the LR grid is
    ``resample_grid(grid_hr, lr_vol.shape)``."""
    grid_lr = resample_grid(grid_hr, np.asarray(lr_vol).shape)
    return init_lattice_on(lr_vol, grid_lr, grid_hr, n_target, t_act, t_init)


def init_lattice_on(lr_vol, grid_lr: Grid, grid_hr: Grid, n_target: int, t_act: int = 1,
                    t_init: float = 0.5):
    """The lattice of ``init_lattice`` over the HR field of view, amplitudes sampled from
    ``lr_vol`` on ``grid_lr``."""
    n, L = lattice_dims(grid_hr, n_target)
    ell = [L[a] / n[a] for a in range(3)]
    xs = [grid_hr.origin[a] + (np.arange(n[a]) + 0.5) * ell[a] for a in range(3)]
    zz, yy, xx = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    pts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    A = trilinear(lr_vol, grid_lr, pts)
    N = pts.shape[0]
    out = np.zeros((N, 12), np.float64)
    out[:, 0:3] = pts
    out[:, 3:6] = np.log(0.5 * np.array(ell))[None, :]
    out[:, 6] = 1.0
    out[:, 10] = A
    out[:, 11] = math.log(t_init / (1.0 - t_init)) if t_act else t_init
    return out.astype(np.float32)


# ---------------------------------------------------------------- phantom (oracle side)

def phantom_from_draws(ph: dict, TR: float, TE: float):
    """HR phantom from the seeded draws of ``inputs.phantom_draws``: intensity of ellipsoid
    e = PD_e T(T1_e, T2_e) (Eq. 2 signal), background 0, normalised to [0, 1] by the
    largest tissue intensity (Sec. 4.1 normalises every volume to [0, 1])."""
    tissue = ph["pd"] * signal_proxy(ph["t1"], ph["t2"], TR, TE)
    table = np.concatenate([[0.0], tissue])
    present = np.unique(ph["label"])
    vmax = table[present].max()
    return table[ph["label"]] / (vmax if vmax > 0 else 1.0)


def rician(lr, n1, n2):
    """Magnitude of the complex signal LR + n1 + i n2 (Rician noise on a magnitude image)."""
    lr = np.asarray(lr, np.float64)
    return np.sqrt((lr + n1) ** 2 + n2 ** 2)


# --------------------------------------------------------------------- metrics

def psnr(x, ref, data_range: float = 1.0) -> float:
    """Peak signal-to-noise ratio over the whole volume (data range 1, Sec. 4.1)."""
    mse = float(np.mean((np.asarray(x, np.float64) - np.asarray(ref, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * math.log10(data_range ** 2 / mse)


def ssim3d(x, ref, data_range: float = 1.0, sigma: float = 1.5) -> float:
    """Mean SSIM (Wang et al. 2004, cited in Sec. 4.2) in 3D with a Gaussian window of
    std ``sigma`` voxels, K1 = 0.01, K2 = 0.03 (window and constants are readings)."""
    from scipy.ndimage import gaussian_filter
    x = np.asarray(x, np.float64)
    y = np.asarray(ref, np.float64)
    c1 = (0.01 * data_range) ** 2
    c2 = (0.03 * data_range) ** 2
    f = lambda a: gaussian_filter(a, sigma, mode="reflect", truncate=3.5)
    mx, my = f(x), f(y)
    sxx = f(x * x) - mx * mx
    syy = f(y * y) - my * my
    sxy = f(x * y) - mx * my
    num = (2 * mx * my + c1) * (2 * sxy + c2)
    den = (mx * mx + my * my + c1) * (sxx + syy + c2)
    return float(np.mean(num / den))


# ------------------------------------------------------------------- fitting step

def fit_step(params, lr_target, grid: Grid, s: int, cfg: Config, m, v, step: int,
             acfg: AdamConfig = AdamConfig(), lr_model: str = "zbox"):
    """One zero-shot fitting iteration, composed of the pinned pieces above: render
    (Eq. 3-4), the LR forward model (``lr_model`` "zbox": z box slice profile of factor s;
    "trilinear": trilinear resize to lr_target's shape), L1 against the LR scan, the forward
    model's adjoint, adjoint render (Eq. 5-6 and the chain), Adam.
    Returns dict(loss, grad, params, m, v, I, lr_pred)."""
    p = np.asarray(params, np.float64)
    r = render(p, grid, cfg)
    if lr_model == "trilinear":
        lr_pred = resample(r["I"], np.asarray(lr_target).shape)
    else:
        lr_pred = downsample(r["I"], s)
    loss, dlr = l1_loss(lr_pred, lr_target)
    if lr_model == "trilinear":
        dI = resample_adjoint(dlr, r["I"].shape)
    else:
        dI = downsample_adjoint(dlr, grid.nz, s)
    grad = render_grad(p, grid, dI, cfg)
    p2, m2, v2 = adam_step(p, grad, m, v, step, acfg)
    return dict(loss=loss, grad=grad, params=p2, m=m2, v=v2, I=r["I"], lr_pred=lr_pred,
                amb=r["amb"])


# ------------------------------------------------ validating a renderer's tie decisions

def _subset_masks(n: int) -> np.ndarray:
    """[2^n, n] 0/1 matrix: row s lists which of n items subset s includes (bit k of s)."""
    s = np.arange(1 << n)[:, None]
    return ((s >> np.arange(n)[None, :]) & 1).astype(np.float64)


def forward_subset_check(I, W, ref, tol: float = 1e-5, tol_w=1e-5, w_min: float = 1e-6,
                         eps: float = 1e-12, max_unenum_frac: float = 1e-3):
    """Check a rendered (I, W) against ``render(..., want_amb=True)`` output ``ref``, voxel by
    voxel, accepting any include/exclude decision on the ambiguous pairs (Sec. 3.3 truncation
    read as d^2 <= sigma_t^2; a pair within the band may be decided either way by rounding).

    A voxel passes if some subset s of its ambiguous pairs gives W_s = W_sure + sum_{k in s} w_k
    with |W - W_s| <= tol_w max(W_s, w_min) and, where W_s > w_min, I_s = S_s / max(W_s, eps)
    with |I - I_s| <= tol |I_s|. Voxels with no ambiguous pair must match the FP64 decision
    (a voxel no Gaussian reaches renders exactly zero). ``tol`` and ``tol_w`` may be arrays
    (per voxel).
    Voxels with more than AMB_SLOTS ambiguous pairs cannot be enumerated; their share of the
    voxels with W > w_min must stay below ``max_unenum_frac``.

    Returns a dict of statistics, including ``flips`` (ambiguous pairs whose matched decision
    differs from the FP64 one) and ``max_flip_rel`` (the largest |d^2 - sigma_t^2| /
    sum_ab |C_ab d_a d_b| among them). Raises AssertionError on failure."""
    I = np.asarray(I, np.float64)
    W = np.asarray(W, np.float64)
    amb = ref["amb"]
    tw = np.broadcast_to(np.asarray(tol_w, np.float64), amb.shape)
    ti = np.broadcast_to(np.asarray(tol, np.float64), amb.shape)
    live = ref["W"] > w_min
    stats = dict(n_live=int(live.sum()), n_plain=0, n_tie=0, n_unenum=0, flips=0,
                 tie_pairs=0, max_flip_rel=0.0, max_relI=0.0, max_relW=0.0)
    # voxels without ambiguous pairs: the FP64 decision is the only valid one
    m = live & (amb == 0)
    Io, Wo = ref["I"][m], ref["W"][m]
    relI = np.abs(I[m] - Io) / np.maximum(np.abs(Io), 1e-30)
    relW = np.abs(W[m] - Wo) / Wo
    stats["n_plain"] = int(m.sum())
    if m.any():
        stats["max_relI"] = float(relI.max())
        stats["max_relW"] = float(relW.max())
        stats["max_relW_over_tol"] = float((relW / tw[m]).max())
        stats["max_relI_over_tol"] = float((relI / ti[m]).max())
        bad = (relI > ti[m]) | (relW > tw[m])
        assert not bad.any(), ("plain voxels", int(bad.sum()), float(relI.max()),
                               float(relW.max()))
    none = (ref["W"] == 0) & (amb == 0)
    assert np.all(W[none] == 0) and np.all(I[none] == 0), "voxels nobody reaches"
    # voxels with 1..AMB_SLOTS ambiguous pairs: some subset must match
    for n in range(1, AMB_SLOTS + 1):
        sel = amb == n
        if not sel.any():
            continue
        masks = _subset_masks(n)
        vw = ref["amb_vw"][sel][:, :n]
        w = ref["amb_w"][sel][:, :n]
        Ws = ref["W_sure"][sel][:, None] + w @ masks.T
        Ss = ref["S_sure"][sel][:, None] + vw @ masks.T
        Is = Ss / np.maximum(Ws, eps)
        Wg, Ig, twv, tiv = W[sel][:, None], I[sel][:, None], tw[sel][:, None], ti[sel][:, None]
        errW = np.abs(Wg - Ws) / np.maximum(Ws, w_min)
        errI = np.abs(Ig - Is) / np.maximum(np.abs(Is), 1e-30)
        okI = (Ws <= w_min) | (errI <= tiv)
        ok = (errW <= twv) & okI
        good = ok.any(axis=1)
        assert good.all(), ("tie voxels", int((~good).sum()), n)
        # the matching subset with the smallest error, against the FP64 decisions
        score = np.where(ok, errW + np.where(Ws > w_min, errI, 0.0), np.inf)
        best = masks[np.argmin(score, axis=1)]
        fp64 = (ref["amb_rel"][sel][:, :n] <= 0).astype(np.float64)
        flip = best != fp64
        rel = np.abs(ref["amb_rel"][sel][:, :n])
        stats["n_tie"] += int(sel.sum())
        stats["tie_pairs"] += int(n * sel.sum())
        stats["flips"] += int(flip.sum())
        if flip.any():
            stats["max_flip_rel"] = max(stats["max_flip_rel"], float(rel[flip].max()))
    un = live & (amb > AMB_SLOTS)
    stats["n_unenum"] = int(un.sum())
    assert stats["n_unenum"] <= max_unenum_frac * max(stats["n_live"], 1), stats
    return stats


def gradient_box_check(got, box, tol: float = 1e-4, group_tol: float = 1e-3):
    """Check a gradient ``got`` [N, 12] against ``render_grad(..., want_box=True)`` output:
    the distance from ``got`` to the box [lo, hi] (the gradients of every decision on the
    ambiguous pairs) must be at most ``tol`` of the FP64 gradient's norm (relative L2), and per
    parameter group (means, log-scales, quaternion, a, t) at most ``group_tol`` of the group's
    norm (floored at 1e-3 of the total: rotation gradients of isotropic Gaussians vanish).
    Returns (distance, relative box width)."""
    got = np.asarray(got, np.float64)
    ref, lo, hi = box["grad"], box["lo"], box["hi"]
    assert box["n_unenum"] == 0, box["n_unenum"]
    proj = np.clip(got, lo, hi)
    tot = float(np.linalg.norm(ref))
    den = tot if tot > 0 else 1.0
    dist = float(np.linalg.norm(got - proj)) / den
    assert dist <= tol, dist
    for a, b in ((0, 3), (3, 6), (6, 10), (10, 11), (11, 12)):
        diff = np.linalg.norm(got[:, a:b] - proj[:, a:b])
        gden = max(np.linalg.norm(ref[:, a:b]), 1e-3 * tot)
        assert diff <= group_tol * gden, (a, b, diff / gden)
    return dist, float(np.linalg.norm(hi - lo)) / den
