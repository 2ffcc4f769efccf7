"""Workload builders for the tests: seeded draws from paper_2603_09621_gb300.inputs turned
into oracle-side parameters and volumes (the oracle applies the method's arithmetic; nothing
here comes from the CUDA path)."""
import functools

import numpy as np

from paper_2603_09621_gb300 import inputs

TR, TE = inputs.TR_MS, inputs.TE_MS


def cloud_params(d: dict, signal="eq2") -> np.ndarray:
    """Raw float32 params from cloud draws: a = PD, t = T(T1, T2) by the oracle's Eq. 2
    (identity activations)."""
    import oracle
    T = oracle.signal_proxy(d["t1"], d["t2"], TR, TE)
    return inputs.assemble_params(d["mu"], d["log_s"], d["q"], d["pd"], T)


@functools.lru_cache(maxsize=None)
def c1():
    """Forward-only workload: 32^3 grid at 1 mm, 4,096 Gaussians, seed 0."""
    import oracle
    d = inputs.gaussian_cloud(0, 4096, (32, 32, 32))
    return cloud_params(d), oracle.Grid(32, 32, 32)


@functools.lru_cache(maxsize=None)
def phantom_fit(shape=(128, 256, 256), s=4, n_gauss=500_000, seed=0, n_ell=12,
                semi=(10.0, 80.0)):
    """Fitting workload: ellipsoid phantom, LR by the z box profile (factor s) with Rician
    noise, lattice init of n_gauss Gaussians (sigmoid relaxation activation).
    Returns dict(grid, hr, lr, params0, s)."""
    import oracle
    nz, ny, nx = shape
    ph = inputs.phantom_draws(seed, shape, n_ell=n_ell, s=s, semi_axes=semi)
    hr = oracle.phantom_from_draws(ph, TR, TE)
    lr_clean = oracle.downsample(hr, s)
    lr = oracle.rician(lr_clean, ph["n1"], ph["n2"]).astype(np.float32)
    grid = oracle.Grid(nx, ny, nz)
    params0 = oracle.init_lattice(lr, grid, s, n_gauss, t_act=1)
    return dict(grid=grid, hr=hr.astype(np.float32), lr=lr, params0=params0, s=s)


def rel_l2(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def to_dev(x, device="cuda"):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x)).to(device)


@functools.lru_cache(maxsize=None)
def phantom_fit_trilinear(shape=(40, 48, 56), lr_shape=(17, 20, 23), n_gauss=6000, seed=2,
                          n_ell=5, semi=(5.0, 16.0)):
    """Fitting workload with the trilinear LR model: ellipsoid phantom, LR by the oracle's
    trilinear resize to lr_shape with Rician noise, lattice init from it."""
    import oracle
    nz, ny, nx = shape
    ph = inputs.phantom_draws(seed, shape, n_ell=n_ell, semi_axes=semi, lr_shape=lr_shape)
    hr = oracle.phantom_from_draws(ph, TR, TE)
    lr = oracle.rician(oracle.resample(hr, lr_shape), ph["n1"], ph["n2"]).astype(np.float32)
    grid = oracle.Grid(nx, ny, nz)
    params0 = oracle.init_lattice_lr(lr, grid, n_gauss, t_act=1)
    return dict(grid=grid, hr=hr, lr=lr, params0=params0)
