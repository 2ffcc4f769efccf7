"""GPU-side assembly of the synthetic workloads from the seeded draws of ``inputs``.

The method's arithmetic (Eq. 2 relaxation proxy, slice profile, lattice initialisation) runs
in libgsmri; torch does data movement (table lookup, copies) and the Rician noise of the
synthetic LR scan (noise synthesis, not a step of the method).
"""
from __future__ import annotations

import numpy as np
import torch

from . import gs, inputs

TR, TE = inputs.TR_MS, inputs.TE_MS


def cloud_params(d: dict, device="cuda") -> torch.Tensor:
    """Raw [N, 12] params on the device: a = PD, t = T(T1, T2) by the library's Eq. 2."""
    t1 = torch.as_tensor(d["t1"], dtype=torch.float32, device=device)
    t2 = torch.as_tensor(d["t2"], dtype=torch.float32, device=device)
    T = gs.gs_signal_proxy(t1, t2, TR, TE)
    n = t1.numel()
    out = torch.empty((n, 12), dtype=torch.float32, device=device)
    out[:, 0:3] = torch.as_tensor(d["mu"], device=device)
    out[:, 3:6] = torch.as_tensor(d["log_s"], device=device)
    out[:, 6:10] = torch.as_tensor(d["q"], device=device)
    out[:, 10] = torch.as_tensor(d["pd"], dtype=torch.float32, device=device)
    out[:, 11] = T
    return out


def lattice_dims(grid: gs.Grid, n_target: int):
    """Axis lattice of about n_target points with isotropic spacing (V / n_target)^(1/3)."""
    L = np.array([grid.nx * grid.h[0], grid.ny * grid.h[1], grid.nz * grid.h[2]])
    ell = (L.prod() / n_target) ** (1.0 / 3.0)
    return [max(1, int(round(L[a] / ell))) for a in range(3)]


def phantom_fit(shape=(128, 256, 256), s=4, n_gauss=500_000, seed=0, n_ell=12,
                semi=(10.0, 80.0), device="cuda"):
    """Fitting workload on the device: HR phantom (for quality metrics), noisy LR scan by the
    z box profile, and the lattice-initialised cloud. Returns dict(grid, hr, lr, params0, s)."""
    nz, ny, nx = shape
    ph = inputs.phantom_draws(seed, shape, n_ell=n_ell, s=s, semi_axes=semi)
    t1 = torch.as_tensor(ph["t1"], dtype=torch.float32, device=device)
    t2 = torch.as_tensor(ph["t2"], dtype=torch.float32, device=device)
    tissue = torch.as_tensor(ph["pd"], dtype=torch.float32, device=device) * gs.gs_signal_proxy(
        t1, t2, TR, TE)
    table = torch.cat([torch.zeros(1, device=device), tissue])
    label = torch.as_tensor(ph["label"], device=device).long()
    present = torch.unique(label)
    vmax = table[present].max()
    hr = (table[label] / torch.where(vmax > 0, vmax, torch.ones_like(vmax))).contiguous()
    lr_clean = gs.gs_downsample_fwd(hr, s)
    n1 = torch.as_tensor(ph["n1"], device=device)
    n2 = torch.as_tensor(ph["n2"], device=device)
    lr = torch.sqrt((lr_clean + n1) ** 2 + n2 ** 2).contiguous()
    grid = gs.Grid(nx, ny, nz)
    nl = lattice_dims(grid, n_gauss)
    params0 = gs.gs_init_lattice(lr, grid, s, nl, t_act=1, t_init=0.5)
    return dict(grid=grid, hr=hr, lr=lr, params0=params0, s=s, nl=nl)


def phantom_fit_trilinear(shape=(155, 240, 240), lr_shape=(100, 100, 100), n_gauss=500_000,
                          seed=0, n_ell=12, semi=(10.0, 80.0), noise_sigma=0.02, device="cuda"):
    """Fitting workload with the trilinear LR model (Sec. 4.1-4.2: LR by trilinear
    downsampling, super-resolution to an arbitrary target shape): HR phantom, noisy LR scan of
    ``lr_shape`` by gs_resample_fwd, lattice init from it. Returns dict(grid, hr, lr,
    params0, nl)."""
    nz, ny, nx = shape
    ph = inputs.phantom_draws(seed, shape, n_ell=n_ell, semi_axes=semi, lr_shape=lr_shape,
                              noise_sigma=noise_sigma)
    t1 = torch.as_tensor(ph["t1"], dtype=torch.float32, device=device)
    t2 = torch.as_tensor(ph["t2"], dtype=torch.float32, device=device)
    tissue = torch.as_tensor(ph["pd"], dtype=torch.float32, device=device) * gs.gs_signal_proxy(
        t1, t2, TR, TE)
    table = torch.cat([torch.zeros(1, device=device), tissue])
    label = torch.as_tensor(ph["label"], device=device).long()
    vmax = table[torch.unique(label)].max()
    hr = (table[label] / torch.where(vmax > 0, vmax, torch.ones_like(vmax))).contiguous()
    lr_clean = gs.gs_resample_fwd(hr, lr_shape)
    n1 = torch.as_tensor(ph["n1"], device=device)
    n2 = torch.as_tensor(ph["n2"], device=device)
    lr = torch.sqrt((lr_clean + n1) ** 2 + n2 ** 2).contiguous()
    grid = gs.Grid(nx, ny, nz)
    nl = lattice_dims(grid, n_gauss)
    params0 = gs.gs_init_lattice_lr(lr, grid, nl, t_act=1, t_init=0.5)
    return dict(grid=grid, hr=hr, lr=lr, params0=params0, nl=nl)


def serving_workload(draws: list, device="cuda", keep_hr: bool = False) -> list:
    """Device inputs of a serving request stream (``inputs.serving_draws``): each fit gets its
    own phantom scan (seeded by its draw), noisy LR target and lattice-initialised cloud; each
    render gets its output grid. Returns the draws with ``grid`` added, and ``params0``,
    ``lr`` (and with ``keep_hr`` the clean HR phantom ``hr``) for fits."""
    out = []
    for d in draws:
        e = dict(d)
        if d["kind"] == "fit":
            w = phantom_fit(shape=d["shape"], s=d["s"], n_gauss=d["n_gauss"], seed=d["seed"],
                            device=device)
            e.update(grid=w["grid"], params0=w["params0"], lr=w["lr"],
                     n_gauss=int(w["params0"].shape[0]))
            if keep_hr:
                e["hr"] = w["hr"]
            del w
        else:
            nz, ny, nx = d["shape"]
            h = float(d["spacing"])
            e.update(grid=gs.Grid(nx, ny, nz, (h, h, h)))
        out.append(e)
    return out
