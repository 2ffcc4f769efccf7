"""Adjoint render on the GPU (Eq. 5-6 and the chain to raw parameters) against the FP64
oracle gradient (relative L2 <= 1e-4), plus determinism, fast (atomic) mode, and central
finite differences through the autograd Function."""
import numpy as np
import pytest

from helpers import c1, cloud_params, phantom_fit, rel_l2, to_dev
from paper_2603_09621_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _gs():
    from paper_2603_09621_gb300 import gs
    return gs


def _grid(og):
    return _gs().Grid(og.nx, og.ny, og.nz, tuple(og.h), tuple(og.origin))


def gpu_grad(params_np, og, dI_np, deterministic=1, brick=(8, 8, 8), signal_mode=0, a_act=0,
             t_act=0):
    import torch
    gs = _gs()
    cfg = gs.Config(brick=brick, deterministic=deterministic, signal_mode=signal_mode,
                    a_act=a_act, t_act=t_act)
    g = _grid(og)
    p = to_dev(params_np.astype(np.float32))
    I, W, bins, ws = gs.render(p, g, cfg)
    dp = gs.gs_render_bwd(p, bins, g, cfg, I, W, to_dev(dI_np.astype(np.float32)), ws)
    torch.cuda.synchronize()
    return dp.cpu().numpy()


def masked_dI(seed, og, ref_amb):
    """Random dL/dI, zero where a pair is on the truncation boundary (ambiguous voxels)."""
    dI = inputs.crop_dI(seed, (og.nz, og.ny, og.nx))
    dI[ref_amb > 0] = 0.0
    return dI


def check_grad(got, ref, tol=TOL):
    err = rel_l2(got, ref)
    assert err <= tol, err
    # per parameter group (means, log-scales, quaternion, a, t), looser; a group whose exact
    # gradient vanishes (e.g. rotations of isotropic Gaussians) is held to the overall scale
    tot = np.linalg.norm(ref)
    for a, b in ((0, 3), (3, 6), (6, 10), (10, 11), (11, 12)):
        diff = np.linalg.norm(got[:, a:b] - ref[:, a:b])
        den = max(np.linalg.norm(ref[:, a:b]), 1e-3 * tot)
        assert diff <= 10 * tol * den, (a, b, diff / den)
    return err


@pytest.mark.parametrize("det", [1, 0])
def test_grad_forward_workload(det):
    """32^3, 4,096 Gaussians: GPU adjoint vs FP64 oracle, both reduction modes."""
    import oracle
    params, og = c1()
    ref_f = oracle.render(params.astype(np.float64), og)
    dI = masked_dI(1, og, ref_f["amb"])
    ref = oracle.render_grad(params.astype(np.float64), og, dI.astype(np.float64))
    got = gpu_grad(params, og, dI, deterministic=det)
    check_grad(got, ref)


def test_grad_deterministic_bitwise():
    params, og = c1()
    dI = inputs.crop_dI(2, (og.nz, og.ny, og.nx))
    a = gpu_grad(params, og, dI, deterministic=1)
    b = gpu_grad(params, og, dI, deterministic=1)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("mode,a_act,t_act,brick", [(1, 0, 0, (8, 8, 8)), (0, 1, 1, (8, 8, 4)),
                                                    (1, 1, 1, (4, 4, 4)), (0, 0, 1, (16, 8, 4))])
def test_grad_modes_activations_bricks(mode, a_act, t_act, brick):
    import oracle
    og = oracle.Grid(33, 27, 19, (1.1, 0.9, 1.3), (0.5, -1.0, 2.0))
    d = inputs.gaussian_cloud(9, 1500, (19, 27, 33), h=og.h)
    d["mu"] = d["mu"] + np.array(og.origin, np.float32)
    p = cloud_params(d)
    rng = np.random.default_rng(4)
    if a_act:
        p[:, 10] = rng.normal(0, 1.5, p.shape[0])
    if t_act:
        p[:, 11] = rng.normal(-0.5, 1.5, p.shape[0])
    cfg = oracle.Config(signal_mode=mode, a_act=a_act, t_act=t_act, brick=brick)
    ref_f = oracle.render(p.astype(np.float64), og, cfg)
    dI = masked_dI(3, og, ref_f["amb"])
    ref = oracle.render_grad(p.astype(np.float64), og, dI.astype(np.float64), cfg)
    got = gpu_grad(p, og, dI, signal_mode=mode, a_act=a_act, t_act=t_act, brick=brick)
    check_grad(got, ref)


def test_grad_fit_workload_crop():
    """Fitting workload (256 x 256 x 128, 500k Gaussians): dL/dI random on a 24^3 crop and
    zero elsewhere; every Gaussian's gradient compared with the oracle's."""
    import oracle
    w = phantom_fit()
    og = w["grid"]
    x0, y0, z0 = 116, 116, 52
    crop = (x0, x0 + 24, y0, y0 + 24, z0, z0 + 24)
    p64 = w["params0"].astype(np.float64)
    cfg = oracle.Config(t_act=1)
    ref_f = oracle.render(p64, og, cfg, crop=crop)
    dIc = inputs.crop_dI(5, (24, 24, 24)).astype(np.float64)
    dIc[ref_f["amb"] > 0] = 0.0
    ref = oracle.render_grad(p64, og, dIc, cfg, crop=crop)
    dI = np.zeros((og.nz, og.ny, og.nx), np.float32)
    dI[z0:z0 + 24, y0:y0 + 24, x0:x0 + 24] = dIc
    got = gpu_grad(w["params0"], og, dI, t_act=1)
    touched = np.abs(ref).sum(1) > 0
    assert touched.sum() > 1000
    assert np.all(got[~touched] == 0)
    check_grad(got, ref)


def test_grad_clustered_anisotropic():
    import oracle
    og = oracle.Grid(48, 48, 48)
    d = inputs.gmm_cloud(8, 6000, (48, 48, 48), n_blobs=3, blob_std=6.0)
    p = cloud_params(d)
    ref_f = oracle.render(p.astype(np.float64), og)
    dI = masked_dI(6, og, ref_f["amb"])
    ref = oracle.render_grad(p.astype(np.float64), og, dI.astype(np.float64))
    for det in (1, 0):
        check_grad(gpu_grad(p, og, dI, deterministic=det), ref)


def test_autograd_function_central_differences():
    """torch.autograd.Function around the library: FP32 central differences of
    L = sum(dI * I) on a well-conditioned cloud (loose tolerance: FP32 differencing)."""
    import torch
    gs = _gs()
    og = gs.Grid(16, 16, 16)
    d = inputs.gaussian_cloud(12, 40, (16, 16, 16), scale_range=(1.0, 2.0))
    import oracle  # noqa: F401
    p = to_dev(cloud_params(d)).requires_grad_(True)
    w = to_dev(inputs.crop_dI(13, og.shape))
    cfg = gs.Config(trunc_sigma=6.0)
    I = gs.GaussianRender.apply(p, og, cfg)
    (I * w).sum().backward()
    ana = p.grad.detach().cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(0)
    idx = [(int(i), int(k)) for i, k in zip(rng.integers(0, 40, 24), rng.integers(0, 12, 24))]
    for i, k in idx:
        h = 2e-2 if k < 6 else 1e-2
        pp = p.detach().clone()
        pm = p.detach().clone()
        pp[i, k] += h
        pm[i, k] -= h
        lp = float((gs.GaussianRender.apply(pp, og, cfg) * w).double().sum())
        lm = float((gs.GaussianRender.apply(pm, og, cfg) * w).double().sum())
        num = (lp - lm) / (2 * h)
        assert abs(ana[i, k] - num) <= 3e-2 * max(abs(num), 1e-2 * np.abs(ana).max()), (i, k)


def test_grad_sparse_cloud_unstaged_bricks():
    """A sparse cloud (about two pairs per brick): each 256-pair adjoint block spans many
    bricks, so most pairs read their per-voxel factors from the volume instead of the block's
    four staged bricks. Both reduction modes against the FP64 oracle."""
    import torch
    import oracle
    gs = _gs()
    og = oracle.Grid(61, 64, 57)
    d = inputs.gaussian_cloud(21, 350, (57, 64, 61), scale_range=(0.5, 1.5))
    p = cloud_params(d)
    # the path is exercised: blocks of 256 consecutive brick-major pairs span > 4 bricks
    g = _grid(og)
    _, _, bins, _ = gs.render(to_dev(p), g, gs.Config())
    torch.cuda.synchronize()
    pb = bins.pair_brick(bins.npairs()).cpu().numpy()
    spans = [len(np.unique(pb[i:i + 256])) for i in range(0, len(pb), 256)]
    assert max(spans) > 4, spans
    ref_f = oracle.render(p.astype(np.float64), og)
    dI = masked_dI(22, og, ref_f["amb"])
    ref = oracle.render_grad(p.astype(np.float64), og, dI.astype(np.float64))
    for det in (1, 0):
        check_grad(gpu_grad(p, og, dI, deterministic=det), ref)
