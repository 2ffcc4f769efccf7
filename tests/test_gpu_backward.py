"""Adjoint render on the GPU (Eq. 5-6 and the chain to raw parameters) against the FP64
oracle gradient (relative L2 <= 1e-4), plus determinism, fast (atomic) mode, and central
finite differences through the autograd Function.

dL/dI is nonzero at every voxel, those with pairs in the ambiguity band of the truncation
boundary included: the oracle bounds the gradient of every include/exclude decision on such
pairs (a box per Gaussian and parameter), and the GPU gradient must lie within 1e-4 (relative
L2) of that box. Where no tie is involved the box is the FP64 gradient itself."""
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


def oracle_box(p, og, dI, cfg=None, crop=None):
    import oracle
    return oracle.render_grad(np.asarray(p, np.float64), og, np.asarray(dI, np.float64),
                              cfg or oracle.Config(), crop=crop, want_box=True)


def check_grad(got, box, tol=TOL):
    import oracle
    dist, width = oracle.gradient_box_check(got, box, tol=tol, group_tol=10 * tol)
    print(f"gradient check: distance to the box {dist:.2e} (relative L2), box width {width:.2e}")
    return dist


@pytest.mark.parametrize("det", [1, 0])
def test_grad_forward_workload(det):
    """32^3, 4,096 Gaussians: GPU adjoint vs FP64 oracle, both reduction modes."""
    import oracle
    params, og = c1()
    dI = inputs.crop_dI(1, (og.nz, og.ny, og.nx))
    got = gpu_grad(params, og, dI, deterministic=det)
    check_grad(got, oracle_box(params, og, dI))
    # and strictly against the FP64 decisions where dL/dI avoids every tie voxel
    ref_f = oracle.render(params.astype(np.float64), og)
    dIm = masked_dI(1, og, ref_f["amb"])
    ref = oracle.render_grad(params.astype(np.float64), og, dIm.astype(np.float64))
    err = rel_l2(gpu_grad(params, og, dIm, deterministic=det), ref)
    assert err <= TOL, err


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
    dI = inputs.crop_dI(3, (og.nz, og.ny, og.nx))
    got = gpu_grad(p, og, dI, signal_mode=mode, a_act=a_act, t_act=t_act, brick=brick)
    check_grad(got, oracle_box(p, og, dI, cfg))


@pytest.mark.parametrize("brick", [(8, 8, 8), (8, 8, 4)])
def test_grad_fit_workload_crop(brick):
    """Fitting workload (256 x 256 x 128, 500k Gaussians): dL/dI random on a 24^3 crop and
    zero elsewhere; every Gaussian's gradient compared with the oracle's, with the fitting
    workload's bricks and the paper's."""
    import oracle
    w = phantom_fit()
    og = w["grid"]
    x0, y0, z0 = 116, 116, 52
    crop = (x0, x0 + 24, y0, y0 + 24, z0, z0 + 24)
    cfg = oracle.Config(t_act=1)
    dIc = inputs.crop_dI(5, (24, 24, 24)).astype(np.float64)
    box = oracle_box(w["params0"], og, dIc, cfg, crop=crop)
    dI = np.zeros((og.nz, og.ny, og.nx), np.float32)
    dI[z0:z0 + 24, y0:y0 + 24, x0:x0 + 24] = dIc
    got = gpu_grad(w["params0"], og, dI, t_act=1, brick=brick)
    touched = (np.abs(box["lo"]).sum(1) + np.abs(box["hi"]).sum(1)) > 0
    assert touched.sum() > 1000
    assert np.all(got[~touched] == 0)
    check_grad(got, box)


def test_grad_clustered_anisotropic():
    import oracle
    og = oracle.Grid(48, 48, 48)
    d = inputs.gmm_cloud(8, 6000, (48, 48, 48), n_blobs=3, blob_std=6.0)
    p = cloud_params(d)
    dI = inputs.crop_dI(6, (og.nz, og.ny, og.nx))
    box = oracle_box(p, og, dI)
    for det in (1, 0):
        check_grad(gpu_grad(p, og, dI, deterministic=det), box)
    # and strictly against the FP64 decisions where dL/dI avoids every tie voxel
    ref_f = oracle.render(p.astype(np.float64), og)
    dIm = masked_dI(6, og, ref_f["amb"])
    ref = oracle.render_grad(p.astype(np.float64), og, dIm.astype(np.float64))
    err = rel_l2(gpu_grad(p, og, dIm), ref)
    assert err <= TOL, err


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
    dI = inputs.crop_dI(22, (og.nz, og.ny, og.nx))
    box = oracle_box(p, og, dI)
    for det in (1, 0):
        check_grad(gpu_grad(p, og, dI, deterministic=det), box)
