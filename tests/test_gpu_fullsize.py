"""Parity at full workload sizes, on sampled crops the FP64 oracle computes from every Gaussian:
the stress workload (512 x 512 x 256 grid, 4M clustered, strongly anisotropic Gaussians in 20
blobs: one axis scale 4-8 voxels, the others 0.5-1.5), forward and adjoint in both reduction
modes, and the full fit's size (256 x 256 x 160 phantom, 1M lattice Gaussians), forward. The
GPU renders the whole volume in the launch configuration the benchmarks time; the oracle
renders 24^3 crops (a dense blob core and a sparse edge) with the same tie handling as the
smaller parity tests."""
import functools

import numpy as np
import pytest

from helpers import cloud_params, phantom_fit, to_dev
from paper_2603_09621_gb300 import inputs

pytestmark = pytest.mark.gpu
STRESS = (256, 512, 512)   # (nz, ny, nx)


def _gs():
    from paper_2603_09621_gb300 import gs
    return gs


@functools.lru_cache(maxsize=None)
def _stress():
    import oracle
    d = inputs.gmm_cloud(0, 4_000_000, STRESS)
    p = cloud_params(d)
    nz, ny, nx = STRESS
    # the densest 24^3 cell of means (a blob core) and a corner cell
    h, edges = np.histogramdd(p[:, [2, 1, 0]], bins=(nz // 24, ny // 24, nx // 24),
                              range=((0, nz // 24 * 24), (0, ny // 24 * 24), (0, nx // 24 * 24)))
    cz, cy, cx = np.unravel_index(np.argmax(h), h.shape)
    dense = (24 * cx, 24 * cy, 24 * cz)
    return p, oracle.Grid(nx, ny, nz), dense


def _crop(c):
    x0, y0, z0 = c
    return (x0, x0 + 24, y0, y0 + 24, z0, z0 + 24), (slice(z0, z0 + 24), slice(y0, y0 + 24),
                                                     slice(x0, x0 + 24))


def _check_forward(I, W, ref):
    import oracle
    from test_gpu_render import tol_i, tol_w
    st = oracle.forward_subset_check(I, W, ref, tol=tol_i(ref), tol_w=tol_w(ref))
    print("forward check:", st)
    return st


def test_stress_forward_crops():
    import torch
    import oracle
    gs = _gs()
    p, og, dense = _stress()
    g = gs.Grid(og.nx, og.ny, og.nz)
    I, W, bins, _ = gs.render(to_dev(p), g, gs.Config())
    torch.cuda.synchronize()
    assert bins.status() == 0
    It, Wt = I.cpu().numpy(), W.cpu().numpy()
    for c in (dense, (488, 0, 232)):
        crop, sl = _crop(c)
        ref = oracle.render(p.astype(np.float64), og, crop=crop, want_amb=True)
        st = _check_forward(It[sl], Wt[sl], ref)
        assert st["n_live"] > 0
    # the dense crop really is dense: hundreds of pairs per voxel
    ref = oracle.render(p.astype(np.float64), og, crop=_crop(dense)[0])
    assert ref["npair"].mean() > 100


@pytest.mark.parametrize("det", [1, 0])
def test_stress_gradient_dense_crop(det):
    """dL/dI random on the dense 24^3 crop and zero elsewhere; the gradient of all 4M
    Gaussians against the oracle's box over the crop's tie decisions."""
    import torch
    import oracle
    from test_gpu_backward import check_grad, oracle_box
    gs = _gs()
    p, og, dense = _stress()
    crop, sl = _crop(dense)
    dIc = inputs.crop_dI(31, (24, 24, 24)).astype(np.float64)
    box = oracle_box(p, og, dIc, crop=crop)
    g = gs.Grid(og.nx, og.ny, og.nz)
    cfg = gs.Config(deterministic=det)
    pd = to_dev(p)
    I, W, bins, ws = gs.render(pd, g, cfg)
    dI = torch.zeros(STRESS, device="cuda")
    dI[sl] = to_dev(dIc.astype(np.float32))
    got = gs.gs_render_bwd(pd, bins, g, cfg, I, W, dI, ws)
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    touched = (np.abs(box["lo"]).sum(1) + np.abs(box["hi"]).sum(1)) > 0
    assert touched.sum() > 10000
    assert np.all(got[~touched] == 0)
    check_grad(got, box)


def test_full_fit_size_forward_crops():
    """256 x 256 x 160 phantom, 1M lattice Gaussians (the full fit's size): the GPU render of
    the initial cloud on two crops."""
    import torch
    import oracle
    gs = _gs()
    w = phantom_fit(shape=(160, 256, 256), s=2, n_gauss=1_000_000, seed=0)
    og = w["grid"]
    I, W, bins, _ = gs.render(to_dev(w["params0"]), gs.Grid(og.nx, og.ny, og.nz),
                              gs.Config(t_act=1))
    torch.cuda.synchronize()
    assert bins.status() == 0
    It, Wt = I.cpu().numpy(), W.cpu().numpy()
    for c in ((120, 60, 70), (232, 232, 136)):
        crop, sl = _crop(c)
        ref = oracle.render(w["params0"].astype(np.float64), og, oracle.Config(t_act=1),
                            crop=crop, want_amb=True)
        _check_forward(It[sl], Wt[sl], ref)
