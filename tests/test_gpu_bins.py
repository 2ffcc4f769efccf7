"""Brick binning on the GPU (Sec. 3.3) against the oracle's FP32 binning specification:
brick lists, offsets and ranges must match bit for bit (integer results)."""
import numpy as np
import pytest

from helpers import c1, cloud_params, phantom_fit, to_dev
from paper_2603_09621_gb300 import inputs

pytestmark = pytest.mark.gpu


def _gs():
    from paper_2603_09621_gb300 import gs
    return gs


def _grid(og):
    return _gs().Grid(og.nx, og.ny, og.nz, tuple(og.h), tuple(og.origin))


def _bin(params_np, og, brick=(8, 8, 8), capacity=None):
    import torch
    gs = _gs()
    cfg = gs.Config(brick=brick)
    g = _grid(og)
    p = to_dev(params_np.astype(np.float32))
    n = p.shape[0]
    cap = capacity if capacity is not None else max(1024, 40 * n)
    bins = gs.Bins(n, cap, g, cfg)
    ws = gs.Workspace(n, cap, g, cfg)
    gs.gs_bin_bricks(p, g, cfg, bins, ws)
    torch.cuda.synchronize()
    return bins


def _compare(params_np, og, brick=(8, 8, 8)):
    import oracle
    ref = oracle.brick_lists(params_np, og, oracle.Config(brick=brick))
    bins = _bin(params_np, og, brick)
    P = bins.npairs()
    assert P == ref["pair_gid"].size
    assert bins.status() == 0
    np.testing.assert_array_equal(bins.brick_off().cpu().numpy(), ref["brick_off"])
    np.testing.assert_array_equal(bins.pair_gid(P).cpu().numpy(), ref["pair_gid"])
    np.testing.assert_array_equal(bins.gm_off().cpu().numpy(), ref["gm_off"])
    br = bins.brange().cpu().numpy()
    ok = ref["ranges"][:, 6] == 1
    np.testing.assert_array_equal(br[ok, :6], ref["ranges"][ok, :6])
    # pair_gmj maps every brick-major pair to its Gaussian-major slot (a permutation whose
    # target brick matches)
    gmj = bins.pair_gmj(P).cpu().numpy()
    assert np.array_equal(np.sort(gmj), np.arange(P))
    bm_brick = np.repeat(np.arange(ref["brick_off"].size - 1), np.diff(ref["brick_off"]))
    np.testing.assert_array_equal(ref["gm_brick"][gmj], bm_brick)
    return P


def test_bins_forward_workload_bit_exact():
    """32^3 grid, 4,096 Gaussians: every list identical to the FP32 specification."""
    params, og = c1()
    assert _compare(params, og) > 4096


@pytest.mark.parametrize("brick", [(8, 8, 8), (8, 8, 4), (4, 4, 4), (16, 8, 4)])
def test_bins_ragged_offset_grid(brick):
    """Ragged dims (partial edge bricks), non-unit spacing, offset origin, brick shapes."""
    import oracle
    og = oracle.Grid(37, 29, 21, (0.9, 1.2, 1.5), (-3.0, 2.5, 1.0))
    d = inputs.gaussian_cloud(5, 3000, (21, 29, 37), h=og.h)
    d["mu"] = d["mu"] + np.array(og.origin, np.float32)
    # a few Gaussians partly or wholly outside the grid
    d["mu"][:50] = d["mu"][:50] * 1.6 - 10.0
    _compare(cloud_params(d), og, brick)


def test_bins_fit_workload_full_size():
    """256 x 256 x 128 grid, 500k lattice Gaussians: full lists bit-exact."""
    w = phantom_fit()
    P = _compare(w["params0"], w["grid"])
    assert P > 500_000


def test_bins_three_radix_passes():
    """512 x 512 x 128 grid with 4^3 bricks: 524,288 bricks, so the brick keys take three 8-bit
    radix passes (the third reuses the first pass's look-back words); 20,000 Gaussians."""
    import oracle
    og = oracle.Grid(512, 512, 128)
    d = inputs.gaussian_cloud(9, 20000, (128, 512, 512))
    assert _compare(cloud_params(d), og, brick=(4, 4, 4)) > 20000


def test_bins_capacity_overflow_reports_and_empties():
    params, og = c1()
    bins = _bin(params, og, capacity=1000)
    assert bins.status() & _gs().GS_STATUS_CAPACITY
    assert bins.npairs() > 1000
    assert int(bins.brick_off().abs().sum().item()) == 0


def test_bins_invalid_gaussians_flagged_and_dropped():
    import oracle
    params, og = c1()
    p = params.copy()
    p[3, 0] = np.nan
    p[7, 6:10] = 0.0
    p[11, 4] = 31.0
    bins = _bin(p, og)
    assert bins.status() & _gs().GS_STATUS_NONFINITE
    gid = bins.pair_gid(bins.npairs()).cpu().numpy()
    assert not np.isin([3, 7, 11], gid).any()
    ref = oracle.brick_lists(p, og)
    np.testing.assert_array_equal(gid, ref["pair_gid"])


def test_bins_empty_and_single():
    import oracle
    og = oracle.Grid(16, 16, 16)
    bins = _bin(np.zeros((0, 12), np.float32), og)
    assert bins.npairs() == 0 and int(bins.brick_off().abs().sum().item()) == 0
    one = np.array([[8.0, 8.0, 8.0, 0, 0, 0, 1, 0, 0, 0, 0.5, 0.5]], np.float32)
    _compare(one, og)


def test_bins_deterministic():
    params, og = c1()
    a = _bin(params, og)
    b = _bin(params, og)
    P = a.npairs()
    assert np.array_equal(a.pair_gid(P).cpu().numpy(), b.pair_gid(P).cpu().numpy())
    assert np.array_equal(a.pair_gmj(P).cpu().numpy(), b.pair_gmj(P).cpu().numpy())
