"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test names the passage it pins and the plausible mistake it would catch. Nothing here
re-types the oracle's formulas: the checks are closed forms for special configurations,
invariants, limits, finite differences, brute force on tiny inputs, or library routines.
"""
import math

import numpy as np
import pytest

from paper_2603_09621_gb300 import inputs

G32 = None


def _grid(n=16, h=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0), ny=None, nz=None):
    import oracle
    return oracle.Grid(n, ny or n, nz or n, h, origin)


def _one(mu, log_s=(0.0, 0.0, 0.0), q=(1.0, 0.0, 0.0, 0.0), a=1.0, t=1.0):
    """One Gaussian's raw parameters in FP64 (the oracle's input precision)."""
    return np.array([list(mu) + list(log_s) + list(q) + [a, t]], dtype=np.float64)


# ------------------------------------------------------------------ Eq. 2

def test_signal_proxy_limits(oracle_mod):
    """Eq. 2: TE = 0 leaves only longitudinal recovery; T1 -> 0 leaves only transverse decay;
    T2 -> inf removes the decay; T1 -> inf kills the signal. Catches swapped T1/T2 roles,
    TR/TE swaps and sign errors in either exponent."""
    o = oracle_mod
    assert o.signal_proxy([1000.0], [50.0], 2000.0, 0.0)[0] == pytest.approx(
        1.0 - math.exp(-2.0), rel=1e-15)
    assert o.signal_proxy([1e-9], [80.0], 2000.0, 100.0)[0] == pytest.approx(
        math.exp(-1.25), rel=1e-15)
    assert o.signal_proxy([500.0], [1e300], 2000.0, 100.0)[0] == pytest.approx(
        1.0 - math.exp(-4.0), rel=1e-15)
    assert o.signal_proxy([1e300], [80.0], 2000.0, 100.0)[0] == 0.0


def test_signal_proxy_monotone_and_range(oracle_mod):
    """Eq. 2 over the paper's tissue ranges (T1 in [300, 2000] ms, T2 in [30, 200] ms,
    TR = 2000 ms, TE = 100 ms): decreasing in T1, increasing in T2, and spanning
    [(1 - e^-1) e^(-10/3), (1 - e^(-20/3)) e^(-1/2)] at the corners."""
    o = oracle_mod
    t1 = np.linspace(300, 2000, 50)
    t2 = np.linspace(30, 200, 50)
    T_t1 = o.signal_proxy(t1, np.full_like(t1, 100.0), 2000.0, 100.0)
    T_t2 = o.signal_proxy(np.full_like(t2, 1000.0), t2, 2000.0, 100.0)
    assert np.all(np.diff(T_t1) < 0) and np.all(np.diff(T_t2) > 0)
    lo = o.signal_proxy([2000.0], [30.0], 2000.0, 100.0)[0]
    hi = o.signal_proxy([300.0], [200.0], 2000.0, 100.0)[0]
    assert lo == pytest.approx(0.022550, abs=1e-5) and hi == pytest.approx(0.605759, abs=1e-5)


# --------------------------------------------------------------- Eq. 3-4

def test_single_gaussian_weights_closed_form(oracle_mod):
    """Eq. 4 for an axis-aligned Gaussian centred on a voxel centre with scales (1, 2, 3):
    along each principal axis, a voxel at t voxels has d^2 = (t / s)^2, so
    W = r exp(-d^2 / 2). Catches a dropped r, a wrong exponent sign or factor, swapped axes."""
    o = oracle_mod
    r = 0.37
    mu = (8.5, 8.5, 8.5)  # centre of voxel (8, 8, 8)
    p = _one(mu, log_s=(0.0, math.log(2.0), math.log(3.0)), a=0.8, t=r)
    out = o.render(p, _grid(17))
    W = out["W"]
    assert W[8, 8, 8] == pytest.approx(r, rel=1e-15)
    assert W[8, 8, 9] == pytest.approx(r * math.exp(-0.5), rel=1e-14)    # x: d^2 = 1
    assert W[8, 8, 10] == pytest.approx(r * math.exp(-2.0), rel=1e-14)   # x: d^2 = 4
    assert W[8, 10, 8] == pytest.approx(r * math.exp(-0.5), rel=1e-14)   # y: (2/2)^2
    assert W[8, 9, 8] == pytest.approx(r * math.exp(-0.125), rel=1e-14)  # y: (1/2)^2
    assert W[11, 8, 8] == pytest.approx(r * math.exp(-0.5), rel=1e-14)   # z: (3/3)^2
    assert W[8, 9, 9] == pytest.approx(r * math.exp(-0.5 * 1.25), rel=1e-14)


def test_truncation_is_inclusive_at_three_sigma(oracle_mod):
    """Sec. 3.3 truncates at the 3-sigma ellipsoid. With s = 1 a voxel 3 voxels away has
    d^2 = 9 exactly and contributes (inclusive); 4 voxels away it does not. Catches < vs <=,
    sigma vs sigma^2 and a missing truncation."""
    o = oracle_mod
    p = _one((8.5, 8.5, 8.5), t=1.0)
    W = o.render(p, _grid(17))["W"]
    assert W[8, 8, 11] == pytest.approx(math.exp(-4.5), rel=1e-14)
    assert W[8, 8, 12] == 0.0
    assert W[8, 8, 5] == pytest.approx(math.exp(-4.5), rel=1e-14)
    assert W[8, 8, 4] == 0.0


def test_truncation_diagonal_neighbours(oracle_mod):
    """d^2 = 8 (offset (2, 2, 0)) is inside the 3-sigma ellipsoid, d^2 = 13 is not."""
    o = oracle_mod
    W = o.render(_one((8.5, 8.5, 8.5)), _grid(17))["W"]
    assert W[8, 10, 10] == pytest.approx(math.exp(-4.0), rel=1e-14)
    assert W[8, 10, 11] == 0.0
    assert W[10, 10, 9] == pytest.approx(math.exp(-4.5), rel=1e-14)  # (1, 2, 2): d^2 = 9


def test_single_gaussian_reproduces_its_signal(oracle_mod):
    """Eq. 3 normalisation (Sec. 3.2): a lone Gaussian renders I = A wherever W > 0 and 0
    elsewhere, whatever its shape, r or rotation."""
    o = oracle_mod
    rng = np.random.default_rng(3)
    for _ in range(5):
        mu = rng.uniform(4, 12, 3)
        p = _one(mu, log_s=rng.uniform(-0.5, 1.0, 3), q=rng.standard_normal(4),
                 a=rng.uniform(0.1, 2.0), t=rng.uniform(0.05, 1.0))
        out = o.render(p, _grid(16))
        sup = out["W"] > 0
        assert sup.sum() > 0
        np.testing.assert_allclose(out["I"][sup], p[0, 10], rtol=1e-14)
        assert np.all(out["I"][~sup] == 0.0)
        assert np.array_equal(out["npair"], sup.astype(np.int32))


def test_two_symmetric_gaussians_average(oracle_mod):
    """Two equal-shape Gaussians mirrored about a voxel give equal weights there, so Eq. 3
    returns the mean of their amplitudes (weighted by r). Catches a missing normalisation or
    a normalisation by the wrong sum."""
    o = oracle_mod
    p = np.concatenate([_one((7.5, 8.5, 8.5), a=0.2, t=0.5),
                        _one((9.5, 8.5, 8.5), a=1.0, t=0.5)])
    I = o.render(p, _grid(17))["I"]
    assert I[8, 8, 8] == pytest.approx(0.6, rel=1e-14)
    p[1, 11] = 1.5  # r2 = 3 r1: weights 1:3
    I = o.render(p, _grid(17))["I"]
    assert I[8, 8, 8] == pytest.approx((0.2 * 0.5 + 1.0 * 1.5) / 2.0, rel=1e-14)


def test_uniform_signal_gives_constant_volume(oracle_mod):
    """'signal linearity' (Sec. 3.2): a cloud whose Gaussians all carry the same A renders
    the constant A wherever it has support."""
    o = oracle_mod
    d = inputs.gaussian_cloud(5, 300, (16, 16, 16))
    p = inputs.assemble_params(d["mu"], d["log_s"], d["q"], np.full(300, 0.7),
                               d["pd"] * 0.9 + 0.05).astype(np.float64)
    out = o.render(p, _grid(16))
    sup = out["W"] > 0
    np.testing.assert_allclose(out["I"][sup], float(np.float32(0.7)), rtol=1e-13)


def test_permutation_invariance(oracle_mod):
    """Order independence (Sec. 3.3: blending is commutative): permuting the Gaussians
    changes the result only by FP64 rounding."""
    o = oracle_mod
    d = inputs.gaussian_cloud(7, 400, (16, 16, 16))
    p = inputs.assemble_params(d["mu"], d["log_s"], d["q"], d["pd"], d["pd"] * 0.5 + 0.1)
    perm = np.random.default_rng(1).permutation(400)
    a = o.render(p.astype(np.float64), _grid(16))
    b = o.render(p[perm].astype(np.float64), _grid(16))
    np.testing.assert_allclose(b["I"], a["I"], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(b["W"], a["W"], rtol=1e-13, atol=1e-300)


def test_rotation_convention_against_scipy(oracle_mod):
    """Covariance Sigma = R diag(s^2) R^T with R the active rotation of the unit quaternion
    (w, x, y, z). The 120-degree turn about (1,1,1) maps x -> y -> z -> x (scipy agrees), so
    the long axis (s = 2) must lie along y, s = 1 along z and s = 0.5 along x. Catches a
    transposed R, a (x, y, z, w) ordering slip and a covariance/precision mix-up."""
    from scipy.spatial.transform import Rotation
    o = oracle_mod
    q = (0.5, 0.5, 0.5, 0.5)
    Rs = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    np.testing.assert_allclose(Rs @ np.array([1.0, 0, 0]), [0, 1, 0], atol=1e-15)
    p = _one((8.5, 8.5, 8.5), log_s=(math.log(2.0), 0.0, math.log(0.5)), q=q, t=1.0)
    W = o.render(p, _grid(17))["W"]
    assert W[8, 10, 8] == pytest.approx(math.exp(-0.5), rel=1e-12)   # y, t = 2, s = 2
    assert W[9, 8, 8] == pytest.approx(math.exp(-0.5), rel=1e-12)    # z, t = 1, s = 1
    assert W[8, 8, 9] == pytest.approx(math.exp(-2.0), rel=1e-12)    # x, t = 1, s = 0.5


def test_ninety_degree_turn_swaps_scales(oracle_mod):
    """A 90-degree turn about z of scales (a, b, c) is the axis-aligned Gaussian with scales
    (b, a, c): the two renders agree to rounding (off-diagonal conic path vs diagonal)."""
    o = oracle_mod
    c45 = math.cos(math.pi / 4)
    ls = (math.log(2.2), math.log(0.7), math.log(1.3))
    p1 = _one((8.3, 8.6, 8.4), log_s=ls, q=(c45, 0.0, 0.0, c45), a=0.4, t=0.9)
    p2 = _one((8.3, 8.6, 8.4), log_s=(ls[1], ls[0], ls[2]), a=0.4, t=0.9)
    a = o.render(p1, _grid(17))
    b = o.render(p2, _grid(17))
    np.testing.assert_allclose(a["W"], b["W"], rtol=1e-7, atol=1e-9)


def test_signal_modes_related_by_common_T(oracle_mod):
    """With one shared relaxation proxy c, mode 0 (r_i = T_i) gives I0 = sum A g / sum g and
    mode 1 (v_i = A_i T_i, r = 1) gives I1 = c I0."""
    import oracle
    o = oracle_mod
    d = inputs.gaussian_cloud(11, 200, (16, 16, 16))
    p = inputs.assemble_params(d["mu"], d["log_s"], d["q"], d["pd"], np.full(200, 0.3))
    a = o.render(p.astype(np.float64), _grid(16), oracle.Config(signal_mode=0))["I"]
    b = o.render(p.astype(np.float64), _grid(16), oracle.Config(signal_mode=1))["I"]
    np.testing.assert_allclose(b, float(np.float32(0.3)) * a, rtol=1e-13, atol=1e-300)


def test_prune_equals_brute_force(oracle_mod):
    """The exact bounding-box shortcut skips only pairs with d^2 > sigma_t^2: results equal
    the unpruned brute force bit for bit (forward) and to rounding (gradient)."""
    o = oracle_mod
    d = inputs.gaussian_cloud(13, 150, (12, 14, 10))
    p = inputs.assemble_params(d["mu"], d["log_s"], d["q"], d["pd"], d["pd"] * 0.5 + 0.1)
    g = _grid(14, ny=14, nz=12)
    p = p.astype(np.float64)
    a = o.render(p, g, prune=True)
    b = o.render(p, g, prune=False)
    for k in ("I", "W", "S", "amb"):
        assert np.array_equal(a[k], b[k]), k
    dI = inputs.crop_dI(2, g.shape).astype(np.float64)
    ga = o.render_grad(p, g, dI, prune=True)
    gb = o.render_grad(p, g, dI, prune=False)
    np.testing.assert_array_equal(ga, gb)


def test_crop_matches_full_render(oracle_mod):
    """Rendering a crop gives exactly the corresponding voxels of the full render."""
    o = oracle_mod
    d = inputs.gaussian_cloud(17, 200, (16, 16, 16))
    p = inputs.assemble_params(d["mu"], d["log_s"], d["q"], d["pd"], d["pd"] + 0.1)
    full = o.render(p.astype(np.float64), _grid(16))
    cr = o.render(p.astype(np.float64), _grid(16), crop=(3, 11, 2, 9, 5, 16))
    assert np.array_equal(cr["I"], full["I"][5:16, 2:9, 3:11])


def test_empty_voxels_render_zero(oracle_mod):
    """No Gaussian near a voxel: W = 0 and I = S / max(W, eps) = 0."""
    o = oracle_mod
    out = o.render(_one((2.5, 2.5, 2.5), a=5.0), _grid(16))
    assert out["W"][12, 12, 12] == 0.0 and out["I"][12, 12, 12] == 0.0
    empty = o.render(np.zeros((0, 12)), _grid(4))
    assert np.all(empty["I"] == 0.0)


def test_invalid_gaussians_are_dropped(oracle_mod):
    """Non-finite parameters, a zero quaternion or |log_s| > 30 make a Gaussian invalid."""
    o = oracle_mod
    p = np.concatenate([_one((8.5, 8.5, 8.5)), _one((8.5, 8.5, 8.5), q=(0, 0, 0, 0)),
                        _one((np.nan, 8.5, 8.5)), _one((8.5, 8.5, 8.5), log_s=(31, 0, 0))])
    out = o.render(p, _grid(17))
    assert out["n_invalid"] == 3
    ref = o.render(p[:1], _grid(17))
    assert np.array_equal(out["W"], ref["W"])


# --------------------------------------------------------------- Eq. 5-6

def _loss(o, p, g, dI, cfg):
    return float((o.render(p, g, cfg)["I"] * dI).sum())


@pytest.mark.parametrize("acts", [(0, 0, 0), (1, 1, 0), (0, 0, 1)])
def test_gradient_matches_central_differences(oracle_mod, acts):
    """Eq. 5-6 and the chain to the raw parameters (log-scale, quaternion with its
    normalisation, amplitude / relaxation activations, both signal modes) against central
    finite differences of the FP64 forward. A wide truncation (10 sigma) keeps the loss
    smooth so that every parameter can be differenced."""
    import oracle
    o = oracle_mod
    a_act, t_act, mode = acts
    cfg = oracle.Config(trunc_sigma=10.0, signal_mode=mode, a_act=a_act, t_act=t_act)
    g = oracle.Grid(9, 8, 7, (1.0, 1.1, 0.9), (0.3, -0.2, 0.1))
    d = inputs.gaussian_cloud(21, 5, (7, 8, 9), scale_range=(0.8, 2.0))
    t = d["pd"] * 0.8 + 0.1 if not t_act else np.random.default_rng(0).normal(0, 1, 5)
    a = d["pd"] if not a_act else np.random.default_rng(1).normal(0, 1, 5)
    p = inputs.assemble_params(d["mu"], d["log_s"], d["q"], a, t).astype(np.float64)
    dI = inputs.crop_dI(3, g.shape).astype(np.float64)
    ana = o.render_grad(p, g, dI, cfg)
    num = np.zeros_like(ana)
    hstep = 1e-5
    for i in range(p.shape[0]):
        for k in range(12):
            pp, pm = p.copy(), p.copy()
            pp[i, k] += hstep
            pm[i, k] -= hstep
            num[i, k] = (_loss(o, pp, g, dI, cfg) - _loss(o, pm, g, dI, cfg)) / (2 * hstep)
    scale = np.abs(num).max()
    np.testing.assert_allclose(ana, num, rtol=2e-6, atol=2e-7 * scale)


def test_gradient_fd_at_three_sigma_away_from_boundary(oracle_mod):
    """Same FD check with the paper's 3-sigma truncation, on a configuration whose pairs all
    stay clear of the truncation boundary under the perturbation (amb count 0 at a wide
    band), so the truncated loss is smooth there."""
    import oracle
    o = oracle_mod
    cfg = oracle.Config()
    g = oracle.Grid(10, 10, 10)
    for seed in range(4, 40):
        d = inputs.gaussian_cloud(seed, 6, (10, 10, 10), scale_range=(0.9, 1.8))
        p = inputs.assemble_params(d["mu"], d["log_s"], d["q"], d["pd"],
                                   d["pd"] * 0.5 + 0.2).astype(np.float64)
        if o.render(p, g, cfg, amb_tol=1e-3)["amb"].sum() == 0:  # band 1e-3 |terms|
            break
    else:
        pytest.fail("no boundary-free configuration found")
    dI = inputs.crop_dI(8, g.shape).astype(np.float64)
    ana = o.render_grad(p, g, dI, cfg)
    hstep = 1e-6
    for i in range(p.shape[0]):
        for k in range(12):
            pp, pm = p.copy(), p.copy()
            pp[i, k] += hstep
            pm[i, k] -= hstep
            num = (_loss(o, pp, g, dI, cfg) - _loss(o, pm, g, dI, cfg)) / (2 * hstep)
            assert ana[i, k] == pytest.approx(num, rel=1e-5, abs=1e-7), (i, k)


def test_single_gaussian_gradient_closed_form(oracle_mod):
    """A lone Gaussian renders I = A on its support, so dI/dmu = dI/dSigma = dI/dr = 0
    there (the (A_i - I)/W factor of Eq. 5 vanishes) and Eq. 6 gives
    dL/dA = sum over the support of dL/dI."""
    o = oracle_mod
    p = _one((8.2, 8.7, 7.9), log_s=(0.3, -0.2, 0.5), q=(0.9, 0.1, -0.3, 0.2), a=0.6, t=0.4)
    g = _grid(16)
    out = o.render(p, g)
    dI = inputs.crop_dI(5, g.shape).astype(np.float64)
    gr, geo = o.render_grad(p, g, dI, want_geo=True)
    sup = out["W"] > 0
    assert gr[0, 10] == pytest.approx(dI[sup].sum(), rel=1e-12)
    scale = np.abs(dI[sup]).sum()
    assert np.all(np.abs(gr[0, :10]) <= 1e-12 * scale)
    assert abs(gr[0, 11]) <= 1e-12 * scale
    assert geo[0, 9] == pytest.approx(gr[0, 10], rel=1e-15)


def test_gradient_below_eps_floor(oracle_mod):
    """Where W < eps the render is I = S / eps and dI/dw_i = v_i / eps (reading of the
    normalisation's floor); checked by differencing at a voxel whose weight is tiny."""
    import oracle
    o = oracle_mod
    cfg = oracle.Config(eps=1e-3)
    p = _one((8.5, 8.5, 8.5), log_s=(0.0, 0.0, 0.0), a=0.7, t=2e-4)
    g = _grid(17)
    dI = np.zeros(g.shape)
    dI[8, 8, 9] = 1.0   # W = 2e-4 e^-0.5 < eps
    ana = o.render_grad(p, g, dI, cfg)
    for k in (0, 3, 10, 11):
        pp, pm = p.copy(), p.copy()
        pp[0, k] += 1e-7
        pm[0, k] -= 1e-7
        num = (_loss(o, pp, g, dI, cfg) - _loss(o, pm, g, dI, cfg)) / 2e-7
        assert ana[0, k] == pytest.approx(num, rel=1e-6, abs=1e-12)


# ------------------------------------------------------- FP32 binning specification

def test_exp_cw_error_bound(oracle_mod):
    """The binning specification's Cody-Waite exponential is within 2 ulp of exp over the
    admissible log-scale range [-30, 30]."""
    o = oracle_mod
    xs = np.concatenate([np.linspace(-30, 30, 4001), np.random.default_rng(0).uniform(-30, 30, 4000)])
    for x in xs.astype(np.float32):
        got = np.float32(o.exp_cw(float(x)))
        ref = math.exp(float(x))
        ulp = np.spacing(np.float32(ref))
        assert abs(float(got) - ref) <= 2.0 * float(ulp), (x, got, ref)


def test_brick_range_axis_aligned(oracle_mod):
    """For q = (1, 0, 0, 0) the 3-sigma box half-extent is sigma_t (1 + 2^-13) s_k exactly
    (Sec. 3.3); voxel and brick ranges follow from it (values chosen away from integers)."""
    import oracle
    o = oracle_mod
    g = oracle.Grid(64, 48, 40)
    p = _one((20.3, 30.7, 10.2), log_s=(math.log(2.0), math.log(1.1), math.log(4.0)))
    rng = o.brick_ranges_fp32(p.astype(np.float32), g)
    e = np.array([2.0, 1.1, 4.0]) * 3.0 * (1 + 2.0 ** -13)
    mu = np.array([20.3, 30.7, 10.2])
    lo = np.maximum(np.ceil(mu - e - 0.5), 0)
    hi = np.minimum(np.floor(mu + e - 0.5), [63, 47, 39])
    assert list(rng[0, :3]) == list((lo // 8).astype(int))
    assert list(rng[0, 3:6]) == list((hi // 8).astype(int))
    assert rng[0, 6] == 1


def test_brick_ranges_cover_the_support(oracle_mod):
    """Brute force on tiny inputs: every voxel a Gaussian reaches in the FP64 render (W > 0,
    i.e. d^2 <= 9) lies in one of its FP32 bricks, for both brick shapes and a non-unit,
    offset grid. Catches a box that is too small, an off-by-one or a wrong axis."""
    import oracle
    o = oracle_mod
    for brick in ((8, 8, 8), (8, 8, 4), (4, 4, 4)):
        g = oracle.Grid(21, 19, 17, (1.0, 0.8, 1.3), (-1.0, 0.5, 2.0))
        cfg = oracle.Config(brick=brick)
        d = inputs.gaussian_cloud(31, 120, (17, 19, 21), h=g.h)
        d["mu"] = d["mu"] + np.array(g.origin, np.float32)[None, :]
        p = inputs.assemble_params(d["mu"], d["log_s"], d["q"], d["pd"], np.ones(120))
        rng = o.brick_ranges_fp32(p, g, cfg)
        for i in range(p.shape[0]):
            W = o.render(p[i:i + 1].astype(np.float64), g, cfg, amb_tol=0.0)["W"]
            zz, yy, xx = np.nonzero(W > 0)
            if zz.size == 0:
                continue
            assert rng[i, 6] == 1
            b = np.stack([xx // brick[0], yy // brick[1], zz // brick[2]], 1)
            assert np.all(b >= rng[i, :3]) and np.all(b <= rng[i, 3:6]), i


def test_brick_lists_structure(oracle_mod):
    """Brick-major lists: offsets are a prefix sum, ids ascend inside each brick, and every
    (Gaussian, brick) pair of the Gaussian-major enumeration appears exactly once."""
    import oracle
    o = oracle_mod
    g = oracle.Grid(24, 20, 16)
    d = inputs.gaussian_cloud(9, 300, (16, 20, 24))
    p = inputs.assemble_params(d["mu"], d["log_s"], d["q"], d["pd"], np.ones(300))
    L = o.brick_lists(p, g)
    off, gid = L["brick_off"], L["pair_gid"]
    assert off[0] == 0 and off[-1] == gid.size == L["gm_off"][-1]
    for b in range(off.size - 1):
        seg = gid[off[b]:off[b + 1]]
        assert np.all(np.diff(seg) > 0)
    pairs_bm = set()
    for b in range(off.size - 1):
        for gg in gid[off[b]:off[b + 1]]:
            pairs_bm.add((int(gg), b))
    pairs_gm = set()
    for gg in range(300):
        for b in L["gm_brick"][L["gm_off"][gg]:L["gm_off"][gg + 1]]:
            pairs_gm.add((gg, int(b)))
    assert pairs_bm == pairs_gm


# ------------------------------------------------- slice profile, loss, optimiser

def test_downsample_exact_means():
    """Box slice profile: integer-valued slices average exactly; non-divisible depth drops
    the trailing slices."""
    import oracle
    nz, s = 11, 3
    hr = np.broadcast_to(np.arange(nz, dtype=np.float64)[:, None, None], (nz, 2, 3))
    lr = oracle.downsample(hr, s)
    assert lr.shape == (3, 2, 3)
    np.testing.assert_array_equal(lr[:, 0, 0], [1.0, 4.0, 7.0])


def test_downsample_adjoint_identity():
    """<D x, y> = <x, D^T y> for the slice profile and its adjoint (catches a missing 1/s,
    an index shift, or gradient leaking into dropped trailing slices)."""
    import oracle
    rng = np.random.default_rng(0)
    for nz, s in ((12, 4), (13, 3), (8, 2), (7, 7)):
        x = rng.standard_normal((nz, 3, 5))
        y = rng.standard_normal((nz // s, 3, 5))
        lhs = float((oracle.downsample(x, s) * y).sum())
        adj = oracle.downsample_adjoint(y, nz, s)
        rhs = float((x * adj).sum())
        assert lhs == pytest.approx(rhs, rel=1e-12)
        assert np.all(adj[s * (nz // s):] == 0)


# ------------------------------------------------------------- trilinear resize (Sec. 4.1)

def test_resample_factor_two_is_block_mean():
    """Halving every axis puts each LR sample at the centre of a 2 x 2 x 2 block with all
    weights 1/2: the closed form is the block mean (catches a half-pixel shift or a wrong
    scale direction)."""
    import oracle
    rng = np.random.default_rng(1)
    v = rng.standard_normal((6, 8, 10))
    got = oracle.resample(v, (3, 4, 5))
    ref = v.reshape(3, 2, 4, 2, 5, 2).mean(axis=(1, 3, 5))
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)


def test_resample_matches_map_coordinates():
    """Any factor (down, up, mixed) equals scipy.ndimage.map_coordinates(order=1,
    mode='nearest') at the half-pixel-centre positions c = (n_src/n_dst)(j + 1/2) - 1/2
    (clamped at 0) computed in FP64 (the oracle takes them in FP32, hence the tolerance)."""
    import oracle
    from scipy.ndimage import map_coordinates
    rng = np.random.default_rng(2)
    for src, dst in (((24, 31, 20), (10, 13, 9)), ((155, 24, 24), (100, 10, 10)),
                     ((7, 9, 5), (16, 9, 12))):
        v = rng.standard_normal(src)
        got = oracle.resample(v, dst)
        pos = []
        for a in range(3):
            c = (src[a] / dst[a]) * (np.arange(dst[a]) + 0.5) - 0.5
            pos.append(np.maximum(c, 0.0))
        Z, Y, X = np.meshgrid(*pos, indexing="ij")
        ref = map_coordinates(v, [Z.ravel(), Y.ravel(), X.ravel()], order=1,
                              mode="nearest").reshape(dst)
        # FP32 positions are off by at most a few ulp of c; the value moves by at most the
        # largest neighbour difference per unit of c along each of the three axes
        slope = max(float(np.abs(np.diff(v, axis=a)).max()) for a in range(3))
        tol = 3 * 4 * 2.0 ** -23 * max(src) * slope
        np.testing.assert_allclose(got, ref, rtol=0, atol=tol)


def test_resample_identity_and_adjoint():
    """Equal shapes copy exactly; <R x, y> = <x, R^T y> for the resize and its adjoint
    (catches a transposed weight, a dropped corner or a wrong clamp in the adjoint)."""
    import oracle
    rng = np.random.default_rng(3)
    v = rng.standard_normal((5, 6, 7))
    np.testing.assert_array_equal(oracle.resample(v, v.shape), v)
    for src, dst in (((9, 13, 17), (4, 6, 7)), ((20, 20, 20), (8, 11, 20)),
                     ((5, 6, 4), (9, 13, 8))):
        x = rng.standard_normal(src)
        y = rng.standard_normal(dst)
        lhs = float((oracle.resample(x, dst) * y).sum())
        rhs = float((x * oracle.resample_adjoint(y, src)).sum())
        assert lhs == pytest.approx(rhs, rel=1e-12)


def test_resample_grid_centres():
    """LR voxel j of ``resample_grid`` has its centre at the HR continuous index c_j of
    ``resample_map`` (the LR grid covers the HR field of view)."""
    import oracle
    g = oracle.Grid(240, 240, 155, (0.9, 0.9, 1.2), (-5.0, 3.0, 1.0))
    lg = oracle.resample_grid(g, (100, 100, 100))
    for a, (n_hr, n_lr) in enumerate(((240, 100), (240, 100), (155, 100))):
        j = np.arange(n_lr)
        lr_centre = lg.origin[a] + (j + 0.5) * lg.h[a]
        c = (n_hr / n_lr) * (j + 0.5) - 0.5
        hr_point = g.origin[a] + (c + 0.5) * g.h[a]
        np.testing.assert_allclose(lr_centre, hr_point, rtol=1e-13, atol=1e-12)


def test_l1_loss_values():
    import oracle
    pred = np.array([0.5, 0.2, 0.3, 0.9])
    tgt = np.array([0.1, 0.2, 0.6, 0.4])
    loss, g = oracle.l1_loss(pred, tgt)
    assert loss == pytest.approx((0.4 + 0.0 + 0.3 + 0.5) / 4, rel=1e-15)
    np.testing.assert_array_equal(g, np.array([1.0, 0.0, -1.0, 1.0]) / 4)


def test_adam_matches_torch():
    """Bias-corrected Adam with per-column learning rates equals torch.optim.Adam with one
    parameter group per column group."""
    import oracle
    import torch
    rng = np.random.default_rng(0)
    p0 = rng.standard_normal((7, 12))
    acfg = oracle.AdamConfig()
    lrs = acfg.lr_vector()
    cols = [(0, 3), (3, 6), (6, 10), (10, 11), (11, 12)]
    tp = [torch.tensor(p0[:, a:b].copy(), dtype=torch.float64, requires_grad=True)
          for a, b in cols]
    opt = torch.optim.Adam([{"params": [t], "lr": float(lrs[a])} for t, (a, _) in zip(tp, cols)],
                           betas=(acfg.beta1, acfg.beta2), eps=acfg.eps)
    p, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    for step in range(1, 5):
        g = rng.standard_normal((7, 12))
        p, m, v = oracle.adam_step(p, g, m, v, step, acfg)
        for t, (a, b) in zip(tp, cols):
            t.grad = torch.tensor(g[:, a:b].copy(), dtype=torch.float64)
        opt.step()
    ref = np.concatenate([t.detach().numpy() for t in tp], axis=1)
    np.testing.assert_allclose(p, ref, rtol=1e-13, atol=1e-15)


# ----------------------------------------------------------------- initialisation

def test_lattice_dims_for_fit_workload():
    """500k Gaussians over 256 x 256 x 128 mm give spacing 2.56 mm and a 100 x 100 x 50
    lattice (N = 500,000 exactly)."""
    import oracle
    n, _ = oracle.lattice_dims(oracle.Grid(256, 256, 128), 500_000)
    assert n == [100, 100, 50]


def test_trilinear_matches_scipy_and_nodes():
    """Trilinear sampling equals scipy.ndimage.map_coordinates(order=1, mode='nearest') on
    the continuous index, and returns the node value at voxel centres."""
    import oracle
    from scipy.ndimage import map_coordinates
    rng = np.random.default_rng(0)
    vol = rng.standard_normal((5, 6, 7))
    g = oracle.Grid(7, 6, 5, (1.0, 1.0, 4.0))
    pts = rng.uniform(-1, 1, (200, 3)) * np.array([8, 7, 24]) + np.array([3.5, 3.0, 10.0])
    got = oracle.trilinear(vol, g, pts)
    u = np.stack([(pts[:, 2] / 4.0 - 0.5), pts[:, 1] - 0.5, pts[:, 0] - 0.5])
    for a, n in enumerate((5, 6, 7)):
        u[a] = np.clip(u[a], 0, n - 1)
    ref = map_coordinates(vol, u, order=1, mode="nearest")
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
    nodes = np.array([[2.5, 3.5, 4 * 1.5]])
    assert oracle.trilinear(vol, g, nodes)[0] == pytest.approx(vol[1, 3, 2], rel=1e-14)


def test_phantom_normalisation():
    import oracle
    ph = inputs.phantom_draws(0, (24, 32, 32), n_ell=4, semi_axes=(4.0, 10.0), s=4)
    hr = oracle.phantom_from_draws(ph, inputs.TR_MS, inputs.TE_MS)
    assert hr.max() == pytest.approx(1.0) and hr.min() == 0.0
    assert np.all(hr[ph["label"] == 0] == 0.0)


# ------------------------------------------------------------------------ metrics

def test_psnr_ssim_basic():
    import oracle
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, (16, 16, 16))
    assert oracle.psnr(x + 0.1, x) == pytest.approx(20.0, rel=1e-12)
    assert oracle.ssim3d(x, x) == pytest.approx(1.0, rel=1e-12)
    y = x + rng.normal(0, 0.1, x.shape)
    assert oracle.ssim3d(x, y) == pytest.approx(oracle.ssim3d(y, x), rel=1e-12)
    assert oracle.ssim3d(x, y) < 0.99


def test_ssim_closed_forms():
    """SSIM (Wang et al. 2004, cited in Sec. 4.2) in closed form for two configurations:
    * constant volumes a and b: the variances vanish, so SSIM = (2ab + C1) / (a^2 + b^2 + C1);
    * a unit impulse against zero: at offset q from the impulse the local mean is the window
      weight w(q) and the variance w - w^2, so SSIM(q) = C1 / (w^2 + C1) * C2 / (w - w^2 + C2),
      with w the separable Gaussian window (std 1.5 voxels, radius 5 voxels, each axis
      normalised) written out here; the mean runs over the whole volume.
    A wrong constant (K1, K2), a dropped factor 2 or another window fails one of them."""
    import oracle
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    for a, b in ((0.2, 0.7), (0.5, 0.5), (0.9, 0.1)):
        x = np.full((12, 12, 12), a)
        y = np.full((12, 12, 12), b)
        assert oracle.ssim3d(x, y) == pytest.approx((2 * a * b + c1) / (a * a + b * b + c1),
                                                    rel=1e-10)
    n = 21
    x = np.zeros((n, n, n))
    x[n // 2, n // 2, n // 2] = 1.0
    k = np.arange(-5, 6, dtype=np.float64)
    g1 = np.exp(-k * k / (2 * 1.5 ** 2))
    g1 /= g1.sum()
    w = np.zeros((n, n, n))
    c = n // 2
    w[c - 5:c + 6, c - 5:c + 6, c - 5:c + 6] = g1[:, None, None] * g1[None, :, None] * g1[None, None, :]
    expect = np.mean(c1 / (w * w + c1) * c2 / (w - w * w + c2))
    assert oracle.ssim3d(x, np.zeros_like(x)) == pytest.approx(expect, rel=1e-9)


# ----------------------------------------------------------- composed pieces: closed forms

def test_rician_closed_forms():
    """Magnitude of LR + n1 + i n2: |LR| without noise, sqrt(n1^2 + n2^2) on a zero signal,
    and the 3-4-5 triangle (catches a dropped channel or a missing square root)."""
    import oracle
    x = np.array([0.3, -0.7, 0.0])
    np.testing.assert_array_equal(oracle.rician(x, 0.0, 0.0), np.abs(x))
    assert oracle.rician(np.array([0.0]), 0.6, 0.8)[0] == pytest.approx(1.0, rel=1e-15)
    assert oracle.rician(np.array([1.0]), 2.0, 4.0)[0] == pytest.approx(5.0, rel=1e-15)


@pytest.mark.parametrize("trilinear_grid", [False, True])
def test_init_lattice_closed_form(trilinear_grid):
    """Lattice init on a constant LR volume gives every Gaussian that amplitude; on a volume
    linear in the LR continuous index it gives the linear function at each centre's LR
    index (interior centres). Centres sit at cell centres of the field of view, log-scales
    are log(l / 2), rotations identity, t = logit(t_init). Catches a half-cell shift, a wrong
    LR spacing or a swapped axis."""
    import oracle
    g = oracle.Grid(24, 20, 16, (1.0, 1.5, 2.0), (-3.0, 2.0, 5.0))
    if trilinear_grid:
        lr_shape = (7, 9, 10)
        lg = oracle.resample_grid(g, lr_shape)
        init = lambda v: oracle.init_lattice_lr(v, g, 480, t_act=1, t_init=0.3)
    else:
        s = 2
        lr_shape = (g.nz // s, g.ny, g.nx)
        lg = oracle.Grid(g.nx, g.ny, g.nz // s, (g.h[0], g.h[1], g.h[2] * s), g.origin)
        init = lambda v: oracle.init_lattice(v, g, s, 480, t_act=1, t_init=0.3)
    n, L = oracle.lattice_dims(g, 480)
    p = init(np.full(lr_shape, 0.625))
    np.testing.assert_allclose(p[:, 10], 0.625, rtol=1e-6)
    ell = [L[a] / n[a] for a in range(3)]
    ix = np.arange(p.shape[0])
    idx = [ix % n[0], (ix // n[0]) % n[1], ix // (n[0] * n[1])]
    for a in range(3):
        np.testing.assert_allclose(p[:, a], g.origin[a] + (idx[a] + 0.5) * ell[a], rtol=1e-6,
                                   atol=1e-5)
        np.testing.assert_allclose(p[:, 3 + a], np.log(ell[a] / 2.0), rtol=1e-6)
    np.testing.assert_allclose(p[:, 6:10], np.tile([1.0, 0.0, 0.0, 0.0], (p.shape[0], 1)))
    np.testing.assert_allclose(p[:, 11], np.log(0.3 / 0.7), rtol=1e-6)
    # linear LR volume: value = 1 + 0.1 i + 0.2 j + 0.3 k at LR index (i, j, k) = (x, y, z)
    K, J, I = np.meshgrid(np.arange(lr_shape[0]), np.arange(lr_shape[1]), np.arange(lr_shape[2]),
                          indexing="ij")
    p = init(1.0 + 0.1 * I + 0.2 * J + 0.3 * K)
    u = [(p[:, a].astype(np.float64) - lg.origin[a]) / lg.h[a] - 0.5 for a in range(3)]
    nl = (lr_shape[2], lr_shape[1], lr_shape[0])
    inner = np.all([(u[a] >= 0) & (u[a] <= nl[a] - 1) for a in range(3)], axis=0)
    assert inner.sum() > 50
    ref = 1.0 + 0.1 * u[0] + 0.2 * u[1] + 0.3 * u[2]
    np.testing.assert_allclose(p[inner, 10], ref[inner], rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("lr_model", ["zbox", "trilinear"])
def test_fit_step_gradient_finite_differences(lr_model):
    """The composed fitting step's gradient is dL/d(raw params) of the L1 loss through the
    render and the LR forward model: central differences of that loss (FP64, wide
    truncation so the render is smooth, a target kept clear of ties) match it. Catches a
    wrong sign or 1/n in the L1 gradient, or a forward model and adjoint that disagree."""
    import oracle
    cfg = oracle.Config(trunc_sigma=10.0, t_act=1)
    g = oracle.Grid(8, 7, 6, (1.0, 1.2, 0.9), (0.2, 0.1, -0.3))
    d = inputs.gaussian_cloud(31, 4, (6, 7, 8), scale_range=(0.9, 1.8))
    t = np.random.default_rng(2).normal(0, 1, 4)
    p = inputs.assemble_params(d["mu"], d["log_s"], d["q"], d["pd"], t).astype(np.float64)
    r = oracle.render(p, g, cfg)["I"]
    if lr_model == "zbox":
        pred = oracle.downsample(r, 2)
        fwd = lambda I: oracle.downsample(I, 2)
    else:
        pred = oracle.resample(r, (4, 5, 5))
        fwd = lambda I: oracle.resample(I, (4, 5, 5))
    rng = np.random.default_rng(5)
    target = pred + rng.choice([-1.0, 1.0], pred.shape) * rng.uniform(0.05, 0.1, pred.shape)
    n = p.shape[0]
    out = oracle.fit_step(p, target, g, 2, cfg, np.zeros((n, 12)), np.zeros((n, 12)), 1,
                          lr_model=lr_model)
    loss = lambda q: float(np.abs(fwd(oracle.render(q, g, cfg)["I"]) - target).mean())
    assert out["loss"] == pytest.approx(loss(p), rel=1e-12)
    num = np.zeros_like(out["grad"])
    hstep = 1e-6
    for i in range(n):
        for k in range(12):
            pp, pm = p.copy(), p.copy()
            pp[i, k] += hstep
            pm[i, k] -= hstep
            num[i, k] = (loss(pp) - loss(pm)) / (2 * hstep)
    np.testing.assert_allclose(out["grad"], num, rtol=1e-5, atol=1e-6 * np.abs(num).max())
