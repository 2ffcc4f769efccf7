"""Pins of the oracle's truncation-boundary outputs (CPU only).

The Sec. 3.3 truncation (a pair contributes when d^2 <= sigma_t^2) is decided in FP64 by the
oracle and in FP32 by a renderer; pairs inside a narrow band around the boundary may go either
way. The oracle therefore reports, per voxel, the sums over the pairs clear of the band and the
terms of each ambiguous pair, and bounds every gradient the possible decisions give. These
tests pin those outputs against brute force in numpy, against constructed exact ties, and
against renders with the truncation radius moved to either side of a tie; and they pin the
acceptance checks built on them (a planted error must be rejected).
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2603_09621_gb300 import inputs


def _brute(p, grid, sigma_t=3.0, band=0.0):
    """Every (voxel, Gaussian) pair in numpy: d^2, sum_ab |C_ab d_a d_b|, w = exp(-d^2/2) r,
    v (identity activations, signal mode 0: v = a, r = t). Arrays [V, N], voxels z-major."""
    mu = p[:, 0:3]
    s = np.exp(p[:, 3:6])
    R = Rotation.from_quat(p[:, [7, 8, 9, 6]]).as_matrix()          # scalar-last order
    C = np.einsum("nam,nm,nbm->nab", R, 1.0 / s ** 2, R)
    zz, yy, xx = np.meshgrid(np.arange(grid.nz), np.arange(grid.ny), np.arange(grid.nx),
                             indexing="ij")
    ctr = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1).astype(np.float64) + 0.5
    ctr = ctr * np.array(grid.h) + np.array(grid.origin)
    d = ctr[:, None, :] - mu[None, :, :]
    d2 = np.einsum("vna,nab,vnb->vn", d, C, d)
    dabs = np.einsum("vna,nab,vnb->vn", np.abs(d), np.abs(C), np.abs(d))
    w = np.exp(-0.5 * d2) * p[None, :, 11]
    amb = np.abs(d2 - sigma_t ** 2) <= band * dabs
    return d2, dabs, w, p[None, :, 10] * np.ones_like(w), amb


def test_ambiguity_outputs_against_brute_force(oracle_mod):
    """A widened band (1e-2 of the absolute terms) puts hundreds of pairs in it. Per voxel the
    count, the slots (Gaussian, v w, w, relative distance to the boundary, in Gaussian order),
    the sure sums and the conditioning sums must equal numpy brute force over all pairs.
    Catches a sure sum that keeps band pairs, a slot that stores w only inside the boundary, a
    wrong sign or scale of the relative distance, and slots out of order."""
    import oracle
    o = oracle_mod
    g = oracle.Grid(11, 10, 9, (1.0, 1.1, 0.9), (0.3, -0.2, 0.1))
    d = inputs.gaussian_cloud(21, 80, (9, 10, 11), h=g.h, scale_range=(0.6, 2.0))
    d["mu"] = d["mu"] + np.array(g.origin, np.float32)
    p = inputs.assemble_params(d["mu"], d["log_s"], d["q"], d["pd"],
                               d["pd"] * 0.5 + 0.2).astype(np.float64)
    band = 1e-2
    r = o.render(p, g, amb_tol=band, want_amb=True, prune=False)
    d2, dabs, w, v, amb = _brute(p, g, band=band)
    inside = d2 <= 9.0
    assert amb.sum() > 100
    np.testing.assert_array_equal(r["amb"].ravel(), amb.sum(1))
    sure = inside & ~amb
    np.testing.assert_allclose(r["W_sure"].ravel(), (w * sure).sum(1), rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(r["S_sure"].ravel(), (v * w * sure).sum(1), rtol=1e-12,
                               atol=1e-300)
    np.testing.assert_allclose(r["cond_w"].ravel(), (w * dabs * inside).sum(1), rtol=1e-12,
                               atol=1e-300)
    Ib = (v * w * inside).sum(1) / np.maximum((w * inside).sum(1), 1e-12)
    np.testing.assert_allclose(r["cond_i"].ravel(),
                               (w * dabs * np.abs(v - Ib[:, None]) * inside).sum(1),
                               rtol=1e-9, atol=1e-14)
    ids = r["amb_id"].reshape(-1, oracle.AMB_SLOTS)
    for vox in np.nonzero(amb.any(1))[0]:
        want = np.nonzero(amb[vox])[0][:oracle.AMB_SLOTS]
        k = want.size
        np.testing.assert_array_equal(ids[vox, :k], want)
        assert np.all(ids[vox, k:] == -1)
        np.testing.assert_allclose(r["amb_w"].reshape(-1, 8)[vox, :k], w[vox, want], rtol=1e-13)
        np.testing.assert_allclose(r["amb_vw"].reshape(-1, 8)[vox, :k],
                                   v[vox, want] * w[vox, want], rtol=1e-13)
        np.testing.assert_allclose(r["amb_rel"].reshape(-1, 8)[vox, :k],
                                   (d2[vox, want] - 9.0) / dabs[vox, want], rtol=1e-9,
                                   atol=1e-12)
    # the FP64 decision is one subset: sure sums + included slots give S and W
    rel = r["amb_rel"].reshape(-1, 8)
    used = ids >= 0
    inc = used & (rel <= 0)
    few = r["amb"].ravel() <= oracle.AMB_SLOTS
    Wrec = r["W_sure"].ravel() + (r["amb_w"].reshape(-1, 8) * inc).sum(1)
    np.testing.assert_allclose(Wrec[few], r["W"].ravel()[few], rtol=1e-12, atol=1e-300)


def _tie_cloud():
    """Gaussian A is axis-aligned with scales (1, 1.3, 1.7) and its mean 3 voxels from the
    centre of voxel (5, 6, 6) along x, so d^2 = 9 exactly there (exactly representable; the
    mirror voxel at x = -1 is outside the grid); Gaussian B, rotated and wider, overlaps it so
    the tie voxel has other content."""
    pa = [2.5, 6.5, 6.5, 0.0, np.log(1.3), np.log(1.7), 1.0, 0.0, 0.0, 0.0, 0.8, 0.6]
    pb = [6.1, 5.3, 6.9, np.log(2.1), np.log(1.6), np.log(2.4), 0.9, 0.3, -0.2, 0.25, 0.3, 0.4]
    return np.array([pa, pb], np.float64)


def test_exact_tie_is_ambiguous_and_included(oracle_mod):
    """A pair exactly on the boundary (d^2 = 9) is the only ambiguous pair, sits at relative
    distance 0, carries w = r e^{-9/2}, and is included by the inclusive truncation."""
    import oracle
    o = oracle_mod
    p = _tie_cloud()
    g = oracle.Grid(12, 12, 12)
    r = o.render(p, g, want_amb=True)
    assert r["amb"].sum() == 1 and r["amb"][6, 6, 5] == 1
    assert r["amb_id"][6, 6, 5, 0] == 0 and r["amb_rel"][6, 6, 5, 0] == 0.0
    assert r["amb_w"][6, 6, 5, 0] == pytest.approx(0.6 * np.exp(-4.5), rel=1e-15)
    assert r["amb_vw"][6, 6, 5, 0] == pytest.approx(0.8 * 0.6 * np.exp(-4.5), rel=1e-15)
    assert r["W"][6, 6, 5] == pytest.approx(r["W_sure"][6, 6, 5] + r["amb_w"][6, 6, 5, 0],
                                            rel=1e-14)


def test_gradient_box_brackets_both_decisions(oracle_mod):
    """With one ambiguous pair there are two valid renders: the tie pair in (truncation radius
    3 (1 + 1e-9)) or out (3 (1 - 1e-9)). Their FP64 gradients are exactly the componentwise
    ends of the box reported at radius 3, and the FP64 decision (inclusive) equals the first.
    Catches a box built from the wrong sure sums, a subset whose I or W drops a term, a sign
    error in the range, and an exclusive truncation."""
    import oracle
    o = oracle_mod
    p = _tie_cloud()
    g = oracle.Grid(12, 12, 12)
    dI = inputs.crop_dI(3, g.shape).astype(np.float64)
    box = o.render_grad(p, g, dI, want_box=True)
    g_in = o.render_grad(p, g, dI, oracle.Config(trunc_sigma=3.0 * (1 + 1e-9)))
    g_out = o.render_grad(p, g, dI, oracle.Config(trunc_sigma=3.0 * (1 - 1e-9)))
    assert not np.allclose(g_in, g_out, rtol=1e-6)
    np.testing.assert_allclose(box["grad"], g_in, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(box["lo"], np.minimum(g_in, g_out), rtol=1e-10, atol=1e-15)
    np.testing.assert_allclose(box["hi"], np.maximum(g_in, g_out), rtol=1e-10, atol=1e-15)
    assert box["n_unenum"] == 0


def test_gradient_box_collapses_without_ties(oracle_mod):
    """With no pair in the band the box is the FP64 gradient itself."""
    import oracle
    o = oracle_mod
    g = oracle.Grid(10, 10, 10)
    for seed in range(4, 60):
        dd = inputs.gaussian_cloud(seed, 6, (10, 10, 10), scale_range=(0.9, 1.8))
        p = inputs.assemble_params(dd["mu"], dd["log_s"], dd["q"], dd["pd"],
                                   dd["pd"] * 0.5 + 0.2).astype(np.float64)
        if o.render(p, g)["amb"].sum() == 0:
            break
    dI = inputs.crop_dI(8, g.shape).astype(np.float64)
    box = o.render_grad(p, g, dI, want_box=True)
    np.testing.assert_array_equal(box["lo"], box["grad"])
    np.testing.assert_array_equal(box["hi"], box["grad"])
    np.testing.assert_array_equal(box["grad"], o.render_grad(p, g, dI))


def _tie_ref():
    import oracle
    d = inputs.gaussian_cloud(0, 300, (16, 16, 16))
    p = inputs.assemble_params(d["mu"], d["log_s"], d["q"], d["pd"],
                               d["pd"] * 0.5 + 0.2).astype(np.float64)
    g = oracle.Grid(16, 16, 16)
    # a wide band so that many voxels hold ambiguous pairs
    return oracle.render(p, g, amb_tol=2e-3, want_amb=True), p, g


def test_forward_subset_check_accepts_either_decision():
    """The FP64 decision passes; so does a result that flips the decision on one ambiguous pair
    of every tie voxel (rebuilt from the reported terms)."""
    import oracle
    ref, _, _ = _tie_ref()
    assert (ref["amb"] > 0).sum() > 50
    st = oracle.forward_subset_check(ref["I"], ref["W"], ref)
    assert st["flips"] == 0 and st["n_tie"] > 50
    I2, W2 = ref["I"].copy(), ref["W"].copy()
    sel = (ref["amb"] > 0) & (ref["amb"] <= oracle.AMB_SLOTS)
    inc = (ref["amb_rel"] <= 0) & (ref["amb_id"] >= 0)
    inc[..., 0] = ~inc[..., 0]                       # flip the first slot
    inc &= ref["amb_id"] >= 0
    Wf = ref["W_sure"] + (ref["amb_w"] * inc).sum(-1)
    Sf = ref["S_sure"] + (ref["amb_vw"] * inc).sum(-1)
    W2[sel] = Wf[sel]
    I2[sel] = (Sf / np.maximum(Wf, 1e-12))[sel]
    st = oracle.forward_subset_check(I2, W2, ref)
    assert st["flips"] >= (sel & (ref["W"] > 1e-6)).sum() * 0.9


def test_forward_subset_check_rejects_planted_errors():
    """A 1e-4 relative error in I on a plain voxel, or a tie voxel whose W matches no subset,
    is rejected."""
    import oracle
    ref, _, _ = _tie_ref()
    plain = np.argwhere((ref["amb"] == 0) & (ref["W"] > 1e-3))[0]
    I2 = ref["I"].copy()
    I2[tuple(plain)] *= 1 + 1e-4
    with pytest.raises(AssertionError):
        oracle.forward_subset_check(I2, ref["W"], ref)
    tie = np.argwhere((ref["amb"] == 1) & (ref["W"] > 1e-3))[0]
    W2 = ref["W"].copy()
    W2[tuple(tie)] += 0.5 * ref["amb_w"][tuple(tie)][0]   # half a pair: no subset
    with pytest.raises(AssertionError):
        oracle.forward_subset_check(ref["I"], W2, ref)


def test_gradient_box_check_projects_onto_the_box(oracle_mod):
    """Any point of the box passes (distance 0); a point 1e-3 of the norm outside fails."""
    import oracle
    o = oracle_mod
    p = _tie_cloud()
    g = oracle.Grid(12, 12, 12)
    dI = inputs.crop_dI(3, g.shape).astype(np.float64)
    box = o.render_grad(p, g, dI, want_box=True)
    dist, width = oracle.gradient_box_check(box["lo"], box)
    assert dist == 0.0 and width > 0
    dist, _ = oracle.gradient_box_check(0.5 * (box["lo"] + box["hi"]), box)
    assert dist == 0.0
    off = box["hi"].copy()
    off[0, 0] += 1e-3 * np.linalg.norm(box["grad"])
    with pytest.raises(AssertionError):
        oracle.gradient_box_check(off, box)
