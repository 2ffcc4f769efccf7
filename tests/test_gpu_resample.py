"""Trilinear resize (Sec. 4.1 LR degradation) and its adjoint on the GPU against the oracle;
lattice init on a resize grid; the fitting step with the trilinear LR model (Sec. 4.2:
super-resolution to an arbitrary target shape) against the oracle's composed step."""
import numpy as np
import pytest

from helpers import phantom_fit_trilinear, rel_l2, to_dev

pytestmark = pytest.mark.gpu

SHAPES = [((21, 29, 37), (9, 13, 16)),      # ragged downsampling, every axis
          ((32, 48, 64), (16, 24, 32)),     # factor 2 (block means)
          ((7, 9, 11), (16, 13, 20)),       # upsampling
          ((40, 30, 50), (40, 12, 77)),     # mixed: identity, down, up
          ((20, 24, 30), (26, 30, 40)),     # mild upsampling (four-slot adjoint runs)
          ((20, 64, 100), (19, 62, 96)),    # near-identity downsampling (four-slot runs)
          ((1, 5, 6), (3, 1, 2))]           # degenerate single-slice axes


def _gs():
    from paper_2603_09621_gb300 import gs
    return gs


@pytest.mark.parametrize("src,dst", SHAPES)
def test_resample_fwd_matches_oracle(src, dst):
    import oracle
    import torch
    gs = _gs()
    rng = np.random.default_rng(sum(src) + sum(dst))
    v = rng.uniform(-1, 1, src).astype(np.float32)
    got = gs.gs_resample_fwd(to_dev(v), dst)
    torch.cuda.synchronize()
    ref = oracle.resample(v.astype(np.float64), dst)
    # the same FP32 sample positions on both sides; FP32 blends of three lerps
    np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=0, atol=1e-6)


@pytest.mark.parametrize("src,dst", SHAPES)
def test_resample_bwd_matches_oracle(src, dst):
    import oracle
    import torch
    gs = _gs()
    rng = np.random.default_rng(7 + sum(src))
    d = rng.uniform(-1, 1, dst).astype(np.float32)
    got = gs.gs_resample_bwd(to_dev(d), src)
    torch.cuda.synchronize()
    ref = oracle.resample_adjoint(d.astype(np.float64), src)
    fan = max(1.0, max(dst[a] / src[a] for a in range(3))) ** 3 * 8
    np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=0, atol=2e-7 * fan)


def test_resample_adjoint_identity_gpu():
    """<R x, y> = <x, R^T y> with the GPU's forward and adjoint (FP64 dot products)."""
    import torch
    gs = _gs()
    rng = np.random.default_rng(11)
    for src, dst in SHAPES[:4]:
        x = rng.uniform(-1, 1, src).astype(np.float32)
        y = rng.uniform(-1, 1, dst).astype(np.float32)
        Rx = gs.gs_resample_fwd(to_dev(x), dst)
        Rty = gs.gs_resample_bwd(to_dev(y), src)
        torch.cuda.synchronize()
        lhs = float((Rx.cpu().numpy().astype(np.float64) * y).sum())
        rhs = float((x.astype(np.float64) * Rty.cpu().numpy()).sum())
        assert lhs == pytest.approx(rhs, rel=1e-5, abs=1e-4)


def test_resample_arbitrary_shape_full_size():
    """Sec. 4.2's arbitrary-shape case at full size: 240 x 240 x 155 <-> 100^3, every output
    against the oracle."""
    import oracle
    import torch
    gs = _gs()
    rng = np.random.default_rng(5)
    hr = rng.uniform(0, 1, (155, 240, 240)).astype(np.float32)
    lr = gs.gs_resample_fwd(to_dev(hr), (100, 100, 100))
    torch.cuda.synchronize()
    np.testing.assert_allclose(lr.cpu().numpy(), oracle.resample(hr.astype(np.float64), (100,) * 3),
                               rtol=0, atol=1e-6)
    d = rng.uniform(-1, 1, (100, 100, 100)).astype(np.float32)
    back = gs.gs_resample_bwd(to_dev(d), (155, 240, 240))
    torch.cuda.synchronize()
    np.testing.assert_allclose(back.cpu().numpy(),
                               oracle.resample_adjoint(d.astype(np.float64), (155, 240, 240)),
                               rtol=0, atol=2e-6)


def test_resample_rejects_bad_sizes():
    gs = _gs()
    import torch
    v = torch.zeros((4, 4, 4), device="cuda")
    with pytest.raises(gs.GsError):
        gs.gs_resample_fwd(v, (0, 4, 4))


def test_init_lattice_lr_matches_oracle():
    import oracle
    import torch
    gs = _gs()
    og = oracle.Grid(64, 48, 40, (0.9, 1.1, 1.3), (-2.0, 1.0, 0.5))
    rng = np.random.default_rng(4)
    lr = rng.uniform(0, 1, (17, 23, 29)).astype(np.float32)
    n, _ = oracle.lattice_dims(og, 20000)
    ref = oracle.init_lattice_lr(lr, og, 20000, t_act=1)
    got = gs.gs_init_lattice_lr(to_dev(lr), gs.Grid(64, 48, 40, og.h, og.origin), n, t_act=1,
                                t_init=0.5)
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    assert got.shape == ref.shape
    np.testing.assert_allclose(got[:, :10], ref[:, :10], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(got[:, 10], ref[:, 10], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(got[:, 11], ref[:, 11], atol=1e-7)


def _tie_free_target(w, cfg_o):
    """LR target = the oracle's trilinear prediction at the initial params shifted by
    +-[0.01, 0.05] (random signs): sign(pred - target) of the L1 gradient has no ties."""
    import oracle
    r = oracle.render(w["params0"].astype(np.float64), w["grid"], cfg_o)
    pred = oracle.resample(r["I"], w["lr"].shape)
    rng = np.random.default_rng(8)
    shift = rng.choice([-1.0, 1.0], pred.shape) * rng.uniform(0.01, 0.05, pred.shape)
    return (pred + shift).astype(np.float32)


def test_fit_step_trilinear_matches_oracle():
    import oracle
    import torch
    gs = _gs()
    w = phantom_fit_trilinear()
    og = w["grid"]
    cfg_o = oracle.Config(t_act=1)
    target = _tie_free_target(w, cfg_o)
    n = w["params0"].shape[0]
    ref = oracle.fit_step(w["params0"], target, og, 1, cfg_o, np.zeros((n, 12)),
                          np.zeros((n, 12)), 1, lr_model="trilinear")
    st = gs.FitState(to_dev(w["params0"]), to_dev(target), gs.Grid(og.nx, og.ny, og.nz), 1,
                     gs.Config(t_act=1), lr_model=gs.GS_LR_TRILINEAR)
    st.step()
    torch.cuda.synchronize()
    rc, bits = st.check()
    assert rc == 0 and bits == 0
    assert float(st.d_loss) == pytest.approx(ref["loss"], rel=1e-5)
    assert rel_l2(st.grad.cpu().numpy(), ref["grad"]) <= 1e-4
    assert int(st.d_step) == 1


def test_fit_trilinear_loss_decreases_and_serving_matches():
    """Thirty steps of the trilinear-model fit lower the loss; the same fit through the
    serving runtime is bit-identical (deterministic mode)."""
    import torch
    from paper_2603_09621_gb300 import serve, workloads
    gs = _gs()
    wk = workloads.phantom_fit_trilinear(shape=(48, 64, 72), lr_shape=(20, 26, 29),
                                         n_gauss=12000, seed=3)
    st = gs.FitState(wk["params0"], wk["lr"], wk["grid"], 1, gs.Config(t_act=1),
                     lr_model=gs.GS_LR_TRILINEAR)
    losses = []
    for _ in range(30):
        st.step()
        losses.append(float(st.d_loss))
    torch.cuda.synchronize()
    assert min(losses[-5:]) < 0.95 * losses[0]
    with serve.Server(1 << 30, max_active=2, chunk_steps=8) as sv:
        rid = sv.submit_fit(wk["params0"], wk["lr"], wk["grid"], 1, 30,
                            lr_model=gs.GS_LR_TRILINEAR)
        sv.run(timeout_s=120)
        assert sv.result(rid)["state"] == "done"
        out = sv.output(rid)
    assert torch.equal(out.view(torch.int32), st.params.view(torch.int32))
