"""The split fitting step (gs_fit_grad + gs_fit_apply) and the z-slab sharding of one volume on
the GPU. One GPU plays both slabs in turn (each slab's step runs to completion before the
other's; their gradients are summed by the test in place of the all-reduce), and the result is
checked against the FP64 oracle's single-process step of the whole volume."""
import numpy as np
import pytest

from helpers import phantom_fit, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _gs():
    from paper_2603_09621_gb300 import gs
    return gs


def _small():
    """The fitting test's workload (32 x 48 x 48, 6,000 Gaussians, z box x4), with an LR target
    shifted from the oracle's prediction by +-[0.01, 0.05] so that the L1 gradient's signs are
    the same in FP32 and FP64."""
    import oracle
    w = phantom_fit(shape=(32, 48, 48), s=4, n_gauss=6000, seed=1, n_ell=5, semi=(5.0, 16.0))
    cfg_o = oracle.Config(t_act=1)
    r = oracle.render(w["params0"].astype(np.float64), w["grid"], cfg_o)
    pred = oracle.downsample(r["I"], w["s"])
    rng = np.random.default_rng(7)
    shift = rng.choice([-1.0, 1.0], pred.shape) * rng.uniform(0.01, 0.05, pred.shape)
    return w, (pred + shift).astype(np.float32), cfg_o


def test_split_step_equals_fused_step():
    """gs_fit_grad(st, 0) then gs_fit_apply(st, overflow flag) = gs_fit_step, bit for bit, over
    three steps (loss, gradient, parameters, moments, step counter)."""
    import torch
    gs = _gs()
    w, target, _ = _small()
    og = w["grid"]
    g = gs.Grid(og.nx, og.ny, og.nz)
    a = gs.FitState(to_dev(w["params0"]), to_dev(target), g, w["s"], gs.Config(t_act=1))
    b = gs.FitState(to_dev(w["params0"]), to_dev(target), g, w["s"], gs.Config(t_act=1),
                    capacity=a.capacity)
    for _ in range(3):
        a.step()
        b.grad_step(0)
        b.apply(b.overflow_flag())
    torch.cuda.synchronize()
    for x, y in ((a.params, b.params), (a.grad, b.grad), (a.m, b.m), (a.v, b.v),
                 (a.d_loss, b.d_loss)):
        assert torch.equal(x.view(torch.int32), y.view(torch.int32))
    assert int(a.d_step) == int(b.d_step) == 3


def test_apply_skips_on_flag():
    import torch
    gs = _gs()
    w, target, _ = _small()
    og = w["grid"]
    st = gs.FitState(to_dev(w["params0"]), to_dev(target), gs.Grid(og.nx, og.ny, og.nz), w["s"],
                     gs.Config(t_act=1))
    st.grad_step(0)
    st.apply(torch.ones(1, dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    assert torch.equal(st.params, to_dev(w["params0"]))
    assert int(st.d_step) == 0 and int(torch.count_nonzero(st.m)) == 0


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_reproduce_the_whole_volume_step(world):
    """`world` z-slabs of the 32-slice volume (whole LR slices each), stepped with the sum of
    their gradients: every slab ends with the same parameters; the summed gradient and loss
    match the FP64 oracle's step of the whole volume (relative L2 1e-4, loss 1e-5), and the
    parameters match where every gradient is clearly nonzero; the summed gradient also
    matches the single-volume GPU step."""
    import torch
    import oracle
    from paper_2603_09621_gb300 import shard
    gs = _gs()
    w, target, cfg_o = _small()
    og, s = w["grid"], w["s"]
    n = w["params0"].shape[0]
    ref = oracle.fit_step(w["params0"], target, og, s, cfg_o, np.zeros((n, 12)),
                          np.zeros((n, 12)), 1)
    grid = gs.Grid(og.nx, og.ny, og.nz)
    p0, lr = to_dev(w["params0"]), to_dev(target)
    fits = [shard.SlabFit(p0, lr, grid, s, r, world, reduce=lambda g, f: None)
            for r in range(world)]
    assert sum(f.z1 - f.z0 for f in fits) == og.nz
    for f in fits:
        f.state.grad_step(f.n_lr_total)
    total = sum(f.state.grad for f in fits)
    flag = torch.stack([f.state.overflow_flag() for f in fits]).amax(0)
    loss = float(sum(f.state.d_loss for f in fits))
    for f in fits:
        f.state.grad.copy_(total)
        f.state.apply(flag)
    torch.cuda.synchronize()
    assert int(flag) == 0
    for f in fits[1:]:
        assert torch.equal(f.state.params, fits[0].state.params)
    assert loss == pytest.approx(ref["loss"], rel=1e-5)
    assert rel_l2(total.cpu().numpy(), ref["grad"]) <= 1e-4
    got = fits[0].state.params.cpu().numpy().astype(np.float64)
    gr = np.abs(ref["grad"])
    clear = gr > 1e-3 * np.sqrt((ref["grad"] ** 2).mean(0))[None, :]
    np.testing.assert_allclose(got[clear], ref["params"][clear], rtol=1e-6, atol=2e-6)
    whole = gs.FitState(p0, lr, grid, s, gs.Config(t_act=1))
    whole.step()
    torch.cuda.synchronize()
    assert rel_l2(total.cpu().numpy(), whole.grad.cpu().numpy()) <= 1e-5
