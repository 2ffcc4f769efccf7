"""One zero-shot fitting step (bin, render, slice profile, L1, adjoints, Adam) on the GPU
against the oracle's composed step; multi-step behaviour; CUDA-graph replay."""
import numpy as np
import pytest

from helpers import phantom_fit, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _gs():
    from paper_2603_09621_gb300 import gs
    return gs


def small_fit():
    return phantom_fit(shape=(32, 48, 48), s=4, n_gauss=6000, seed=1, n_ell=5, semi=(5.0, 16.0))


def _tie_free_target(w, cfg_o):
    """LR target = the oracle's prediction at the initial params shifted by +-[0.01, 0.05]
    (random signs), so that sign(pred - target) of the L1 gradient has no ties."""
    import oracle
    r = oracle.render(w["params0"].astype(np.float64), w["grid"], cfg_o)
    pred = oracle.downsample(r["I"], w["s"])
    rng = np.random.default_rng(7)
    shift = rng.choice([-1.0, 1.0], pred.shape) * rng.uniform(0.01, 0.05, pred.shape)
    return (pred + shift).astype(np.float32)


def test_fit_step_matches_oracle():
    import oracle
    import torch
    gs = _gs()
    w = small_fit()
    og = w["grid"]
    cfg_o = oracle.Config(t_act=1)
    target = _tie_free_target(w, cfg_o)
    n = w["params0"].shape[0]
    ref = oracle.fit_step(w["params0"], target, og, w["s"], cfg_o, np.zeros((n, 12)),
                          np.zeros((n, 12)), 1)
    st = gs.FitState(to_dev(w["params0"]), to_dev(target), gs.Grid(og.nx, og.ny, og.nz), w["s"],
                     gs.Config(t_act=1))
    st.step()
    torch.cuda.synchronize()
    rc, bits = st.check()
    assert rc == 0 and bits == 0
    assert float(st.d_loss) == pytest.approx(ref["loss"], rel=1e-5)
    grad = st.grad.cpu().numpy()
    assert rel_l2(grad, ref["grad"]) <= 1e-4
    assert rel_l2(st.m.cpu().numpy(), ref["m"]) <= 1e-4
    # Adam's first step moves each parameter by lr * g / (|g| + eps): compare where the
    # oracle gradient is clearly non-zero; elsewhere the step is bounded by the rate.
    p_new = st.params.cpu().numpy().astype(np.float64)
    g = np.abs(ref["grad"])
    clear = g > 1e-3 * np.sqrt((ref["grad"] ** 2).mean(0))[None, :]
    np.testing.assert_allclose(p_new[clear], ref["params"][clear], rtol=1e-6, atol=2e-6)
    lrs = oracle.AdamConfig().lr_vector()[None, :] * np.ones_like(g)
    assert np.all(np.abs(p_new - w["params0"]) <= 1.0001 * lrs + 1e-6)
    assert int(st.d_step) == 1


def test_fit_loss_decreases_and_psnr_rises():
    """Forty steps on the phantom: the L1 loss falls and the HR render moves towards the
    clean phantom (PSNR against it rises)."""
    import oracle
    import torch
    gs = _gs()
    w = small_fit()
    og = w["grid"]
    st = gs.FitState(to_dev(w["params0"]), to_dev(w["lr"]), gs.Grid(og.nx, og.ny, og.nz), w["s"],
                     gs.Config(t_act=1))
    losses = []
    st.step()
    torch.cuda.synchronize()
    psnr0 = oracle.psnr(st.I.cpu().numpy(), w["hr"])
    for _ in range(40):
        st.step()
        losses.append(float(st.d_loss))
    torch.cuda.synchronize()
    psnr1 = oracle.psnr(st.I.cpu().numpy(), w["hr"])
    assert losses[-1] < 0.8 * losses[0]
    assert psnr1 > psnr0


def test_fit_step_graph_replay_matches_eager():
    """The step has no host synchronisation: a CUDA graph of it replays to the same
    parameters as eager steps (deterministic mode, bit for bit)."""
    import torch
    gs = _gs()
    w = small_fit()
    og = w["grid"]
    g = gs.Grid(og.nx, og.ny, og.nz)
    eager = gs.FitState(to_dev(w["params0"]), to_dev(w["lr"]), g, w["s"], gs.Config(t_act=1))
    graphed = gs.FitState(to_dev(w["params0"]), to_dev(w["lr"]), g, w["s"], gs.Config(t_act=1),
                          capacity=eager.capacity)
    for _ in range(3):
        eager.step()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        graphed.step(stream=s)  # warm-up step outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=s):
        graphed.step(stream=s)
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(eager.params, graphed.params)
    assert int(graphed.d_step) == 3


@pytest.mark.parametrize("deterministic", [1, 0])
def test_fit_step_overflow_is_a_no_op(deterministic):
    """A step whose binning overflows the pair capacity leaves params, moments and the step
    counter unchanged and reports GS_STATUS_CAPACITY; after growing, the fit continues as if
    the capacity had sufficed."""
    import torch
    gs = _gs()
    w = small_fit()
    og = w["grid"]
    g = gs.Grid(og.nx, og.ny, og.nz)
    cfg = gs.Config(t_act=1, deterministic=deterministic)
    ref = gs.FitState(to_dev(w["params0"]), to_dev(w["lr"]), g, w["s"], cfg)
    tiny = gs.FitState(to_dev(w["params0"]), to_dev(w["lr"]), g, w["s"], cfg, capacity=1000)
    ref.step()
    tiny.step()
    tiny.step()
    torch.cuda.synchronize()
    rc, bits = tiny.check()
    assert bits & gs.GS_STATUS_CAPACITY
    assert int(tiny.d_step) == 0
    assert torch.equal(tiny.params, to_dev(w["params0"]))
    assert int(torch.count_nonzero(tiny.m)) == 0 and int(torch.count_nonzero(tiny.v)) == 0
    assert int(torch.count_nonzero(tiny.grad)) == 0
    if deterministic:
        grown = gs.FitState(tiny.params, to_dev(w["lr"]), g, w["s"], cfg, capacity=ref.capacity)
        grown.step()
        torch.cuda.synchronize()
        assert torch.equal(grown.params, ref.params)


@pytest.mark.parametrize("lr_model", ["zbox", "trilinear"])
def test_fit_step_full_size_equals_composed_entry_points(lr_model):
    """At full size, in the bench's configuration (graph-capturable fused step, 8^3 bricks,
    deterministic), one gs_fit_step equals the composition of the public entry points that
    the parity tests check against the oracle: render, LR forward model, L1, its adjoint,
    adjoint render, Adam. Loss, gradient and updated parameters must agree bit for bit."""
    import torch
    from paper_2603_09621_gb300 import workloads
    gs = _gs()
    cfg = gs.Config(t_act=1)
    if lr_model == "zbox":
        w = workloads.phantom_fit()
        st = gs.FitState(w["params0"], w["lr"], w["grid"], w["s"], cfg)
    else:
        w = workloads.phantom_fit_trilinear()
        st = gs.FitState(w["params0"], w["lr"], w["grid"], 1, cfg, lr_model=gs.GS_LR_TRILINEAR)
    g = w["grid"]
    st.step()
    torch.cuda.synchronize()
    assert st.check()[0] == 0
    # composed: every step through its own entry point
    p0 = w["params0"]
    I, W, bins, ws = gs.render(p0, g, cfg)
    if lr_model == "zbox":
        pred = gs.gs_downsample_fwd(I, w["s"])
    else:
        pred = gs.gs_resample_fwd(I, tuple(w["lr"].shape))
    dpred = torch.empty_like(pred)
    loss = gs.gs_l1_loss(pred, w["lr"], ws, dpred=dpred)
    if lr_model == "zbox":
        dI = gs.gs_downsample_bwd(dpred, g.nz, w["s"])
    else:
        dI = gs.gs_resample_bwd(dpred, tuple(I.shape))
    grad = gs.gs_render_bwd(p0, bins, g, cfg, I, W, dI, ws)
    params = p0.clone()
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    d_step = torch.zeros((), dtype=torch.int32, device=params.device)
    gs.gs_adam_step(params, grad, m, v, gs.Adam(), d_step)
    torch.cuda.synchronize()
    assert torch.equal(st.d_loss, loss)
    assert torch.equal(st.grad.view(torch.int32), grad.view(torch.int32))
    assert torch.equal(st.params.view(torch.int32), params.view(torch.int32))
    assert torch.equal(st.m.view(torch.int32), m.view(torch.int32))
    assert int(st.d_step) == int(d_step) == 1


@pytest.mark.parametrize("pinned", [True, False])
def test_fit_steps_host_equal_device_steps(pinned):
    """Three steps through gs_fit_step_host, from page-locked or ordinary host memory, each
    uploading the step's parameters and LR target, equal three device steps that start from
    the same uploads (the side-stream copy of the LR target must not overtake the step before
    it), bit for bit, with every step's loss read back."""
    import torch
    gs = _gs()
    w = small_fit()
    og = w["grid"]
    g = gs.Grid(og.nx, og.ny, og.nz)
    a = gs.FitState(to_dev(w["params0"]), to_dev(w["lr"]), g, w["s"], gs.Config(t_act=1))
    b = gs.FitState(torch.zeros_like(a.params), torch.zeros_like(a.lr_target), g, w["s"],
                    gs.Config(t_act=1), capacity=a.capacity)
    rng = np.random.default_rng(11)
    for k in range(3):
        # each step gets its own inputs: perturbed parameters and LR target
        p = (w["params0"] + rng.normal(0.0, 1e-3, w["params0"].shape)).astype(np.float32)
        lr = (w["lr"] + rng.normal(0.0, 1e-2, w["lr"].shape)).astype(np.float32)
        h_params, h_lr = torch.as_tensor(p).contiguous(), torch.as_tensor(lr).contiguous()
        h_loss = torch.full((), -1.0)
        if pinned:
            h_params, h_lr, h_loss = h_params.pin_memory(), h_lr.pin_memory(), h_loss.pin_memory()
        a.params.copy_(to_dev(p))
        a.lr_target.copy_(to_dev(lr))
        a.step()
        b.step_host(h_params, h_lr, h_loss)
        torch.cuda.synchronize()
        assert torch.equal(a.params, b.params) and torch.equal(a.grad, b.grad)
        assert torch.equal(a.m, b.m) and torch.equal(a.v, b.v)
        assert float(h_loss) == float(a.d_loss)


def test_fit_step_host_equals_device_step():
    """gs_fit_step_host (inputs copied from page-locked host memory inside the call, loss copied
    back) gives the device step's result bit for bit."""
    import torch
    gs = _gs()
    w = small_fit()
    og = w["grid"]
    g = gs.Grid(og.nx, og.ny, og.nz)
    a = gs.FitState(to_dev(w["params0"]), to_dev(w["lr"]), g, w["s"], gs.Config(t_act=1))
    b = gs.FitState(torch.zeros_like(a.params), torch.zeros_like(a.lr_target), g, w["s"],
                    gs.Config(t_act=1), capacity=a.capacity)
    h_params = torch.as_tensor(w["params0"]).contiguous().pin_memory()
    h_lr = torch.as_tensor(w["lr"]).contiguous().pin_memory()
    h_loss = torch.full((), -1.0).pin_memory()
    a.step()
    b.step_host(h_params, h_lr, h_loss)
    torch.cuda.synchronize()
    assert torch.equal(a.params, b.params) and torch.equal(a.grad, b.grad)
    assert float(h_loss) == float(a.d_loss)
    with pytest.raises(ValueError):
        b.step_host(h_params[:10].contiguous())
