"""Serving runtime on the GPU: a request's result does not depend on what else is resident,
on chunking, graphs or pair capacity (deterministic mode: bit-identical to stepping one
FitState), admission keeps to the arena budget, renders wait for their source fit."""
import functools

import pytest

pytestmark = pytest.mark.gpu

MB = 1 << 20


def _mods():
    import torch
    from paper_2603_09621_gb300 import gs, serve, workloads
    return torch, gs, serve, workloads


@functools.lru_cache(maxsize=None)
def _scan(seed, shape=(48, 64, 64), s=2, n=12000):
    _, _, _, workloads = _mods()
    w = workloads.phantom_fit(shape=shape, s=s, n_gauss=n, seed=seed)
    return w["params0"], w["lr"], w["grid"], s


def _fit_reference(seed, iters, **scan_kw):
    """The plain path: one FitState stepped `iters` times on the current stream."""
    torch, gs, _, _ = _mods()
    p0, lr, grid, s = _scan(seed, **scan_kw)
    st = gs.FitState(p0, lr, grid, s, gs.Config(t_act=1))
    for _ in range(iters):
        st.step()
    torch.cuda.synchronize()
    assert st.check()[0] == 0
    return st.params.clone()


def _equal(a, b):
    torch = _mods()[0]
    return torch.equal(a.view(torch.int32), b.view(torch.int32))


def test_fit_matches_fitstate_graph_chunks_and_eager_tail():
    """30 steps in chunks of 8: three graph replays and a 6-step eager tail."""
    _, gs, serve, _ = _mods()
    p0, lr, grid, s = _scan(1)
    ref = _fit_reference(1, 30)
    with serve.Server(512 * MB, max_active=2, chunk_steps=8) as sv:
        rid = sv.submit_fit(p0, lr, grid, s, 30)
        sv.run(timeout_s=120)
        r = sv.result(rid)
        assert r["state"] == "done" and r["steps_done"] == 30 and r["chunks"] == 4
        assert _equal(sv.output(rid), ref)
        assert sv.stats()["graphs_captured"] == 1


def test_alone_equals_in_mix():
    """A fit run alone, and inside a mix of four fits of other scans and a render, resident
    together on four streams: identical bits (and identical to eager steps)."""
    _, gs, serve, _ = _mods()
    p0, lr, grid, s = _scan(2)
    with serve.Server(512 * MB, max_active=1, chunk_steps=10) as sv:
        a = sv.submit_fit(p0, lr, grid, s, 40)
        sv.run(timeout_s=120)
        alone = sv.output(a)
    with serve.Server(2048 * MB, max_active=4, chunk_steps=7, use_graphs=False) as sv:
        b = sv.submit_fit(p0, lr, grid, s, 40)
        sv.run(timeout_s=120)
        eager = sv.output(b)
    with serve.Server(4096 * MB, max_active=4, chunk_steps=10) as sv:
        others = []
        for k, seed in enumerate((3, 4, 5)):
            q0, qlr, qg, qs = _scan(seed, shape=(40 + 8 * k, 72, 56), s=2 + k % 2,
                                    n=9000 + 3000 * k)
            others.append(sv.submit_fit(q0, qlr, qg, qs, 25 + 10 * k, arrival_s=0.0))
        mid = sv.submit_fit(p0, lr, grid, s, 40, arrival_s=0.0)
        rend = sv.submit_render(gs.Grid(80, 80, 60, (0.8, 0.8, 0.8)), source=others[0])
        sv.run(timeout_s=300)
        st = sv.stats()
        assert st["n_done"] == 5 and st["n_failed"] == 0
        mixed = sv.output(mid)
        assert sv.result(rend)["state"] == "done"
    assert _equal(alone, eager)
    assert _equal(alone, mixed)


def test_capacity_growth_is_invisible():
    """Starting at 0.25 pairs per Gaussian, the bins grow between chunks (overflowed steps
    are no-ops); the result equals the plain path's."""
    _, gs, serve, _ = _mods()
    p0, lr, grid, s = _scan(6)
    ref = _fit_reference(6, 20)
    with serve.Server(512 * MB, max_active=1, chunk_steps=5, pairs_per_gauss=0.25) as sv:
        rid = sv.submit_fit(p0, lr, grid, s, 20)
        sv.run(timeout_s=120)
        r = sv.result(rid)
        assert r["state"] == "done" and r["grows"] >= 1
        assert r["status_bits"] & gs.GS_STATUS_CAPACITY
        assert _equal(sv.output(rid), ref)


def test_render_of_fitted_cloud_matches_render_fwd():
    """A render request of a finished fit on a finer grid equals gs_render_fwd of the fitted
    cloud; it waits for its source although it arrived first in the queue order."""
    torch, gs, serve, _ = _mods()
    p0, lr, grid, s = _scan(7)
    g2 = gs.Grid(70, 70, 52, (0.9, 0.9, 0.9), (0.5, 0.25, 0.0))
    with serve.Server(1024 * MB, max_active=2, chunk_steps=5) as sv:
        f = sv.submit_fit(p0, lr, grid, s, 15)
        r = sv.submit_render(g2, source=f, arrival_s=0.0)
        sv.run(timeout_s=120)
        rf, rr = sv.result(f), sv.result(r)
        assert rr["admit_s"] >= rf["done_s"]
        fitted = sv.output(f)
        vol = sv.output(r)
        with pytest.raises(gs.GsError):
            sv.release(10)                   # unknown id
        sv.release(r)
        sv.release(f)
    cfg = gs.Config(t_act=1)
    I = gs.render(fitted, g2, cfg)[0]
    torch.cuda.synchronize()
    assert vol.shape == I.shape and _equal(vol, I)


def test_admission_keeps_to_budget():
    """An arena that holds one of these fits at a time: they run one after another, the arena
    high-water mark stays within the budget, and arrival order is kept."""
    _, gs, serve, _ = _mods()
    p0, lr, grid, s = _scan(8)
    probe = serve.Server(64 * MB, max_active=4)
    need = probe.request_bytes(serve.fit_request(p0, lr, grid, s, 10))
    probe.close()
    budget = int(need * 1.5)
    with serve.Server(budget, max_active=4, chunk_steps=5) as sv:
        ids = [sv.submit_fit(p0, lr, grid, s, 10, arrival_s=0.0) for _ in range(3)]
        sv.run(timeout_s=120)
        res = [sv.result(i) for i in ids]
        st = sv.stats()
    assert all(r["state"] == "done" for r in res)
    assert st["peak_bytes"] <= budget
    for a, b in zip(res, res[1:]):
        assert b["admit_s"] >= a["done_s"]


def test_bypass_bound_and_oversized_request():
    """A request larger than the arena is refused at submission; with max_bypass = 0 a blocked
    request is not overtaken, with max_bypass >= 1 a smaller later one runs first."""
    _, gs, serve, _ = _mods()
    small = _scan(9, shape=(32, 48, 48), n=4000)
    big = _scan(10, shape=(64, 96, 96), n=30000)
    probe = serve.Server(64 * MB, max_active=4)
    nb = probe.request_bytes(serve.fit_request(big[0], big[1], big[2], big[3], 10))
    ns = probe.request_bytes(serve.fit_request(small[0], small[1], small[2], small[3], 10))
    probe.close()
    assert nb > 2 * ns
    with serve.Server(nb + ns // 2, max_active=4) as sv:
        with pytest.raises(gs.GsError):
            sv.submit_fit(*_scan(11, shape=(128, 192, 192), n=200000)[:3], 2, 10)
    for bypass, small_first in ((0, False), (2, True)):
        with serve.Server(nb + ns // 2, max_active=4, chunk_steps=5, max_bypass=bypass) as sv:
            a = sv.submit_fit(small[0], small[1], small[2], small[3], 30, arrival_s=0.0)
            b = sv.submit_fit(big[0], big[1], big[2], big[3], 10, arrival_s=0.0)
            c = sv.submit_fit(small[0], small[1], small[2], small[3], 10, arrival_s=0.0)
            sv.run(timeout_s=120)
            rb, rc = sv.result(b), sv.result(c)
            assert rb["state"] == "done" and rc["state"] == "done"
            assert (rc["admit_s"] < rb["admit_s"]) == small_first, (bypass, rb, rc)


def test_held_outputs_block_until_released():
    """With the arena full of finished outputs and nothing resident, run() reports
    GS_ERR_CAPACITY instead of waiting; releasing an output lets the queue go on."""
    _, gs, serve, _ = _mods()
    p0, lr, grid, s = _scan(12)
    probe = serve.Server(64 * MB, max_active=4)
    need = probe.request_bytes(serve.fit_request(p0, lr, grid, s, 5))
    probe.close()
    out_bytes = p0.numel() * 4
    with serve.Server(need + out_bytes // 2, max_active=2, chunk_steps=5) as sv:
        a = sv.submit_fit(p0, lr, grid, s, 5)
        sv.run(timeout_s=60)
        assert sv.result(a)["state"] == "done"
        b = sv.submit_fit(p0, lr, grid, s, 5)
        with pytest.raises(gs.GsError, match="CAPACITY"):
            sv.run(timeout_s=60)
        assert sv.result(b)["state"] == "pending"
        first = sv.output(a)
        sv.release(a)
        sv.run(timeout_s=60)
        assert sv.result(b)["state"] == "done"
        assert _equal(sv.output(b), first)


def _tie_free_scan(seed=1, margin=(0.04, 0.08)):
    """Small fitting workload built by the oracle (phantom, LR scan, lattice init), with an LR
    target shifted from the oracle's initial prediction by +-[0.04, 0.08]: three Adam steps
    move the prediction by less than that, so no residual of the L1 loss crosses zero and the
    sign of its gradient is the same in FP32 and FP64."""
    import numpy as np
    import oracle
    from helpers import phantom_fit
    w = phantom_fit(shape=(32, 48, 48), s=4, n_gauss=6000, seed=seed, n_ell=5, semi=(5.0, 16.0))
    cfg_o = oracle.Config(t_act=1)
    r = oracle.render(w["params0"].astype(np.float64), w["grid"], cfg_o)
    pred = oracle.downsample(r["I"], w["s"])
    rng = np.random.default_rng(11)
    shift = rng.choice([-1.0, 1.0], pred.shape) * rng.uniform(margin[0], margin[1], pred.shape)
    return w, (pred + shift).astype(np.float32), cfg_o


def test_served_fit_matches_oracle_alone_and_in_mix():
    """A fit served alone (a graph chunk of 2 steps and an eager tail) and the same fit served
    among two other scans' fits give identical bits, and both agree with the FP64 oracle's
    composed fitting step (render, z box profile, L1, adjoints, Adam) iterated 3 times: the
    last step's loss to 1e-5, and the parameters to the fit step's tolerance wherever every
    step's gradient is clearly nonzero (elsewhere Adam's move is bounded by its rate)."""
    import numpy as np
    import oracle
    from helpers import to_dev
    torch, gs, serve, _ = _mods()
    K = 3
    w, target, cfg_o = _tie_free_scan()
    og, s = w["grid"], w["s"]
    n = w["params0"].shape[0]
    p, m, v = w["params0"].astype(np.float64), np.zeros((n, 12)), np.zeros((n, 12))
    grads, loss = [], None
    for t in range(1, K + 1):
        ref = oracle.fit_step(p, target, og, s, cfg_o, m, v, t)
        grads.append(ref["grad"])
        p, m, v, loss = ref["params"], ref["m"], ref["v"], ref["loss"]
    grid = gs.Grid(og.nx, og.ny, og.nz)
    p0, lr = to_dev(w["params0"]), to_dev(target)
    with serve.Server(512 * MB, max_active=1, chunk_steps=2) as sv:
        rid = sv.submit_fit(p0, lr, grid, s, K)
        sv.run(timeout_s=120)
        r = sv.result(rid)
        assert r["state"] == "done" and r["steps_done"] == K
        alone, alone_loss = sv.output(rid).clone(), r["loss"]
    with serve.Server(2048 * MB, max_active=3, chunk_steps=2) as sv:
        for seed in (3, 4):
            q0, qlr, qg, qs = _scan(seed)
            sv.submit_fit(q0, qlr, qg, qs, 7, arrival_s=0.0)
        mid = sv.submit_fit(p0, lr, grid, s, K, arrival_s=0.0)
        sv.run(timeout_s=300)
        assert sv.stats()["n_done"] == 3
        mixed = sv.output(mid).clone()
    assert _equal(alone, mixed)
    assert alone_loss == pytest.approx(loss, rel=1e-5)
    got = alone.cpu().numpy().astype(np.float64)
    clear = np.ones_like(got, dtype=bool)
    for g in grads:
        clear &= np.abs(g) > 1e-3 * np.sqrt((g ** 2).mean(0))[None, :]
    assert clear.mean() > 0.5
    np.testing.assert_allclose(got[clear], p[clear], rtol=1e-6, atol=K * 2e-6)
    lrs = oracle.AdamConfig().lr_vector()[None, :] * np.ones_like(got)
    assert np.all(np.abs(got - p) <= 2 * K * lrs + 1e-5)
