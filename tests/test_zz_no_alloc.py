"""The workspace-free L1 entry point (for callers that cannot allocate device memory) matches
the workspace entry point and the FP64 oracle.

Collected last on purpose: it uses the library's static scratch array, and if it fails, a
run that stops at the first failure has already run every other test. It must pass both in a
fresh process and after the other tests."""
import ctypes

import numpy as np
import pytest

from helpers import to_dev

pytestmark = pytest.mark.gpu

# A fixed-order FP32 sum of n values in [0, 1] (32 strided values per thread, a 256-way tree,
# then a tree over at most 4,096 partials) is within about 60 units in the last place of the
# exact mean; 1e-5 relative leaves a wide margin.
TOL_LOSS = 1e-5


def _call_static(lib, pred, tgt, loss, dpred):
    import torch
    rc = lib.gs_l1_loss_static(ctypes.c_void_p(pred.data_ptr()), ctypes.c_void_p(tgt.data_ptr()),
                               pred.numel(), ctypes.c_void_p(loss.data_ptr()),
                               None if dpred is None else ctypes.c_void_p(dpred.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0


def _check_against_oracle(loss, dpred, pred_np, tgt_np):
    import oracle
    ref_loss, ref_d = oracle.l1_loss(pred_np, tgt_np)
    assert float(loss) == pytest.approx(ref_loss, rel=TOL_LOSS)
    if dpred is not None:
        d = dpred.cpu().numpy().astype(np.float64)
        # the sign of an FP32 difference is exact; 1/n is rounded once to FP32
        assert np.array_equal(np.sign(d), np.sign(ref_d))
        assert np.allclose(d, ref_d, rtol=1e-7, atol=0)


def test_static_l1_matches_workspace_l1_twice():
    import torch
    from paper_2603_09621_gb300 import gs
    lib = gs.load()
    ws = gs.Workspace(1, 1, gs.Grid(4, 4, 4), gs.Config())
    rng = np.random.default_rng(11)
    for n in (2_097_152 + 333, 5000):  # two calls in a row, different sizes
        pred_np = rng.uniform(0, 1, n).astype(np.float32)
        tgt_np = rng.uniform(0, 1, n).astype(np.float32)
        tgt_np[:7] = pred_np[:7]  # sign(0) = 0
        pred, tgt = to_dev(pred_np), to_dev(tgt_np)
        ref_d = torch.empty(n, device="cuda")
        ref = gs.gs_l1_loss(pred, tgt, ws, dpred=ref_d)
        loss = torch.full((), -1.0, device="cuda")
        dpred = torch.full((n,), 7.0, device="cuda")
        _call_static(lib, pred, tgt, loss, dpred)
        torch.cuda.synchronize()
        assert float(loss) == pytest.approx(float(ref), rel=TOL_LOSS)
        assert torch.equal(dpred, ref_d)
        _check_against_oracle(loss, dpred, pred_np, tgt_np)


def test_static_l1_full_scratch_and_no_gradient():
    """The largest accepted size (every one of the 4,096 partial sums written and read),
    then a call without the gradient output."""
    import torch
    from paper_2603_09621_gb300 import gs
    lib = gs.load()
    n = gs.GS_L1_STATIC_MAX_N
    gen = torch.Generator(device="cuda").manual_seed(5)
    pred = torch.rand(n, device="cuda", generator=gen)
    tgt = torch.rand(n, device="cuda", generator=gen)
    ws = gs.Workspace(1, 1, gs.Grid(4, 4, 4), gs.Config())
    ref_d = torch.empty(n, device="cuda")
    ref = gs.gs_l1_loss(pred, tgt, ws, dpred=ref_d)
    loss = torch.full((), -1.0, device="cuda")
    dpred = torch.empty(n, device="cuda")
    _call_static(lib, pred, tgt, loss, dpred)
    torch.cuda.synchronize()
    assert float(loss) == pytest.approx(float(ref), rel=TOL_LOSS)
    assert torch.equal(dpred, ref_d)
    # the last block's partial decides the tail: compare with the FP64 mean
    exact = (pred.double() - tgt.double()).abs().mean().item()
    assert float(loss) == pytest.approx(exact, rel=TOL_LOSS)
    del dpred, ref_d
    # without the gradient output, on a small case checked against the oracle
    rng = np.random.default_rng(12)
    pred_np = rng.uniform(0, 1, 70_001).astype(np.float32)
    tgt_np = rng.uniform(0, 1, 70_001).astype(np.float32)
    loss2 = torch.full((), -1.0, device="cuda")
    _call_static(lib, to_dev(pred_np), to_dev(tgt_np), loss2, None)
    torch.cuda.synchronize()
    _check_against_oracle(loss2, None, pred_np, tgt_np)


def test_static_l1_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2603_09621_gb300 import gs
    lib = gs.load()
    x = torch.zeros(4, device="cuda")
    too_many = gs.GS_L1_STATIC_MAX_N + 1
    rc = lib.gs_l1_loss_static(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                               too_many, ctypes.c_void_p(x.data_ptr()), None, None)
    assert rc == -1
    # the binding checks sizes and layouts before calling
    with pytest.raises(ValueError):
        gs.gs_l1_loss_static(x, torch.zeros(5, device="cuda"))
    with pytest.raises(ValueError):
        gs.gs_l1_loss_static(x, x.double())
