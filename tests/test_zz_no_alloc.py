"""The workspace-free L1 entry point (for callers that cannot allocate device memory) matches
the workspace entry point.

Collected last on purpose: it uses the library's static scratch array, and if it fails, a
run that stops at the first failure has already run every other test. It must pass both in a
fresh process and after the other tests."""
import ctypes

import numpy as np
import pytest

from helpers import to_dev

pytestmark = pytest.mark.gpu


def _call_static(lib, pred, tgt, loss, dpred):
    import torch
    rc = lib.gs_l1_loss_static(ctypes.c_void_p(pred.data_ptr()), ctypes.c_void_p(tgt.data_ptr()),
                               pred.numel(), ctypes.c_void_p(loss.data_ptr()),
                               ctypes.c_void_p(dpred.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0


def test_static_l1_matches_workspace_l1_twice():
    import torch
    from paper_2603_09621_gb300 import gs
    lib = gs.load()
    ws = gs.Workspace(1, 1, gs.Grid(4, 4, 4), gs.Config())
    rng = np.random.default_rng(11)
    for n in (2_097_152 + 333, 5000):  # two calls in a row, different sizes
        pred = to_dev(rng.uniform(0, 1, n).astype(np.float32))
        tgt = to_dev(rng.uniform(0, 1, n).astype(np.float32))
        ref_d = torch.empty(n, device="cuda")
        ref = gs.gs_l1_loss(pred, tgt, ws, dpred=ref_d)
        loss = torch.full((), -1.0, device="cuda")
        dpred = torch.full((n,), 7.0, device="cuda")
        _call_static(lib, pred, tgt, loss, dpred)
        torch.cuda.synchronize()
        assert float(loss) == pytest.approx(float(ref), rel=1e-5)
        assert torch.equal(dpred, ref_d)


def test_static_l1_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2603_09621_gb300 import gs
    lib = gs.load()
    x = torch.zeros(4, device="cuda")
    too_many = gs.GS_L1_STATIC_MAX_N + 1
    rc = lib.gs_l1_loss_static(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                               too_many, ctypes.c_void_p(x.data_ptr()), None, None)
    assert rc == -1
