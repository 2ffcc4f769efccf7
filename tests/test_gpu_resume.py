"""Checkpoint and resume of a fit: the fitting step reads no state besides the caller-owned
parameters, Adam moments and step counter (bins and workspace are rebuilt every step), so a
fit copied out to host memory and restored into a fresh FitState continues bit for bit."""
import numpy as np
import pytest

from helpers import phantom_fit, to_dev

pytestmark = pytest.mark.gpu


def test_fit_resumes_bit_for_bit_from_host_copies():
    import torch
    from paper_2603_09621_gb300 import gs
    w = phantom_fit(shape=(32, 48, 48), s=4, n_gauss=6000, seed=3, n_ell=5, semi=(5.0, 16.0))
    og = w["grid"]
    g = gs.Grid(og.nx, og.ny, og.nz)
    cfg = gs.Config(t_act=1)
    a = gs.FitState(to_dev(w["params0"]), to_dev(w["lr"]), g, w["s"], cfg)
    for _ in range(12):
        a.step()
    torch.cuda.synchronize()
    saved = {k: getattr(a, k).detach().cpu().clone() for k in ("params", "m", "v", "d_step")}
    for _ in range(8):
        a.step()
    torch.cuda.synchronize()
    # a fresh state restored from the host copies
    b = gs.FitState(saved["params"].cuda(), to_dev(w["lr"]), g, w["s"], cfg,
                    capacity=a.capacity)
    for k in ("m", "v", "d_step"):
        getattr(b, k).copy_(saved[k].cuda())
    for _ in range(8):
        b.step()
    torch.cuda.synchronize()
    assert a.check() == (0, 0) and b.check() == (0, 0)
    assert int(b.d_step) == int(a.d_step) == 20
    for k in ("params", "m", "v"):
        assert np.array_equal(getattr(a, k).cpu().numpy(), getattr(b, k).cpu().numpy()), k
    assert float(a.d_loss) == float(b.d_loss)
