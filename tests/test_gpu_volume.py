"""Slice-profile model, L1 loss, Adam, Eq. 2 and lattice initialisation on the GPU against
the oracle."""
import numpy as np
import pytest

from helpers import TR, TE, rel_l2, to_dev
from paper_2603_09621_gb300 import inputs

pytestmark = pytest.mark.gpu


def _gs():
    from paper_2603_09621_gb300 import gs
    return gs


@pytest.mark.parametrize("shape,s", [((128, 64, 48), 4), ((13, 7, 9), 3), ((8, 5, 3), 2),
                                     ((5, 4, 4), 7)])
def test_downsample_fwd_bwd(shape, s):
    import oracle
    import torch
    gs = _gs()
    rng = np.random.default_rng(0)
    hr = rng.uniform(0, 1, shape).astype(np.float32)
    nz = shape[0]
    if nz // s == 0:
        return
    lr = gs.gs_downsample_fwd(to_dev(hr), s)
    dlr = rng.standard_normal((nz // s,) + shape[1:]).astype(np.float32)
    dhr = gs.gs_downsample_bwd(to_dev(dlr), nz, s)
    torch.cuda.synchronize()
    np.testing.assert_allclose(lr.cpu().numpy(), oracle.downsample(hr, s), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(dhr.cpu().numpy(), oracle.downsample_adjoint(dlr, nz, s),
                               rtol=1e-6, atol=0)


def test_l1_loss_and_gradient():
    import oracle
    import torch
    gs = _gs()
    rng = np.random.default_rng(1)
    n = 2_097_152 + 77
    pred = rng.uniform(0, 1, n).astype(np.float32)
    tgt = (pred + rng.choice([-1, 1], n) * rng.uniform(1e-3, 0.2, n)).astype(np.float32)
    tgt[:10] = pred[:10]  # exact ties: sign(0) = 0
    ws = gs.Workspace(1, 1, gs.Grid(4, 4, 4), gs.Config())
    dpred = torch.empty(n, device="cuda")
    loss = gs.gs_l1_loss(to_dev(pred), to_dev(tgt), ws, dpred=dpred)
    loss2 = gs.gs_l1_loss(to_dev(pred), to_dev(tgt), ws)
    torch.cuda.synchronize()
    ref_loss, ref_g = oracle.l1_loss(pred, tgt)
    assert float(loss) == pytest.approx(ref_loss, rel=1e-5)
    assert float(loss) == float(loss2)  # deterministic reduction
    np.testing.assert_allclose(dpred.cpu().numpy(), ref_g, rtol=1e-6, atol=0)


def test_adam_matches_oracle():
    import oracle
    import torch
    gs = _gs()
    rng = np.random.default_rng(2)
    n = 10007
    p = rng.standard_normal((n, 12)).astype(np.float32)
    m = np.zeros_like(p, dtype=np.float64)
    v = np.zeros_like(p, dtype=np.float64)
    pd, md, vd = to_dev(p), torch.zeros((n, 12), device="cuda"), torch.zeros((n, 12), device="cuda")
    step = torch.zeros((), dtype=torch.int32, device="cuda")
    ref = p.astype(np.float64)
    hp = gs.Adam()
    for t in range(1, 6):
        g = (rng.standard_normal((n, 12)) * 10 ** rng.uniform(-3, 1, (n, 12))).astype(np.float32)
        gs.gs_adam_step(pd, to_dev(g), md, vd, hp, step)
        ref, m, v = oracle.adam_step(ref, g, m, v, t)
    torch.cuda.synchronize()
    assert int(step) == 5
    np.testing.assert_allclose(pd.cpu().numpy(), ref, rtol=1e-5, atol=1e-6)
    assert rel_l2(md.cpu().numpy(), m) < 1e-6 and rel_l2(vd.cpu().numpy(), v) < 1e-6


def test_signal_proxy_matches_oracle():
    import oracle
    import torch
    gs = _gs()
    rng = np.random.default_rng(3)
    t1 = rng.uniform(*inputs.T1_RANGE, 100000).astype(np.float32)
    t2 = rng.uniform(*inputs.T2_RANGE, 100000).astype(np.float32)
    T = gs.gs_signal_proxy(to_dev(t1), to_dev(t2), TR, TE)
    torch.cuda.synchronize()
    np.testing.assert_allclose(T.cpu().numpy(), oracle.signal_proxy(t1, t2, TR, TE), rtol=2e-6)


def test_init_lattice_matches_oracle():
    import oracle
    import torch
    gs = _gs()
    og = oracle.Grid(64, 48, 40)
    s = 4
    rng = np.random.default_rng(4)
    lr = rng.uniform(0, 1, (10, 48, 64)).astype(np.float32)
    n, _ = oracle.lattice_dims(og, 20000)
    ref = oracle.init_lattice(lr, og, s, 20000, t_act=1)
    got = gs.gs_init_lattice(to_dev(lr), gs.Grid(64, 48, 40), s, n, t_act=1, t_init=0.5)
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    assert got.shape == ref.shape
    np.testing.assert_allclose(got[:, :10], ref[:, :10], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(got[:, 10], ref[:, 10], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(got[:, 11], ref[:, 11], atol=1e-7)
