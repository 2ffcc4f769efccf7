"""Z-slab sharding of one volume's fit (shard.SlabFit) on the host: two gloo ranks, each
computing its slab with the FP64 oracle as the compute backend, reproduce the oracle's
single-process fitting step of the whole volume (gradient after the all-reduce, loss, updated
parameters); an overflow on one rank makes the step a no-op on both. Pins the slab bounds
(whole LR slices, trailing HR slices on the last slab), the sub-grid origins, the LR slab
slicing and the whole-volume L1 normaliser."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NZ, NY, NX, S = 14, 12, 16, 3       # 4 LR slices; HR slices 12 and 13 have none


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    import oracle
    from paper_2603_09621_gb300 import inputs
    d = inputs.gaussian_cloud(4, 160, (NZ, NY, NX), scale_range=(0.6, 2.2))
    p = inputs.assemble_params(d["mu"], d["log_s"], d["q"], d["pd"],
                               np.random.default_rng(5).normal(0.0, 1.0, 160)).astype(np.float64)
    rng = np.random.default_rng(6)
    lr = rng.uniform(0.0, 0.8, (NZ // S, NY, NX))
    return p, lr, oracle.Grid(NX, NY, NZ), oracle.Config(t_act=1)


class OracleSlab:
    """FP64 oracle stand-in for gs.FitState (the interface shard.SlabFit drives)."""

    def __init__(self, params, lr, grid, s, force_overflow=0):
        import torch
        import oracle
        self.o = oracle
        self.params = params.clone()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.d_loss = torch.zeros(1, dtype=torch.float64)
        self.step_no = 0
        self.lr, self.s, self.force = lr.numpy(), s, force_overflow
        self.grid = self.o.Grid(grid.nx, grid.ny, grid.nz, tuple(grid.h), tuple(grid.origin))
        self.cfg = self.o.Config(t_act=1)

    def grad_step(self, n_lr_total):
        import torch
        o = self.o
        p = self.params.numpy()
        I = o.render(p, self.grid, self.cfg)["I"]
        pred = o.downsample(I, self.s)
        diff = pred - self.lr
        self.d_loss[0] = np.abs(diff).sum() / n_lr_total
        dI = o.downsample_adjoint(np.sign(diff) / n_lr_total, self.grid.nz, self.s)
        self.grad.copy_(torch.as_tensor(o.render_grad(p, self.grid, dI, self.cfg)))

    def overflow_flag(self):
        import torch
        return torch.tensor([self.force], dtype=torch.int32)

    def apply(self, flag):
        import torch
        if int(flag.item()) != 0:
            return
        self.step_no += 1
        p, m, v = self.o.adam_step(self.params.numpy(), self.grad.numpy(), self.m.numpy(),
                                   self.v.numpy(), self.step_no)
        self.params.copy_(torch.as_tensor(p))
        self.m.copy_(torch.as_tensor(m))
        self.v.copy_(torch.as_tensor(v))


def _worker(rank, world, port, force_rank, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import torch.distributed as dist
    from paper_2603_09621_gb300 import gs, shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p, lr, og, _ = _problem()
    grid = gs.Grid(og.nx, og.ny, og.nz)

    def make(params, lr_slab, g, s):
        return OracleSlab(params, lr_slab, g, s, force_overflow=int(rank == force_rank))

    fit = shard.SlabFit(torch.as_tensor(p), torch.as_tensor(lr), grid, S, rank, world,
                        make_state=make)
    flag = fit.step()
    loss = fit.state.d_loss.clone()
    dist.all_reduce(loss)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, (fit.z0, fit.z1), tuple(fit.grid.origin), fit.lr.shape[0], int(flag.item()),
           float(loss.item()), fit.state.grad.numpy().copy(), fit.state.params.numpy().copy()))


def _run(force_rank=-1, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, force_rank, q))
             for r in range(world)]
    for pr in procs:
        pr.start()
    res = {}
    for _ in range(world):
        item = q.get(timeout=300)
        res[item[0]] = item[1:]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    return res


def test_slab_bounds_and_grids():
    from paper_2603_09621_gb300 import gs, shard
    assert shard.slab_bounds(128, 4, 2) == [(0, 64), (64, 128)]
    assert shard.slab_bounds(130, 3, 3) == [(0, 45), (45, 87), (87, 130)]
    assert shard.slab_bounds(14, 3, 2) == [(0, 6), (6, 14)]
    with pytest.raises(ValueError):
        shard.slab_bounds(8, 4, 3)
    g = shard.slab_grid(gs.Grid(10, 9, 20, (1.0, 1.0, 1.5), (0.5, 0.0, -2.0)), 8, 20)
    assert g.nz == 12 and g.origin == (0.5, 0.0, -2.0 + 8 * 1.5)


def test_sharded_step_matches_single_process_oracle_gloo_world2(oracle_mod):
    import oracle
    p, lr, og, cfg = _problem()
    n = p.shape[0]
    ref = oracle.fit_step(p, lr, og, S, cfg, np.zeros((n, 12)), np.zeros((n, 12)), 1)
    res = _run()
    assert res[0][0] == (0, 6) and res[1][0] == (6, 14)
    assert res[1][1] == (0.0, 0.0, 6.0) and res[0][2] == 2 and res[1][2] == 2
    for r in (0, 1):
        _, _, _, flag, loss, grad, params = res[r]
        assert flag == 0
        assert loss == pytest.approx(ref["loss"], rel=1e-12)
        np.testing.assert_allclose(grad, ref["grad"], rtol=1e-9,
                                   atol=1e-12 * np.abs(ref["grad"]).max())
        np.testing.assert_allclose(params, ref["params"], rtol=1e-12, atol=1e-12)
    # Gaussians straddling the cut get contributions from both slabs
    assert np.array_equal(res[0][5], res[1][5])


def test_overflow_on_one_rank_is_a_no_op_everywhere(oracle_mod):
    p, _, _, _ = _problem()
    res = _run(force_rank=1)
    for r in (0, 1):
        _, _, _, flag, _, _, params = res[r]
        assert flag == 1
        np.testing.assert_array_equal(params, p)
