"""Z-slab sharding of one volume's zero-shot fit over several processes, one GPU each.

The fitting loss (L1 over the LR scan, a mean over LR voxels) and its gradient (Eq. 5-6: a sum
over voxels of per-voxel terms) split over any partition of the voxels. Cutting the HR volume
along z into slabs of whole LR slices (multiples of the slice factor s, so that every LR slice
of the z box profile lies in one slab) gives each process a complete sub-problem on its own
sub-grid: it bins only the Gaussians whose box meets its slab, renders the slab, and forms the
slab's share of the loss and of every Gaussian's gradient (the L1 mean normalised by the whole
volume's LR count). The forward needs no exchange. The one exchange step is a sum-reduction
of the raw-parameter gradient [N, 12] (indexed by Gaussian id: Gaussians that straddle slabs
get contributions from several processes, the others from one), after which every process
holds the same gradient and applies the same Adam update to its replica of the parameters and
moments. An overflow of any process's pair capacity makes the step a no-op on all of them (a
max-reduction of one flag), as a single-process step is.

The compute backend is any object with the FitState interface used here (``grad_step``,
``overflow_flag``, ``apply``, ``grad``, ``d_loss``); the reduction is a function of
(grad, flag), by default torch.distributed all-reduces (NCCL on GPUs). Argument marshalling
only: every step of the fit runs in libgsmri.
"""
from __future__ import annotations

import torch

from . import gs


def slab_bounds(nz: int, s: int, world: int):
    """HR z-ranges [z0, z1) of `world` slabs: the floor(nz / s) LR slices split as evenly as
    possible (the first slabs take one more when they do not divide), each slab s times its LR
    slices; the last slab also takes the trailing nz - s floor(nz / s) HR slices, which no LR
    slice covers (zero gradient there, as in the single-process step)."""
    nl = nz // s
    if s < 1 or world < 1 or nl < world:
        raise ValueError(f"cannot cut {nz} slices (factor {s}) into {world} slabs")
    base, extra = divmod(nl, world)
    out, l0 = [], 0
    for r in range(world):
        l1 = l0 + base + (1 if r < extra else 0)
        out.append((l0 * s, nz if r == world - 1 else l1 * s))
        l0 = l1
    return out


def slab_grid(grid: gs.Grid, z0: int, z1: int) -> gs.Grid:
    """The sub-grid of slices [z0, z1): same x-y layout and spacing, origin moved by z0 slices,
    so that its voxel centres are the whole grid's."""
    o = tuple(grid.origin)
    return gs.Grid(grid.nx, grid.ny, z1 - z0, tuple(grid.h),
                   (o[0], o[1], o[2] + z0 * grid.h[2]))


def dist_reduce(grad: torch.Tensor, flag: torch.Tensor, group=None):
    """Sum of the gradients and maximum of the overflow flags over the process group."""
    import torch.distributed as dist
    dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(flag, op=dist.ReduceOp.MAX, group=group)


class SlabFit:
    """One process's part of a z-slab-sharded fit of one volume.

    params0: the whole initial cloud [N, 12] (every process holds a replica); lr_target: the
    whole LR scan [nz // s, ny, nx]; grid: the whole HR grid. The slab's state is built by
    ``make_state(params0, lr_slab, sub_grid, s)`` (default: a gs.FitState with ``cfg``)."""

    def __init__(self, params0, lr_target, grid: gs.Grid, s: int, rank: int, world: int,
                 cfg: gs.Config = gs.Config(t_act=1), make_state=None, reduce=None):
        self.rank, self.world = rank, world
        self.z0, self.z1 = slab_bounds(grid.nz, s, world)[rank]
        self.grid = slab_grid(grid, self.z0, self.z1)
        l0, nl = self.z0 // s, (self.z1 - self.z0) // s
        self.lr = lr_target[l0:l0 + nl].contiguous()
        self.n_lr_total = (grid.nz // s) * grid.ny * grid.nx
        if make_state is None:
            def make_state(p, lr, g, s_):
                return gs.FitState(p, lr, g, s_, cfg)
        self.state = make_state(params0, self.lr, self.grid, s)
        self.reduce = reduce or dist_reduce

    def step(self):
        """One fitting step of the whole volume: this slab's gradient, the reductions, Adam.
        Returns the overflow flag (device): nonzero means the step changed nothing anywhere
        and every process should grow its bins and repeat it."""
        st = self.state
        st.grad_step(self.n_lr_total)
        flag = st.overflow_flag()
        self.reduce(st.grad, flag)
        st.apply(flag)
        return flag
