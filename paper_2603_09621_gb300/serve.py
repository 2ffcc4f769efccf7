"""Thin Python binding of the serving runtime (C ABI in include/gs_serve.h).

A ``Server`` owns one device arena and runs many scans' fitting loops and re-renders at once
(continuous batching, admission by the arena budget). Argument marshalling only: the
scheduler, the allocator and every kernel run in libgsmri.
"""
from __future__ import annotations

import ctypes

import torch

from . import gs
from .gs import Adam, Config, Grid, _check

STATE_NAMES = {gs.GS_REQ_PENDING: "pending", gs.GS_REQ_ACTIVE: "active",
               gs.GS_REQ_DONE: "done", gs.GS_REQ_FAILED: "failed"}


class _DeviceView:
    """Zero-copy view of arena memory for torch (CUDA array interface)."""

    def __init__(self, ptr: int, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f4",
                                         "data": (ptr, False), "version": 2}


def server_config(budget_bytes: int, max_active: int = 4, chunk_steps: int = 25,
                  use_graphs: bool = True, max_bypass: int = 4, pairs_per_gauss: float = 8.0,
                  cfg: Config = Config(t_act=1), adam: Adam = Adam()) -> gs.gs_server_config:
    c = gs.gs_server_config()
    c.hbm_budget = int(budget_bytes)
    c.max_active, c.chunk_steps = max_active, chunk_steps
    c.use_graphs, c.max_bypass = int(use_graphs), max_bypass
    c.pairs_per_gauss = pairs_per_gauss
    c.cfg, c.adam = cfg.c(), adam.c()
    return c


def fit_request(params0: torch.Tensor, lr_target: torch.Tensor, grid: Grid, s: int, iters: int,
                arrival_s: float = 0.0, lr_model: int = gs.GS_LR_ZBOX) -> gs.gs_request:
    """lr_model GS_LR_ZBOX: lr_target is [nz // s, ny, nx]; GS_LR_TRILINEAR: any LR shape (s
    unused)."""
    r = gs.gs_request()
    r.kind, r.grid, r.s, r.iters = gs.GS_REQ_FIT, grid.c(), s, iters
    r.n_gauss = params0.shape[0]
    r.params, r.lr_target = params0.data_ptr(), lr_target.data_ptr()
    r.source, r.arrival_s = -1, arrival_s
    r.lr_model = lr_model
    if lr_model == gs.GS_LR_TRILINEAR:
        r.lr_nz, r.lr_ny, r.lr_nx = lr_target.shape
    return r


def render_request(grid: Grid, n_gauss: int, source: int = -1,
                   params: torch.Tensor | None = None, arrival_s: float = 0.0) -> gs.gs_request:
    r = gs.gs_request()
    r.kind, r.grid, r.s, r.iters = gs.GS_REQ_RENDER, grid.c(), 1, 1
    r.n_gauss = n_gauss
    r.params = params.data_ptr() if params is not None else None
    r.lr_target, r.source, r.arrival_s = None, source, arrival_s
    return r


class Server:
    def __init__(self, budget_bytes: int, **kw):
        self.lib = gs.load()
        self.cfg = server_config(budget_bytes, **kw)
        self._h = ctypes.c_void_p()
        _check(self.lib.gs_server_create(ctypes.byref(self.cfg), ctypes.byref(self._h)),
               "gs_server_create")
        self._keep = {}    # caller tensors, alive until the request is admitted
        self._shape = {}   # output shapes

    def close(self):
        if self._h:
            self.lib.gs_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def request_bytes(self, req: gs.gs_request) -> int:
        return int(self.lib.gs_server_request_bytes(ctypes.byref(self.cfg), ctypes.byref(req)))

    def _submit(self, req, keep, shape) -> int:
        # the inputs are read on the server's streams: finish the work that produced them
        torch.cuda.current_stream().synchronize()
        rid = ctypes.c_int64()
        _check(self.lib.gs_server_submit(self._h, ctypes.byref(req), ctypes.byref(rid)),
               "gs_server_submit")
        self._keep[rid.value] = keep
        self._shape[rid.value] = shape
        return rid.value

    def submit_fit(self, params0, lr_target, grid: Grid, s: int, iters: int,
                   arrival_s: float = 0.0, lr_model: int = gs.GS_LR_ZBOX) -> int:
        params0, lr_target = params0.contiguous(), lr_target.contiguous()
        req = fit_request(params0, lr_target, grid, s, iters, arrival_s, lr_model)
        return self._submit(req, (params0, lr_target), (params0.shape[0], 12))

    def submit_render(self, grid: Grid, source: int | None = None, params=None,
                      n_gauss: int | None = None, arrival_s: float = 0.0) -> int:
        if source is not None:
            n = n_gauss if n_gauss is not None else self._shape[source][0]
            req = render_request(grid, n, source=source, arrival_s=arrival_s)
            keep = None
        else:
            params = params.contiguous()
            req = render_request(grid, params.shape[0], params=params, arrival_s=arrival_s)
            keep = params
        return self._submit(req, keep, grid.shape)

    def poll(self) -> int:
        n = ctypes.c_int32()
        _check(self.lib.gs_server_poll(self._h, ctypes.byref(n)), "gs_server_poll")
        return n.value

    def run(self, timeout_s: float = 600.0, poll_us: int = 50):
        _check(self.lib.gs_server_run(self._h, timeout_s, poll_us), "gs_server_run")

    def result(self, rid: int) -> dict:
        r = gs.gs_result()
        _check(self.lib.gs_server_result(self._h, rid, ctypes.byref(r)), "gs_server_result")
        return dict(state=STATE_NAMES[r.state], error=gs.STATUS.get(r.error, r.error),
                    status_bits=r.status_bits, steps_done=r.steps_done, capacity=r.capacity,
                    grows=r.grows, chunks=r.chunks, loss=r.loss, arrival_s=r.arrival_s,
                    admit_s=r.admit_s, done_s=r.done_s, output=r.output, bytes=r.bytes)

    def output(self, rid: int) -> torch.Tensor:
        """A copy of a finished request's output (fitted cloud [N, 12] or volume [nz, ny, nx])."""
        r = self.result(rid)
        if r["state"] != "done" or not r["output"]:
            raise gs.GsError(f"request {rid} has no output ({r['state']}, {r['error']})")
        view = torch.as_tensor(_DeviceView(r["output"], self._shape[rid]), device="cuda")
        return view.clone()

    def release(self, rid: int):
        _check(self.lib.gs_server_release(self._h, rid), "gs_server_release")
        self._keep.pop(rid, None)

    def stats(self) -> dict:
        s = gs.gs_server_stats()
        _check(self.lib.gs_server_stats_read(self._h, ctypes.byref(s)), "gs_server_stats_read")
        return {k: getattr(s, k) for k, _ in gs.gs_server_stats._fields_}
