"""Thin Python binding of libgsmri (C ABI in include/gs_api.h and include/gs_serve.h).

Argument marshalling only: every step of the rendering path runs in the CUDA library; torch
provides device memory and streams. Importing this module loads the library and raises if it
is missing (there is no fallback path). Function names follow the C ABI.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import torch

from . import build as _build

_lib = None


class GsError(RuntimeError):
    pass


# ---------------------------------------------------------------------- C structs
class gs_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("h", ctypes.c_float * 3), ("origin", ctypes.c_float * 3)]


class gs_config(ctypes.Structure):
    _fields_ = [("brick", ctypes.c_int32 * 3), ("trunc_sigma", ctypes.c_float),
                ("eps", ctypes.c_float), ("deterministic", ctypes.c_int32),
                ("signal_mode", ctypes.c_int32), ("a_act", ctypes.c_int32),
                ("t_act", ctypes.c_int32)]


class gs_bins(ctypes.Structure):
    _fields_ = [("n_gauss", ctypes.c_int64), ("capacity", ctypes.c_int64),
                ("n_bricks", ctypes.c_int32), ("nbx", ctypes.c_int32), ("nby", ctypes.c_int32),
                ("nbz", ctypes.c_int32), ("brick_off", ctypes.c_void_p),
                ("pair_gid", ctypes.c_void_p), ("pair_gmj", ctypes.c_void_p),
                ("pair_brick", ctypes.c_void_p), ("gm_off", ctypes.c_void_p),
                ("rec", ctypes.c_void_p),
                ("brange", ctypes.c_void_p), ("d_npairs", ctypes.c_void_p),
                ("d_status", ctypes.c_void_p)]


class gs_adam(ctypes.Structure):
    _fields_ = [("lr_mu", ctypes.c_float), ("lr_scale", ctypes.c_float),
                ("lr_rot", ctypes.c_float), ("lr_a", ctypes.c_float), ("lr_t", ctypes.c_float),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double)]


class gs_fit_state(ctypes.Structure):
    _fields_ = [("grid", gs_grid), ("cfg", gs_config), ("adam", gs_adam),
                ("n_gauss", ctypes.c_int64), ("s", ctypes.c_int32),
                ("params", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("m", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("d_step", ctypes.c_void_p), ("bins", gs_bins),
                ("I", ctypes.c_void_p), ("W", ctypes.c_void_p), ("lr_pred", ctypes.c_void_p), ("lr_target", ctypes.c_void_p),
                ("d_loss", ctypes.c_void_p), ("ws", ctypes.c_void_p),
                ("ws_bytes", ctypes.c_size_t), ("phase_events", ctypes.c_void_p),
                ("n_phase_events", ctypes.c_int32), ("lr_model", ctypes.c_int32),
                ("lr_nx", ctypes.c_int32), ("lr_ny", ctypes.c_int32), ("lr_nz", ctypes.c_int32)]


GS_LR_ZBOX, GS_LR_TRILINEAR = 0, 1


GS_FIT_PHASES = 7


# serving runtime (include/gs_serve.h)
class gs_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_active", ctypes.c_int32),
                ("chunk_steps", ctypes.c_int32), ("use_graphs", ctypes.c_int32),
                ("max_bypass", ctypes.c_int32), ("pairs_per_gauss", ctypes.c_float),
                ("cfg", gs_config), ("adam", gs_adam)]


class gs_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("grid", gs_grid), ("s", ctypes.c_int32),
                ("iters", ctypes.c_int32), ("n_gauss", ctypes.c_int64),
                ("params", ctypes.c_void_p), ("lr_target", ctypes.c_void_p),
                ("source", ctypes.c_int64), ("arrival_s", ctypes.c_double),
                ("lr_model", ctypes.c_int32), ("lr_nx", ctypes.c_int32),
                ("lr_ny", ctypes.c_int32), ("lr_nz", ctypes.c_int32)]


class gs_result(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("error", ctypes.c_int), ("status_bits", ctypes.c_int32),
                ("steps_done", ctypes.c_int32), ("capacity", ctypes.c_int64),
                ("grows", ctypes.c_int32), ("chunks", ctypes.c_int32), ("loss", ctypes.c_float),
                ("arrival_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("output", ctypes.c_void_p),
                ("bytes", ctypes.c_size_t)]


class gs_server_stats(ctypes.Structure):
    _fields_ = [("now_s", ctypes.c_double), ("n_pending", ctypes.c_int32),
                ("n_active", ctypes.c_int32), ("n_done", ctypes.c_int32),
                ("n_failed", ctypes.c_int32), ("arena_bytes", ctypes.c_size_t),
                ("used_bytes", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t),
                ("chunks_launched", ctypes.c_int64), ("graphs_captured", ctypes.c_int64),
                ("grows", ctypes.c_int64)]


GS_REQ_FIT, GS_REQ_RENDER = 0, 1
GS_REQ_PENDING, GS_REQ_ACTIVE, GS_REQ_DONE, GS_REQ_FAILED = 0, 1, 2, 3


STATUS = {0: "GS_OK", -1: "GS_ERR_INVALID_ARG", -2: "GS_ERR_CAPACITY", -3: "GS_ERR_WORKSPACE",
          -4: "GS_ERR_CUDA", -5: "GS_ERR_TIMEOUT", -6: "GS_ERR_NONFINITE"}
GS_STATUS_CAPACITY = 1
GS_STATUS_NONFINITE = 2

# Exported entry points and their ctypes signatures (checked against include/gs_api.h by
# the CPU test suite).
_P, _I32, _I64, _F, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t
SIGNATURES = {
    "gs_bins_bytes": (_SZ, [_I64, _I64, _P, _P]),
    "gs_bins_bind": (ctypes.c_int, [_P, _SZ, _I64, _I64, _P, _P, _P]),
    "gs_workspace_bytes": (_SZ, [_I64, _I64, _P, _P]),
    "gs_signal_proxy": (ctypes.c_int, [_P, _P, _I64, _F, _F, _P, _P]),
    "gs_bin_bricks": (ctypes.c_int, [_P, _P, _P, _P, _P, _SZ, _P]),
    "gs_render_fwd": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "gs_render_bwd": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "gs_downsample_fwd": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32, _P, _P]),
    "gs_downsample_bwd": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32, _P, _P]),
    "gs_l1_loss": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P, _SZ, _P]),
    "gs_l1_loss_static": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P]),
    "gs_adam_step": (ctypes.c_int, [_P, _P, _P, _P, _I64, _P, _P, _P]),
    "gs_init_lattice": (ctypes.c_int, [_P, _P, _I32, _I32, _I32, _I32, _I32, _F, _P, _P]),
    "gs_init_lattice_lr": (ctypes.c_int, [_P, _I32, _I32, _I32, _P, _I32, _I32, _I32, _I32, _F,
                                          _P, _P]),
    "gs_resample_fwd": (ctypes.c_int, [_P, _I32, _I32, _I32, _P, _I32, _I32, _I32, _P]),
    "gs_resample_bwd": (ctypes.c_int, [_P, _I32, _I32, _I32, _P, _I32, _I32, _I32, _P]),
    "gs_fit_step": (ctypes.c_int, [_P, _P]),
    "gs_fit_grad": (ctypes.c_int, [_P, _I64, _P]),
    "gs_fit_step_host": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "gs_fit_apply": (ctypes.c_int, [_P, _P, _P]),
    "gs_status_read": (ctypes.c_int, [_P, _P, _P]),
    "gs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gs_launch_count": (ctypes.c_ulonglong, []),
    "gs_version": (ctypes.c_char_p, []),
    # serving runtime
    "gs_arena_create": (ctypes.c_int, [_P, _SZ, _P]),
    "gs_arena_alloc": (ctypes.c_int, [_P, _SZ, _P]),
    "gs_arena_alloc_top": (ctypes.c_int, [_P, _SZ, _P]),
    "gs_arena_free": (ctypes.c_int, [_P, _P]),
    "gs_arena_stats": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "gs_arena_destroy": (None, [_P]),
    "gs_server_request_bytes": (_SZ, [_P, _P]),
    "gs_server_create": (ctypes.c_int, [_P, _P]),
    "gs_server_submit": (ctypes.c_int, [_P, _P, _P]),
    "gs_server_poll": (ctypes.c_int, [_P, _P]),
    "gs_server_run": (ctypes.c_int, [_P, ctypes.c_double, _I32]),
    "gs_server_result": (ctypes.c_int, [_P, _I64, _P]),
    "gs_server_release": (ctypes.c_int, [_P, _I64]),
    "gs_server_stats_read": (ctypes.c_int, [_P, _P]),
    "gs_server_destroy": (None, [_P]),
}


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libgsmri.so (built in-tree). Raises GsError if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise GsError(f"libgsmri.so not found at {path}: build it with "
                      "`python -m paper_2603_09621_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, what: str):
    if rc != 0:
        raise GsError(f"{what}: {STATUS.get(rc, rc)}")


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------- value types
@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    h: tuple = (1.0, 1.0, 1.0)
    origin: tuple = (0.0, 0.0, 0.0)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def c(self) -> gs_grid:
        g = gs_grid()
        g.nx, g.ny, g.nz = self.nx, self.ny, self.nz
        for k in range(3):
            g.h[k] = self.h[k]
            g.origin[k] = self.origin[k]
        return g


@dataclass
class Config:
    brick: tuple = (8, 8, 8)
    trunc_sigma: float = 3.0
    eps: float = 1e-12
    deterministic: int = 1
    signal_mode: int = 0
    a_act: int = 0
    t_act: int = 0

    def c(self) -> gs_config:
        c = gs_config()
        for k in range(3):
            c.brick[k] = self.brick[k]
        c.trunc_sigma = self.trunc_sigma
        c.eps = self.eps
        c.deterministic = self.deterministic
        c.signal_mode = self.signal_mode
        c.a_act = self.a_act
        c.t_act = self.t_act
        return c


@dataclass
class Adam:
    lr_mu: float = 1e-3
    lr_scale: float = 5e-3
    lr_rot: float = 5e-3
    lr_a: float = 5e-3
    lr_t: float = 5e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8

    def c(self) -> gs_adam:
        a = gs_adam()
        for k in ("lr_mu", "lr_scale", "lr_rot", "lr_a", "lr_t", "beta1", "beta2", "eps"):
            setattr(a, k, getattr(self, k))
        return a


def _empty_bytes(nbytes: int, device) -> torch.Tensor:
    # torch's caching allocator returns 512-byte aligned blocks; the ABI needs 256.
    t = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
    assert t.data_ptr() % 256 == 0
    return t


class Bins:
    """Device arena + bound gs_bins for a cloud of n_gauss Gaussians on one grid."""

    def __init__(self, n_gauss: int, capacity: int, grid: Grid, cfg: Config, device="cuda"):
        lib = load()
        self.grid, self.cfg = grid, cfg
        self._g, self._c = grid.c(), cfg.c()
        nbytes = lib.gs_bins_bytes(n_gauss, capacity, ctypes.byref(self._g), ctypes.byref(self._c))
        if nbytes == 0:
            raise GsError("gs_bins_bytes: invalid arguments")
        self.arena = _empty_bytes(nbytes, device)
        self.c = gs_bins()
        _check(lib.gs_bins_bind(_ptr(self.arena), nbytes, n_gauss, capacity,
                                ctypes.byref(self._g), ctypes.byref(self._c),
                                ctypes.byref(self.c)), "gs_bins_bind")
        self.n_gauss, self.capacity = n_gauss, capacity

    def _view(self, addr, count, dtype):
        base = self.arena.data_ptr()
        off = addr - base
        esz = torch.empty((), dtype=dtype).element_size()
        return self.arena[off:off + count * esz].view(dtype)

    def brick_off(self):
        return self._view(self.c.brick_off, self.c.n_bricks + 1, torch.int32)

    def pair_gid(self, n=None):
        return self._view(self.c.pair_gid, self.capacity if n is None else n, torch.int32)

    def pair_gmj(self, n=None):
        return self._view(self.c.pair_gmj, self.capacity if n is None else n, torch.int32)

    def pair_brick(self, n=None):
        return self._view(self.c.pair_brick, self.capacity if n is None else n, torch.int32)

    def gm_off(self):
        return self._view(self.c.gm_off, self.n_gauss + 1, torch.int32)

    def rec(self):
        return self._view(self.c.rec, self.n_gauss * 20, torch.float32).view(-1, 20)

    def brange(self):
        return self._view(self.c.brange, self.n_gauss * 8, torch.int32).view(-1, 8)

    def npairs(self) -> int:
        return int(self._view(self.c.d_npairs, 1, torch.int64).item())

    def npairs_dev(self) -> torch.Tensor:
        """Device int64 [1]: pairs needed by the last binning (no host synchronisation)."""
        return self._view(self.c.d_npairs, 1, torch.int64)

    def status(self) -> int:
        return int(self._view(self.c.d_status, 1, torch.int32).item())


class Workspace:
    def __init__(self, n_gauss: int, capacity: int, grid: Grid, cfg: Config, device="cuda"):
        lib = load()
        g, c = grid.c(), cfg.c()
        self.nbytes = lib.gs_workspace_bytes(n_gauss, capacity, ctypes.byref(g), ctypes.byref(c))
        if self.nbytes == 0:
            raise GsError("gs_workspace_bytes: invalid arguments")
        self.buf = _empty_bytes(self.nbytes, device)


# ---------------------------------------------------------------------- entry points
def gs_signal_proxy(T1: torch.Tensor, T2: torch.Tensor, TR: float, TE: float, out=None, stream=None):
    out = torch.empty_like(T1) if out is None else out
    _check(load().gs_signal_proxy(_ptr(T1), _ptr(T2), T1.numel(), TR, TE, _ptr(out),
                                  _stream(stream)), "gs_signal_proxy")
    return out


def gs_bin_bricks(params: torch.Tensor, grid: Grid, cfg: Config, bins: Bins, ws: Workspace,
                  stream=None):
    assert params.is_contiguous() and params.dtype == torch.float32
    g, c = grid.c(), cfg.c()
    _check(load().gs_bin_bricks(_ptr(params), ctypes.byref(g), ctypes.byref(c),
                                ctypes.byref(bins.c), _ptr(ws.buf), ws.nbytes, _stream(stream)),
           "gs_bin_bricks")


def gs_render_fwd(bins: Bins, grid: Grid, cfg: Config, I=None, W=None, stats=None, stream=None):
    dev = bins.arena.device
    I = torch.empty(grid.shape, dtype=torch.float32, device=dev) if I is None else I
    W = torch.empty(grid.shape, dtype=torch.float32, device=dev) if W is None else W
    g, c = grid.c(), cfg.c()
    _check(load().gs_render_fwd(ctypes.byref(bins.c), ctypes.byref(g), ctypes.byref(c), _ptr(I),
                                _ptr(W), _ptr(stats), _stream(stream)), "gs_render_fwd")
    return I, W


def gs_render_bwd(params, bins: Bins, grid: Grid, cfg: Config, I, W, dI, ws: Workspace,
                  dparams=None, stream=None):
    dparams = torch.empty_like(params) if dparams is None else dparams
    g, c = grid.c(), cfg.c()
    _check(load().gs_render_bwd(_ptr(params), ctypes.byref(bins.c), ctypes.byref(g),
                                ctypes.byref(c), _ptr(I), _ptr(W), _ptr(dI), _ptr(dparams),
                                _ptr(ws.buf), ws.nbytes, _stream(stream)), "gs_render_bwd")
    return dparams


def gs_downsample_fwd(hr: torch.Tensor, s: int, lr=None, stream=None):
    nz, ny, nx = hr.shape
    lr = torch.empty((nz // s, ny, nx), dtype=torch.float32, device=hr.device) if lr is None else lr
    _check(load().gs_downsample_fwd(_ptr(hr), nz, ny, nx, s, _ptr(lr), _stream(stream)),
           "gs_downsample_fwd")
    return lr


def gs_downsample_bwd(dlr: torch.Tensor, nz: int, s: int, dhr=None, stream=None):
    _, ny, nx = dlr.shape
    dhr = torch.empty((nz, ny, nx), dtype=torch.float32, device=dlr.device) if dhr is None else dhr
    _check(load().gs_downsample_bwd(_ptr(dlr), nz, ny, nx, s, _ptr(dhr), _stream(stream)),
           "gs_downsample_bwd")
    return dhr


def gs_resample_fwd(src: torch.Tensor, out_shape, dst=None, stream=None):
    """Trilinear resize (half-pixel centres) of a [z, y, x] volume to out_shape."""
    snz, sny, snx = src.shape
    dnz, dny, dnx = out_shape
    dst = torch.empty(tuple(out_shape), dtype=torch.float32, device=src.device) if dst is None else dst
    _check(load().gs_resample_fwd(_ptr(src), snz, sny, snx, _ptr(dst), dnz, dny, dnx,
                                  _stream(stream)), "gs_resample_fwd")
    return dst


def gs_resample_bwd(ddst: torch.Tensor, src_shape, dsrc=None, stream=None):
    """Adjoint of gs_resample_fwd: R^T ddst on the source shape."""
    dnz, dny, dnx = ddst.shape
    snz, sny, snx = src_shape
    dsrc = torch.empty(tuple(src_shape), dtype=torch.float32, device=ddst.device) if dsrc is None else dsrc
    _check(load().gs_resample_bwd(_ptr(ddst), dnz, dny, dnx, _ptr(dsrc), snz, sny, snx,
                                  _stream(stream)), "gs_resample_bwd")
    return dsrc


def gs_l1_loss(pred, target, ws: Workspace, d_loss=None, dpred=None, stream=None):
    d_loss = torch.empty((), dtype=torch.float32, device=pred.device) if d_loss is None else d_loss
    _check(load().gs_l1_loss(_ptr(pred), _ptr(target), pred.numel(), _ptr(d_loss), _ptr(dpred),
                             _ptr(ws.buf), ws.nbytes, _stream(stream)), "gs_l1_loss")
    return d_loss


GS_L1_STATIC_MAX_N = 33554432


def _check_f32_cuda(name, t, n):
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} values, expected {n}")


def gs_l1_loss_static(pred, target, d_loss=None, dpred=None, stream=None):
    """L1 loss without a workspace (for callers that cannot allocate device memory).

    pred, target (and dpred, if given) are contiguous float32 CUDA tensors of equal size,
    at most GS_L1_STATIC_MAX_N values; d_loss, if given, is a float32 CUDA scalar."""
    n = pred.numel()
    _check_f32_cuda("pred", pred, None)
    _check_f32_cuda("target", target, n)
    if dpred is not None:
        _check_f32_cuda("dpred", dpred, n)
    if n < 1 or n > GS_L1_STATIC_MAX_N:
        raise ValueError(f"gs_l1_loss_static takes 1 to {GS_L1_STATIC_MAX_N} values, got {n}")
    if d_loss is not None:
        _check_f32_cuda("d_loss", d_loss, 1)
    d_loss = torch.empty((), dtype=torch.float32, device=pred.device) if d_loss is None else d_loss
    _check(load().gs_l1_loss_static(_ptr(pred), _ptr(target), pred.numel(), _ptr(d_loss),
                                    _ptr(dpred), _stream(stream)), "gs_l1_loss_static")
    return d_loss


def gs_adam_step(params, grad, m, v, hp: Adam, d_step, stream=None):
    a = hp.c()
    _check(load().gs_adam_step(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), params.shape[0],
                               ctypes.byref(a), _ptr(d_step), _stream(stream)), "gs_adam_step")


def gs_init_lattice(lr, grid: Grid, s: int, nl, t_act: int = 1, t_init: float = 0.5, out=None,
                    stream=None):
    n = nl[0] * nl[1] * nl[2]
    out = torch.empty((n, 12), dtype=torch.float32, device=lr.device) if out is None else out
    g = grid.c()
    _check(load().gs_init_lattice(_ptr(lr), ctypes.byref(g), s, nl[0], nl[1], nl[2], t_act,
                                  t_init, _ptr(out), _stream(stream)), "gs_init_lattice")
    return out


def gs_init_lattice_lr(lr, grid: Grid, nl, t_act: int = 1, t_init: float = 0.5, out=None,
                       stream=None):
    """Lattice init from an LR volume made by gs_resample_fwd on ``grid``'s field of view."""
    lnz, lny, lnx = lr.shape
    n = nl[0] * nl[1] * nl[2]
    out = torch.empty((n, 12), dtype=torch.float32, device=lr.device) if out is None else out
    g = grid.c()
    _check(load().gs_init_lattice_lr(_ptr(lr), lnz, lny, lnx, ctypes.byref(g), nl[0], nl[1],
                                     nl[2], t_act, t_init, _ptr(out), _stream(stream)),
           "gs_init_lattice_lr")
    return out


def gs_launch_count() -> int:
    return int(load().gs_launch_count())


def gs_status_read(bins: Bins, stream=None) -> tuple[int, int]:
    h = ctypes.c_int32(0)
    rc = load().gs_status_read(ctypes.c_void_p(bins.c.d_status), ctypes.byref(h), _stream(stream))
    return rc, h.value


# ---------------------------------------------------------------------- composite helpers
def render(params: torch.Tensor, grid: Grid, cfg: Config = Config(), capacity: int | None = None,
           stats: torch.Tensor | None = None, stream=None):
    """Bin and render a cloud. Grows the pair capacity (one host read) if it overflows.
    Returns (I, W, bins, workspace)."""
    n = params.shape[0]
    cap = capacity if capacity is not None else max(1024, 16 * n)
    while True:
        bins = Bins(n, cap, grid, cfg, params.device)
        ws = Workspace(n, cap, grid, cfg, params.device)
        gs_bin_bricks(params, grid, cfg, bins, ws, stream)
        need = bins.npairs()
        if need <= cap:
            break
        cap = int(need * 1.25) + 1024
    I, W = gs_render_fwd(bins, grid, cfg, stats=stats, stream=stream)
    return I, W, bins, ws


class GaussianRender(torch.autograd.Function):
    """I = render(params) with the library's adjoint as backward (Eq. 5-6)."""

    @staticmethod
    def forward(ctx, params, grid: Grid, cfg: Config):
        params = params.contiguous()
        I, W, bins, ws = render(params, grid, cfg)
        ctx.save_for_backward(params, I, W)
        ctx.bins, ctx.ws, ctx.grid, ctx.cfg = bins, ws, grid, cfg
        return I

    @staticmethod
    def backward(ctx, dI):
        params, I, W = ctx.saved_tensors
        dparams = gs_render_bwd(params, ctx.bins, ctx.grid, ctx.cfg, I, W, dI.contiguous(), ctx.ws)
        return dparams, None, None


# ---------------------------------------------------------------------- fitting state
class FitState:
    """Device-resident zero-shot fitting state for one scan (params, Adam moments, bins,
    volumes, workspace) driving gs_fit_step."""

    def __init__(self, params0: torch.Tensor, lr_target: torch.Tensor, grid: Grid, s: int,
                 cfg: Config = Config(t_act=1), adam: Adam = Adam(), capacity: int | None = None,
                 lr_model: int = GS_LR_ZBOX):
        """lr_model GS_LR_ZBOX: lr_target is [nz // s, ny, nx]; GS_LR_TRILINEAR: lr_target has
        any shape and s is unused."""
        dev = params0.device
        n = params0.shape[0]
        self.grid, self.cfg, self.adam, self.s = grid, cfg, adam, s
        self.params = params0.clone().contiguous()
        self.grad = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.d_step = torch.zeros((), dtype=torch.int32, device=dev)
        self.I = torch.zeros(grid.shape, dtype=torch.float32, device=dev)
        self.W = torch.zeros_like(self.I)
        self.lr_target = lr_target.contiguous()
        self.lr_pred = torch.zeros_like(self.lr_target)
        self.d_loss = torch.zeros((), dtype=torch.float32, device=dev)
        if capacity is None:
            tmp_bins = Bins(n, max(1024, 64 * n), grid, cfg, dev)
            tmp_ws = Workspace(n, max(1024, 64 * n), grid, cfg, dev)
            gs_bin_bricks(self.params, grid, cfg, tmp_bins, tmp_ws)
            capacity = int(tmp_bins.npairs() * 1.5) + 4096
            del tmp_bins, tmp_ws
        self.capacity = capacity
        self.bins = Bins(n, capacity, grid, cfg, dev)
        self.ws = Workspace(n, capacity, grid, cfg, dev)
        st = gs_fit_state()
        st.grid, st.cfg, st.adam = grid.c(), cfg.c(), adam.c()
        st.n_gauss, st.s = n, s
        st.params, st.grad = self.params.data_ptr(), self.grad.data_ptr()
        st.m, st.v, st.d_step = self.m.data_ptr(), self.v.data_ptr(), self.d_step.data_ptr()
        st.bins = self.bins.c
        st.I, st.W = self.I.data_ptr(), self.W.data_ptr()
        st.lr_pred, st.lr_target = self.lr_pred.data_ptr(), self.lr_target.data_ptr()
        st.d_loss, st.ws, st.ws_bytes = self.d_loss.data_ptr(), self.ws.buf.data_ptr(), self.ws.nbytes
        st.lr_model = lr_model
        if lr_model == GS_LR_TRILINEAR:
            st.lr_nz, st.lr_ny, st.lr_nx = self.lr_target.shape
        self.c = st

    def set_phase_events(self, events):
        """Record the GS_FIT_PHASES torch.cuda.Event objects at the step's phase boundaries
        (None: stop recording). Each event must have been recorded once (so it exists)."""
        if events is None:
            self._ev_arr = None
            self.c.phase_events, self.c.n_phase_events = None, 0
            return
        assert len(events) == GS_FIT_PHASES
        self._ev_arr = (ctypes.c_void_p * GS_FIT_PHASES)(*[e.cuda_event for e in events])
        self.c.phase_events = ctypes.cast(self._ev_arr, ctypes.c_void_p)
        self.c.n_phase_events = GS_FIT_PHASES

    def step(self, stream=None):
        _check(load().gs_fit_step(ctypes.byref(self.c), _stream(stream)), "gs_fit_step")

    def step_host(self, h_params=None, h_lr_target=None, h_loss=None, stream=None):
        """gs_fit_step_host: one step with its inputs (and loss) in host memory: h_params
        [n_gauss, 12] and h_lr_target (LR shape) float32 CPU tensors (page-locked for
        asynchronous copies) or None to keep the device copies; h_loss a float32 CPU scalar
        tensor or None. Synchronise the stream before reading h_loss."""
        for name, t in (("h_params", h_params), ("h_lr_target", h_lr_target), ("h_loss", h_loss)):
            if t is not None and (t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous float32 host tensor")
        if h_params is not None and h_params.numel() != self.params.numel():
            raise ValueError("h_params has the wrong size")
        if h_lr_target is not None and h_lr_target.numel() != self.lr_target.numel():
            raise ValueError("h_lr_target has the wrong size")
        _check(load().gs_fit_step_host(ctypes.byref(self.c), _ptr(h_params), _ptr(h_lr_target),
                                       _ptr(h_loss), _stream(stream)), "gs_fit_step_host")

    def grad_step(self, n_lr_total: int = 0, stream=None):
        """gs_fit_grad: this state's gradient into self.grad, no Adam; the L1 mean is taken over
        n_lr_total LR values when > 0 (a slab's share of a whole volume's loss)."""
        _check(load().gs_fit_grad(ctypes.byref(self.c), int(n_lr_total), _stream(stream)),
               "gs_fit_grad")

    def apply(self, d_skip: torch.Tensor | None = None, stream=None):
        """gs_fit_apply: Adam from self.grad, skipped when d_skip (device int32) is nonzero."""
        _check(load().gs_fit_apply(ctypes.byref(self.c), _ptr(d_skip), _stream(stream)),
               "gs_fit_apply")

    def overflow_flag(self) -> torch.Tensor:
        """Device int32 [1]: 1 when the last binning needed more pairs than the capacity."""
        return (self.bins.npairs_dev() > self.capacity).to(torch.int32)

    def grow(self, capacity: int | None = None):
        """New bins and workspace for `capacity` pairs (default: 1.125 x the last binning's
        count); parameters, moments and the step counter are kept."""
        if capacity is None:
            capacity = int(self.bins.npairs() * 1.125) + 4096
        dev = self.params.device
        n = self.params.shape[0]
        self.capacity = capacity
        self.bins = Bins(n, capacity, self.grid, self.cfg, dev)
        self.ws = Workspace(n, capacity, self.grid, self.cfg, dev)
        self.c.bins = self.bins.c
        self.c.ws, self.c.ws_bytes = self.ws.buf.data_ptr(), self.ws.nbytes

    def check(self, stream=None):
        rc, bits = gs_status_read(self.bins, stream)
        return rc, bits
