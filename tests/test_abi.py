"""The C-ABI library builds for sm_103a, loads, and exports every entry point declared in
include/*.h; host-only entry points validate their arguments (no GPU needed)."""
import glob
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def declared_functions():
    src = "\n".join(open(h).read() for h in HEADERS)
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(gs_[a-z0-9_]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import torch  # noqa: F401  (loads the CUDA runtime the library links against)
    from paper_2603_09621_gb300 import build, gs
    build.build()
    gs._lib = None
    return gs.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gs_bin_bricks", "gs_render_fwd", "gs_render_bwd", "gs_downsample_fwd",
                     "gs_downsample_bwd", "gs_fit_step"):
        assert required in names
    assert len(names) >= 15


def test_library_exports_every_declared_symbol(lib):
    from paper_2603_09621_gb300 import gs
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in gs.SIGNATURES, name


def test_library_targets_sm103a():
    from paper_2603_09621_gb300 import build
    flags = " ".join(build.ARCH)
    assert "compute_103a" in flags and "sm_103a" in flags


def test_host_only_sizes_and_binding(lib):
    from paper_2603_09621_gb300 import gs
    g = gs.Grid(256, 256, 128).c()
    c = gs.Config().c()
    nb = lib.gs_bins_bytes(500_000, 5_000_000, ctypes.byref(g), ctypes.byref(c))
    assert nb > 5_000_000 * 8
    assert lib.gs_workspace_bytes(500_000, 5_000_000, ctypes.byref(g), ctypes.byref(c)) > 0
    bins = gs.gs_bins()
    fake = ctypes.c_void_p(1 << 40)  # host-side carving only: nothing is dereferenced
    rc = lib.gs_bins_bind(fake, nb, 500_000, 5_000_000, ctypes.byref(g), ctypes.byref(c),
                          ctypes.byref(bins))
    assert rc == 0
    assert (bins.nbx, bins.nby, bins.nbz, bins.n_bricks) == (32, 32, 16, 32 * 32 * 16)
    for f in ("brick_off", "pair_gid", "pair_gmj", "gm_off", "rec", "brange", "d_npairs",
              "d_status"):
        off = getattr(bins, f) - (1 << 40)
        assert 0 <= off < nb and off % 256 == 0, f
    # arena too small / misaligned
    assert lib.gs_bins_bind(fake, nb - 1, 500_000, 5_000_000, ctypes.byref(g), ctypes.byref(c),
                            ctypes.byref(bins)) == -3
    assert lib.gs_bins_bind(ctypes.c_void_p((1 << 40) + 16), nb, 500_000, 5_000_000,
                            ctypes.byref(g), ctypes.byref(c), ctypes.byref(bins)) == -1


@pytest.mark.parametrize("field,value", [("brick", (6, 8, 8)), ("trunc_sigma", 0.0),
                                         ("eps", 0.0), ("signal_mode", 2), ("t_act", 3)])
def test_invalid_config_rejected(lib, field, value):
    from paper_2603_09621_gb300 import gs
    cfg = gs.Config(**{field: value})
    g = gs.Grid(32, 32, 32).c()
    assert lib.gs_bins_bytes(100, 1000, ctypes.byref(g), ctypes.byref(cfg.c())) == 0


def test_invalid_grid_rejected(lib):
    from paper_2603_09621_gb300 import gs
    c = gs.Config().c()
    for grid in (gs.Grid(0, 4, 4), gs.Grid(4, 4, 4, h=(0.0, 1.0, 1.0))):
        g = grid.c()
        assert lib.gs_bins_bytes(10, 100, ctypes.byref(g), ctypes.byref(c)) == 0
    g = gs.Grid(8, 8, 8).c()
    assert lib.gs_bins_bytes(10, 1 << 40, ctypes.byref(g), ctypes.byref(c)) == 0


def test_null_arguments_rejected_before_launch(lib):
    """Argument errors come back synchronously without touching the device."""
    from paper_2603_09621_gb300 import gs
    g, c = gs.Grid(16, 16, 16).c(), gs.Config().c()
    assert lib.gs_bin_bricks(None, ctypes.byref(g), ctypes.byref(c), None, None, 0, None) == -1
    assert lib.gs_render_fwd(None, ctypes.byref(g), ctypes.byref(c), None, None, None, None) == -1
    assert lib.gs_downsample_fwd(None, 8, 8, 8, 2, None, None) == -1
    assert lib.gs_downsample_bwd(None, 8, 8, 8, 0, None, None) == -1
    assert lib.gs_l1_loss(None, None, 10, None, None, None, 0, None) == -1
    assert lib.gs_fit_step(None, None) == -1
    assert lib.gs_signal_proxy(None, None, 0, 2000.0, 100.0, None, None) == 0
    assert lib.gs_signal_proxy(None, None, 5, 2000.0, 100.0, None, None) == -1


def test_status_strings(lib):
    assert lib.gs_status_string(0) == b"ok"
    assert lib.gs_status_string(-2) == b"pair capacity exceeded"
    assert b"sm_103a" in lib.gs_version()
