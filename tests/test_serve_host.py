"""Host side of the serving runtime (no GPU): the best-fit arena allocator, request sizing,
configuration checks and the seeded request stream."""
import ctypes

import numpy as np
import pytest

from paper_2603_09621_gb300 import inputs

BASE = 1 << 40  # host bookkeeping only: the arena never dereferences its range


@pytest.fixture(scope="module")
def lib():
    import torch  # noqa: F401  (loads the CUDA runtime the library links against)
    from paper_2603_09621_gb300 import build, gs
    build.build()
    gs._lib = None
    return gs.load()


def _arena(lib, nbytes):
    a = ctypes.c_void_p()
    assert lib.gs_arena_create(ctypes.c_void_p(BASE), nbytes, ctypes.byref(a)) == 0
    return a


def _alloc(lib, a, n):
    p = ctypes.c_void_p()
    rc = lib.gs_arena_alloc(a, n, ctypes.byref(p))
    return rc, (p.value or 0) - BASE if rc == 0 else None


def _stats(lib, a):
    u, pk, lf, nl = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int64()
    assert lib.gs_arena_stats(a, ctypes.byref(u), ctypes.byref(pk), ctypes.byref(lf),
                              ctypes.byref(nl)) == 0
    return u.value, pk.value, lf.value, nl.value


def test_arena_alignment_and_rounding(lib):
    a = _arena(lib, 1 << 20)
    offs = [_alloc(lib, a, n)[1] for n in (1, 255, 256, 257, 1000)]
    assert offs == [0, 256, 512, 768, 1280]
    assert all(o % 256 == 0 for o in offs)
    used, peak, largest, n_live = _stats(lib, a)
    assert used == 256 * (1 + 1 + 1 + 2 + 4) and peak == used and n_live == 5
    assert largest == (1 << 20) - used
    lib.gs_arena_destroy(a)


def test_arena_best_fit_and_coalescing(lib):
    a = _arena(lib, 16 * 256)
    blocks = [_alloc(lib, a, 256)[1] for _ in range(16)]
    assert _alloc(lib, a, 1)[0] == -2          # full: GS_ERR_CAPACITY
    # holes of 2, 1 and 3 granules
    for i in (2, 3, 6, 10, 11, 12):
        assert lib.gs_arena_free(a, ctypes.c_void_p(BASE + blocks[i])) == 0
    rc, off = _alloc(lib, a, 256)
    assert rc == 0 and off == blocks[6]        # the smallest hole that fits
    rc, off = _alloc(lib, a, 512)
    assert rc == 0 and off == blocks[2]        # exact fit before the larger hole
    rc, off = _alloc(lib, a, 3 * 256)
    assert rc == 0 and off == blocks[10]
    assert _stats(lib, a)[2] == 0
    # free everything: neighbours merge back into one hole
    for i in range(16):
        lib.gs_arena_free(a, ctypes.c_void_p(BASE + blocks[i]))
    used, peak, largest, n_live = _stats(lib, a)
    assert used == 0 and n_live == 0 and largest == 16 * 256 and peak == 16 * 256
    lib.gs_arena_destroy(a)


def _alloc_top(lib, a, n):
    p = ctypes.c_void_p()
    rc = lib.gs_arena_alloc_top(a, n, ctypes.byref(p))
    return rc, (p.value or 0) - BASE if rc == 0 else None


def test_arena_top_allocation_keeps_free_space_whole(lib):
    """Long-lived blocks from the top, short-lived from the bottom: after the short-lived ones
    are freed, the free space is one hole."""
    size = 64 * 256
    a = _arena(lib, size)
    assert _alloc_top(lib, a, 256) == (0, size - 256)
    assert _alloc_top(lib, a, 300) == (0, size - 3 * 256)
    lows = [_alloc(lib, a, 1000)[1] for _ in range(4)]
    assert lows == [0, 1024, 2048, 3072]
    tops = [_alloc_top(lib, a, 256)[1] for _ in range(3)]
    assert tops == [size - 4 * 256, size - 5 * 256, size - 6 * 256]
    for off in lows:
        assert lib.gs_arena_free(a, ctypes.c_void_p(BASE + off)) == 0
    used, _, largest, n_live = _stats(lib, a)
    assert n_live == 5 and largest == size - used
    # the top allocation takes the highest hole that fits, not the largest
    assert lib.gs_arena_free(a, ctypes.c_void_p(BASE + tops[1])) == 0
    assert _alloc_top(lib, a, 256) == (0, tops[1])
    assert _alloc_top(lib, a, size)[0] == -2
    lib.gs_arena_destroy(a)


def test_arena_random_alloc_free_invariants(lib):
    rng = np.random.default_rng(3)
    size = 1 << 16
    a = _arena(lib, size)
    live = {}
    for _ in range(2000):
        if live and rng.uniform() < 0.45:
            off = list(live)[int(rng.integers(len(live)))]
            assert lib.gs_arena_free(a, ctypes.c_void_p(BASE + off)) == 0
            del live[off]
        else:
            n = int(rng.integers(1, 3000))
            rc, off = (_alloc_top if rng.uniform() < 0.3 else _alloc)(lib, a, n)
            if rc == 0:
                need = (n + 255) // 256 * 256
                for o, m in live.items():      # no overlap with any live block
                    assert off + need <= o or o + m <= off
                assert off + need <= size
                live[off] = need
            else:
                assert rc == -2
        used, _, largest, n_live = _stats(lib, a)
        assert used == sum(live.values()) and n_live == len(live)
        assert largest <= size - used
    lib.gs_arena_destroy(a)


def test_arena_rejects_bad_calls(lib):
    a = ctypes.c_void_p()
    assert lib.gs_arena_create(ctypes.c_void_p(BASE + 8), 4096, ctypes.byref(a)) == -1
    assert lib.gs_arena_create(None, 4096, ctypes.byref(a)) == -1
    a = _arena(lib, 4096)
    assert _alloc(lib, a, 0)[0] == -1
    assert _alloc(lib, a, 8192)[0] == -2
    rc, off = _alloc(lib, a, 100)
    assert lib.gs_arena_free(a, ctypes.c_void_p(BASE + off + 256)) == -1   # not a block
    assert lib.gs_arena_free(a, ctypes.c_void_p(BASE + off)) == 0
    assert lib.gs_arena_free(a, ctypes.c_void_p(BASE + off)) == -1         # double free
    lib.gs_arena_destroy(a)


def _fake_fit(gs, serve, nx=64, ny=64, nz=48, n=20000, s=2):
    r = gs.gs_request()
    r.kind, r.grid, r.s, r.iters, r.n_gauss = gs.GS_REQ_FIT, gs.Grid(nx, ny, nz).c(), s, 10, n
    r.params, r.lr_target, r.source, r.arrival_s = 1 << 40, 1 << 41, -1, 0.0
    return r


def test_request_bytes(lib):
    from paper_2603_09621_gb300 import gs, serve
    cfg = serve.server_config(1 << 30)
    r = _fake_fit(gs, serve)
    b = lib.gs_server_request_bytes(ctypes.byref(cfg), ctypes.byref(r))
    # at least params + grad + m + v, I, W and the two LR volumes
    assert b >= 4 * 20000 * 48 + 2 * 64 * 64 * 48 * 4 + 2 * 64 * 64 * 24 * 4
    big = _fake_fit(gs, serve, n=40000)
    assert lib.gs_server_request_bytes(ctypes.byref(cfg), ctypes.byref(big)) > b
    cfg2 = serve.server_config(1 << 30, pairs_per_gauss=32.0)
    assert lib.gs_server_request_bytes(ctypes.byref(cfg2), ctypes.byref(r)) > b
    rend = serve.render_request(gs.Grid(80, 80, 60), 20000, source=0)
    assert lib.gs_server_request_bytes(ctypes.byref(cfg), ctypes.byref(rend)) >= 2 * 80 * 80 * 60 * 4
    for bad in ("s", "iters", "n_gauss", "params"):
        x = _fake_fit(gs, serve)
        setattr(x, bad, 0 if bad != "params" else None)
        assert lib.gs_server_request_bytes(ctypes.byref(cfg), ctypes.byref(x)) == 0, bad
    x = _fake_fit(gs, serve)
    x.kind = 7
    assert lib.gs_server_request_bytes(ctypes.byref(cfg), ctypes.byref(x)) == 0


def test_server_config_checked_before_any_device_call(lib):
    from paper_2603_09621_gb300 import serve
    out = ctypes.c_void_p()
    for kw in (dict(max_active=0), dict(max_active=65), dict(chunk_steps=0),
               dict(max_bypass=-1), dict(pairs_per_gauss=0.0)):
        cfg = serve.server_config(1 << 30, **kw)
        assert lib.gs_server_create(ctypes.byref(cfg), ctypes.byref(out)) == -1, kw
    cfg = serve.server_config(0)
    assert lib.gs_server_create(ctypes.byref(cfg), ctypes.byref(out)) == -1


def test_serving_draws_stream():
    a = inputs.serving_draws(seed=0)
    b = inputs.serving_draws(seed=0)
    assert a == b and len(a) == 32
    assert a[0]["kind"] == "fit" and a[0]["arrival_s"] == 0.0
    t = [d["arrival_s"] for d in a]
    assert all(x <= y for x, y in zip(t, t[1:]))
    # mean inter-arrival near 1 / rate over a long stream
    long = inputs.serving_draws(seed=1, n=4000)
    gaps = np.diff([d["arrival_s"] for d in long])
    assert abs(gaps.mean() - 0.5) < 0.03
    frac = np.mean([d["kind"] == "fit" for d in long])
    assert abs(frac - 0.75) < 0.03
    for i, d in enumerate(a):
        if d["kind"] == "fit":
            assert d["shape"] in inputs.SERVE_SHAPES and d["s"] in (2, 3, 4)
            assert d["n_gauss"] == inputs.serve_n_gauss(d["shape"])
        else:
            src = a[d["source"]]
            assert d["source"] < i and src["kind"] == "fit"
            assert d["shape"] == tuple(int(round(x / d["spacing"])) for x in src["shape"])
    assert inputs.serve_n_gauss((192, 256, 256)) == 1_000_000
    assert inputs.serve_n_gauss((128, 128, 128)) == 166_667
    assert inputs.serve_n_gauss((8, 8, 8)) == 100_000
