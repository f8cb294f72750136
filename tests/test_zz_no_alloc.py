"""tg_backproject_noalloc: the backprojection entry point for callers that
cannot allocate device memory (a host that fixes its device-memory budget at
start-up, real-time paths that cannot afford an allocator's latency or
failure).  It must give the results of tg_backproject through the C ABI,
call after call, while using only its static scratch, and must take no
memory from the device allocator.  This file runs last so that a stop at the
first failure has already run every other test."""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

from conftest import max_rel, rel_l2
from paper_2412_10129_gb300 import build, inputs, tg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_L2 = 1e-6   # same kernels, same inputs: agreement to rounding or better


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return tg.load()


def _geo():
    return inputs.random_geometry((37, 29, 23), (1.0, 1.2, 0.9), (45, 31), (1.3, 1.1), 13, seed=41,
                                  DSO=300.0, DSD=520.0)


def _raw(lib, g, proj, vol, method, batch):
    G = tg._Geo(g)
    code = {"matched": tg.TG_MATCHED, "fdk": tg.TG_FDK_WEIGHT, "siddon": tg.TG_SIDDON_BP}[method]
    return lib.tg_backproject_noalloc(G.ref, G.ang, G.n, ctypes.c_void_p(proj.data_ptr()),
                                      ctypes.c_void_p(vol.data_ptr()), code, batch,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("method", ["matched", "fdk", "siddon"])
def test_noalloc_matches_backproject_on_consecutive_calls(lib, method):
    g = _geo()
    for seed in (1, 2):   # two calls in a row: the shared scratch is refilled
        y = torch.from_numpy(inputs.random_projections(g, seed=seed)).cuda()
        ref = tg.backproject(g, y, method)
        out = torch.full(g.vol_shape, float("nan"), device="cuda")
        assert _raw(lib, g, y, out, method, 1) == 0
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert rel_l2(a, b) <= TOL_L2
        assert max_rel(a, b) <= 10 * TOL_L2


def test_noalloc_batched_and_full_circle(lib):
    g = inputs.config_small()
    ys = torch.from_numpy(np.stack([inputs.random_projections(g, seed=s) for s in (3, 4)])).cuda()
    ref = tg.backproject(g, ys, "matched")
    out = tg.backproject_noalloc(g, ys, "matched")
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) <= TOL_L2


def test_noalloc_rejects_what_it_cannot_serve(lib):
    g = _geo()
    y = torch.from_numpy(inputs.random_projections(g, seed=5)).cuda()
    out = torch.empty(g.vol_shape, device="cuda")
    # host buffers would need staging memory
    G = tg._Geo(g)
    yh = inputs.random_projections(g, seed=5)
    vh = np.empty(g.vol_shape, np.float32)
    assert lib.tg_backproject_noalloc(G.ref, G.ang, G.n, yh.ctypes.data, vh.ctypes.data, 0, 1, None) == 1
    # more angles than the static scratch holds
    big = inputs.circular_geometry((8, 8, 8), (1.0,) * 3, (4, 4), (4.0, 4.0), 4097, 100.0, 160.0)
    yb = torch.zeros(big.proj_shape, device="cuda")
    vb = torch.empty(big.vol_shape, device="cuda")
    assert _raw(lib, big, yb, vb, "matched", 1) == 6
    with pytest.raises(tg.TgError):
        tg.backproject_noalloc(big, yb)
    # the call that follows a rejection still works
    assert _raw(lib, g, y, out, "matched", 1) == 0
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), tg.backproject(g, y, "matched").cpu().numpy()) <= TOL_L2


def _cudart():
    for name in (ctypes.util.find_library("cudart"), "/usr/local/cuda/lib64/libcudart.so", "libcudart.so"):
        if name:
            try:
                return ctypes.CDLL(name)
            except OSError:
                continue
    pytest.skip("libcudart not found")


USED_MEM_HIGH = 8   # cudaMemPoolAttrUsedMemHigh


def _pool_high(rt, pool):
    v = ctypes.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, USED_MEM_HIGH, ctypes.byref(v)) == 0
    return v.value


def _pool_reset(rt, pool):
    zero = ctypes.c_uint64(0)
    assert rt.cudaMemPoolSetAttribute(pool, USED_MEM_HIGH, ctypes.byref(zero)) == 0


def test_noalloc_takes_no_device_memory(lib):
    """The device's default memory pool (where cudaMallocAsync draws from)
    keeps its high-water mark and the free device memory stays the same
    across warmed-up calls of every method; tg_backproject, which takes its
    scratch from that pool, raises the mark (the check can see an
    allocation)."""
    rt = _cudart()
    dev = torch.cuda.current_device()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    g = _geo()
    y = torch.from_numpy(inputs.random_projections(g, seed=7)).cuda()
    out = torch.empty(g.vol_shape, device="cuda")
    for method in ("matched", "fdk", "siddon"):
        assert _raw(lib, g, y, out, method, 1) == 0   # warm-up (first-call set-up)
    torch.cuda.synchronize()
    _pool_reset(rt, pool)
    base = _pool_high(rt, pool)
    free0 = torch.cuda.mem_get_info()[0]
    for method in ("matched", "fdk", "siddon"):
        assert _raw(lib, g, y, out, method, 1) == 0
        torch.cuda.synchronize()
        assert _pool_high(rt, pool) == base, method
    assert torch.cuda.mem_get_info()[0] == free0
    tg.backproject(g, y, "matched", out=out)
    torch.cuda.synchronize()
    assert _pool_high(rt, pool) > base
