"""tg_backproject_noalloc: the backprojection entry point for callers that
cannot allocate device memory (code being captured into a CUDA graph, hosts
with a fixed device-memory budget, latency-bound paths).  It must give the
results of tg_backproject through the C ABI, call after call, while using
only its static scratch.  This file runs last so that a stop at the first
failure has already run every other test."""
import ctypes

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
    code = {"matched": tg.TG_MATCHED, "fdk": tg.TG_FDK_WEIGHT}[method]
    return lib.tg_backproject_noalloc(G.ref, G.ang, G.n, ctypes.c_void_p(proj.data_ptr()),
                                      ctypes.c_void_p(vol.data_ptr()), code, batch,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("method", ["matched", "fdk"])
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
