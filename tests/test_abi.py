"""The C ABI: libtg builds, loads and exports every function include/tg.h
declares; host-side argument and geometry validation runs before any CUDA
call, so it is checked here without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2412_10129_gb300 import build, inputs, tg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return tg.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tg_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("tg_forward", "tg_backproject", "tg_fdk", "tg_sirt", "tg_ossart", "tg_cgls",
              "tg_workspace_size", "tg_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_probe_library_exports_its_header():
    """libtgprobe (the gather-rate microbenchmarks of include/tg_probe.h)
    builds and exports what its header declares."""
    from paper_2412_10129_gb300 import probe
    build.build()
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "tg_probe.h")).read(), flags=re.S)
    names = sorted(set(re.findall(r"\b(tgp_[a-z0-9_]+)\s*\(", text)))
    assert names == ["tgp_sector_gather", "tgp_smem_atomic", "tgp_smem_atomic_kind", "tgp_tex_gather"]
    lib = probe.load()
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    assert tg.status_string(0) == "ok"
    assert tg.status_string(2) == "invalid geometry"
    assert "unknown" in tg.status_string(99)


def _geo():
    return inputs.circular_geometry((8, 8, 8), (1.0,) * 3, (10, 10), (1.5, 1.5), 4, 100.0, 160.0)


def _call_forward(geo, vol=None, proj=None, method=0, batch=1):
    G = tg._Geo(geo)
    v = vol if vol is not None else np.zeros(geo.vol_shape, np.float32)
    p = proj if proj is not None else np.zeros(geo.proj_shape, np.float32)
    return tg.load().tg_forward(G.ref, G.ang, G.n, v.ctypes.data, p.ctypes.data, method, batch, None)


@pytest.mark.parametrize("mutate,code", [
    (lambda g: setattr(g, "nVoxel", (0, 8, 8)), 2),
    (lambda g: setattr(g, "dVoxel", (1.0, -1.0, 1.0)), 2),
    (lambda g: setattr(g, "nDetector", (10, 0)), 2),
    (lambda g: setattr(g, "dDetector", (float("nan"), 1.0)), 2),
    (lambda g: setattr(g, "DSO", np.full(4, -5.0)), 2),
    (lambda g: setattr(g, "DSD", np.full(4, 0.0)), 2),
    # source inside the volume
    (lambda g: setattr(g, "DSO", np.full(4, 3.0)), 2),
    # detector plane cutting through the volume
    (lambda g: setattr(g, "DSD", np.full(4, 101.0)), 2),
    (lambda g: g.angles.__setitem__((1, 0), float("inf")), 2),
])
def test_invalid_geometry_is_rejected_on_the_host(lib, mutate, code):
    g = _geo()
    mutate(g)
    assert _call_forward(g) == code


def test_invalid_arguments_are_rejected(lib):
    g = _geo()
    G = tg._Geo(g)
    p = np.zeros(g.proj_shape, np.float32)
    assert lib.tg_forward(G.ref, G.ang, G.n, None, p.ctypes.data, 0, 1, None) == 1
    assert _call_forward(g, method=7) == 1
    assert _call_forward(g, batch=-1) == 1
    assert lib.tg_forward(None, G.ang, G.n, None, None, 0, 1, None) == 1
    assert lib.tg_forward(G.ref, None, 3, None, None, 0, 1, None) == 1
    v = np.zeros(g.vol_shape, np.float32)
    assert lib.tg_backproject(G.ref, G.ang, G.n, p.ctypes.data, v.ctypes.data, 5, 1, None) == 1
    assert lib.tg_fdk(G.ref, G.ang, G.n, p.ctypes.data, v.ctypes.data, 5, None) == 1
    assert lib.tg_fdk(G.ref, G.ang, G.n, p.ctypes.data, v.ctypes.data, -1, None) == 1
    assert lib.tg_fdk_ex(G.ref, G.ang, G.n, p.ctypes.data, v.ctypes.data, 0, 4, None) == 1
    assert lib.tg_fdk_filter(G.ref, G.ang, G.n, p.ctypes.data, p.ctypes.data, 0, 0, None) == 1
    assert lib.tg_sirt(G.ref, G.ang, G.n, p.ctypes.data, v.ctypes.data, -1, 1.0, 1, None, None) == 1
    assert lib.tg_ossart(G.ref, G.ang, G.n, p.ctypes.data, v.ctypes.data, 2, 0, 0, 0, 1.0, 1, None, None) == 1
    assert lib.tg_ossart(G.ref, G.ang, G.n, p.ctypes.data, v.ctypes.data, 2, 2, 9, 0, 1.0, 1, None, None) == 1
    assert lib.tg_cgls(G.ref, G.ang, G.n, p.ctypes.data, None, 2, None, None) == 1


def test_empty_requests_are_no_ops(lib):
    """nAngles == 0 or batch == 0 returns before touching the device."""
    g = _geo()
    G = tg._Geo(g)
    assert lib.tg_forward(G.ref, G.ang, 0, None, None, 0, 1, None) == 0
    assert lib.tg_forward(G.ref, G.ang, G.n, None, None, 0, 0, None) == 0
    assert lib.tg_backproject(G.ref, G.ang, G.n, None, None, 0, 0, None) == 0
    one = np.zeros(1, np.float32)
    assert lib.tg_cgls(G.ref, G.ang, G.n, one.ctypes.data, one.ctypes.data, 0, None, None) == 0
    assert lib.tg_sirt(G.ref, G.ang, G.n, one.ctypes.data, one.ctypes.data, 0, 1.0, 1, None, None) == 0


def test_workspace_size(lib):
    g = inputs.config_clinical()
    nvox, nray = 512 ** 3, 720 * 768 * 1024
    assert tg.workspace_size(g, "cgls") >= 4 * (2 * nray + 2 * nvox)
    assert tg.workspace_size(g, "ossart", blocksize=20) >= 4 * nvox * 36
    assert tg.workspace_size(g, "forward") < 1 << 20
    # the matched backprojection's brick rims: 2129 upper-face voxels per
    # 32 x 32 x 16 brick (16 x 16 x 32 bricks), owned sums in place
    rims = 4 * 2129 * 16 * 16 * 32
    assert rims <= tg.workspace_size(g, "backproject") < rims + (1 << 20)
    # SIRT-type epilogues keep the owned sums in a volume of their own
    assert tg.workspace_size(g, "sirt") >= 4 * (2 * nray + 2 * nvox) + rims


def test_fdk_weight_options_are_checked_on_the_host(lib):
    """Parker needs increasing angles over more than pi, Wang a detector that
    reaches across the central ray, and the two are not combined; all are
    refused before any CUDA call."""
    import math
    g = _geo()  # full orbit of 4 angles: 0 .. 3/2 pi
    G = tg._Geo(g)
    p = np.zeros(g.proj_shape, np.float32)
    v = np.zeros(g.vol_shape, np.float32)
    assert lib.tg_fdk_ex(G.ref, G.ang, G.n, p.ctypes.data, v.ctypes.data, 0, 3, None) == 6
    short = inputs.circular_geometry((8, 8, 8), (1.0,) * 3, (10, 10), (1.5, 1.5), 4, 100.0, 160.0,
                                     arc=0.9 * math.pi)
    S = tg._Geo(short)
    assert lib.tg_fdk_ex(S.ref, S.ang, S.n, p.ctypes.data, v.ctypes.data, 0, 1, None) == 2
    back = inputs.circular_geometry((8, 8, 8), (1.0,) * 3, (10, 10), (1.5, 1.5), 4, 100.0, 160.0)
    back.angles[:, 0] = back.angles[::-1, 0]
    B = tg._Geo(back)
    assert lib.tg_fdk_filter(B.ref, B.ang, B.n, p.ctypes.data, v.ctypes.data, 0, 1, None) == 2
    off = _geo()
    off.offDetector[:, 0] = 9 * 1.5
    O = tg._Geo(off)
    assert lib.tg_fdk_ex(O.ref, O.ang, O.n, p.ctypes.data, v.ctypes.data, 0, 2, None) == 2
    with pytest.raises(ValueError):
        tg.fdk(g, p, "gaussian")


def test_solver_arguments_are_checked_on_the_host(lib):
    """Invalid counts, methods, orders and parameters of the EM, Krylov and
    POCS solvers are refused before any CUDA call; niter = 0 is a no-op."""
    import math
    g = _geo()
    G = tg._Geo(g)
    p = np.zeros(g.proj_shape, np.float32)
    v = np.zeros(g.vol_shape, np.float32)
    P, V = p.ctypes.data, v.ctypes.data
    assert lib.tg_mlem(G.ref, G.ang, G.n, P, V, -1, 0, None, None) == 1
    assert lib.tg_mlem(G.ref, G.ang, G.n, P, V, 2, 5, None, None) == 1
    assert lib.tg_mlem(G.ref, G.ang, G.n, P, V, 0, 0, None, None) == 0
    assert lib.tg_osem(G.ref, G.ang, G.n, P, V, 2, 0, 0, 0, 0, None, None) == 1
    assert lib.tg_osem(G.ref, G.ang, G.n, P, V, 2, 2, 7, 0, 0, None, None) == 1
    assert lib.tg_lsqr(G.ref, G.ang, G.n, P, None, 2, None, None) == 1
    assert lib.tg_lsmr(G.ref, G.ang, G.n, P, V, -3, None, None) == 1
    assert lib.tg_lsqr(G.ref, G.ang, G.n, P, V, 0, None, None) == 0
    good = dict(niter=2, blocksize=1, tv_steps=20, alpha=0.002, alpha_red=0.95, r_max=0.95, data_tol=0.0,
                beta=1.0, beta_red=0.995, delta=math.inf, eps=1e-8)
    for bad in (dict(niter=-1), dict(blocksize=0), dict(tv_steps=-2), dict(eps=0.0), dict(delta=-1.0),
                dict(alpha=math.nan)):
        prm = tg._PocsParams(**{**good, **bad})
        assert lib.tg_asd_pocs(G.ref, G.ang, G.n, P, V, ctypes.byref(prm), None, None) == 1, bad
    assert lib.tg_asd_pocs(G.ref, G.ang, G.n, P, V, None, None, None) == 1
    zero = tg._PocsParams(**{**good, "niter": 0})
    assert lib.tg_asd_pocs(G.ref, G.ang, G.n, P, V, ctypes.byref(zero), None, None) == 0
    dims = (ctypes.c_int32 * 3)(8, 8, 8)
    assert lib.tg_tv_gradient(V, V, dims, ctypes.c_float(math.inf), ctypes.c_float(1e-8), None) == 1
    assert lib.tg_tv_descent(None, dims, 3, ctypes.c_float(0.1), ctypes.c_float(math.inf), ctypes.c_float(1e-8),
                             None) == 1
    bad_dims = (ctypes.c_int32 * 3)(8, 0, 8)
    assert lib.tg_tv_descent(V, bad_dims, 3, ctypes.c_float(0.1), ctypes.c_float(math.inf), ctypes.c_float(1e-8),
                             None) == 1


def test_workspace_sizes_of_the_solvers(lib):
    g = _geo()
    for op in ("mlem", "osem", "asd_pocs", "lsqr", "lsmr"):
        assert tg.workspace_size(g, op, blocksize=2) > 4 * int(np.prod(g.vol_shape))


def test_parallel_beam_refusals_on_the_host(lib):
    """Parker / Wang weights are not defined for a parallel scan; the call
    is refused before any CUDA call."""
    import math
    g = inputs.parallel_geometry((8, 8, 8), (1.0,) * 3, (10, 10), (1.5, 1.5), 6, arc=1.2 * math.pi,
                                 DSO=100.0, DSD=160.0)
    G = tg._Geo(g)
    assert G.g.parallel == 1
    p = np.zeros(g.proj_shape, np.float32)
    v = np.zeros(g.vol_shape, np.float32)
    assert lib.tg_fdk_ex(G.ref, G.ang, G.n, p.ctypes.data, v.ctypes.data, 0, 1, None) == 6
    assert lib.tg_fdk_filter(G.ref, G.ang, G.n, p.ctypes.data, v.ctypes.data, 0, 2, None) == 6
    assert tg._Geo(_geo()).g.parallel == 0
