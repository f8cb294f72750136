"""Python binding of libtg (include/tg.h): argument marshalling only.

Every function takes a :class:`~paper_2412_10129_gb300.inputs.Geometry` and
torch tensors (CUDA tensors run asynchronously on the current stream; CPU
tensors and numpy arrays are host buffers that libtg stages itself) and calls
the C ABI of the same name.  There is no fallback: if ``lib/libtg.so`` has not
been built, or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libtg.so")

TG_INTERP, TG_SIDDON = 0, 1
TG_MATCHED, TG_FDK_WEIGHT, TG_SIDDON_BP = 0, 1, 2
TG_RAMLAK, TG_SHEPP_LOGAN, TG_COSINE, TG_HAMMING, TG_HANN = 0, 1, 2, 3, 4
FILTERS = {"ram-lak": TG_RAMLAK, "shepp-logan": TG_SHEPP_LOGAN, "cosine": TG_COSINE, "hamming": TG_HAMMING,
           "hann": TG_HANN}
TG_FDK_PARKER, TG_FDK_WANG = 1, 2
TG_ORDER_SEQUENTIAL, TG_ORDER_RANDOM = 0, 1

_STATUS = {0: "ok", 1: "invalid argument", 2: "invalid geometry", 3: "device out of memory",
           4: "CUDA error", 5: "device wait timed out", 6: "unsupported request"}


class _PocsParams(ctypes.Structure):
    _fields_ = [("niter", ctypes.c_int), ("blocksize", ctypes.c_int), ("tv_steps", ctypes.c_int),
                ("alpha", ctypes.c_float), ("alpha_red", ctypes.c_float), ("r_max", ctypes.c_float),
                ("data_tol", ctypes.c_float), ("beta", ctypes.c_float), ("beta_red", ctypes.c_float),
                ("delta", ctypes.c_float), ("eps", ctypes.c_float)]


class TgError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} failed: {_STATUS.get(code, code)} (status {code})")
        self.code = code


class _CGeometry(ctypes.Structure):
    _fields_ = [
        ("nVoxel", ctypes.c_int32 * 3),
        ("dVoxel", ctypes.c_double * 3),
        ("nDetector", ctypes.c_int32 * 2),
        ("dDetector", ctypes.c_double * 2),
        ("accuracy", ctypes.c_double),
        ("DSO0", ctypes.c_double),
        ("DSD0", ctypes.c_double),
        ("DSO", ctypes.POINTER(ctypes.c_double)),
        ("DSD", ctypes.POINTER(ctypes.c_double)),
        ("offOrigin", ctypes.POINTER(ctypes.c_double)),
        ("offDetector", ctypes.POINTER(ctypes.c_double)),
        ("rotDetector", ctypes.POINTER(ctypes.c_double)),
        ("COR", ctypes.POINTER(ctypes.c_double)),
        ("parallel", ctypes.c_int32),
    ]


_lib = None
_DP = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p


def load():
    """Load libtg; raises if it is missing (no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libtg is not built ({LIB_PATH}); run paper_2412_10129_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        G = ctypes.POINTER(_CGeometry)
        sig = {
            "tg_forward": [G, _DP, ctypes.c_int, _VP, _VP, ctypes.c_int, ctypes.c_int, _VP],
            "tg_backproject": [G, _DP, ctypes.c_int, _VP, _VP, ctypes.c_int, ctypes.c_int, _VP],
            "tg_fdk": [G, _DP, ctypes.c_int, _VP, _VP, ctypes.c_int, _VP],
            "tg_fdk_ex": [G, _DP, ctypes.c_int, _VP, _VP, ctypes.c_int, ctypes.c_int, _VP],
            "tg_fdk_filter": [G, _DP, ctypes.c_int, _VP, _VP, ctypes.c_int, ctypes.c_int, _VP],
            "tg_sirt": [G, _DP, ctypes.c_int, _VP, _VP, ctypes.c_int, ctypes.c_float, ctypes.c_int, _DP, _VP],
            "tg_ossart": [G, _DP, ctypes.c_int, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                          ctypes.c_uint64, ctypes.c_float, ctypes.c_int, _DP, _VP],
            "tg_cgls": [G, _DP, ctypes.c_int, _VP, _VP, ctypes.c_int, _DP, _VP],
            "tg_mlem": [G, _DP, ctypes.c_int, _VP, _VP, ctypes.c_int, ctypes.c_int, _DP, _VP],
            "tg_lsqr": [G, _DP, ctypes.c_int, _VP, _VP, ctypes.c_int, _DP, _VP],
            "tg_lsmr": [G, _DP, ctypes.c_int, _VP, _VP, ctypes.c_int, _DP, _VP],
            "tg_asd_pocs": [G, _DP, ctypes.c_int, _VP, _VP, ctypes.POINTER(_PocsParams), _DP, _VP],
            "tg_tv_gradient": [_VP, _VP, ctypes.POINTER(ctypes.c_int32), ctypes.c_float, ctypes.c_float, _VP],
            "tg_tv_descent": [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.c_int, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, _VP],
            "tg_osem": [G, _DP, ctypes.c_int, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                        ctypes.c_int, _DP, _VP],
            "tg_workspace_size": [G, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_size_t)],
            "tg_count_samples": [G, _DP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), _VP],
            "tg_backproject_noalloc": [G, _DP, ctypes.c_int, _VP, _VP, ctypes.c_int, ctypes.c_int, _VP],
            "tg_gradient": [G, _DP, ctypes.c_int, _VP, _VP, _VP, ctypes.c_int, ctypes.c_int, _VP],
            "tg_conv3d_forward": [_VP, _VP, _VP, _VP] + [ctypes.c_int] * 8 + [_VP],
            "tg_conv3d_forward_ragged": [_VP, _VP, _VP, _VP, ctypes.POINTER(ctypes.c_int32)] + [ctypes.c_int] * 5
                                        + [_VP],
            "tg_conv3d_backward_data": [_VP, _VP, _VP] + [ctypes.c_int] * 6 + [_VP],
            "tg_conv3d_backward_weight": [_VP, _VP, _VP] + [ctypes.c_int] * 6 + [_VP],
            "tg_conv3d_backward_bias": [_VP, _VP, ctypes.c_size_t, ctypes.c_int, _VP],
            "tg_relu_backward": [_VP, _VP, _VP, ctypes.c_size_t, _VP],
            "tg_lg_pack": [_VP, _VP, _VP, ctypes.c_size_t, ctypes.c_int, ctypes.c_float, ctypes.c_float, _VP],
            "tg_lg_unpack": [_VP, ctypes.c_int, _VP, _VP, ctypes.c_size_t, ctypes.c_float, ctypes.c_float,
                             ctypes.c_int, _VP],
            "tg_lg_update": [_VP, _VP, _VP, ctypes.c_size_t, ctypes.c_int, ctypes.c_float, _VP],
            "tg_grad_split": [_VP, _VP, _VP, _VP, ctypes.c_size_t, _VP],
            "tg_lg_pack_split": [_VP, _VP, _VP, ctypes.c_size_t, ctypes.c_int, ctypes.c_float, _VP],
            "tg_lg_unpack_f32": [_VP, ctypes.c_int, _VP, _VP, ctypes.c_size_t, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_int, _VP],
            "tg_conv3d_backward_data_split": [_VP, _VP, _VP, _VP] + [ctypes.c_int] * 6 + [_VP],
            "tg_conv3d_backward_weight_split": [_VP, _VP, _VP, _VP] + [ctypes.c_int] * 6 + [_VP],
            "tg_conv3d_backward_bias_split": [_VP, _VP, _VP, ctypes.c_size_t, ctypes.c_int, _VP],
            "tg_device_status": [_VP],
            "tg_test_conv_wait": [ctypes.c_int, ctypes.c_longlong],
            "tg_kernel_timing": [ctypes.c_int],
            "tg_kernel_timing_read": [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)],
            "tg_forward_batched": [G, ctypes.POINTER(_DP), ctypes.POINTER(ctypes.c_int), ctypes.c_int, _VP, _VP, _VP],
            "tg_backproject_batched": [G, ctypes.POINTER(_DP), ctypes.POINTER(ctypes.c_int), ctypes.c_int, _VP, _VP,
                                       _VP],
            "tg_gradient_batched": [G, ctypes.POINTER(_DP), ctypes.POINTER(ctypes.c_int), ctypes.c_int, _VP, _VP, _VP,
                                    ctypes.c_int, _VP],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.tg_status_string.argtypes = [ctypes.c_int]
        lib.tg_status_string.restype = ctypes.c_char_p
        lib.tg_launch_count.argtypes = []
        lib.tg_launch_count.restype = ctypes.c_uint64
        _lib = lib
    return _lib


class _Geo:
    """tg_geometry plus the FP64 arrays it points into (kept alive)."""

    def __init__(self, geo):
        n = int(geo.nAngles)
        c = lambda a, shape: np.ascontiguousarray(np.asarray(a, np.float64).reshape(shape))  # noqa: E731
        self.angles = c(geo.angles, (n, 3))
        self.arrs = [c(geo.DSO, (n,)), c(geo.DSD, (n,)), c(geo.offOrigin, (n, 3)), c(geo.offDetector, (n, 2)),
                     c(geo.rotDetector, (n, 3)), c(geo.COR, (n,))]
        g = _CGeometry()
        g.nVoxel[:] = [int(v) for v in geo.nVoxel]
        g.dVoxel[:] = [float(v) for v in geo.dVoxel]
        g.nDetector[:] = [int(v) for v in geo.nDetector]
        g.dDetector[:] = [float(v) for v in geo.dDetector]
        g.accuracy = float(geo.accuracy)
        g.DSO0 = float(self.arrs[0][0]) if n else 1000.0
        g.DSD0 = float(self.arrs[1][0]) if n else 1536.0
        for name, arr in zip(("DSO", "DSD", "offOrigin", "offDetector", "rotDetector", "COR"), self.arrs):
            setattr(g, name, arr.ctypes.data_as(_DP))
        g.parallel = 1 if getattr(geo, "parallel", False) else 0
        self.g = g
        self.n = n

    @property
    def ref(self):
        return ctypes.byref(self.g)

    @property
    def ang(self):
        return self.angles.ctypes.data_as(_DP)


def _check(fn, code):
    if code != 0:
        raise TgError(fn, code)


def _torch():
    import torch
    return torch


def _ptr(t):
    """Data pointer of a contiguous float32 tensor / array."""
    if isinstance(t, np.ndarray):
        if t.dtype != np.float32 or not t.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a C-contiguous float32 array")
        return t.ctypes.data
    if t.dtype != _torch().float32 or not t.is_contiguous():
        raise ValueError("expected a contiguous float32 tensor")
    return t.data_ptr()


def _stream(t, stream):
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    if not isinstance(t, np.ndarray) and t.is_cuda:
        return _torch().cuda.current_stream(t.device).cuda_stream
    return None


def _empty_like_kind(ref, shape):
    if isinstance(ref, np.ndarray):
        return np.empty(shape, np.float32)
    return _torch().empty(shape, dtype=_torch().float32, device=ref.device)


def _batch(x, base_ndim):
    if x.ndim == base_ndim:
        return 1, False
    if x.ndim == base_ndim + 1:
        return int(x.shape[0]), True
    raise ValueError(f"expected {base_ndim} or {base_ndim + 1} dimensions, got {x.ndim}")


_METHOD_FP = {"interp": TG_INTERP, "siddon": TG_SIDDON}
_METHOD_BP = {"matched": TG_MATCHED, "fdk": TG_FDK_WEIGHT, "siddon": TG_SIDDON_BP}


def forward(geo, vol, method: str = "interp", out=None, stream=None):
    """A x: vol [(B,) nz, ny, nx] -> proj [(B,) nA, nv, nu]."""
    G = _Geo(geo)
    B, batched = _batch(vol, 3)
    shape = ((B,) if batched else ()) + tuple(geo.proj_shape)
    if out is None:
        out = _empty_like_kind(vol, shape)
    _check("tg_forward", load().tg_forward(G.ref, G.ang, G.n, _ptr(vol), _ptr(out), _METHOD_FP[method], B,
                                           _stream(vol, stream)))
    return out


def backproject(geo, proj, method: str = "matched", out=None, stream=None):
    """A^T y (matched: transpose of the interpolated projector; siddon: of
    the Siddon projector) or the FDK backprojection: proj [(B,) nA, nv, nu] -> vol."""
    G = _Geo(geo)
    B, batched = _batch(proj, 3)
    shape = ((B,) if batched else ()) + tuple(geo.vol_shape)
    if out is None:
        out = _empty_like_kind(proj, shape)
    _check("tg_backproject", load().tg_backproject(G.ref, G.ang, G.n, _ptr(proj), _ptr(out), _METHOD_BP[method], B,
                                                   _stream(proj, stream)))
    return out


def backproject_noalloc(geo, proj, method: str = "matched", out=None, stream=None):
    """tg_backproject_noalloc: the backprojection for callers that cannot
    allocate device memory.  ``proj`` (and ``out``, if given) must be CUDA
    tensors; the library allocates nothing (its scratch is a static device
    array), so calls that overlap on the GPU must be serialised."""
    G = _Geo(geo)
    B, batched = _batch(proj, 3)
    shape = ((B,) if batched else ()) + tuple(geo.vol_shape)
    if out is None:
        out = _empty_like_kind(proj, shape)
    _check("tg_backproject_noalloc", load().tg_backproject_noalloc(G.ref, G.ang, G.n, _ptr(proj), _ptr(out),
                                                                   _METHOD_BP[method], B, _stream(proj, stream)))
    return out


def gradient(geo, vol, proj=None, out=None, accumulate: bool = False, stream=None):
    """A^T (A x - b) (Eq. 4's data-fit gradient; b = 0 when ``proj`` is None):
    vol [(B,) nz, ny, nx] -> [(B,) nz, ny, nx]; ``accumulate`` adds into ``out``."""
    G = _Geo(geo)
    B, batched = _batch(vol, 3)
    if out is None:
        if accumulate:
            raise ValueError("accumulate needs out")
        out = _empty_like_kind(vol, vol.shape)
    _check("tg_gradient", load().tg_gradient(G.ref, G.ang, G.n, _ptr(vol), None if proj is None else _ptr(proj),
                                             _ptr(out), int(bool(accumulate)), B, _stream(vol, stream)))
    return out


class _Geos:
    """An array of tg_geometry (and the arrays they point into) for the
    *_batched calls."""

    def __init__(self, geos):
        self.items = [_Geo(g) for g in geos]
        n = len(self.items)
        self.arr = (_CGeometry * n)(*[it.g for it in self.items])
        self.angles = (_DP * n)(*[it.ang for it in self.items])
        self.nang = (ctypes.c_int * n)(*[it.n for it in self.items])
        self.n = n


def _packed_sizes(geos, which):
    if which == "vol":
        return [int(np.prod(g.vol_shape)) for g in geos]
    return [int(np.prod(g.proj_shape)) for g in geos]


def forward_batched(geos, vol, out=None, stream=None):
    """A_v x_v for volumes of different geometries in one launch: ``vol`` is
    the packed FP32 CUDA buffer of all volumes (back to back), the result the
    packed projection sets."""
    G = _Geos(geos)
    if out is None:
        out = _torch().empty(sum(_packed_sizes(geos, "proj")), dtype=_torch().float32, device=vol.device)
    _check("tg_forward_batched", load().tg_forward_batched(G.arr, G.angles, G.nang, G.n, _ptr(vol), _ptr(out),
                                                           _stream(vol, stream)))
    return out


def backproject_batched(geos, proj, out=None, stream=None):
    """A_v^T y_v (matched) for volumes of different geometries, packed buffers."""
    G = _Geos(geos)
    if out is None:
        out = _torch().empty(sum(_packed_sizes(geos, "vol")), dtype=_torch().float32, device=proj.device)
    _check("tg_backproject_batched", load().tg_backproject_batched(G.arr, G.angles, G.nang, G.n, _ptr(proj),
                                                                   _ptr(out), _stream(proj, stream)))
    return out


def gradient_batched(geos, vol, proj=None, out=None, accumulate: bool = False, stream=None):
    """A_v^T (A_v x_v - b_v) for volumes of different geometries (packed)."""
    G = _Geos(geos)
    if out is None:
        if accumulate:
            raise ValueError("accumulate needs out")
        out = _torch().empty_like(vol)
    _check("tg_gradient_batched", load().tg_gradient_batched(
        G.arr, G.angles, G.nang, G.n, _ptr(vol), None if proj is None else _ptr(proj), _ptr(out),
        int(bool(accumulate)), _stream(vol, stream)))
    return out


def _fdk_options(filter, parker, wang):
    if filter not in FILTERS:
        raise ValueError(f"unknown filter {filter!r}; one of {sorted(FILTERS)}")
    return FILTERS[filter], (TG_FDK_PARKER if parker else 0) | (TG_FDK_WANG if wang else 0)


def fdk(geo, proj, filter: str = "ram-lak", parker: bool = False, wang: bool = False, out=None, stream=None):
    """FDK reconstruction (tg_fdk_ex): cosine pre-weight, optional Parker
    (short scan) or Wang (displaced detector) weights, row filter ``filter``
    (ram-lak, shepp-logan, cosine, hamming, hann), weighted backprojection."""
    G = _Geo(geo)
    f, w = _fdk_options(filter, parker, wang)
    if out is None:
        out = _empty_like_kind(proj, geo.vol_shape)
    _check("tg_fdk_ex", load().tg_fdk_ex(G.ref, G.ang, G.n, _ptr(proj), _ptr(out), f, w, _stream(proj, stream)))
    return out


def fdk_filter(geo, proj, filter: str = "ram-lak", parker: bool = False, wang: bool = False, out=None,
               stream=None):
    """The pre-weighted, row-filtered projections of tg_fdk_ex (tg_fdk_filter)."""
    G = _Geo(geo)
    f, w = _fdk_options(filter, parker, wang)
    if out is None:
        out = _empty_like_kind(proj, geo.proj_shape)
    _check("tg_fdk_filter", load().tg_fdk_filter(G.ref, G.ang, G.n, _ptr(proj), _ptr(out), f, w,
                                                 _stream(proj, stream)))
    return out


def _x0(geo, proj, x0):
    if x0 is not None:
        return x0
    if isinstance(proj, np.ndarray):
        return np.zeros(geo.vol_shape, np.float32)
    return _torch().zeros(geo.vol_shape, dtype=_torch().float32, device=proj.device)


def _hist(niter, want):
    if not want:
        return None, None
    h = np.zeros(max(niter, 1), np.float64)
    return h, h.ctypes.data_as(_DP)


def sirt(geo, proj, niter: int, x0=None, lam: float = 1.0, nonneg: bool = True, resid: bool = False, stream=None):
    """SIRT; returns x (and the residual history when ``resid``)."""
    G = _Geo(geo)
    x = _x0(geo, proj, x0)
    h, hp = _hist(niter, resid)
    _check("tg_sirt", load().tg_sirt(G.ref, G.ang, G.n, _ptr(proj), _ptr(x), int(niter), float(lam), int(bool(nonneg)),
                                     hp, _stream(proj, stream)))
    if resid:
        _sync(proj)
        return x, h[:niter]
    return x


def ossart(geo, proj, niter: int, blocksize: int = 20, order: str = "sequential", seed: int = 0, x0=None,
           lam: float = 1.0, nonneg: bool = True, resid: bool = False, stream=None):
    """OS-SART; returns x (and the residual history when ``resid``)."""
    G = _Geo(geo)
    x = _x0(geo, proj, x0)
    h, hp = _hist(niter, resid)
    o = {"sequential": TG_ORDER_SEQUENTIAL, "random": TG_ORDER_RANDOM}[order]
    _check("tg_ossart", load().tg_ossart(G.ref, G.ang, G.n, _ptr(proj), _ptr(x), int(niter), int(blocksize), o,
                                         int(seed), float(lam), int(bool(nonneg)), hp, _stream(proj, stream)))
    if resid:
        _sync(proj)
        return x, h[:niter]
    return x


def cgls(geo, proj, niter: int, x0=None, resid: bool = False, stream=None):
    """CGLS; returns x (and the recurrence residual history when ``resid``)."""
    G = _Geo(geo)
    x = _x0(geo, proj, x0)
    h, hp = _hist(niter, resid)
    _check("tg_cgls", load().tg_cgls(G.ref, G.ang, G.n, _ptr(proj), _ptr(x), int(niter), hp, _stream(proj, stream)))
    if resid:
        _sync(proj)
        return x, h[:niter]
    return x


def lsqr(geo, proj, niter: int, x0=None, resid: bool = False, stream=None):
    """LSQR; returns x (and the recurrence's ||b - A x_k|| when ``resid``)."""
    G = _Geo(geo)
    x = _x0(geo, proj, x0)
    h, hp = _hist(niter, resid)
    _check("tg_lsqr", load().tg_lsqr(G.ref, G.ang, G.n, _ptr(proj), _ptr(x), int(niter), hp, _stream(proj, stream)))
    if resid:
        _sync(proj)
        return x, h[:niter]
    return x


def lsmr(geo, proj, niter: int, x0=None, resid: bool = False, stream=None):
    """LSMR; returns x (and ||A x_k - b|| when ``resid``)."""
    G = _Geo(geo)
    x = _x0(geo, proj, x0)
    h, hp = _hist(niter, resid)
    _check("tg_lsmr", load().tg_lsmr(G.ref, G.ang, G.n, _ptr(proj), _ptr(x), int(niter), hp, _stream(proj, stream)))
    if resid:
        _sync(proj)
        return x, h[:niter]
    return x


def _ones_like_vol(geo, proj):
    if isinstance(proj, np.ndarray):
        return np.ones(geo.vol_shape, np.float32)
    return _torch().ones(geo.vol_shape, dtype=_torch().float32, device=proj.device)


def mlem(geo, proj, niter: int, x0=None, method: str = "interp", resid: bool = False, stream=None):
    """MLEM (Eq. 5) with the (interp, matched) or (siddon, siddon transpose)
    pair; x0 = 1 unless given.  Returns x (and the residual history)."""
    G = _Geo(geo)
    x = x0 if x0 is not None else _ones_like_vol(geo, proj)
    h, hp = _hist(niter, resid)
    _check("tg_mlem", load().tg_mlem(G.ref, G.ang, G.n, _ptr(proj), _ptr(x), int(niter), _METHOD_FP[method], hp,
                                     _stream(proj, stream)))
    if resid:
        _sync(proj)
        return x, h[:niter]
    return x


def osem(geo, proj, niter: int, blocksize: int = 20, order: str = "sequential", seed: int = 0, x0=None,
         method: str = "interp", resid: bool = False, stream=None):
    """OS-EM: MLEM updates over blocks of consecutive angles."""
    G = _Geo(geo)
    x = x0 if x0 is not None else _ones_like_vol(geo, proj)
    h, hp = _hist(niter, resid)
    o = {"sequential": TG_ORDER_SEQUENTIAL, "random": TG_ORDER_RANDOM}[order]
    _check("tg_osem", load().tg_osem(G.ref, G.ang, G.n, _ptr(proj), _ptr(x), int(niter), int(blocksize), o,
                                     int(seed), _METHOD_FP[method], hp, _stream(proj, stream)))
    if resid:
        _sync(proj)
        return x, h[:niter]
    return x


def asd_pocs(geo, proj, niter: int, blocksize: int = 1, tv_steps: int = 20, alpha: float = 0.002,
             alpha_red: float = 0.95, r_max: float = 0.95, data_tol: float = 0.0, beta: float = 1.0,
             beta_red: float = 0.995, delta: float = float("inf"), eps: float = 1e-8, x0=None,
             resid: bool = False, stream=None):
    """ASD-POCS (blocksize 1) / OS-ASD-POCS with plain TV or AwTV (finite
    ``delta``); returns x (and ||A x_k - b|| after each data step)."""
    G = _Geo(geo)
    x = _x0(geo, proj, x0)
    h, hp = _hist(niter, resid)
    P = _PocsParams(int(niter), int(blocksize), int(tv_steps), alpha, alpha_red, r_max, data_tol, beta, beta_red,
                    delta, eps)
    _check("tg_asd_pocs", load().tg_asd_pocs(G.ref, G.ang, G.n, _ptr(proj), _ptr(x), ctypes.byref(P), hp,
                                             _stream(proj, stream)))
    if resid:
        _sync(proj)
        return x, h[:niter]
    return x


def _dims(vol):
    nz, ny, nx = vol.shape[-3:]
    return (ctypes.c_int32 * 3)(int(nx), int(ny), int(nz))


def tv_gradient(vol, delta: float = float("inf"), eps: float = 1e-8, out=None, stream=None):
    """Gradient of (Aw)TV with frozen weights; CUDA tensors [nz, ny, nx]."""
    if out is None:
        out = _torch().empty_like(vol)
    _check("tg_tv_gradient", load().tg_tv_gradient(_ptr(vol), _ptr(out), _dims(vol), delta, eps,
                                                   _stream(vol, stream)))
    return out


def tv_descent(vol, steps: int, step: float, delta: float = float("inf"), eps: float = 1e-8, stream=None):
    """``steps`` normalised (Aw)TV descent steps on a CUDA tensor, in place."""
    _check("tg_tv_descent", load().tg_tv_descent(_ptr(vol), _dims(vol), int(steps), step, delta, eps,
                                                 _stream(vol, stream)))
    return vol


def workspace_size(geo, op: str, batch: int = 1, blocksize: int = 20) -> int:
    ops = {"forward": 0, "backproject": 1, "fdk": 2, "sirt": 3, "ossart": 4, "cgls": 5, "mlem": 6, "osem": 7,
           "asd_pocs": 8, "lsqr": 9, "lsmr": 10}
    G = _Geo(geo)
    out = ctypes.c_size_t(0)
    _check("tg_workspace_size", load().tg_workspace_size(G.ref, G.n, ops[op], int(batch), int(blocksize),
                                                         ctypes.byref(out)))
    return int(out.value)


def count_samples(geo, method: str = "interp", stream=None) -> int:
    """Samples (interp) or voxel segments (siddon) of one forward projection."""
    G = _Geo(geo)
    out = ctypes.c_uint64(0)
    s = getattr(stream, "cuda_stream", stream)
    _check("tg_count_samples", load().tg_count_samples(G.ref, G.ang, G.n, _METHOD_FP[method], ctypes.byref(out), s))
    return int(out.value)


def device_status(stream=None) -> None:
    """Waits for the stream and raises TgError(TG_ERR_TIMEOUT) when a
    bounded device-side wait of the tensor-core kernels gave up."""
    torch = _torch()
    st = getattr(stream, "cuda_stream", stream)
    if st is None and torch.cuda.is_available():
        st = torch.cuda.current_stream().cuda_stream
    _check("tg_device_status", load().tg_device_status(st))


def test_conv_wait(stall: bool, budget_cycles: int = 0) -> None:
    """tg_test_conv_wait: test hook of the tensor-core convolutions' bounded
    waits (budget in SM clocks, 0 = default; ``stall`` makes their epilogue
    wait on a barrier that nothing arrives at)."""
    _check("tg_test_conv_wait", load().tg_test_conv_wait(1 if stall else 0, int(budget_cycles)))


KERNEL_CLASSES = {"fp_interp": 0, "fp_siddon": 1, "bp_matched": 2, "bp_fdk": 3, "bp_siddon": 4, "fdk_filter": 5,
                  "bp_matched_split": 6}


def kernel_timing(enable: bool) -> None:
    """tg_kernel_timing: start (or stop) recording per-kernel launch times; clears the totals."""
    _check("tg_kernel_timing", load().tg_kernel_timing(1 if enable else 0))


def kernel_timing_read() -> dict:
    """tg_kernel_timing_read for every class: {name: (total ms, launches)}."""
    out = {}
    for name, cls in KERNEL_CLASSES.items():
        ms, n = ctypes.c_double(), ctypes.c_uint64()
        _check("tg_kernel_timing_read", load().tg_kernel_timing_read(cls, ctypes.byref(ms), ctypes.byref(n)))
        out[name] = (ms.value, int(n.value))
    return out


def launch_count() -> int:
    """Kernel launches libtg has issued in this process."""
    return int(load().tg_launch_count())


def status_string(code: int) -> str:
    return load().tg_status_string(int(code)).decode()


def _sync(t):
    if not isinstance(t, np.ndarray) and t.is_cuda:
        _torch().cuda.current_stream(t.device).synchronize()


# ---------------------------------------------------------------------------
# Learned-gradient network kernels: activations are bfloat16 CUDA tensors,
# channels last [n, nz, ny, nx, c]; weights float32 [27, cout, cin].
# ---------------------------------------------------------------------------

def _dptr(t, dtype):
    """Data pointer of a contiguous CUDA tensor of the given torch dtype."""
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"expected a contiguous CUDA tensor of {dtype}")
    return t.data_ptr()


def _cs(t, stream):
    return _stream(t, stream)


def conv3d(x, w, bias=None, relu: bool = False, out_f32: bool = False, out=None, accumulate: bool = False,
           stream=None):
    """tg_conv3d_forward: x [n, nz, ny, nx, cin] bf16 -> [n, nz, ny, nx, cout]
    (FP32 with ``out_f32``; ``accumulate`` adds the result to the FP32 ``out``)."""
    torch = _torch()
    n, nz, ny, nx, cin = x.shape
    cout = int(w.shape[1])
    if tuple(w.shape) != (27, cout, cin):
        raise ValueError("weights must be [27, cout, cin]")
    if accumulate and (out is None or relu):
        raise ValueError("accumulate needs an FP32 out and no ReLU")
    f32 = bool(out_f32) or bool(accumulate)
    if out is None:
        out = torch.empty((n, nz, ny, nx, cout), dtype=torch.float32 if f32 else torch.bfloat16, device=x.device)
    _check("tg_conv3d_forward", load().tg_conv3d_forward(
        _dptr(x, torch.bfloat16), _dptr(w, torch.float32), None if bias is None else _dptr(bias, torch.float32),
        _dptr(out, torch.float32 if f32 else torch.bfloat16), n, nz, ny, nx, cin, cout, int(bool(relu)),
        2 if accumulate else int(f32), _cs(x, stream)))
    return out


def conv3d_ragged(x, dims, w, bias=None, relu: bool = False, out_f32: bool = False, out=None, stream=None):
    """tg_conv3d_forward_ragged: volumes of sizes ``dims`` [(nz, ny, nx), ...]
    packed back to back in x [sum voxels, cin] (bf16) -> [sum voxels, cout]."""
    torch = _torch()
    cout, cin = int(w.shape[1]), int(w.shape[2])
    d = np.ascontiguousarray(np.asarray(dims, np.int32).reshape(-1, 3))
    nvox = int(np.sum(np.prod(d.astype(np.int64), axis=1)))
    if x.numel() != nvox * cin:
        raise ValueError("x does not hold the voxels of dims")
    if out is None:
        out = torch.empty((nvox, cout), dtype=torch.float32 if out_f32 else torch.bfloat16, device=x.device)
    _check("tg_conv3d_forward_ragged", load().tg_conv3d_forward_ragged(
        _dptr(x, torch.bfloat16), _dptr(w, torch.float32), None if bias is None else _dptr(bias, torch.float32),
        _dptr(out, torch.float32 if out_f32 else torch.bfloat16), d.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
        int(d.shape[0]), cin, cout, int(bool(relu)), int(bool(out_f32)), _cs(x, stream)))
    return out


def conv3d_backward_data(gy, w, out=None, stream=None):
    """tg_conv3d_backward_data: gy [n, nz, ny, nx, cout] bf16 -> gx [.., cin] bf16."""
    torch = _torch()
    n, nz, ny, nx, cout = gy.shape
    cin = int(w.shape[2])
    if out is None:
        out = torch.empty((n, nz, ny, nx, cin), dtype=torch.bfloat16, device=gy.device)
    _check("tg_conv3d_backward_data", load().tg_conv3d_backward_data(
        _dptr(gy, torch.bfloat16), _dptr(w, torch.float32), _dptr(out, torch.bfloat16), n, nz, ny, nx, cin, cout,
        _cs(gy, stream)))
    return out


def conv3d_backward_weight(x, gy, out=None, stream=None):
    """tg_conv3d_backward_weight: dw [27, cout, cin] float32."""
    torch = _torch()
    n, nz, ny, nx, cin = x.shape
    cout = int(gy.shape[4])
    if out is None:
        out = torch.empty((27, cout, cin), dtype=torch.float32, device=x.device)
    _check("tg_conv3d_backward_weight", load().tg_conv3d_backward_weight(
        _dptr(x, torch.bfloat16), _dptr(gy, torch.bfloat16), _dptr(out, torch.float32), n, nz, ny, nx, cin, cout,
        _cs(x, stream)))
    return out


def conv3d_backward_bias(gy, out=None, stream=None):
    """tg_conv3d_backward_bias: db [cout] float32."""
    torch = _torch()
    cout = int(gy.shape[-1])
    if out is None:
        out = torch.empty((cout,), dtype=torch.float32, device=gy.device)
    _check("tg_conv3d_backward_bias", load().tg_conv3d_backward_bias(
        _dptr(gy, torch.bfloat16), _dptr(out, torch.float32), gy.numel() // cout, cout, _cs(gy, stream)))
    return out


def relu_backward(g, act, out=None, stream=None):
    """tg_relu_backward (bf16); ``out`` may be ``g``."""
    torch = _torch()
    if out is None:
        out = torch.empty_like(g)
    _check("tg_relu_backward", load().tg_relu_backward(
        _dptr(g, torch.bfloat16), _dptr(act, torch.bfloat16), _dptr(out, torch.bfloat16), g.numel(), _cs(g, stream)))
    return out


def lg_pack(x, grad, channels: int, sx: float = 1.0, sg: float = 1.0, out=None, stream=None):
    """tg_lg_pack: FP32 volume(s) -> bf16 [..., channels] = (sx x, sg grad, 0, ...)."""
    torch = _torch()
    if out is None:
        out = torch.empty(tuple(x.shape) + (channels,), dtype=torch.bfloat16, device=x.device)
    _check("tg_lg_pack", load().tg_lg_pack(
        _dptr(x, torch.float32), None if grad is None else _dptr(grad, torch.float32), _dptr(out, torch.bfloat16),
        x.numel(), int(channels), float(sx), float(sg), _cs(x, stream)))
    return out


def lg_unpack(t, a, b=None, sa: float = 1.0, sb: float = 1.0, accumulate: bool = False, stream=None):
    """tg_lg_unpack: a (=|+=) sa t[..., 0]; b = sb t[..., 1]."""
    torch = _torch()
    _check("tg_lg_unpack", load().tg_lg_unpack(
        _dptr(t, torch.bfloat16), int(t.shape[-1]), _dptr(a, torch.float32),
        None if b is None else _dptr(b, torch.float32), a.numel(), float(sa), float(sb), int(bool(accumulate)),
        _cs(t, stream)))
    return a


def grad_split(g, act=None, out=None, stream=None):
    """tg_grad_split: FP32 gradient g -> (hi, lo) bf16 with hi + lo = m g,
    m the ReLU mask act > 0 (1 without ``act``)."""
    torch = _torch()
    if out is None:
        out = (torch.empty(g.shape, dtype=torch.bfloat16, device=g.device),
               torch.empty(g.shape, dtype=torch.bfloat16, device=g.device))
    hi, lo = out
    if act is not None and act.shape != g.shape:
        raise ValueError("act must have the shape of g")
    _check("tg_grad_split", load().tg_grad_split(
        _dptr(g, torch.float32), None if act is None else _dptr(act, torch.bfloat16), _dptr(hi, torch.bfloat16),
        _dptr(lo, torch.bfloat16), g.numel(), _cs(g, stream)))
    return hi, lo


def lg_pack_split(x, channels: int, s: float = 1.0, stream=None):
    """tg_lg_pack_split: FP32 volume(s) -> (hi, lo) bf16 [..., channels] with
    hi + lo = (s x, 0, ..., 0)."""
    torch = _torch()
    shape = tuple(x.shape) + (channels,)
    hi = torch.empty(shape, dtype=torch.bfloat16, device=x.device)
    lo = torch.empty(shape, dtype=torch.bfloat16, device=x.device)
    _check("tg_lg_pack_split", load().tg_lg_pack_split(
        _dptr(x, torch.float32), _dptr(hi, torch.bfloat16), _dptr(lo, torch.bfloat16), x.numel(), int(channels),
        float(s), _cs(x, stream)))
    return hi, lo


def lg_unpack_f32(t, a, b=None, sa: float = 1.0, sb: float = 1.0, accumulate: bool = False, stream=None):
    """tg_lg_unpack_f32: a (=|+=) sa t[..., 0]; b = sb t[..., 1] (t FP32)."""
    torch = _torch()
    _check("tg_lg_unpack_f32", load().tg_lg_unpack_f32(
        _dptr(t, torch.float32), int(t.shape[-1]), _dptr(a, torch.float32),
        None if b is None else _dptr(b, torch.float32), a.numel(), float(sa), float(sb), int(bool(accumulate)),
        _cs(t, stream)))
    return a


def conv3d_backward_data_split(hi, lo, w, out=None, stream=None):
    """tg_conv3d_backward_data_split: gy = hi + lo [n, nz, ny, nx, cout] bf16
    pair -> gx [.., cin] FP32."""
    torch = _torch()
    n, nz, ny, nx, cout = hi.shape
    cin = int(w.shape[2])
    if lo.shape != hi.shape:
        raise ValueError("hi and lo must have one shape")
    if out is None:
        out = torch.empty((n, nz, ny, nx, cin), dtype=torch.float32, device=hi.device)
    _check("tg_conv3d_backward_data_split", load().tg_conv3d_backward_data_split(
        _dptr(hi, torch.bfloat16), _dptr(lo, torch.bfloat16), _dptr(w, torch.float32), _dptr(out, torch.float32), n,
        nz, ny, nx, cin, cout, _cs(hi, stream)))
    return out


def conv3d_backward_weight_split(x, hi, lo, out=None, stream=None):
    """tg_conv3d_backward_weight_split: dw [27, cout, cin] FP32 for gy = hi + lo."""
    torch = _torch()
    n, nz, ny, nx, cin = x.shape
    cout = int(hi.shape[4])
    if lo.shape != hi.shape:
        raise ValueError("hi and lo must have one shape")
    if out is None:
        out = torch.empty((27, cout, cin), dtype=torch.float32, device=x.device)
    _check("tg_conv3d_backward_weight_split", load().tg_conv3d_backward_weight_split(
        _dptr(x, torch.bfloat16), _dptr(hi, torch.bfloat16), _dptr(lo, torch.bfloat16), _dptr(out, torch.float32), n,
        nz, ny, nx, cin, cout, _cs(x, stream)))
    return out


def conv3d_backward_bias_split(hi, lo, out=None, stream=None):
    """tg_conv3d_backward_bias_split: db [cout] FP32 for gy = hi + lo."""
    torch = _torch()
    cout = int(hi.shape[-1])
    if out is None:
        out = torch.empty((cout,), dtype=torch.float32, device=hi.device)
    _check("tg_conv3d_backward_bias_split", load().tg_conv3d_backward_bias_split(
        _dptr(hi, torch.bfloat16), _dptr(lo, torch.bfloat16), _dptr(out, torch.float32), hi.numel() // cout, cout,
        _cs(hi, stream)))
    return out


def lg_update(x, net, so: float = 1.0, out=None, stream=None):
    """tg_lg_update: x + so net[..., 0] (FP32); ``out`` may be ``x``."""
    torch = _torch()
    if out is None:
        out = torch.empty_like(x)
    _check("tg_lg_update", load().tg_lg_update(
        _dptr(x, torch.float32), _dptr(net, torch.float32), _dptr(out, torch.float32), x.numel(), int(net.shape[-1]),
        float(so), _cs(x, stream)))
    return out
