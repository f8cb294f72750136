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
TG_MATCHED, TG_FDK_WEIGHT = 0, 1
TG_RAMLAK = 0
TG_ORDER_SEQUENTIAL, TG_ORDER_RANDOM = 0, 1

_STATUS = {0: "ok", 1: "invalid argument", 2: "invalid geometry", 3: "device out of memory",
           4: "CUDA error", 5: "device wait timed out", 6: "unsupported request"}


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
            "tg_sirt": [G, _DP, ctypes.c_int, _VP, _VP, ctypes.c_int, ctypes.c_float, ctypes.c_int, _DP, _VP],
            "tg_ossart": [G, _DP, ctypes.c_int, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                          ctypes.c_uint64, ctypes.c_float, ctypes.c_int, _DP, _VP],
            "tg_cgls": [G, _DP, ctypes.c_int, _VP, _VP, ctypes.c_int, _DP, _VP],
            "tg_workspace_size": [G, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_size_t)],
            "tg_count_samples": [G, _DP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), _VP],
            "tg_backproject_noalloc": [G, _DP, ctypes.c_int, _VP, _VP, ctypes.c_int, ctypes.c_int, _VP],
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
_METHOD_BP = {"matched": TG_MATCHED, "fdk": TG_FDK_WEIGHT}


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
    """A^T y (matched) or the FDK backprojection: proj [(B,) nA, nv, nu] -> vol."""
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


def fdk(geo, proj, out=None, stream=None):
    """FDK reconstruction (Ram-Lak)."""
    G = _Geo(geo)
    if out is None:
        out = _empty_like_kind(proj, geo.vol_shape)
    _check("tg_fdk", load().tg_fdk(G.ref, G.ang, G.n, _ptr(proj), _ptr(out), TG_RAMLAK, _stream(proj, stream)))
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


def workspace_size(geo, op: str, batch: int = 1, blocksize: int = 20) -> int:
    ops = {"forward": 0, "backproject": 1, "fdk": 2, "sirt": 3, "ossart": 4, "cgls": 5}
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


def launch_count() -> int:
    """Kernel launches libtg has issued in this process."""
    return int(load().tg_launch_count())


def status_string(code: int) -> str:
    return load().tg_status_string(int(code)).decode()


def _sync(t):
    if not isinstance(t, np.ndarray) and t.is_cuda:
        _torch().cuda.current_stream(t.device).synchronize()
