"""GB300-native cone-beam CT projectors and iterative reconstruction.

The compute path is the CUDA library ``libtg`` (``csrc/``, C-ABI declared in
``include/tg.h``); ``tg`` is its thin Python binding (argument marshalling
only).  ``inputs`` draws seeded synthetic scans and phantoms.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "tg"]


def __getattr__(name):
    if name == "tg":
        from . import tg as _tg
        return _tg
    raise AttributeError(name)
