"""GB300-native cone-beam CT projectors and iterative reconstruction.

The compute path is the CUDA library ``libtg`` (``csrc/``, C ABI declared in
``include/tg.h``); ``tg`` is its thin Python binding (argument marshalling
only; the library is loaded on first use).  ``inputs`` draws seeded
synthetic scans and phantoms.
"""
from . import inputs, tg  # noqa: F401

__all__ = ["inputs", "tg"]
