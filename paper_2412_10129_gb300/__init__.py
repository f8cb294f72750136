"""GB300-native cone- and parallel-beam CT projectors, iterative and learned
reconstruction.

The compute path is the CUDA library ``libtg`` (``csrc/``, C ABI declared in
``include/tg.h``); ``tg`` is its thin Python binding (argument marshalling
only; the library is loaded on first use).  ``inputs`` draws seeded
synthetic scans and phantoms; ``autograd`` wraps the projector pair as
``torch.autograd.Function``s; ``learned`` is the learned-gradient scheme;
``build`` compiles the library in-tree; ``probe`` measures the gather and
scatter rates the projectors are reported against.
"""
from . import inputs, tg  # noqa: F401

__all__ = ["inputs", "tg"]
