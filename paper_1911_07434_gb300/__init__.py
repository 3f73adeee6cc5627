"""GB300-native fast-MUSIC angle-of-arrival estimator (arXiv 1911.07434).

The compute path is the C-ABI CUDA library built from ``csrc/`` (see
``include/fastmusic.h``); ``binding`` is a thin ctypes layer over it.  ``synth``
is the seeded synthetic-frame generator.  Submodules are imported lazily so that
``synth`` can be used without the CUDA library.
"""
__all__ = ["binding", "synth"]
