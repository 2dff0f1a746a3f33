"""GB300-native MDFS information-gain scan (arXiv 1811.00631).

The compute path lives in ``csrc/`` (CUDA for sm_103a behind a C ABI declared
in ``include/mdfs.h``); ``mdfs`` is the thin ctypes binding over it and
``synth`` draws the seeded synthetic inputs.  Importing this package does not
load the CUDA library; the first call into ``mdfs`` does, and fails loudly if
the library has not been built.
"""
__all__ = ["mdfs", "synth"]
