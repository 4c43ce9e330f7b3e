"""GB300 (sm_103a) implementation of fast adaptive bilateral filtering
(Gavaskar & Chaudhury): the C ABI of include/fabf.h backed by hand-written
CUDA kernels, with a thin ctypes binding (``fabf``), the in-tree build
(``build``) and the seeded synthetic inputs (``synth``).

Importing the package does not load the CUDA library; the first call into
``fabf`` does, and raises if it is missing.
"""
__all__ = ["fabf", "build", "synth"]
