"""GB300 (sm_103a) implementation of the FFT momentum power-spectrum estimator of
Pan (arXiv:2005.06170).

Modules:
    pkmom     - ctypes binding of libpkmom.so (the C-ABI in include/pkmom.h)
    catalogs  - seeded synthetic particle catalogues (inputs only)
    build     - in-tree nvcc build of libpkmom.so for sm_103a

Importing the package loads nothing; ``pkmom.lib()`` loads (and if needed builds)
the CUDA library and raises if it cannot.
"""
__all__ = ["pkmom", "catalogs", "build"]
