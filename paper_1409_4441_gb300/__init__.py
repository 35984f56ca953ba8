"""GB300-native compact-kernel spherical convolution (arXiv:1409.4441 hot path).

The compute lives in the CUDA/C++ library ``libksconv.so`` built from ``csrc/``
and declared in ``include/ksconv.h``; ``ksconv`` is its thin ctypes binding.
Importing this package loads nothing: ``inputs`` (seeded synthetic inputs) is
importable on machines without the library or a GPU.
"""

__all__ = ["ksconv", "inputs"]
