"""GB300 (sm_103a) library for the data-parallel hot path of the Astrometric Global Iterative
Solution (Lindegren et al. 2012, arXiv:1112.4139).

The compute lives in libagis.so (CUDA kernels behind the C ABI of include/agis.h); this
package holds the build script and the ctypes binding.
"""
from . import _build  # noqa: F401

__all__ = ["agis", "build"]


def build(force=False):
    """Compile libagis.so for sm_103a in-tree and return its path."""
    return _build.build(force=force)
