"""DIST differentiable sphere tracing on NVIDIA B300 (sm_103a).

The compute lives in ``libdist.so`` (hand-written CUDA behind the C ABI of
``include/dist.h``); this package is its thin Python binding.  Importing the
package does not load the library; the first call does, and fails loudly if
it has not been built.
"""

__all__ = ["api", "serve"]
