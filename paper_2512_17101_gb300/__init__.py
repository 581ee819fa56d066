"""GB300-native nodal DG hot path: libdg.so (CUDA for sm_103a behind a C ABI) and its Python binding.

The binding is loaded lazily: ``from paper_2512_17101_gb300 import dg`` loads
libdg.so and raises ImportError if it has not been built.
"""

__all__ = ["dg", "capi", "build"]
