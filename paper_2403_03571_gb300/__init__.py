"""GB300-native anisotropic power diagrams (arXiv 2403.03571): C-ABI library
(libapd.so, hand-written sm_103a kernels) with a thin ctypes binding.

``capi`` loads the library lazily and fails loudly when it is missing;
``synth`` draws seeded inputs; ``build`` compiles the library with nvcc.
"""
__all__ = ["capi", "synth", "build"]
