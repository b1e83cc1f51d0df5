"""GB300-native gradient anisotropic diffusion for H I cubes (arXiv:1609.03782).

The compute path is ``libafd.so`` (hand-written sm_103a CUDA kernels behind the
C ABI in ``include/afd.h``); ``afd`` is its Python binding.  Build with
``paper_1609_03782_gb300._build.build()``.
"""
__all__ = ["afd"]
