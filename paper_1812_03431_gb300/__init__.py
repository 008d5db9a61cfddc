"""GB300-native T-REXI step for the linear shallow-water equations on the rotating sphere.

The compute path is the C-ABI library ``librexi`` (hand-written sm_103a CUDA
kernels plus host plan setup in C++), declared in ``include/rexi.h``.
``paper_1812_03431_gb300.rexi`` is its Python binding; ``inputs`` holds the
seeded synthetic-state generators.  Submodules are imported lazily so that the
input generators can be used without loading the CUDA library.
"""

__all__ = ["rexi", "inputs", "build"]
