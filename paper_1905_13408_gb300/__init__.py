"""GB300-native reweighted smoothing-proximal-gradient solver for the
regularized real-space refinement objective of Luo, "Improving the resolution
of Cryo-EM single particle analysis" (arXiv 1905.13408), Sec. 2.1-2.5.

The compute path is the CUDA library ``libspg.so`` (C ABI in include/spg.h);
``spg`` is its ctypes binding and ``synth`` the seeded input generator.
Nothing is loaded at import time; the first call into ``spg`` builds (if
needed) and loads the library and raises if it cannot.
"""
__all__ = ["spg", "synth", "build"]
