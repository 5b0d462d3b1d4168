"""GB300-native solver for the radial step of the neutrino bulb model (arXiv:1912.10596).

The compute path is libxflat.so (CUDA, sm_103a) behind the C ABI in include/xflat.h; the Python
module ``paper_1912_10596_gb300.xflat`` is a ctypes binding of it.  Build with
``paper_1912_10596_gb300.build.build()``.
"""
