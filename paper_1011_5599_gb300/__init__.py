"""GB300-native HyperANF: HyperLogLog neighbourhood-function iteration on CUDA.

The compute path is a C-ABI CUDA library (``include/hanf.h``); this package
holds its sources (``csrc/``), the thin ctypes binding (``hanf``) and the
seeded input generators (``graphs``).  Nothing is imported eagerly so that
the package can be inspected on machines without a GPU.
"""
