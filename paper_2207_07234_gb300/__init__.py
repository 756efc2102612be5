"""GB300-native space-time PDHG solver for implicit schemes of scalar
conservation laws (Liu, Osher, Li, Shu, arXiv 2207.07234).

The compute path is the CUDA library ``libpdhg.so`` (C ABI in
``include/pdhg.h``); ``paper_2207_07234_gb300.binding`` is its ctypes
binding (imported explicitly; importing the package itself loads nothing).
"""
