"""GB300-native tight-binding eigen-solver and Schrödinger–Poisson hot path (OMEN 3-D method).

The compute path is the CUDA library libomen.so (C ABI in include/omen.h); `omen` is its
ctypes binding.  Import `paper_1003_4570_gb300.omen` to use it.
"""
