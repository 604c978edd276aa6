"""B300-native KCM step (Protofold II): C-ABI library `libkcm.so` plus a thin ctypes binding.

Importing the package loads nothing; `paper_1712_05012_b300.kcm` loads the CUDA library.
"""
