"""GB300-native (sm_103a) particle-decomposition Gamma-SPH-ALE hot path.

The compute path lives in the CUDA library libgsph.so (csrc/), reached through the C-ABI declared in
include/gsph.h; gsph.py is its thin ctypes binding. scenes.py holds the seeded input generators.
Importing the package loads nothing; gsph.load() loads the CUDA library and fails loudly if it is
missing.
"""
