"""GB300-native (sm_103a, FP64) BSSN + fluid evolution for PBH formation.

The compute path is the CUDA library ``libcosmos_gb300.so`` (C ABI in
``include/cosmos.h``); ``cosmos`` is its ctypes binding, ``evolve`` holds the
torch-level helpers that allocate device buffers and call the binding, and
``inputs`` the seeded synthetic-input generators.  Importing the package
loads nothing; the library is loaded on first use and its absence raises.
"""
