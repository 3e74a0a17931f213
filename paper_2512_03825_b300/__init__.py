"""B300-native Parallel Tempering for the periodic 2D Ising model (arXiv 2512.03825).

The compute path lives in ``libpt.so`` (hand-written sm_103a CUDA behind a C ABI declared in
``include/pt.h``); this package is its thin ctypes binding. Importing the package does not
load the library; the first call that needs it does, and fails loudly if it is missing.
"""
