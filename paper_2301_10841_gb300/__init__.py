"""GB300-native Free Join: COLT index building and vectorized plan execution.

The compute path lives in ``libfj.so`` (hand-written CUDA for sm_103a behind a
C ABI, declared in ``include/fj.h``).  :mod:`paper_2301_10841_gb300.fj` is the
thin ctypes binding; :mod:`paper_2301_10841_gb300.datagen` draws seeded
synthetic inputs.  Importing this package does not load the library; importing
``fj`` does, and fails loudly when it is missing.
"""
