"""GB300-native hybrid nodal-staggered PSATD particle-in-cell step.

The compute path lives in the CUDA library ``libpic`` (C ABI declared in
``include/pic.h``); :mod:`paper_2106_12919_gb300.pic` is the thin ctypes binding
and :mod:`paper_2106_12919_gb300.workloads` the seeded synthetic inputs.
Importing the package itself loads nothing; the library is loaded on first use
of :mod:`paper_2106_12919_gb300.pic` and a missing library is a hard error.
"""
