"""GB300 (sm_103a) spectral-element screened-Poisson solver.

The compute path is the C-ABI library libsem.so (include/sem.h), built in-tree
by paper_1506_05996_gb300.build. `from paper_1506_05996_gb300 import sem`
loads it and raises if it is missing: there is no fallback implementation.
"""
